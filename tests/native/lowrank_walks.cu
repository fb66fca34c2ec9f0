// Host-side check of the low-rank step kernels' index logic (no GPU): the
// device helpers of haf_lowrank.cu are __host__ __device__, so this program
// includes the file and runs them on the CPU against brute-force
// enumeration of compositions:
//  - unrank_bars + advance_bars (the bar walk of lowrank_step and of the
//    even sum): every lane's walk through its segment, the bars of every
//    rank, and for_each_pred's predecessor ranks (all in bounds);
//  - CubeWalk (lowrank_step_cube): init, decompose, advance3 and the cube
//    changes along every lane's walk, and the predecessor ranks;
//  - the cube offset decomposition for every offset of every cube size up
//    to bar position 142 (n + r at the largest sizes), and advance3 from
//    every start for steps of 1 and 32;
//  - even_weight's parity test.
// Exit status 0 and "walks ok" on success.
#include "../../paper_1805_12498_gb300/csrc/haf_lowrank.cu"

#include <algorithm>
#include <cstdio>
#include <vector>

namespace hafgb {
int set_error(int code, const std::string&) { return code; }
}  // namespace hafgb

using namespace hafgb;

namespace {

long g_fails = 0;
#define CHECK(cond, ...)                 \
  do {                                   \
    if (!(cond)) {                       \
      if (g_fails++ < 20) {              \
        std::printf(__VA_ARGS__);        \
        std::printf("\n");               \
      }                                  \
    }                                    \
  } while (0)

uint64_t binom(int a, int b) {
  if (b < 0 || a < 0 || b > a) return 0;
  unsigned __int128 r = 1;
  for (int i = 1; i <= b; ++i) r = r * (unsigned __int128)(a - b + i) / (unsigned __int128)i;
  return (uint64_t)r;
}

// rank of a composition e (parts e_0..e_{R-1}): sum_t C(c_t, t+1) over the
// bar positions c_t = e_0 + .. + e_t + t, t < R - 1
uint64_t rank_of(const std::vector<int>& e) {
  uint64_t rk = 0;
  int c = -1;
  for (size_t t = 0; t + 1 < e.size(); ++t) {
    c += e[t] + 1;
    rk += binom(c, (int)t + 1);
  }
  return rk;
}

void compositions(int k, int R, std::vector<int>& cur, std::vector<std::vector<int>>& out) {
  int s = 0;
  for (int x : cur) s += x;
  if ((int)cur.size() == R - 1) {
    cur.push_back(k - s);
    out.push_back(cur);
    cur.pop_back();
    return;
  }
  for (int v = 0; v <= k - s; ++v) {
    cur.push_back(v);
    compositions(k, R, cur, out);
    cur.pop_back();
  }
}

std::vector<std::pair<int, uint64_t>> want_preds(const std::vector<int>& e) {
  std::vector<std::pair<int, uint64_t>> w;
  for (size_t j = 0; j < e.size(); ++j)
    if (e[j] >= 1) {
      auto f = e;
      f[j]--;
      w.push_back({(int)j, rank_of(f)});
    }
  return w;
}

template <int R>
void check_rank(int kmax) {
  constexpr int NB = R > 1 ? R - 1 : 1;
  for (int k = 1; k <= kmax; ++k) {
    std::vector<uint64_t> tb((size_t)(k + R + 1) * (R + 1));
    for (int a = 0; a <= k + R; ++a)
      for (int c = 0; c <= R; ++c) tb[(size_t)a * (R + 1) + c] = binom(a, c);
    std::vector<std::vector<int>> all, byrank;
    std::vector<int> cur;
    compositions(k, R, cur, all);
    const uint64_t count = binom(k + R - 1, R - 1), oldcount = binom(k + R - 2, R - 1);
    CHECK(all.size() == count, "count R=%d k=%d", R, k);
    byrank.assign(count, {});
    for (auto& e : all) {
      const uint64_t rk = rank_of(e);
      CHECK(rk < count, "rank out of range R=%d k=%d", R, k);
      if (rk < count) byrank[rk] = e;
    }
    const int top = k + R - 1;
    std::vector<double> ones(k + 1, 1.0);
    auto check_bars = [&](uint64_t idx, const int* c, const char* what) {
      const auto& e = byrank[idx];
      int cp = -1;
      for (int t = 0; t < R - 1; ++t) {
        cp += e[t] + 1;
        CHECK(c[t] == cp, "%s bars R=%d k=%d idx=%llu t=%d: %d, want %d", what, R, k, (unsigned long long)idx, t,
              c[t], cp);
      }
      std::vector<std::pair<int, uint64_t>> got;
      for_each_pred<R>(c, top, tb.data(), [&](int j, uint64_t o) { got.push_back({j, o}); });
      CHECK(got == want_preds(e), "%s preds R=%d k=%d idx=%llu", what, R, k, (unsigned long long)idx);
      for (auto& p : got) CHECK(p.second < oldcount, "%s pred out of range", what);
      double w;
      bool even = true;
      for (int x : e) even = even && !(x & 1);
      CHECK(even_weight<R>(c, top, ones.data(), &w) == even, "even_weight R=%d k=%d", R, k);
    };
    // the bar walk of lowrank_step: segments of 32 * tiles ranks, lane l
    // from the segment's base + l in steps of 32
    for (int tiles : {1, 3, 16}) {
      const uint64_t seg = 32ull * tiles, nseg = (count + seg - 1) / seg;
      for (uint64_t sg = 0; sg < nseg; ++sg) {
        const uint64_t end = std::min<uint64_t>(count, (sg + 1) * seg);
        for (int lane = 0; lane < 32; ++lane) {
          uint64_t idx = sg * seg + lane;
          if (idx >= end) continue;
          int c[NB];
          if constexpr (R >= 2) unrank_bars<R>(idx, k, tb.data(), c);
          for (;;) {
            check_bars(idx, c, "step");
            idx += 32;
            if (idx >= end) break;
            advance_bars<R>(c, top, 32);
          }
        }
      }
    }
    // the even sum's walk: contiguous ranges, steps of 1
    for (uint64_t T : {1ull, 7ull, 64ull}) {
      const uint64_t per = (count + T - 1) / T;
      for (uint64_t th = 0; th < T; ++th) {
        const uint64_t lo = th * per, hi = std::min(count, lo + per);
        if (lo >= hi) continue;
        int c[NB];
        if constexpr (R >= 2) unrank_bars<R>(lo, k, tb.data(), c);
        for (uint64_t idx = lo;;) {
          check_bars(idx, c, "sum");
          if (++idx >= hi) break;
          advance_bars<R>(c, top, 1);
        }
      }
    }
    // the cube walk of lowrank_step_cube
    if constexpr (R >= 4) {
      for (int tiles : {1, 2, 16}) {
        const uint64_t seg = 32ull * tiles, nseg = (count + seg - 1) / seg;
        for (uint64_t sg = 0; sg < nseg; ++sg) {
          const uint64_t end = std::min<uint64_t>(count, (sg + 1) * seg);
          for (int lane = 0; lane < 32; ++lane) {
            uint64_t idx = sg * seg + lane;
            if (idx >= end) continue;
            CubeWalk<R> w;
            uint32_t o;
            w.init(idx, k, tb.data(), &o);
            CHECK(o < w.size, "cube init offset R=%d k=%d", R, k);
            int c[3];
            w.decompose(o, c);
            for (;;) {
              const auto& e = byrank[idx];
              int cp = -1;
              for (int t = 0; t < 3; ++t) {
                cp += e[t] + 1;
                CHECK(c[t] == cp, "cube bars R=%d k=%d idx=%llu t=%d", R, k, (unsigned long long)idx, t);
              }
              std::vector<std::pair<int, uint64_t>> got;
              w.preds(o, c, [&](int j, uint64_t p) { got.push_back({j, p}); });
              CHECK(got == want_preds(e), "cube preds R=%d k=%d idx=%llu", R, k, (unsigned long long)idx);
              for (auto& p : got) CHECK(p.second < oldcount, "cube pred out of range");
              idx += 32;
              if (idx >= end) break;
              o += 32;
              if (o < w.size) {
                advance3(c, 32);
              } else {
                do {
                  o -= w.size;
                  w.next(tb.data());
                } while (o >= w.size);
                w.decompose(o, c);
              }
            }
          }
        }
      }
    }
  }
}

// every offset of every cube up to bar position 142: decompose, and
// advance3 from each of the first 32 offsets in steps of 1 and 32
void check_cubes_exhaustive() {
  for (int c3top = 3; c3top <= 142; ++c3top) {
    CubeWalk<4> w;  // R = 4: one cube, c3top = top = k + 3
    std::vector<uint64_t> tb((size_t)(c3top + 2) * 5, 0);
    uint32_t o0;
    w.init(0, c3top - 3, tb.data(), &o0);
    CHECK(w.c3top == c3top && w.size == binom(c3top, 3), "cube size %d", c3top);
    std::vector<int> C0, C1, C2;
    for (int c2 = 2; c2 < c3top; ++c2)
      for (int c1 = 1; c1 < c2; ++c1)
        for (int c0 = 0; c0 < c1; ++c0) {
          C0.push_back(c0);
          C1.push_back(c1);
          C2.push_back(c2);
        }
    for (uint32_t o = 0; o < C0.size(); ++o) {
      int c[3];
      w.decompose(o, c);
      CHECK(c[0] == C0[o] && c[1] == C1[o] && c[2] == C2[o], "decompose c3top=%d o=%u", c3top, o);
    }
    for (int d : {1, 32})
      for (size_t start = 0; start < std::min<size_t>(C0.size(), 32); ++start) {
        int c[3] = {C0[start], C1[start], C2[start]};
        for (size_t o = start; o + d < C0.size(); o += d) {
          advance3(c, d);
          if (c[0] != C0[o + d] || c[1] != C1[o + d] || c[2] != C2[o + d]) {
            CHECK(false, "advance3 c3top=%d o=%zu d=%d", c3top, o, d);
            break;
          }
        }
      }
  }
}

}  // namespace

int main() {
  check_rank<1>(20);
  check_rank<2>(40);
  check_rank<3>(30);
  check_rank<4>(40);
  check_rank<5>(20);
  check_rank<6>(14);
  check_rank<7>(11);
  check_rank<8>(11);
  check_rank<10>(7);
  check_rank<12>(6);
  check_rank<16>(4);
  check_cubes_exhaustive();
  std::printf("%s (%ld failures)\n", g_fails ? "walks FAILED" : "walks ok", g_fails);
  return g_fails ? 1 : 0;
}
