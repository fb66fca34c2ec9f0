// haf_lowrank.cu -- hafnian of a low-rank matrix A = G G^T (App. C).
//
// For G with n rows and r columns, haf(G G^T) depends only on the entries
// above the diagonal, and App. C expresses it through the coefficients of
//     q(x_1..x_r) = prod_{i=1}^{n} sum_{j=1}^{r} g_ij x_j            (eq. q)
// as   haf = sum over even exponent vectors e of lambda_e prod_j (e_j - 1)!!
// (eq. qexp and the sum after it; (a)!! = 1 for a <= 0).
//
// GPU form.  The expansion is built one row at a time: after k rows the
// state is the vector of coefficients of all monomials of degree k, one per
// composition e of k into r non-negative parts (C(k+r-1, r-1) of them),
// and row k+1 maps it to degree k+1 by
//     new[e] = sum_{j : e_j >= 1} g_{k+1, j} old[e - u_j].
// Compositions are ranked with the combinatorial number system of their
// "stars and bars" form (bar positions c_t = e_0 + .. + e_t + t, rank =
// sum_t C(c_t, t+1)), so the state is a dense array in HBM and the rank of
// e - u_j follows from the bars of e by lowering the bars t >= j by one.
// One launch per row streams the degree-k array into the degree-(k+1)
// array.  A warp takes a segment of consecutive ranks, 32 at a time (lane l
// the rank base + l), so its writes coalesce and the predecessor reads of
// one term j mostly fall in the same lines.  Each lane finds the bars of
// its first rank by a search in the binomial table and then steps them 32
// ranks forward at a time, so the search is paid once per segment.  Two
// walks do the stepping (the rank r is a template parameter, so the bars
// stay in registers):
//  - the bar walk (small r) steps all r - 1 bars in colex order: the lowest
//    bar moves along its row, a carry moves to the next row;
//  - the cube walk (large r) keeps, per "cube" of compositions that share
//    the upper bars c_3.., the constants that turn the offset in the cube
//    into predecessor ranks, and steps only the three lowest bars.
// On GB300 a step is bound by its FP64 multiply-adds: five DFMA per term
// (a complex multiply-add and the |g| recurrence's), not by its HBM
// traffic.
// The same recurrence on |g_ij| gives, at the end, abs_sum =
// sum_e Lambda_e prod (e_j - 1)!!, the scale of the rounding error (every
// summand's magnitude bound), reported like the subset path's sum |f(Z)|.
// The final sum over even e is a fixed-order double-double reduction.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/hafnian_gb300.h"
#include "haf_internal.h"
#include "haf_nvtx.h"

namespace hafgb {
namespace {

struct __align__(16) zc {
  double re, im;
};

constexpr int kLrThreads = 256;
constexpr int kLowRankMaxR = HAF_LOWRANK_MAX_R;
constexpr int kLrSumBlocks = 1024;  // fixed: the reduction order depends on it
// Ranks from which the step uses the cube walk (both walks give the same
// results bit for bit: the same terms in the same order).  Both kernels are
// bound by the FP64 multiply-adds (5 DFMA per term); the cube walk moves
// less DRAM traffic at r = 8 and is 2 % faster there, the bar walk, with
// twice the resident warps, is faster at r = 6.
constexpr int kLrCubeMinR = 7;

// Binomial table b[a * (R + 1) + c] = C(a, c) (saturating at 2^64 - 1) for
// 0 <= a <= n + R, 0 <= c <= R; (x - 1)!! for x <= n; the degree-0 state.
__global__ void lowrank_tables(uint64_t* __restrict__ b, int A, int R, double* __restrict__ df, int n,
                               zc* __restrict__ z0, double* __restrict__ a0) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int a = 0; a <= A; ++a)
    for (int c = 0; c <= R; ++c) {
      uint64_t v;
      if (c == 0) v = 1;
      else if (a == 0) v = 0;
      else {
        const uint64_t x = b[(a - 1) * (R + 1) + c - 1], y = b[(a - 1) * (R + 1) + c];
        v = x + y < x ? ~0ull : x + y;  // Pascal's rule, saturating
      }
      b[a * (R + 1) + c] = v;
    }
  df[0] = 1.0;
  if (n >= 1) df[1] = 1.0;
  for (int x = 2; x <= n; ++x) df[x] = df[x - 2] * (double)(x - 1);
  z0[0] = zc{1.0, 0.0};
  a0[0] = 1.0;
}

// Bars of the composition with rank `idx` of degree k into R parts:
// c[0] < ... < c[R-2] in [0, k+R-2], rank = sum_t C(c[t], t+1).  Each bar
// is the largest v with C(v, t+1) <= the remaining rank (binary search).
template <int R>
__host__ __device__ __forceinline__ void unrank_bars(uint64_t idx, int k, const uint64_t* b, int* c) {
  int hi = k + R - 2;
#pragma unroll
  for (int t = R - 2; t >= 0; --t) {
    int lo = t;  // C(t, t+1) = 0 <= idx always
    int top = hi;
    while (lo < top) {
      const int mid = (lo + top + 1) >> 1;
      if (b[mid * (R + 1) + t + 1] <= idx) lo = mid;
      else top = mid - 1;
    }
    c[t] = lo;
    idx -= b[lo * (R + 1) + t + 1];
    hi = lo - 1;
  }
}

// Step the bars d ranks forward in colex order (the caller guarantees that
// rank + d is a composition of the same degree; `top` = k + R - 1 is the
// virtual bar above the last).  Within a row (bars 1.. fixed) the lowest bar
// just moves; past the row's end the next row is the colex successor of the
// upper bars: the lowest bar t >= 1 with room above it moves up by one and
// the bars below it go to their least places 0, 1, ...
template <int R>
__host__ __device__ __forceinline__ void advance_bars(int* c, int top, int d) {
  if constexpr (R >= 2) {
    while (d > 0) {
      int nxt;
      if constexpr (R >= 3) nxt = c[1];
      else nxt = top;
      const int room = nxt - 1 - c[0];
      if (d <= room) {
        c[0] += d;
        return;
      }
      d -= room + 1;
      if constexpr (R >= 3) {
        int t = R - 2;
#pragma unroll
        for (int s = R - 3; s >= 1; --s)
          if (c[s] + 1 < c[s + 1]) t = s;
#pragma unroll
        for (int s = 0; s <= R - 2; ++s) {
          if (s == t) c[s] += 1;
          else if (s < t) c[s] = s;
        }
      }
    }
  }
}

// Calls f(j, rank(e - u_j)) for every j with e_j >= 1, in the order
// j = 0..R-1, for the composition e of degree top - R + 1 with bars c.
// The predecessor ranks follow from prefix sums of C(c_t, t+1) and suffix
// sums of C(c_t - 1, t+1):
//   rank(e - u_j) = sum_{t<j} C(c_t, t+1) + sum_{t>=j} C(c_t - 1, t+1).
// C(c, 1) and C(c, 2) are computed; the rest come from the binomial table b.
template <int R, class F>
__host__ __device__ __forceinline__ void for_each_pred(const int* c, int top, const uint64_t* b, F&& f) {
  // C(c_t, t+1) (lo = false) or C(c_t - 1, t+1) (lo = true); c_t >= t
  auto bin = [&](int t, int ct, bool lo) -> uint64_t {
    const uint64_t v = (uint64_t)(lo ? ct - 1 : ct);
    if (t == 0) return ct > 0 ? v : 0;
    if (t == 1) return ct > (lo ? 1 : 0) ? v * (v - 1) / 2 : 0;
    return b[(lo ? ct - 1 : ct) * (R + 1) + t + 1];
  };
  uint64_t suf = 0;  // sum_{t>=j} C(c_t - 1, t+1), from j = 0
#pragma unroll
  for (int t = 0; t < R - 1; ++t) suf += bin(t, c[t], true);
  uint64_t pre = 0;  // sum_{t<j} C(c_t, t+1)
  int cp = -1;
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int cj = j < R - 1 ? c[j] : top;
    if (cj - cp >= 2) f(j, pre + suf);  // e_j = cj - cp - 1 >= 1
    if (j < R - 1) {
      pre += bin(j, cj, false);
      suf -= bin(j, cj, true);
    }
    cp = cj;
  }
}

// C(v, 2) and C(v, 3) for bar positions v <= HAF_LOWRANK_MAX_N +
// HAF_LOWRANK_MAX_R (both fit 32 bits).
__host__ __device__ __forceinline__ uint32_t binom2(int v) { return v < 2 ? 0u : (uint32_t)v * (v - 1) / 2; }
__host__ __device__ __forceinline__ uint32_t binom3(int v) {
  return v < 3 ? 0u : (uint32_t)v * (uint32_t)(v - 1) * (uint32_t)(v - 2) / 6;
}

// Cube walk (R >= 4).  The compositions with the same upper bars
// c_3..c_{R-2} form a "cube" of C(c_3, 3) consecutive ranks (c_3 is the
// virtual top bar when R == 4), in which the offset o = C(c_2, 3) +
// C(c_1, 2) + c_0 fixes the three lowest bars.  Per cube the walk keeps the
// upper bars and the constants K_j (j = 3..R-1) with
//   rank(e - u_j) = o + K_j                       (j >= 3),
//   rank(e - u_j) = [the t <= 2 terms] + K_3      (j <= 2),
// K_3 = sum_{t>=3} C(c_t - 1, t+1), K_{j+1} = K_j + C(c_j, t+1) - C(c_j - 1,
// t+1) at t = j, so K_{R-1} is the cube's first rank.  A lane steps o by 32
// and moves to the next cube when o passes the cube's size; the three
// lowest bars come from o by a cube and a square root and a +-1 correction,
// so the table in shared memory is read only at cube changes.
template <int R>
struct CubeWalk {
  static constexpr int NH = R > 4 ? R - 4 : 1;
  int h[NH];       // c_3..c_{R-2}
  int top;         // the virtual bar above the last
  int c3top;       // c_3, or top when R == 4
  uint32_t size;   // C(c3top, 3)
  uint32_t vmask;  // bit j (4 <= j < R): e_j >= 1 in this cube
  uint64_t K[R - 3];

  // the cube of rank idx (degree k) and the offset of idx in it
  __host__ __device__ __forceinline__ void init(uint64_t idx, int k, const uint64_t* b, uint32_t* o) {
    top = k + R - 1;
    int hi = k + R - 2;
#pragma unroll
    for (int t = R - 2; t >= 3; --t) {
      int lo = t;
      int tp = hi;
      while (lo < tp) {
        const int mid = (lo + tp + 1) >> 1;
        if (b[mid * (R + 1) + t + 1] <= idx) lo = mid;
        else tp = mid - 1;
      }
      h[t - 3] = lo;
      idx -= b[lo * (R + 1) + t + 1];
      hi = lo - 1;
    }
    *o = (uint32_t)idx;
    constants(b);
  }
  __host__ __device__ __forceinline__ int bar(int t) const { return t <= R - 2 ? h[t - 3] : top; }
  __host__ __device__ __forceinline__ void constants(const uint64_t* b) {
    c3top = R > 4 ? h[0] : top;
    size = binom3(c3top);
    uint64_t k3 = 0;
#pragma unroll
    for (int t = 3; t <= R - 2; ++t) k3 += b[(h[t - 3] - 1) * (R + 1) + t + 1];
    K[0] = k3;
#pragma unroll
    for (int j = 3; j <= R - 2; ++j)
      K[j - 2] = K[j - 3] + b[h[j - 3] * (R + 1) + j + 1] - b[(h[j - 3] - 1) * (R + 1) + j + 1];
    vmask = 0;
#pragma unroll
    for (int j = 4; j < R; ++j)
      if (bar(j) - bar(j - 1) >= 2) vmask |= 1u << j;
  }
  // the next cube in rank order: the colex successor of the upper bars
  __host__ __device__ __forceinline__ void next(const uint64_t* b) {
    if constexpr (R > 4) {
      int t = R - 2;
#pragma unroll
      for (int s = R - 3; s >= 3; --s)
        if (h[s - 3] + 1 < h[s - 2]) t = s;
#pragma unroll
      for (int s = 3; s <= R - 2; ++s) {
        if (s == t) h[s - 3] += 1;
        else if (s < t) h[s - 3] = s;
      }
      constants(b);
    }
  }
  // the three lowest bars of the composition at offset o of this cube:
  // c2 the largest v < c3top with C(v, 3) <= o, then c1 and c0 likewise
  // (estimates by a cube and a square root, corrected exactly)
  __host__ __device__ __forceinline__ void decompose(uint32_t o, int* c) const {
    int v = (int)cbrtf(6.0f * (float)o) + 1;
    v = v < 2 ? 2 : (v > c3top - 1 ? c3top - 1 : v);
    while (binom3(v) > o) --v;
    while (v + 1 < c3top && binom3(v + 1) <= o) ++v;
    const uint32_t rem = o - binom3(v);
    int u = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)rem)) * 0.5f);
    u = u < 1 ? 1 : (u > v - 1 ? v - 1 : u);
    while (binom2(u) > rem) --u;
    while (u + 1 < v && binom2(u + 1) <= rem) ++u;
    c[0] = (int)(rem - binom2(u));
    c[1] = u;
    c[2] = v;
  }
  // f(j, rank(e - u_j)) for every j with e_j >= 1, j = 0..R-1, for the
  // composition at offset o of this cube, whose lowest bars are c[0..2]
  template <class F>
  __host__ __device__ __forceinline__ void preds(uint32_t o, const int* c, F&& f) const {
    const int c0 = c[0], c1 = c[1], c2 = c[2];
    const uint64_t b12 = (uint64_t)binom2(c1 - 1) + binom3(c2 - 1) + K[0];
    if (c0 >= 1) f(0, (uint64_t)(c0 - 1) + b12);
    if (c1 - c0 >= 2) f(1, (uint64_t)c0 + b12);
    if (c2 - c1 >= 2) f(2, (uint64_t)c0 + binom2(c1) + binom3(c2 - 1) + K[0]);
    if (c3top - c2 >= 2) f(3, (uint64_t)o + K[0]);
#pragma unroll
    for (int j = 4; j < R; ++j)
      if (vmask >> j & 1u) f(j, (uint64_t)o + K[j - 3]);
  }
};

// Step the three lowest bars d offsets forward inside one cube (the caller
// guarantees the target offset is in the cube): c0 moves along its row of
// length c1; past the row's end, (c1, c2) takes its colex successor.
__host__ __device__ __forceinline__ void advance3(int* c, int d) {
  while (d > 0) {
    const int room = c[1] - 1 - c[0];
    if (d <= room) {
      c[0] += d;
      return;
    }
    d -= room + 1;
    if (c[1] + 1 < c[2]) {
      c[1] += 1;
    } else {
      c[2] += 1;
      c[1] = 1;
    }
    c[0] = 0;
  }
}

// Degree k-1 -> k for R >= 4 by the cube walk; the same segments and the
// same order of the terms (j = 0..R-1) as lowrank_step.
template <int R>
__global__ void __launch_bounds__(kLrThreads, R <= 10 ? 2 : 1)
    lowrank_step_cube(const zc* __restrict__ old, const double* __restrict__ old_abs, zc* __restrict__ nw,
                      double* __restrict__ nw_abs, const zc* __restrict__ grow, int k,
                      const uint64_t* __restrict__ binom, uint64_t count, int seg_tiles) {
  // shared: the binomial table (read at cube changes); the row of G and its
  // moduli stay in registers, so that the up to 2R gathers of a monomial
  // can all be in flight at once
  extern __shared__ __align__(16) uint64_t sbc[];
  const int tab = (k + R + 1) * (R + 1);
  for (int i = threadIdx.x; i < tab; i += blockDim.x) sbc[i] = binom[i];
  __syncthreads();
  zc g[R];
  double ga[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    g[j] = grow[j];
    ga[j] = hypot(g[j].re, g[j].im);
  }
  const int lane = threadIdx.x & 31;
  const uint64_t seg = 32ull * (uint64_t)seg_tiles;
  const uint64_t nseg = (count + seg - 1) / seg;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t sg = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; sg < nseg; sg += nwarps) {
    const uint64_t end = min(count, (sg + 1) * seg);
    uint64_t idx = sg * seg + lane;
    if (idx >= end) continue;
    CubeWalk<R> w;
    uint32_t o;
    w.init(idx, k, sbc, &o);
    while (o >= w.size) {  // (init leaves o inside its cube; kept for symmetry)
      o -= w.size;
      w.next(sbc);
    }
    int c[3];
    w.decompose(o, c);
    for (;;) {
      double ar = 0.0, ai = 0.0, aa = 0.0;
      w.preds(o, c, [&](int j, uint64_t p) {
        const zc v = old[p];
        ar = fma(g[j].re, v.re, fma(-g[j].im, v.im, ar));
        ai = fma(g[j].re, v.im, fma(g[j].im, v.re, ai));
        aa = fma(ga[j], old_abs[p], aa);
      });
      nw[idx] = zc{ar, ai};
      nw_abs[idx] = aa;
      idx += 32;
      if (idx >= end) break;
      o += 32;
      if (o < w.size) {
        advance3(c, 32);
      } else {
        do {
          o -= w.size;
          w.next(sbc);
        } while (o >= w.size);
        w.decompose(o, c);
      }
    }
  }
}

// Degree k-1 -> k for the ranks [0, count): warp w takes the segments
// w, w + W, ... of 32 * seg_tiles ranks.
template <int R>
__global__ void __launch_bounds__(kLrThreads, R <= 8 ? 4 : 2)
    lowrank_step(const zc* __restrict__ old, const double* __restrict__ old_abs, zc* __restrict__ nw,
                 double* __restrict__ nw_abs, const zc* __restrict__ grow, int k, const uint64_t* __restrict__ binom,
                 uint64_t count, int seg_tiles) {
  // shared: the binomial table, then the row of G and its moduli (read by
  // every lane alike: broadcasts, and no registers held for them)
  extern __shared__ __align__(16) uint64_t sb[];
  const int tab = (k + R + 1) * (R + 1);
  zc* const g = reinterpret_cast<zc*>(sb + tab + (tab & 1));
  double* const ga = reinterpret_cast<double*>(g + R);
  for (int i = threadIdx.x; i < tab; i += blockDim.x) sb[i] = binom[i];
  if (threadIdx.x < R) {
    const zc v = grow[threadIdx.x];
    g[threadIdx.x] = v;
    ga[threadIdx.x] = hypot(v.re, v.im);
  }
  __syncthreads();
  constexpr int NB = R > 1 ? R - 1 : 1;
  const int lane = threadIdx.x & 31;
  const int top = k + R - 1;
  const uint64_t seg = 32ull * (uint64_t)seg_tiles;
  const uint64_t nseg = (count + seg - 1) / seg;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t sg = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; sg < nseg; sg += nwarps) {
    const uint64_t end = min(count, (sg + 1) * seg);
    uint64_t idx = sg * seg + lane;
    if (idx >= end) continue;
    int c[NB];
    if constexpr (R >= 2) unrank_bars<R>(idx, k, sb, c);
    for (;;) {
      double ar = 0.0, ai = 0.0, aa = 0.0;
      for_each_pred<R>(c, top, sb, [&](int j, uint64_t o) {
        const zc v = old[o];
        const zc gj = g[j];
        ar = fma(gj.re, v.re, fma(-gj.im, v.im, ar));
        ai = fma(gj.re, v.im, fma(gj.im, v.re, ai));
        aa = fma(ga[j], old_abs[o], aa);
      });
      nw[idx] = zc{ar, ai};
      nw_abs[idx] = aa;
      idx += 32;
      if (idx >= end) break;
      advance_bars<R>(c, top, 32);
    }
  }
}

__device__ __forceinline__ void two_sum_lr(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void dd_add_lr(double& hi, double& lo, double xh, double xl) {
  double s, e;
  two_sum_lr(hi, xh, s, e);
  e += lo + xl;
  hi = s + e;
  lo = e - (hi - s);
}

// For the composition e with bars c (top = its degree + R - 1): whether
// every e_j is even, and then w = prod_j (e_j - 1)!! (df[x] = (x - 1)!!),
// multiplied in the order j = 0..R-1.
template <int R>
__host__ __device__ __forceinline__ bool even_weight(const int* c, int top, const double* df, double* w) {
  double p = 1.0;
  bool even = true;
  int cp = -1;
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int cj = j < R - 1 ? c[j] : top;
    const int e = cj - cp - 1;
    if (e & 1) even = false;
    else if (even) p *= df[e];
    cp = cj;
  }
  *w = p;
  return even;
}

// Fixed-order reduction of lambda_e prod (e_j - 1)!! over the even
// compositions of degree n: thread t of the grid (T threads, T fixed) takes
// the contiguous ranks [t * per, (t + 1) * per), finding the bars of its
// first rank by search and stepping them one rank at a time; blocks combine
// in a fixed tree and block partials go to `part` (re_hi, re_lo, im_hi,
// im_lo, abs).
template <int R>
__global__ void __launch_bounds__(kLrThreads) lowrank_even_sum(const zc* __restrict__ lam,
                                                               const double* __restrict__ lam_abs, int n,
                                                               const uint64_t* __restrict__ binom,
                                                               const double* __restrict__ dfact, uint64_t count,
                                                               double* __restrict__ part) {
  extern __shared__ uint64_t sb[];
  const int tab = (n + R + 1) * (R + 1);
  for (int i = threadIdx.x; i < tab; i += blockDim.x) sb[i] = binom[i];
  __syncthreads();
  __shared__ double red[5][kLrThreads];
  double rh = 0, rl = 0, ih = 0, il = 0, ab = 0;
  auto add = [&](uint64_t idx, double w) {
    const zc v = lam[idx];
    dd_add_lr(rh, rl, v.re * w, fma(v.re, w, -(v.re * w)));
    dd_add_lr(ih, il, v.im * w, fma(v.im, w, -(v.im * w)));
    ab += lam_abs[idx] * w;
  };
  constexpr int NB = R > 1 ? R - 1 : 1;
  const int top = n + R - 1;
  const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t per = (count + T - 1) / T;
  const uint64_t lo = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) * per, hi = min(count, lo + per);
  if (lo < hi) {
    int c[NB];
    if constexpr (R >= 2) unrank_bars<R>(lo, n, sb, c);
    for (uint64_t idx = lo;;) {
      double w;
      if (even_weight<R>(c, top, dfact, &w)) add(idx, w);
      if (++idx >= hi) break;
      advance_bars<R>(c, top, 1);
    }
  }
  red[0][threadIdx.x] = rh;
  red[1][threadIdx.x] = rl;
  red[2][threadIdx.x] = ih;
  red[3][threadIdx.x] = il;
  red[4][threadIdx.x] = ab;
  __syncthreads();
  for (int s = 1; s < blockDim.x; s <<= 1) {
    if ((threadIdx.x & (2 * s - 1)) == 0 && threadIdx.x + s < blockDim.x) {
      double a0 = red[0][threadIdx.x], a1 = red[1][threadIdx.x];
      double b0 = red[2][threadIdx.x], b1 = red[3][threadIdx.x];
      dd_add_lr(a0, a1, red[0][threadIdx.x + s], red[1][threadIdx.x + s]);
      dd_add_lr(b0, b1, red[2][threadIdx.x + s], red[3][threadIdx.x + s]);
      red[0][threadIdx.x] = a0;
      red[1][threadIdx.x] = a1;
      red[2][threadIdx.x] = b0;
      red[3][threadIdx.x] = b1;
      red[4][threadIdx.x] += red[4][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 5; ++q) part[5 * (size_t)blockIdx.x + q] = red[q][0];
}

__global__ void lowrank_finish(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double rh = 0, rl = 0, ih = 0, il = 0, ab = 0;
  for (int b = 0; b < nblocks; ++b) {
    const double* p = part + 5 * (size_t)b;
    dd_add_lr(rh, rl, p[0], p[1]);
    dd_add_lr(ih, il, p[2], p[3]);
    ab += p[4];
  }
  out[0] = rh;
  out[1] = ih;
  out[2] = rl;
  out[3] = il;
  out[4] = ab;
}

int lfail(int code, const std::string& msg) { return set_error(code, msg); }

uint64_t host_binom(int a, int b) {
  if (b < 0 || b > a) return 0;
  unsigned __int128 r = 1;
  for (int i = 1; i <= b; ++i) r = r * (unsigned __int128)(a - b + i) / (unsigned __int128)i;
  return r > (unsigned __int128)UINT64_MAX ? UINT64_MAX : (uint64_t)r;
}

// Workspace of one expansion (byte offsets, 256-aligned): two coefficient
// arrays and two abs arrays of the largest degree, the tables, the block
// partials of the final sum.
struct LrLayout {
  uint64_t maxcount = 0;
  size_t z0 = 0, z1 = 0, a0 = 0, a1 = 0, bt = 0, df = 0, part = 0, total = 0;
};

bool lr_layout(int n, int r, LrLayout* L) {
  L->maxcount = host_binom(n + r - 1, r - 1);
  if (L->maxcount >= ((uint64_t)1 << 40)) return false;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t off = 0;
  L->z0 = off;
  off += al((size_t)L->maxcount * sizeof(zc));
  L->z1 = off;
  off += al((size_t)L->maxcount * sizeof(zc));
  L->a0 = off;
  off += al((size_t)L->maxcount * sizeof(double));
  L->a1 = off;
  off += al((size_t)L->maxcount * sizeof(double));
  L->bt = off;
  off += al((size_t)(n + r + 1) * (r + 1) * sizeof(uint64_t));
  L->df = off;
  off += al((size_t)(n + 1) * sizeof(double));
  L->part = off;
  off += al((size_t)kLrSumBlocks * 5 * sizeof(double));
  L->total = off;
  return true;
}

// Dynamic shared memory of lowrank_step for degree k: the binomial rows
// 0..k+R (padded to 16 bytes), the row of G, its moduli.
template <int R>
size_t step_smem(int k) {
  const size_t tab = (size_t)(k + R + 1) * (R + 1);
  return (tab + (tab & 1)) * sizeof(uint64_t) + R * (sizeof(zc) + sizeof(double));
}

// The whole expansion on one stream: tables, n row steps, the even sum.
template <int R>
cudaError_t run_expansion(const zc* G, int n, char* w, const LrLayout& L, double* d_out, cudaStream_t st) {
  int dev = 0, sms = 0, nb = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem_n = (size_t)(n + R + 1) * (R + 1) * sizeof(uint64_t);
  // R >= kLrCubeMinR: the cube walk; smaller R: the bar walk
  if (e == cudaSuccess) {
    if constexpr (R >= kLrCubeMinR)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, lowrank_step_cube<R>, kLrThreads, step_smem<R>(n));
    else
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, lowrank_step<R>, kLrThreads, step_smem<R>(n));
  }
  if (e != cudaSuccess) return e;
  sms = std::max(sms, 1);
  nb = std::max(nb, 1);
  zc* z[2] = {(zc*)(w + L.z0), (zc*)(w + L.z1)};
  double* za[2] = {(double*)(w + L.a0), (double*)(w + L.a1)};
  const uint64_t* bt = (const uint64_t*)(w + L.bt);
  lowrank_tables<<<1, 1, 0, st>>>((uint64_t*)(w + L.bt), n + R, R, (double*)(w + L.df), n, z[0], za[0]);
  const uint64_t warps = (uint64_t)sms * nb * (kLrThreads / 32);
  int cur = 0;
  for (int k = 1; k <= n; ++k) {
    const uint64_t cnt = host_binom(k + R - 1, R - 1);
    // segments of 32 * seg_tiles ranks, about four per resident warp
    const uint64_t tiles = std::max<uint64_t>(1, std::min<uint64_t>(16, cnt / (32 * warps * 4)));
    const uint64_t nseg = (cnt + 32 * tiles - 1) / (32 * tiles);
    const uint64_t want = (nseg + kLrThreads / 32 - 1) / (kLrThreads / 32);
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sms * nb));
    if constexpr (R >= kLrCubeMinR)
      lowrank_step_cube<R><<<grid, kLrThreads, step_smem<R>(k), st>>>(z[cur], za[cur], z[cur ^ 1], za[cur ^ 1],
                                                                     G + (size_t)(k - 1) * R, k, bt, cnt, (int)tiles);
    else
      lowrank_step<R><<<grid, kLrThreads, step_smem<R>(k), st>>>(z[cur], za[cur], z[cur ^ 1], za[cur ^ 1],
                                                                G + (size_t)(k - 1) * R, k, bt, cnt, (int)tiles);
    cur ^= 1;
  }
  lowrank_even_sum<R><<<kLrSumBlocks, kLrThreads, smem_n, st>>>(z[cur], za[cur], n, bt, (const double*)(w + L.df),
                                                                L.maxcount, (double*)(w + L.part));
  lowrank_finish<<<1, 32, 0, st>>>((const double*)(w + L.part), kLrSumBlocks, d_out);
  return cudaGetLastError();
}

cudaError_t run_rank(int r, const zc* G, int n, char* w, const LrLayout& L, double* d_out, cudaStream_t st) {
  switch (r) {
#define LR_CASE(R) \
  case R:          \
    return run_expansion<R>(G, n, w, L, d_out, st);
    LR_CASE(1) LR_CASE(2) LR_CASE(3) LR_CASE(4) LR_CASE(5) LR_CASE(6) LR_CASE(7) LR_CASE(8)
    LR_CASE(9) LR_CASE(10) LR_CASE(11) LR_CASE(12) LR_CASE(13) LR_CASE(14) LR_CASE(15) LR_CASE(16)
#undef LR_CASE
    default:
      return cudaErrorInvalidValue;
  }
}
static_assert(kLowRankMaxR == 16, "run_rank instantiates r = 1..16");

// Per-device stream and workspace kept between calls of the host entry
// point (calls are serialised by the mutex).  Workspaces up to kLrKeepBytes
// stay allocated, so repeated small expansions pay no cudaMalloc/cudaFree;
// larger ones are released after their call.
constexpr size_t kLrKeepBytes = (size_t)256 << 20;
struct LrDevice {
  cudaStream_t st = nullptr;
  char* buf = nullptr;
  size_t bytes = 0;
};
std::mutex g_lr_mu;
std::map<int, LrDevice> g_lr_dev;

}  // namespace
}  // namespace hafgb

using namespace hafgb;

extern "C" size_t haf_lowrank_workspace_bytes(int64_t n, int64_t r) {
  if (n < 2 || n > HAF_LOWRANK_MAX_N || (n & 1) || r < 1 || r > HAF_LOWRANK_MAX_R) return 0;
  LrLayout L;
  return lr_layout((int)n, (int)r, &L) ? L.total : 0;
}

extern "C" int haf_lowrank_launch(const double* dG, int64_t n64, int64_t r64, double* d_out, void* d_work,
                                  size_t ws_bytes, void* stream) {
  const NvtxRange nvtx_range("haf_lowrank_launch");
  if (!dG || !d_out || !d_work || n64 < 2 || n64 > HAF_LOWRANK_MAX_N || (n64 & 1) || r64 < 1 ||
      r64 > HAF_LOWRANK_MAX_R)
    return lfail(HAF_EINVAL, "haf_lowrank_launch: need device pointers, even 2 <= n <= HAF_LOWRANK_MAX_N, "
                             "1 <= r <= HAF_LOWRANK_MAX_R");
  if (reinterpret_cast<uintptr_t>(d_work) % 256 != 0)
    return lfail(HAF_EINVAL, "haf_lowrank_launch: workspace not 256-byte aligned");
  LrLayout L;
  if (!lr_layout((int)n64, (int)r64, &L)) return lfail(HAF_ENOMEM, "haf_lowrank_launch: expansion too large");
  if (ws_bytes < L.total) return lfail(HAF_ESMALL, "haf_lowrank_launch: workspace too small");
  const cudaError_t e = run_rank((int)r64, reinterpret_cast<const zc*>(dG), (int)n64, static_cast<char*>(d_work), L,
                                 d_out, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return lfail(HAF_ECUDA, std::string("haf_lowrank_launch: ") + cudaGetErrorString(e));
  return HAF_OK;
}

extern "C" int haf_lowrank_c128(const double* G, int64_t n64, int64_t r64, double* out, haf_info* info) {
  const NvtxRange nvtx_range("haf_lowrank");
  if (!out || n64 < 0 || n64 > HAF_LOWRANK_MAX_N || r64 < 1 || r64 > HAF_LOWRANK_MAX_R || (n64 > 0 && !G))
    return lfail(HAF_EINVAL, "haf_lowrank_c128: need 0 <= n <= HAF_LOWRANK_MAX_N, 1 <= r <= HAF_LOWRANK_MAX_R");
  const int n = (int)n64, r = (int)r64;
  const auto t0 = std::chrono::steady_clock::now();
  auto report = [&](double re, double im, double lre, double lim, double abs_sum, int64_t terms, int64_t launches) {
    out[0] = re;
    out[1] = im;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = haf_info{abs_sum, {lre, lim}, terms, secs, launches};
  };
  if (n == 0) {
    report(1.0, 0.0, 0.0, 0.0, 1.0, 0, 0);
    return HAF_OK;
  }
  if (n & 1) {
    report(0.0, 0.0, 0.0, 0.0, 0.0, 0, 0);
    return HAF_OK;
  }
  LrLayout L;
  if (!lr_layout(n, r, &L)) return lfail(HAF_ENOMEM, "haf_lowrank_c128: expansion too large");
  size_t freeb = 0, totalb = 0;
  cudaError_t e = cudaMemGetInfo(&freeb, &totalb);
  if (e != cudaSuccess) return lfail(HAF_ECUDA, std::string("haf_lowrank_c128: ") + cudaGetErrorString(e));
  // G and the 5-double result after the workspace
  const size_t o_g = L.total, o_out = o_g + (((size_t)n * r * sizeof(zc) + 255) & ~(size_t)255);
  const size_t need = o_out + 256;
  std::lock_guard<std::mutex> lk(g_lr_mu);
  int dev = 0;
  cudaGetDevice(&dev);
  LrDevice& ld = g_lr_dev[dev];
  if (ld.bytes < need && need + ((size_t)64 << 20) > (freeb + ld.bytes) / 10 * 9)
    return lfail(HAF_ENOMEM, "haf_lowrank_c128: the expansion does not fit the free device memory");
  if (!ld.st) {
    e = cudaStreamCreateWithFlags(&ld.st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      ld.st = nullptr;
      return lfail(HAF_ECUDA, std::string("haf_lowrank_c128: ") + cudaGetErrorString(e));
    }
  }
  if (ld.bytes < need) {
    if (ld.buf) cudaFree(ld.buf);
    ld.buf = nullptr;
    ld.bytes = 0;
    e = cudaMalloc(&ld.buf, need);
    if (e != cudaSuccess) return lfail(HAF_ENOMEM, std::string("haf_lowrank_c128: ") + cudaGetErrorString(e));
    ld.bytes = need;
  }
  char* dbuf = ld.buf;
  cudaStream_t st = ld.st;
  auto done = [&](int rc) {
    if (ld.bytes > kLrKeepBytes) {  // do not hold a large expansion's memory
      cudaStreamSynchronize(st);
      cudaFree(ld.buf);
      ld.buf = nullptr;
      ld.bytes = 0;
    }
    return rc;
  };
  e = cudaMemcpyAsync(dbuf + o_g, G, (size_t)n * r * sizeof(zc), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = run_rank(r, (const zc*)(dbuf + o_g), n, dbuf, L, (double*)(dbuf + o_out), st);
  double res[5];
  if (e == cudaSuccess) e = cudaMemcpyAsync(res, dbuf + o_out, sizeof(res), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return done(lfail(HAF_ECUDA, std::string("haf_lowrank_c128: ") + cudaGetErrorString(e)));
  report(res[0] + res[2], res[1] + res[3], res[2], res[3], res[4], (int64_t)L.maxcount, (int64_t)n + 3);
  return done(HAF_OK);
}
