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
// array, one entry per thread and grid-stride step (consecutive lanes take
// consecutive ranks, so the writes coalesce and the predecessor reads of a
// warp mostly fall in a few lines).
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

namespace hafgb {
namespace {

struct __align__(16) zc {
  double re, im;
};

constexpr int kLrThreads = 256;
constexpr int kLowRankMaxR = HAF_LOWRANK_MAX_R;

// binomial table b[a * (R + 1) + c] = C(a, c), 0 <= a <= A, 0 <= c <= R
__device__ __forceinline__ uint64_t bnm(const uint64_t* b, int R, int a, int c) {
  return (a < 0 || c < 0 || c > a) ? 0ull : b[a * (R + 1) + c];
}

// Bars of the composition with rank `idx` of degree k into r parts:
// c[0] < ... < c[r-2] in [0, k+r-2], rank = sum_t C(c[t], t+1).  Each bar
// is the largest v with C(v, t+1) <= the remaining rank (binary search).
__device__ __forceinline__ void unrank_bars(uint64_t idx, int k, int r, const uint64_t* b, int R, int* c) {
  int hi = k + r - 2;
  for (int t = r - 2; t >= 0; --t) {
    int lo = t;  // C(t, t+1) = 0 <= idx always
    int top = hi;
    while (lo < top) {
      const int mid = (lo + top + 1) >> 1;
      if (bnm(b, R, mid, t + 1) <= idx) lo = mid;
      else top = mid - 1;
    }
    c[t] = lo;
    idx -= bnm(b, R, lo, t + 1);
    hi = lo - 1;
  }
}

// One entry per thread and grid-stride step, so consecutive lanes write
// (and mostly read) consecutive ranks.  The predecessor ranks follow from
// prefix sums of C(c_t, t+1) and suffix sums of C(c_t - 1, t+1):
//   rank(e - u_j) = sum_{t<j} C(c_t, t+1) + sum_{t>=j} C(c_t - 1, t+1).
__global__ void lowrank_step(const zc* __restrict__ old, const double* __restrict__ old_abs, zc* __restrict__ nw,
                             double* __restrict__ nw_abs, const zc* __restrict__ grow, int k, int r,
                             const uint64_t* __restrict__ binom, int R, uint64_t count) {
  extern __shared__ uint64_t sb[];
  const int tab = (k + r + 1) * (R + 1);
  for (int i = threadIdx.x; i < tab; i += blockDim.x) sb[i] = binom[i];
  __syncthreads();
  zc g[kLowRankMaxR];
  double ga[kLowRankMaxR];
  for (int j = 0; j < r; ++j) {
    g[j] = grow[j];
    ga[j] = hypot(g[j].re, g[j].im);
  }
  for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < count;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    int c[kLowRankMaxR + 1];
    unrank_bars(idx, k, r, sb, R, c);
    c[r - 1] = k + r - 1;  // virtual top bar
    // suffix sums of C(c_t - 1, t+1), t = j..r-2
    uint64_t suf[kLowRankMaxR + 1];
    suf[r - 1] = 0;
    for (int t = r - 2; t >= 0; --t) suf[t] = suf[t + 1] + bnm(sb, R, c[t] - 1, t + 1);
    double ar = 0.0, ai = 0.0, aa = 0.0;
    uint64_t pre = 0;  // sum_{t<j} C(c_t, t+1)
    int cp = -1;
    for (int j = 0; j < r; ++j) {
      const int cj = c[j];
      if (cj - cp - 1 >= 1) {  // e_j >= 1
        const uint64_t o = pre + suf[j];
        const zc v = old[o];
        ar = fma(g[j].re, v.re, fma(-g[j].im, v.im, ar));
        ai = fma(g[j].re, v.im, fma(g[j].im, v.re, ai));
        aa = fma(ga[j], old_abs[o], aa);
      }
      if (j < r - 1) pre += bnm(sb, R, cj, j + 1);
      cp = cj;
    }
    nw[idx] = zc{ar, ai};
    nw_abs[idx] = aa;
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

// Fixed-order reduction of lambda_e prod (e_j - 1)!! over the even
// compositions of degree n: thread t of the grid (T threads, T fixed) takes
// the contiguous ranks [t * per, (t + 1) * per); blocks combine in a fixed
// tree and block partials go to `part` (re_hi, re_lo, im_hi, im_lo, abs).
__global__ void lowrank_even_sum(const zc* __restrict__ lam, const double* __restrict__ lam_abs, int n, int r,
                                 const uint64_t* __restrict__ binom, int R, const double* __restrict__ dfact,
                                 uint64_t count, double* __restrict__ part) {
  extern __shared__ uint64_t sb[];
  const int tab = (n + r + 1) * (R + 1);
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
  const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t per = (count + T - 1) / T;
  const uint64_t lo = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) * per, hi = min(count, lo + per);
  for (uint64_t idx = lo; idx < hi; ++idx) {
    int c[kLowRankMaxR + 1];
    unrank_bars(idx, n, r, sb, R, c);
    c[r - 1] = n + r - 1;
    double w = 1.0;
    bool even = true;
    int cp = -1;
    for (int j = 0; j < r && even; ++j) {
      const int e = c[j] - cp - 1;
      if (e & 1) even = false;
      else w *= dfact[e];
      cp = c[j];
    }
    if (even) add(idx, w);
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

// Per-device stream and workspace kept between calls (calls are serialised
// by the mutex).  Workspaces up to kLrKeepBytes stay allocated, so repeated
// small expansions pay no cudaMalloc/cudaFree; larger ones are released
// after their call.
constexpr size_t kLrKeepBytes = (size_t)256 << 20;
struct LrDevice {
  cudaStream_t st = nullptr;
  char* buf = nullptr;
  size_t bytes = 0;
};
std::mutex g_lr_mu;
std::map<int, LrDevice> g_lr_dev;

uint64_t host_binom(int a, int b) {
  if (b < 0 || b > a) return 0;
  unsigned __int128 r = 1;
  for (int i = 1; i <= b; ++i) r = r * (unsigned __int128)(a - b + i) / (unsigned __int128)i;
  return r > (unsigned __int128)UINT64_MAX ? UINT64_MAX : (uint64_t)r;
}

}  // namespace
}  // namespace hafgb

using namespace hafgb;

extern "C" int haf_lowrank_c128(const double* G, int64_t n64, int64_t r64, double* out, haf_info* info) {
  if (!out || n64 < 0 || n64 > HAF_LOWRANK_MAX_N || r64 < 1 || r64 > HAF_LOWRANK_MAX_R || (n64 > 0 && !G))
    return lfail(HAF_EINVAL, "haf_lowrank_c128: need 0 <= n <= HAF_LOWRANK_MAX_N, 1 <= r <= HAF_LOWRANK_MAX_R");
  const int n = (int)n64, r = (int)r64, R = r;
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
  const uint64_t maxcount = host_binom(n + r - 1, r - 1);
  if (maxcount >= ((uint64_t)1 << 40)) return lfail(HAF_ENOMEM, "haf_lowrank_c128: expansion too large");
  const size_t bytes_state = (size_t)maxcount * (sizeof(zc) + sizeof(double));
  size_t freeb = 0, totalb = 0;
  cudaError_t e = cudaMemGetInfo(&freeb, &totalb);
  if (e != cudaSuccess) return lfail(HAF_ECUDA, std::string("haf_lowrank_c128: ") + cudaGetErrorString(e));
  if (2 * bytes_state + ((size_t)64 << 20) > freeb / 10 * 9)
    return lfail(HAF_ENOMEM, "haf_lowrank_c128: the expansion does not fit the free device memory");
  // host tables: binomials C(a, c) for a <= n + r, c <= r; (e - 1)!! for e <= n
  const int A = n + r;
  std::vector<uint64_t> bt((size_t)(A + 1) * (R + 1), 0);
  for (int a = 0; a <= A; ++a)
    for (int c = 0; c <= R; ++c) bt[(size_t)a * (R + 1) + c] = host_binom(a, c);
  std::vector<double> df(n + 1, 1.0);
  for (int x = 2; x <= n; ++x) df[x] = df[x - 2] * (double)(x - 1);  // df[x] = (x - 1)!!
  df[0] = 1.0;
  const int blocks_sum = 1024;  // fixed: the reduction order depends on it
  // device buffers
  char* dbuf = nullptr;
  size_t off = 0;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t o_z0 = off;
  off += al((size_t)maxcount * sizeof(zc));
  const size_t o_z1 = off;
  off += al((size_t)maxcount * sizeof(zc));
  const size_t o_a0 = off;
  off += al((size_t)maxcount * sizeof(double));
  const size_t o_a1 = off;
  off += al((size_t)maxcount * sizeof(double));
  const size_t o_g = off;
  off += al((size_t)n * r * sizeof(zc));
  const size_t o_b = off;
  off += al(bt.size() * sizeof(uint64_t));
  const size_t o_df = off;
  off += al(df.size() * sizeof(double));
  const size_t o_part = off;
  off += al((size_t)blocks_sum * 5 * sizeof(double));
  const size_t o_out = off;
  off += 256;
  std::lock_guard<std::mutex> lk(g_lr_mu);
  int dev = 0;
  cudaGetDevice(&dev);
  LrDevice& ld = g_lr_dev[dev];
  if (!ld.st) {
    e = cudaStreamCreateWithFlags(&ld.st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      ld.st = nullptr;
      return lfail(HAF_ECUDA, std::string("haf_lowrank_c128: ") + cudaGetErrorString(e));
    }
  }
  if (ld.bytes < off) {
    if (ld.buf) cudaFree(ld.buf);
    ld.buf = nullptr;
    ld.bytes = 0;
    e = cudaMalloc(&ld.buf, off);
    if (e != cudaSuccess) return lfail(HAF_ENOMEM, std::string("haf_lowrank_c128: ") + cudaGetErrorString(e));
    ld.bytes = off;
  }
  dbuf = ld.buf;
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
  zc* z[2] = {(zc*)(dbuf + o_z0), (zc*)(dbuf + o_z1)};
  double* za[2] = {(double*)(dbuf + o_a0), (double*)(dbuf + o_a1)};
  const zc one{1.0, 0.0};
  const double onea = 1.0;
  e = cudaMemcpyAsync(dbuf + o_g, G, (size_t)n * r * sizeof(zc), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dbuf + o_b, bt.data(), bt.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dbuf + o_df, df.data(), df.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(z[0], &one, sizeof(zc), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(za[0], &onea, sizeof(double), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return done(lfail(HAF_ECUDA, std::string("haf_lowrank_c128: ") + cudaGetErrorString(e)));
  const zc* gdev = (const zc*)(dbuf + o_g);
  const uint64_t* bdev = (const uint64_t*)(dbuf + o_b);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int cur = 0;
  int64_t launches = 0;
  for (int k = 1; k <= n; ++k) {
    const uint64_t cnt = host_binom(k + r - 1, r - 1);
    const uint64_t want = (cnt + kLrThreads - 1) / kLrThreads;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)std::max(1, sms) * 16));
    const size_t smem = (size_t)(k + r + 1) * (R + 1) * sizeof(uint64_t);
    lowrank_step<<<grid, kLrThreads, smem, st>>>(z[cur], za[cur], z[cur ^ 1], za[cur ^ 1], gdev + (size_t)(k - 1) * r,
                                                 k, r, bdev, R, cnt);
    ++launches;
    cur ^= 1;
  }
  const size_t smem = (size_t)(n + r + 1) * (R + 1) * sizeof(uint64_t);
  lowrank_even_sum<<<blocks_sum, kLrThreads, smem, st>>>(z[cur], za[cur], n, r, bdev, R, (const double*)(dbuf + o_df),
                                                         maxcount, (double*)(dbuf + o_part));
  lowrank_finish<<<1, 32, 0, st>>>((const double*)(dbuf + o_part), blocks_sum, (double*)(dbuf + o_out));
  launches += 2;
  double res[5];
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(res, dbuf + o_out, sizeof(res), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return done(lfail(HAF_ECUDA, std::string("haf_lowrank_c128: ") + cudaGetErrorString(e)));
  report(res[0] + res[2], res[1] + res[3], res[2], res[3], res[4], (int64_t)maxcount, launches);
  return done(HAF_OK);
}
