// haf_kernels.cu -- sm_103a kernels for the hafnian / loop-hafnian subset sum.
//
// The hafnian of an n x n symmetric matrix is the signed sum over all
// subsets Z of the h = n/2 vertex pairs (Sec. 3.2, eq. main):
//     haf(A) = sum_Z (-1)^{h-|Z|} f(Z),
// with f(Z) the lambda^h coefficient of the trace generating function of
// B = (X A)^{(Z)} (Sec. 3.3, eq. poly / eq. haffinal).  Since
// exp(sum_k tr(B^k) lambda^k / 2k) = det(I - lambda B)^{-1/2}, each summand
// is computed here without eigenvalues (App. B: any route to the power
// traces that stays in the field is admissible):
//   1. gather B (the rows of each kept pair swapped, eq. matA);
//   2. Householder reduction of B to upper Hessenberg form H (unitary
//      similarity, so det(I - lambda B) = det(I - lambda H));
//   3. La Budde's recurrence on the leading principal submatrices of H for
//      the coefficients d_j of det(I - lambda H), truncated at degree h;
//   4. g = det(I - lambda H)^{-1/2} by the recurrence
//      k g_k = -sum_j (k - j/2) d_j g_{k-j}, and f(Z) = g_h.
// For the loop hafnian the exponent gains sum_k u_k lambda^k / 2 with
// u_k = v B^{k-1} X v^T, v = diag(A^{(Z)}) (Sec. 3.3, the q(lambda,B,v)
// function; the printed vector term is garbled and this is the reading that
// agrees with the definition), so f(Z) = [lambda^h] g(lambda) e(lambda),
// e = exp(sum_k u_k lambda^k / 2).  The u_k are formed from H with the
// Householder reflectors applied to v and X v^T during step 2.
//
// Execution model.  GB300's FP64 unit retires one warp-wide DFMA per 64
// cycles per SM sub-partition and charges idle lanes in full, so the kernel
// is organised around lane occupancy of the FP64 pipe: a warp processes
// S = 32/G subsets of the same size |Z| = m in lock step, G lanes per
// subset, every tile in the warp's own slice of shared memory.  A CTA has
// 4, 8 or 16 warps (a template parameter; the slice per warp shrinks
// accordingly), one CTA per SM; two warps per sub-partition keep the FP64
// pipe busier while the other waits on shared memory.  Persistent warps
// pull chunks of colex-ordered subsets of one size from a work list
// (largest tiles first).  Each chunk's signed terms are summed in
// double-double and written to its own slot; a finalize kernel adds the
// slots in a fixed order, so results do not depend on scheduling.  The same
// code runs in single precision for the FP32-bulk mode (bulk type cplxf /
// float, series and sum in FP64).
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "haf_internal.h"

namespace hafgb {

namespace {

constexpr unsigned kFull = 0xffffffffu;

struct __align__(16) cplx {
  double re, im;
};
struct __align__(8) cplxf {
  float re, im;
};

// ---------------------------------------------------------------------------
// Scalar operations for the complex (cplx) and real (double) paths.  Every
// complex multiply-add is four DFMAs.
// ---------------------------------------------------------------------------
template <class T>
struct Ops;

// Block sums over c lanes (defined below).
template <class R>
__device__ __forceinline__ R bsum1(R x, int c);
template <class R>
__device__ __forceinline__ void bsum2(R& x, R& y, int c);
template <class R>
__device__ __forceinline__ void bsum4(R& a, R& b, R& c2, R& d, int c);

// x with its sign bit flipped when `neg` (an integer operation, not an
// FP64 instruction).
__device__ __forceinline__ double neg_if(double x, bool neg) {
  return __longlong_as_double(__double_as_longlong(x) ^ (neg ? (long long)0x8000000000000000ull : 0ll));
}
__device__ __forceinline__ float neg_if(float x, bool neg) {
  return __int_as_float(__float_as_int(x) ^ (neg ? (int)0x80000000u : 0));
}

template <>
struct Ops<cplx> {
  using R = double;
  static constexpr int kMadSlots = 4;  // FP64 instructions per multiply-add
  static __device__ __forceinline__ cplx zero() { return cplx{0.0, 0.0}; }
  static __device__ __forceinline__ cplx one() { return cplx{1.0, 0.0}; }
  // acc + a b
  static __device__ __forceinline__ cplx fma(cplx a, cplx b, cplx acc) {
    acc.re = ::fma(a.re, b.re, acc.re);
    acc.im = ::fma(a.re, b.im, acc.im);
    acc.re = ::fma(-a.im, b.im, acc.re);
    acc.im = ::fma(a.im, b.re, acc.im);
    return acc;
  }
  // acc - a b
  static __device__ __forceinline__ cplx fnma(cplx a, cplx b, cplx acc) {
    acc.re = ::fma(-a.re, b.re, acc.re);
    acc.im = ::fma(-a.re, b.im, acc.im);
    acc.re = ::fma(a.im, b.im, acc.re);
    acc.im = ::fma(-a.im, b.re, acc.im);
    return acc;
  }
  // acc + conj(a) b
  static __device__ __forceinline__ cplx cfma(cplx a, cplx b, cplx acc) {
    acc.re = ::fma(a.re, b.re, acc.re);
    acc.im = ::fma(a.re, b.im, acc.im);
    acc.re = ::fma(a.im, b.im, acc.re);
    acc.im = ::fma(-a.im, b.re, acc.im);
    return acc;
  }
  // acc - a conj(b)
  static __device__ __forceinline__ cplx fnma_cb(cplx a, cplx b, cplx acc) {
    acc.re = ::fma(-a.re, b.re, acc.re);
    acc.im = ::fma(-a.im, b.re, acc.im);
    acc.re = ::fma(-a.im, b.im, acc.re);
    acc.im = ::fma(a.re, b.im, acc.im);
    return acc;
  }
  static __device__ __forceinline__ cplx mul(cplx a, cplx b) {
    cplx r;
    r.re = a.re * b.re;
    r.im = a.re * b.im;
    r.re = ::fma(-a.im, b.im, r.re);
    r.im = ::fma(a.im, b.re, r.im);
    return r;
  }
  static __device__ __forceinline__ cplx scale(cplx a, double s) { return cplx{a.re * s, a.im * s}; }
  // acc + s a   (s real)
  static __device__ __forceinline__ cplx axpy(double s, cplx a, cplx acc) {
    return cplx{::fma(s, a.re, acc.re), ::fma(s, a.im, acc.im)};
  }
  static __device__ __forceinline__ double abs2(cplx a) { return ::fma(a.im, a.im, a.re * a.re); }
  static __device__ __forceinline__ double abs2_acc(cplx a, double acc) {
    return ::fma(a.im, a.im, ::fma(a.re, a.re, acc));
  }
  static __device__ __forceinline__ cplx shfl_xor(cplx a, int o) {
    return cplx{__shfl_xor_sync(kFull, a.re, o), __shfl_xor_sync(kFull, a.im, o)};
  }
  static __device__ __forceinline__ cplx shfl(cplx a, int src) {
    return cplx{__shfl_sync(kFull, a.re, src), __shfl_sync(kFull, a.im, src)};
  }
  static __device__ __forceinline__ cplx add(cplx a, cplx b) { return cplx{a.re + b.re, a.im + b.im}; }
  static __device__ __forceinline__ cplx sub(cplx a, cplx b) { return cplx{a.re - b.re, a.im - b.im}; }
  static __device__ __forceinline__ double re(cplx a) { return a.re; }
  static __device__ __forceinline__ double im(cplx a) { return a.im; }
  static __device__ __forceinline__ double absval(cplx a) { return hypot(a.re, a.im); }
  // Loads of A go through L2 only (ld.global.cg): a job's matrix may sit at
  // an address an earlier job used, written since by a copy engine.
  static __device__ __forceinline__ cplx load(const double* p, size_t i) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p) + i);
    return cplx{v.x, v.y};
  }
  static __device__ __forceinline__ cplx from_re(double x) { return cplx{x, 0.0}; }
  // a, or conj(a) when `c`
  static __device__ __forceinline__ cplx conj_sel(cplx a, bool c) { return cplx{a.re, neg_if(a.im, c)}; }
  static __device__ __forceinline__ cplx block_sum(cplx a, int c) {
    bsum2(a.re, a.im, c);
    return a;
  }
  static __device__ __forceinline__ void block_sum2(cplx& a, cplx& b, int c) { bsum4(a.re, a.im, b.re, b.im, c); }

  // Householder vector for x = (x0, x1, ...), |x|^2 = nrm2, |x0|^2 = s0:
  // H = I - w w^H with w = c (x + e^{i arg x0} |x| e_1), c = 1/sqrt(|x|(|x|+|x0|)),
  // H x = alpha e_1 with alpha = -e^{i arg x0} |x| (Golub & Van Loan's sign
  // choice, which avoids cancellation in the first entry).  With the ratio
  // r = |x| / |x0| = nrm2 / sqrt(nrm2 s0):
  //   w_0 = c (1 + r) x0,  alpha = -r x0,  c = 1 / sqrt(nrm2 + s0 r),
  // two reciprocal square roots (each costs several FP64 instructions).
  // x0 = 0 takes the phase 1: r = |x|, w_0 = 1, alpha = -|x|.  Where the
  // product nrm2 s0 leaves the normal range (tiny or huge columns, e.g. the
  // rounding residue of an exactly cancelling column), r is formed from the
  // separate roots of nrm2 and s0.
  static __device__ __forceinline__ void reflector(cplx x0, double s0, double nrm2, double& c,
                                                   cplx& w0, cplx& alpha) {
    const bool z0 = __double_as_longlong(s0) == 0;
    const bool zz = __double_as_longlong(nrm2) == 0;
    const double pr = z0 ? nrm2 : nrm2 * s0;
    double r;
    if (pr >= 1e-300 && pr <= 1e300)
      r = nrm2 * rsqrt(pr);
    else  // rare: |x| = nrm2 rsqrt(nrm2), 1/|x0| = rsqrt(s0), each in range
      r = (nrm2 * rsqrt(nrm2)) * (z0 ? 1.0 : rsqrt(s0));
    const double cc = rsqrt(z0 ? nrm2 : ::fma(s0, r, nrm2));
    const double t = cc * (1.0 + r);
    c = zz ? 0.0 : cc;
    w0 = zz ? cplx{0.0, 0.0} : (z0 ? cplx{cc * r, 0.0} : cplx{x0.re * t, x0.im * t});
    alpha = zz ? x0 : (z0 ? cplx{-r, 0.0} : cplx{-r * x0.re, -r * x0.im});
  }
};

template <>
struct Ops<double> {
  using R = double;
  static constexpr int kMadSlots = 1;
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double one() { return 1.0; }
  static __device__ __forceinline__ double fma(double a, double b, double acc) { return ::fma(a, b, acc); }
  static __device__ __forceinline__ double fnma(double a, double b, double acc) { return ::fma(-a, b, acc); }
  static __device__ __forceinline__ double cfma(double a, double b, double acc) { return ::fma(a, b, acc); }
  static __device__ __forceinline__ double fnma_cb(double a, double b, double acc) { return ::fma(-a, b, acc); }
  static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
  static __device__ __forceinline__ double scale(double a, double s) { return a * s; }
  static __device__ __forceinline__ double axpy(double s, double a, double acc) { return ::fma(s, a, acc); }
  static __device__ __forceinline__ double abs2(double a) { return a * a; }
  static __device__ __forceinline__ double abs2_acc(double a, double acc) { return ::fma(a, a, acc); }
  static __device__ __forceinline__ double shfl_xor(double a, int o) { return __shfl_xor_sync(kFull, a, o); }
  static __device__ __forceinline__ double shfl(double a, int src) { return __shfl_sync(kFull, a, src); }
  static __device__ __forceinline__ double add(double a, double b) { return a + b; }
  static __device__ __forceinline__ double sub(double a, double b) { return a - b; }
  static __device__ __forceinline__ double re(double a) { return a; }
  static __device__ __forceinline__ double im(double) { return 0.0; }
  static __device__ __forceinline__ double absval(double a) { return fabs(a); }
  static __device__ __forceinline__ double load(const double* p, size_t i) { return __ldcg(p + i); }
  static __device__ __forceinline__ double from_re(double x) { return x; }
  static __device__ __forceinline__ double conj_sel(double a, bool) { return a; }
  static __device__ __forceinline__ double block_sum(double a, int c) { return bsum1(a, c); }
  static __device__ __forceinline__ void block_sum2(double& a, double& b, int c) { bsum2(a, b, c); }

  static __device__ __forceinline__ void reflector(double x0, double s0, double nrm2, double& c,
                                                   double& w0, double& alpha) {
    const bool zz = __double_as_longlong(nrm2) == 0;
    const double rn = rsqrt(nrm2);
    const double nrm = nrm2 * rn;
    const double ax0 = fabs(x0);
    const double ph = copysign(1.0, x0);
    const double cc = rsqrt(nrm * (nrm + ax0));
    c = zz ? 0.0 : cc;
    w0 = zz ? 0.0 : ph * (cc * (ax0 + nrm));
    alpha = zz ? x0 : -nrm * ph;
    (void)s0;
  }
};

// ---------------------------------------------------------------------------
// FP32 arithmetic for the reduced-precision mode: the gather, the Householder
// reduction, the loop moments and La Budde's recurrence run in single
// precision (complex64 / float32); the power series and the subset sum stay
// in FP64 (see process_chunk).  A single-precision complex multiply-add is
// four FFMAs, which GB300 retires ~60x faster than DFMAs.
// ---------------------------------------------------------------------------
template <>
struct Ops<cplxf> {
  using R = float;
  static constexpr int kMadSlots = 4;
  static __device__ __forceinline__ cplxf zero() { return cplxf{0.f, 0.f}; }
  static __device__ __forceinline__ cplxf one() { return cplxf{1.f, 0.f}; }
  static __device__ __forceinline__ cplxf fma(cplxf a, cplxf b, cplxf acc) {
    acc.re = fmaf(a.re, b.re, acc.re);
    acc.im = fmaf(a.re, b.im, acc.im);
    acc.re = fmaf(-a.im, b.im, acc.re);
    acc.im = fmaf(a.im, b.re, acc.im);
    return acc;
  }
  static __device__ __forceinline__ cplxf fnma(cplxf a, cplxf b, cplxf acc) {
    acc.re = fmaf(-a.re, b.re, acc.re);
    acc.im = fmaf(-a.re, b.im, acc.im);
    acc.re = fmaf(a.im, b.im, acc.re);
    acc.im = fmaf(-a.im, b.re, acc.im);
    return acc;
  }
  static __device__ __forceinline__ cplxf cfma(cplxf a, cplxf b, cplxf acc) {
    acc.re = fmaf(a.re, b.re, acc.re);
    acc.im = fmaf(a.re, b.im, acc.im);
    acc.re = fmaf(a.im, b.im, acc.re);
    acc.im = fmaf(-a.im, b.re, acc.im);
    return acc;
  }
  static __device__ __forceinline__ cplxf fnma_cb(cplxf a, cplxf b, cplxf acc) {
    acc.re = fmaf(-a.re, b.re, acc.re);
    acc.im = fmaf(-a.im, b.re, acc.im);
    acc.re = fmaf(-a.im, b.im, acc.re);
    acc.im = fmaf(a.re, b.im, acc.im);
    return acc;
  }
  static __device__ __forceinline__ cplxf mul(cplxf a, cplxf b) {
    cplxf r;
    r.re = a.re * b.re;
    r.im = a.re * b.im;
    r.re = fmaf(-a.im, b.im, r.re);
    r.im = fmaf(a.im, b.re, r.im);
    return r;
  }
  static __device__ __forceinline__ cplxf scale(cplxf a, float s) { return cplxf{a.re * s, a.im * s}; }
  static __device__ __forceinline__ float abs2(cplxf a) { return fmaf(a.im, a.im, a.re * a.re); }
  static __device__ __forceinline__ float abs2_acc(cplxf a, float acc) {
    return fmaf(a.im, a.im, fmaf(a.re, a.re, acc));
  }
  static __device__ __forceinline__ cplxf shfl_xor(cplxf a, int o) {
    return cplxf{__shfl_xor_sync(kFull, a.re, o), __shfl_xor_sync(kFull, a.im, o)};
  }
  static __device__ __forceinline__ cplxf add(cplxf a, cplxf b) { return cplxf{a.re + b.re, a.im + b.im}; }
  static __device__ __forceinline__ cplxf load(const double* p, size_t i) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p) + i);
    return cplxf{(float)v.x, (float)v.y};
  }
  static __device__ __forceinline__ cplx widen(cplxf a) { return cplx{(double)a.re, (double)a.im}; }
  static __device__ __forceinline__ cplxf conj_sel(cplxf a, bool c) { return cplxf{a.re, neg_if(a.im, c)}; }
  static __device__ __forceinline__ cplxf block_sum(cplxf a, int c) {
    bsum2(a.re, a.im, c);
    return a;
  }
  static __device__ __forceinline__ void block_sum2(cplxf& a, cplxf& b, int c) { bsum4(a.re, a.im, b.re, b.im, c); }
  // the reflector of Ops<cplx>, in single precision
  static __device__ __forceinline__ void reflector(cplxf x0, float s0, float nrm2, float& c, cplxf& w0,
                                                   cplxf& alpha) {
    const bool z0 = __float_as_int(s0) == 0;
    const bool zz = __float_as_int(nrm2) == 0;
    const float rn = rsqrtf(nrm2);
    const float nrm = nrm2 * rn;
    const float r0 = rsqrtf(s0);
    const float ax0 = s0 * r0;
    const float phr = z0 ? 1.f : x0.re * r0;
    const float phi = z0 ? 0.f : x0.im * r0;
    const float a0 = z0 ? 0.f : ax0;
    const float cc = rsqrtf(nrm * (nrm + a0));
    const float t = cc * (a0 + nrm);
    c = zz ? 0.f : cc;
    w0 = zz ? cplxf{0.f, 0.f} : cplxf{phr * t, phi * t};
    alpha = zz ? x0 : cplxf{-nrm * phr, -nrm * phi};
  }
};

template <>
struct Ops<float> {
  using R = float;
  static constexpr int kMadSlots = 1;
  static __device__ __forceinline__ float zero() { return 0.f; }
  static __device__ __forceinline__ float one() { return 1.f; }
  static __device__ __forceinline__ float fma(float a, float b, float acc) { return fmaf(a, b, acc); }
  static __device__ __forceinline__ float fnma(float a, float b, float acc) { return fmaf(-a, b, acc); }
  static __device__ __forceinline__ float cfma(float a, float b, float acc) { return fmaf(a, b, acc); }
  static __device__ __forceinline__ float fnma_cb(float a, float b, float acc) { return fmaf(-a, b, acc); }
  static __device__ __forceinline__ float mul(float a, float b) { return a * b; }
  static __device__ __forceinline__ float scale(float a, float s) { return a * s; }
  static __device__ __forceinline__ float abs2(float a) { return a * a; }
  static __device__ __forceinline__ float abs2_acc(float a, float acc) { return fmaf(a, a, acc); }
  static __device__ __forceinline__ float shfl_xor(float a, int o) { return __shfl_xor_sync(kFull, a, o); }
  static __device__ __forceinline__ float add(float a, float b) { return a + b; }
  static __device__ __forceinline__ float load(const double* p, size_t i) { return (float)__ldcg(p + i); }
  static __device__ __forceinline__ double widen(float a) { return (double)a; }
  static __device__ __forceinline__ float conj_sel(float a, bool) { return a; }
  static __device__ __forceinline__ float block_sum(float a, int c) { return bsum1(a, c); }
  static __device__ __forceinline__ void block_sum2(float& a, float& b, int c) { bsum2(a, b, c); }
  static __device__ __forceinline__ void reflector(float x0, float s0, float nrm2, float& c, float& w0,
                                                   float& alpha) {
    const bool zz = __float_as_int(nrm2) == 0;
    const float rn = rsqrtf(nrm2);
    const float nrm = nrm2 * rn;
    const float ax0 = fabsf(x0);
    const float ph = copysignf(1.f, x0);
    const float cc = rsqrtf(nrm * (nrm + ax0));
    c = zz ? 0.f : cc;
    w0 = zz ? 0.f : ph * (cc * (ax0 + nrm));
    alpha = zz ? x0 : -nrm * ph;
    (void)s0;
  }
};

// Block sums over c lanes (c a power of two dividing the group width; the
// block is lanes with equal lane / c).  Every lane of the block ends with
// the bitwise-identical sums: each stage adds a commuting pair.  Two values
// are reduced by splitting them over the two halves of the block first
// (each half keeps one value and adds its partner's copy of it), so the
// pair costs log2(c) additions per lane instead of 2 log2(c); four values
// split twice.
template <class R>
__device__ __forceinline__ R bsum1(R x, int c) {
  for (int o = c >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}
template <class R>
__device__ __forceinline__ void bsum2(R& x, R& y, int c) {
  if (c == 1) return;
  const int h = c >> 1;
  const bool hi = (threadIdx.x & h) != 0;
  R keep = hi ? y : x;
  const R send = hi ? x : y;
  keep += __shfl_xor_sync(kFull, send, h);
  for (int o = h >> 1; o > 0; o >>= 1) keep += __shfl_xor_sync(kFull, keep, o);
  const R other = __shfl_xor_sync(kFull, keep, h);
  x = hi ? other : keep;
  y = hi ? keep : other;
}
template <class R>
__device__ __forceinline__ void bsum4(R& a, R& b, R& c2, R& d, int c) {
  if (c <= 2) {
    bsum2(a, b, c);
    bsum2(c2, d, c);
    return;
  }
  const int h = c >> 1, h2 = c >> 2;
  const bool hi = (threadIdx.x & h) != 0, hi2 = (threadIdx.x & h2) != 0;
  // stage 1: the lower half keeps (a, b), the upper half (c2, d)
  R k0 = hi ? c2 : a, k1 = hi ? d : b;
  const R s0 = hi ? a : c2, s1 = hi ? b : d;
  k0 += __shfl_xor_sync(kFull, s0, h);
  k1 += __shfl_xor_sync(kFull, s1, h);
  // stage 2: each quarter keeps one value
  R z = hi2 ? k1 : k0;
  const R w = hi2 ? k0 : k1;
  z += __shfl_xor_sync(kFull, w, h2);
  for (int o = h2 >> 1; o > 0; o >>= 1) z += __shfl_xor_sync(kFull, z, o);
  // quarter (hi, hi2) holds: (0,0) a, (0,1) b, (1,0) c2, (1,1) d
  const R zh = __shfl_xor_sync(kFull, z, h), zq = __shfl_xor_sync(kFull, z, h2),
          zb = __shfl_xor_sync(kFull, z, h | h2);
  const R v00 = hi ? (hi2 ? zb : zh) : (hi2 ? zq : z);
  const R v01 = hi ? (hi2 ? zh : zb) : (hi2 ? z : zq);
  const R v10 = hi ? (hi2 ? zq : z) : (hi2 ? zb : zh);
  const R v11 = hi ? (hi2 ? z : zq) : (hi2 ? zh : zb);
  a = v00;
  b = v01;
  c2 = v10;
  d = v11;
}

// Sum over the G lanes of a group.
template <class R>
__device__ __forceinline__ R group_sum(R x, int G) {
  return bsum1(x, G);
}
template <class T>
__device__ __forceinline__ T group_sum_t(T x, int G) {
  return Ops<T>::block_sum(x, G);
}

// First index >= lo that lane g of a G-lane group owns (index = g mod G).
__device__ __forceinline__ int first_owned(int lo, int g, int G) {
  return lo + ((g - lo) & (G - 1));
}

// Knuth's TwoSum and its fast variant: (s, e) with s + e = a + b exactly.
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void dd_add(double& hi, double& lo, double x) {
  double s, e;
  two_sum(hi, x, s, e);
  e += lo;
  hi = s + e;
  lo = e - (hi - s);
}
__device__ __forceinline__ void dd_add_dd(double& hi, double& lo, double xhi, double xlo) {
  double s, e;
  two_sum(hi, xhi, s, e);
  e += lo + xlo;
  hi = s + e;
  lo = e - (hi - s);
}

// Next subset of the same size in colex order (Gosper).
__device__ __forceinline__ uint64_t next_comb(uint64_t x) {
  const uint64_t c = x & (~x + 1);
  const uint64_t r = x + c;
  return (((r ^ x) >> 2) >> (__ffsll((long long)c) - 1)) | r;
}

// ---------------------------------------------------------------------------
// The two passes of a Householder step over the active block.  GB300 retires
// one warp-wide FP64 instruction per 64 cycles per SM sub-partition and
// charges idle lanes in full, so both passes spread their multiply-adds
// evenly over the G lanes of a group, whatever the shape of the block.
//
// Dot pass.  The N + L dot products of length L (L = N - k1)
//   p_i  = sum_{j in K} A_ij w_j        (rows i = 0..N-1)
//   t'_j = sum_{i in K} conj(w_i) A_ij  (columns j in K)
// are cut into c pieces each; piece q of product tau is taken by lane
// (tau c + q) mod G in round (tau c + q) / G, so the c pieces of a product
// sit in c adjacent lanes of one round and are added by c-lane block sums.
// c is chosen per step to minimise the rounds times (multiply-adds per piece
// + combine stages).
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ int dot_pieces(int ntask, int L, int G) {
  constexpr int kMad = Ops<T>::kMadSlots;
  int best = 0x7fffffff, best_lc = 0;
  for (int lc = 0; (1 << lc) <= G; ++lc) {
    const int c = 1 << lc;
    const int rounds = (ntask * c + G - 1) / G;
    const int len = (L + c - 1) >> lc;
    const int cost = rounds * (kMad * len + lc);
    if (cost < best) {
      best = cost;
      best_lc = lc;
    }
  }
  return best_lc;
}

template <class T>
__device__ __forceinline__ void dot_pass(const T* __restrict__ tile, int ld, int N, int k1,
                                         const T* __restrict__ W, T* __restrict__ P, T* __restrict__ TV,
                                         int g, int G) {
  using O = Ops<T>;
  const int L = N - k1, ntask = N + L;
  const int lc = dot_pieces<T>(ntask, L, G);
  const int c = 1 << lc;
  const int len = (L + c - 1) >> lc;
  const int npiece = ntask << lc;
  for (int p0 = 0; p0 < npiece; p0 += G) {
    const int piece = p0 + g;
    const bool live = piece < npiece;
    const int tau = live ? (piece >> lc) : 0;
    const int q = piece & (c - 1);
    const bool col = tau >= N;
    const int l0 = q * len;
    const int l1 = live ? min(l0 + len, L) : l0;
    const int a0 = col ? k1 * ld + (k1 + tau - N) : tau * ld + k1;  // >= 0 for every lane
    const T* a = tile + a0;
    const int stride = col ? ld : 1;
    T acc = O::zero();
    // not unrolled: unrolling puts adjacent W entries in one iteration, and a
    // load vectoriser could then join them into one access wider than their
    // 16-byte alignment
#pragma unroll 1
    for (int l = l0; l < l1; ++l) acc = O::fma(a[l * stride], O::conj_sel(W[k1 + l], col), acc);
    acc = O::block_sum(acc, c);
    if (live && q == 0) {
      if (col)
        TV[k1 + tau - N] = acc;
      else
        P[tau] = acc;
    }
  }
}

// Update pass: A_ij -= q_i conj(w_j) for rows i < k1 and
// A_ij -= q_i conj(w_j) + w_i t'_j for rows i in K, columns j in K; the
// elements of each region are dealt to the lanes round robin.
template <class T>
__device__ __forceinline__ void update_pass(T* __restrict__ tile, int ld, int N, int k1, const T* __restrict__ W,
                                            const T* __restrict__ TV, const T* __restrict__ Q, int g, int G) {
  using O = Ops<T>;
  const int L = N - k1;
  BlockWalk w1(g, G, L);  // element e = w1.i * L + w1.j of the rows above K
  for (int e = g; e < k1 * L; e += G, w1.next()) {
    const int i = w1.i, j = k1 + w1.j;
    T* a = tile + i * ld + j;
    *a = O::fnma_cb(Q[i], W[j], *a);
  }
  BlockWalk w2(g, G, L);  // element e = w2.i * L + w2.j of K x K
  for (int e = g; e < L * L; e += G, w2.next()) {
    const int i = k1 + w2.i, j = k1 + w2.j;
    T* a = tile + i * ld + j;
    const T v = O::fnma_cb(Q[i], W[j], *a);
    *a = O::fnma(W[i], TV[j], v);
  }
}

// gamma = w^H p_K and, with loops, aw = va . w (both over K), summed over the
// group; then q_i = p_i - gamma w_i (i in K) and va <- va - aw conj(w).
template <class T>
__device__ __forceinline__ void finish_step(int N, int k1, const T* __restrict__ W, T* __restrict__ P,
                                            T* VA, bool loops, int g, int G) {
  using O = Ops<T>;
  T gam = O::zero(), aw = O::zero();
  for (int i = k1 + g; i < N; i += G) {
    gam = O::cfma(W[i], P[i], gam);
    if (loops) aw = O::fma(VA[i], W[i], aw);
  }
  if (loops)
    O::block_sum2(gam, aw, G);
  else
    gam = O::block_sum(gam, G);
  for (int i = k1 + g; i < N; i += G) {
    P[i] = O::fnma(gam, W[i], P[i]);
    if (loops) VA[i] = O::fnma_cb(aw, W[i], VA[i]);
  }
}

// ---------------------------------------------------------------------------
// Householder reduction to upper Hessenberg form, in place, by one G-lane
// group.  Step k reflects rows/columns K = {k+1, ..., N-1} with
// H = I - w w^H, w from column k:
//   p = A[:, K] w;  t'_j = sum_{i in K} conj(w_i) A_ij;  gamma = w^H p_K;
//   q = p - gamma w (on K);  A_ij -= q_i conj(w_j) + w_i t'_j,
// which is A <- H A H restricted to the active block (the w_i t'_j term only
// on rows in K).  With `loops` the reduction starts from b ("Krylov start"):
// a first reflector on all N indices maps vb to alpha e_0 and is applied to A
// from both sides and to va; the later steps act on indices >= 1, so vb stays
// alpha e_0 while va <- va (I - w w^H) follows every step.  Then H^{k-1} vb
// is supported on its first k entries (H is Hessenberg), which is what makes
// the loop moments cheap.
// ---------------------------------------------------------------------------
template <class T>
__device__ void householder(T* __restrict__ tile, int ld, int N, T* __restrict__ W, T* P,
                            T* __restrict__ TV, T* VA, const T* VB, T* beta, bool loops, int g,
                            int G) {
  using O = Ops<T>;
  using R = typename O::R;
  if (loops) {
    R sig = R(0);
    for (int i = 1 + g; i < N; i += G) sig = O::abs2_acc(VB[i], sig);
    sig = group_sum(sig, G);
    const T x0 = VB[0];
    const R s0 = O::abs2(x0);
    R c;
    T w0, alpha;
    O::reflector(x0, s0, s0 + sig, c, w0, alpha);
    for (int i = 1 + g; i < N; i += G) W[i] = O::scale(VB[i], c);
    if (g == 0) {
      W[0] = w0;
      *beta = alpha;  // b is now alpha e_0
    }
    // VB may share P's storage: every read of it is done before this
    // barrier, and the dot pass below writes P
    __syncwarp();
    dot_pass<T>(tile, ld, N, 0, W, P, TV, g, G);
    __syncwarp();
    finish_step<T>(N, 0, W, P, VA, true, g, G);
    __syncwarp();
    update_pass<T>(tile, ld, N, 0, W, TV, P, g, G);
    __syncwarp();
  }
  for (int k = 0; k + 2 < N; ++k) {
    const int k1 = k + 1;
    const int i2 = k + 2 + g;  // this lane's rows below the first reflected entry
    R sig = R(0);
    for (int i = i2; i < N; i += G) sig = O::abs2_acc(tile[i * ld + k], sig);
    sig = group_sum(sig, G);
    const T x0 = tile[k1 * ld + k];
    const R s0 = O::abs2(x0);
    R c;
    T w0, alpha;
    O::reflector(x0, s0, s0 + sig, c, w0, alpha);
    for (int i = i2; i < N; i += G) W[i] = O::scale(tile[i * ld + k], c);
    if (g == 0) W[k1] = w0;
    __syncwarp();
    // every lane has read x0 by now, so its entry may take alpha (column k
    // is outside the columns the rest of this step reads)
    if (g == 0) tile[k1 * ld + k] = alpha;
    dot_pass<T>(tile, ld, N, k1, W, P, TV, g, G);
    __syncwarp();
    finish_step<T>(N, k1, W, P, VA, loops, g, G);
    __syncwarp();
    update_pass<T>(tile, ld, N, k1, W, TV, P, g, G);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Loop moments u_k = a H^{k-1} b, k = 1..min(h, N), for the loop hafnian
// (a = v Q, b = Q^H X v^T after the reduction, so u_k = v B^{k-1} X v^T).
// The reduction started from b, so b = beta e_0 and y_k = H^{k-1} b is
// supported on entries 0..k-1: step k computes rows 0..k-1 of H y_{k-1}
// from columns 0..k-2 only (row i from column max(i-1, 0)), about k^2/2
// multiply-adds instead of N^2/2.  Y0, Y1: scratch vectors of length N.
// Row i has k - max(i, 1) entries, so rows p and k-1-p together have about
// k + 1: each such pair is one task, cut into c pieces taken by c adjacent
// lanes (c chosen per k as in the dot pass); a piece crosses from the first
// row to the second at most once, and the two partial sums are added over
// the c lanes.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ int moment_pieces(int npair, int k, int G) {
  constexpr int kMad = Ops<T>::kMadSlots;
  int best = 0x7fffffff, best_lc = 0;
  for (int lc = 0; (1 << lc) <= G; ++lc) {
    const int c = 1 << lc;
    const int rounds = (npair * c + G - 1) / G;
    const int len = (k + 1 + c - 1) >> lc;
    const int cost = rounds * (kMad * len + (lc >= 2 ? lc + 1 : 2 * lc) + 2 * kMad);
    if (cost < best) {
      best = cost;
      best_lc = lc;
    }
  }
  return best_lc;
}

template <class T>
__device__ void loop_moments(const T* __restrict__ tile, int ld, int N, int h,
                             const T* __restrict__ VA, const T* __restrict__ VB, T* Y0, T* Y1,
                             T* __restrict__ U, int g, int G) {
  using O = Ops<T>;
  const int kmax = min(h, N);
  if (g == 0) {
    Y0[0] = VB[0];
    U[1] = O::mul(VA[0], VB[0]);
  }
  for (int k = 2; k <= kmax; ++k) {
    __syncwarp();
    const int npair = (k + 1) >> 1;
    const int lc = moment_pieces<T>(npair, k, G);
    const int c = 1 << lc;
    const int len = (k + 1 + c - 1) >> lc;
    T uk = O::zero();
    for (int p0 = 0; p0 < (npair << lc); p0 += G) {
      const int piece = p0 + g;
      const bool live = piece < (npair << lc);
      const int p = live ? (piece >> lc) : 0;
      const int q = piece & (c - 1);
      const int ra = p, rb = k - 1 - p;
      const int la = (ra == 0) ? k - 1 : k - ra;            // entries of row ra
      const int lb = (rb == ra) ? 0 : ((rb == 0) ? k - 1 : k - rb);
      const int ja = ra > 0 ? ra - 1 : 0, jb = rb > 0 ? rb - 1 : 0;
      const int lo = q * len;
      const int hi = live ? min(lo + len, la + lb) : lo;
      T acc = O::zero(), acc_a = O::zero();
      for (int e = lo; e < hi; ++e) {
        if (e == la) {  // the piece passes from row ra to row rb
          acc_a = acc;
          acc = O::zero();
        }
        const bool in_a = e < la;
        const int i = in_a ? ra : rb;
        const int j = in_a ? ja + e : jb + (e - la);
        acc = O::fma(tile[i * ld + j], Y0[j], acc);
      }
      T sa = (lo >= la) ? O::zero() : ((hi <= la) ? acc : acc_a);
      T sb = (hi <= la) ? O::zero() : acc;
      O::block_sum2(sa, sb, c);
      if (live && q == 0) {
        Y1[ra] = sa;
        uk = O::fma(VA[ra], sa, uk);
        if (rb != ra) {
          Y1[rb] = sb;
          uk = O::fma(VA[rb], sb, uk);
        }
      }
    }
    uk = group_sum_t(uk, G);
    if (g == 0) U[k] = uk;
    T* t = Y0;
    Y0 = Y1;
    Y1 = t;
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// La Budde's recurrence (characteristic polynomial of an upper Hessenberg
// matrix from its leading principal submatrices), in the reversed form
// D_i(lambda) = det(I - lambda H_i), truncated at degree h:
//   D_i = (1 - alpha_{i-1} lambda) D_{i-1}
//         - sum_{m=1}^{i-1} c_{i,m} lambda^{m+1} D_{i-1-m},
//   c_{i,m} = H_{i-1-m, i-1} prod_{l=i-m}^{i-1} H_{l, l-1}.
// The products are folded into the upper triangle first (column by column,
// from the diagonal upward), so c_{i,m} = H'_{i-1-m, i-1}.
// The sum is evaluated "right-looking": once D_r is final, its terms
//   D_{r+1}[j]   += D_r[j]                       (j = 1..min(r,h))
//   D_i[t+i-r]   -= H'_{r, i-1} D_r[t]          (i = r+1..N; H'_{r,r} = alpha_r)
// are added to every later polynomial; the (i, t) pairs of one r are dealt
// round robin over the group's lanes.  D_i[1..min(i,h)] for i < N accumulate in
// row i of the tile, columns 0..i-1 (free after the reduction: entries
// below the subdiagonal and, once folded, the subdiagonal); D_N goes to DN.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T* dslot(T* tile, int ld, int N, T* DN, int i, int j) {
  return (i < N) ? tile + i * ld + (j - 1) : DN + j;
}

template <class T>
__device__ void labudde(T* __restrict__ tile, int ld, int N, int h, T* __restrict__ DN, int g,
                        int G) {
  using O = Ops<T>;
  // Fold the subdiagonal products into the upper triangle, row by row:
  // H'_{a,b} = H_{a,b} s_{a+1} s_{a+2} ... s_b (s_l = H_{l,l-1}).  Row a has
  // N-1-a entries, so rows a and N-2-a together have N: each lane takes such
  // a pair (the middle row alone) and walks it as one loop of N entries, so
  // every lane of a round runs the same number of iterations.
  for (int p = g; p < (N >> 1); p += G) {
    const int a0 = p, a1 = N - 2 - p;
    const int l0 = N - 1 - a0, l1 = (a1 != a0) ? N - 1 - a1 : 0;
    int a = a0, b = a0 + 1;
    T rho = O::one();
    for (int e = 0; e < l0 + l1; ++e) {
      if (e == l0) {  // second row of the pair
        a = a1;
        b = a1 + 1;
      }
      const T sub = tile[b * ld + b - 1];
      rho = (b == a + 1) ? sub : O::mul(rho, sub);
      T* h = tile + a * ld + b;
      *h = O::mul(*h, rho);
      ++b;
    }
  }
  __syncwarp();
  // zero the accumulators D_i[1..min(i,h)], i = 1..N
  for (int i = 1; i <= N; ++i) {
    const int J = min(i, h);
    for (int j = 1 + g; j <= J; j += G) *dslot(tile, ld, N, DN, i, j) = O::zero();
  }
  __syncwarp();
  for (int r = 0; r < N; ++r) {
    const T* Dr = tile + r * ld;  // D_r[t] = Dr[t - 1] for 1 <= t <= min(r,h); D_r[0] = 1
    const T* Hr = tile + r * ld;  // H'_{r, i-1} = Hr[i-1]; H'_{r,r} = alpha_r
    // D_i[t+i-r] -= H'_{r,i-1} D_r[t] for rows i = r+1..imax and
    // t = 0..min(ra, h-(i-r)); row i = r+1 also takes D_r[t+1] (the
    // D_{r+1}[j] += D_r[j] term).  The (i, t) units, row by row, are dealt to
    // the lanes round robin (lane g takes units g, g+G, ...), so the lanes'
    // shares differ by at most one and no two lanes write the same entry.
    const int ra = min(r, h);
    const int imax = min(N, h + r);
    int i = r + 1, t = g;
    while (i <= imax && t > min(ra, h - (i - r))) {
      t -= min(ra, h - (i - r)) + 1;
      ++i;
    }
    while (i <= imax) {
      const T dl = Dr[t > 0 ? t - 1 : 0];  // an address inside row r even when t = 0
      const T d = (t == 0) ? O::one() : dl;
      T* a = dslot(tile, ld, N, DN, i, i - r);  // D_i[t + i - r] = a[t]
      T v = a[t];
      if (i == r + 1 && t < ra) v = O::add(v, Dr[t]);
      a[t] = O::fnma(Hr[i - 1], d, v);
      t += G;
      while (i <= imax && t > min(ra, h - (i - r))) {
        t -= min(ra, h - (i - r)) + 1;
        ++i;
      }
    }
    __syncwarp();
  }
  if (g == 0) DN[0] = O::one();
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Power series.  g = D^{-1/2}: k g_k = -sum_{j=1}^{min(k,N)} (k - j/2) d_j g_{k-j}
// (differentiate D g^2 = 1).  With loops, e = exp(sum_k u_k lambda^k / 2):
// k e_k = sum_{j=1}^{k} (j u_j / 2) e_{k-j}.  Both are run "right-looking":
// once g_k, e_k are final, their contributions are added to every later
// coefficient, one per lane.  Returns f = [lambda^h] g e.
// ---------------------------------------------------------------------------
template <class T>
__device__ T series(int N, int h, const T* __restrict__ DN, T* U, T* GS, T* AC,
                    T* ES, T* AC2, bool loops, const double* __restrict__ tables, int g, int G) {
  using O = Ops<T>;
  const double* half = tables;         // half[k] = k/2
  const double* inv = tables + 128;    // inv[k] = 1/k
  const int jmax = min(N, h);
  for (int k = g; k <= h; k += G) {
    AC[k] = O::zero();
    AC2[k] = O::zero();
    if (loops && k >= 1) U[k] = O::scale(U[k], half[k]);  // j u_j / 2
  }
  if (g == 0) {
    GS[0] = O::one();
    ES[0] = O::one();
  }
  __syncwarp();
  for (int k = 0; k < h; ++k) {
    const T gk = GS[k];
    const T ek = ES[k];
    for (int kp = first_owned(k + 1, g, G); kp <= h; kp += G) {
      const int j = kp - k;
      if (j <= jmax) AC[kp] = O::axpy(half[kp + k], O::mul(DN[j], gk), AC[kp]);
      if (loops) AC2[kp] = O::fma(U[j], ek, AC2[kp]);
    }
    __syncwarp();
    if (g == 0) {
      GS[k + 1] = O::scale(AC[k + 1], -inv[k + 1]);
      ES[k + 1] = O::scale(AC2[k + 1], inv[k + 1]);
    }
    __syncwarp();
  }
  if (!loops) return GS[h];
  T f = O::zero();
  for (int k = g; k <= h; k += G) f = O::fma(GS[k], ES[h - k], f);
  return group_sum_t(f, G);
}

// Cayley-Hamilton continuation u_k = -sum_{j=1}^{N} d_j u_{k-j} for N < k <= h.
template <class T>
__device__ void loop_moments_tail(int N, int h, const T* __restrict__ DN, T* U, int g, int G) {
  using O = Ops<T>;
  for (int k = N + 1; k <= h; ++k) {
    T acc = O::zero();
    for (int j = 1 + g; j <= N; j += G) acc = O::fnma(DN[j], U[k - j], acc);
    acc = group_sum_t(acc, G);
    __syncwarp();
    if (g == 0) U[k] = acc;
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// One chunk: ceil(count / S) rounds of S subsets (one per group).
// TB is the type of the bulk steps (gather, Householder, loop moments, La
// Budde), TS the type of the power series and of f(Z).  FP64 runs with
// TB = TS; the FP32 mode runs TB in single precision and widens the
// characteristic-polynomial coefficients (and loop moments) to FP64 before
// the series, so only the O(N^3) part loses precision.
// Per-subset shared-memory layout: subset_layout in haf_internal.h (the
// tile, whose first 4 (h+1) series elements take the power-series arrays
// once La Budde is done; W, P, TV and, with loops, VA, VB; La Budde's output
// and the loop moments; int pos[h]).
// ---------------------------------------------------------------------------
template <class TB, class TS>
__device__ void process_chunk(const Job& job, const Chunk& ch, double* __restrict__ partial_out,
                              const double* __restrict__ tables, const uint64_t* __restrict__ masks,
                              double* __restrict__ terms_out, unsigned char* wbase, int lane) {
  using OB = Ops<TB>;
  using OS = Ops<TS>;
  constexpr bool kMixed = !std::is_same<TB, TS>::value;
  const int n = job.n, h = n >> 1, m = ch.m, N = 2 * m, G = ch.G, S = 32 / G, ld = ch.ld;
  const int s = lane / G, g = lane - s * G;
  const bool loops = job.loops != 0;
  const SubsetLayout lay = subset_layout(N, ld, h, (int)sizeof(TB), (int)sizeof(TS), kMixed, loops);
  unsigned char* base = wbase + s * lay.total;
  TB* tile = reinterpret_cast<TB*>(base);
  TB* W = reinterpret_cast<TB*>(base + lay.vec);
  TB* P = W + N;
  TB* TV = P + N;
  TB* DNb = reinterpret_cast<TB*>(base + lay.dnb);
  TS* DN = reinterpret_cast<TS*>(base + lay.dn);
  // the loop-hafnian arrays exist only with loops; otherwise they alias
  // arrays of the subset (never written then), so that every pointer stays
  // inside the subset's region
  TB* VA = loops ? TV + N : W;
  TB* VB = loops ? P : W;  // b = X v^T: read by the Krylov start before P is written
  TB* beta = reinterpret_cast<TB*>(base + lay.pos);  // b's first entry after the Krylov start
  TB* Ub = loops ? reinterpret_cast<TB*>(base + lay.ub) : DNb;
  TS* U = loops ? reinterpret_cast<TS*>(base + lay.u) : DN;
  TS* GS = reinterpret_cast<TS*>(base);
  TS* AC = GS + (h + 1);
  TS* ES = AC + (h + 1);
  TS* AC2 = ES + (h + 1);
  int* pos = reinterpret_cast<int*>(base + lay.pos);
  const bool neg = ((h - m) & 1) != 0;
  const bool term_mode = terms_out != nullptr;

  double re_hi = 0.0, re_lo = 0.0, im_hi = 0.0, im_lo = 0.0, asum = 0.0;
  uint64_t mask = ch.mask0;
  if (!term_mode)
    for (int q = 0; q < s; ++q) mask = next_comb(mask);

  for (uint32_t base_r = 0; base_r < ch.count; base_r += (uint32_t)S) {
    const uint32_t local = base_r + (uint32_t)s;
    const bool valid = local < ch.count;
    uint64_t zmask;
    if (term_mode) {
      zmask = valid ? masks[ch.rank0 + local] : ((1ull << m) - 1);
    } else {
      zmask = valid ? mask : ((1ull << m) - 1);
      for (int q = 0; q < S; ++q) mask = next_comb(mask);  // this group's next subset
    }
    // pair list: pos[t] = t-th set bit of zmask
    for (int t = g; t < m; t += G) {
      uint64_t x = zmask;
      for (int q = 0; q < t; ++q) x &= x - 1;
      pos[t] = __ffsll((long long)x) - 1;
    }
    __syncwarp();
    // gather B = (X A)^{(Z)}: B[r][c] = At[idx(r)][idx(c)], idx(r) = 2 pos[r/2] + (r&1)
    BlockWalk wg(g, G, N);  // element e = r * N + c
    for (int e = g; e < N * N; e += G, wg.next()) {
      const int r = wg.i, c = wg.j;
      const int ir = 2 * pos[r >> 1] + (r & 1), ic = 2 * pos[c >> 1] + (c & 1);
      tile[r * ld + c] = valid ? OB::load(job.At, (size_t)ir * n + ic) : OB::zero();
    }
    if (loops) {
      for (int r = g; r < N; r += G) {
        const int ir = 2 * pos[r >> 1] + (r & 1);
        const TB v = valid ? OB::load(job.diag, ir) : OB::zero();
        VA[r] = v;      // a = v
        VB[r ^ 1] = v;  // b = X v^T
      }
    }
    __syncwarp();
    householder<TB>(tile, ld, N, W, P, TV, VA, VB, beta, loops, g, G);
    if (loops) loop_moments<TB>(tile, ld, N, h, VA, beta, W, TV, Ub, g, G);
    labudde<TB>(tile, ld, N, h, DNb, g, G);
    if constexpr (kMixed) {
      // widen the coefficients (and loop moments) for the FP64 series
      const int jm = min(N, h);
      for (int j = g; j <= jm; j += G) DN[j] = OB::widen(DNb[j]);
      if (loops)
        for (int k = 1 + g; k <= jm; k += G) U[k] = OB::widen(Ub[k]);
      __syncwarp();
    }
    if (loops && N < h) loop_moments_tail<TS>(N, h, DN, U, g, G);
    const TS f = series<TS>(N, h, DN, U, GS, AC, ES, AC2, loops, tables, g, G);
    if (term_mode) {
      if (valid && g == 0) {
        terms_out[2 * (ch.rank0 + local)] = OS::re(f);
        terms_out[2 * (ch.rank0 + local) + 1] = OS::im(f);
      }
    } else if (valid) {
      const double fr = neg ? -OS::re(f) : OS::re(f);
      const double fi = neg ? -OS::im(f) : OS::im(f);
      dd_add(re_hi, re_lo, fr);
      dd_add(im_hi, im_lo, fi);
      asum += OS::absval(f);
    }
    __syncwarp();
  }
  if (term_mode) return;
  // Combine the S group accumulators in group order.
  double t_re_hi = __shfl_sync(kFull, re_hi, 0), t_re_lo = __shfl_sync(kFull, re_lo, 0);
  double t_im_hi = __shfl_sync(kFull, im_hi, 0), t_im_lo = __shfl_sync(kFull, im_lo, 0);
  double t_abs = __shfl_sync(kFull, asum, 0);
  for (int q = 1; q < S; ++q) {
    const double a = __shfl_sync(kFull, re_hi, q * G), b = __shfl_sync(kFull, re_lo, q * G);
    const double c = __shfl_sync(kFull, im_hi, q * G), d = __shfl_sync(kFull, im_lo, q * G);
    const double e = __shfl_sync(kFull, asum, q * G);
    dd_add_dd(t_re_hi, t_re_lo, a, b);
    dd_add_dd(t_im_hi, t_im_lo, c, d);
    t_abs += e;
  }
  if (lane == 0) {
    double* o = partial_out;
    o[0] = t_re_hi;
    o[1] = t_re_lo;
    o[2] = t_im_hi;
    o[3] = t_im_lo;
    o[4] = t_abs;
  }
}

template <class TB, class TS, int WPB>
__global__ void __launch_bounds__(32 * WPB, 1) subset_kernel(KernelArgs args) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* wbase = smem + warp * args.warp_bytes;
  for (;;) {
    int ci = 0;
    if (lane == 0) ci = atomicAdd(args.counter, 1);
    ci = __shfl_sync(kFull, ci, 0);
    if (ci >= args.nchunks) break;
    const int id = args.order[ci];
    const Chunk ch = args.chunks[id];
    const Job job = args.jobs[ch.job];
    process_chunk<TB, TS>(job, ch, args.partials ? args.partials + 5 * (size_t)id : nullptr, args.tables,
                     args.masks, args.terms_out, wbase, lane);
  }
}

// ---------------------------------------------------------------------------
// Server loop.  Warps claim chunk descriptors from two rings in device
// memory that the host scheduler appends to, by copy-engine transfers, while
// the kernel runs: the host copies the new descriptors and then the new
// published count; a warp reads the count (ld.acquire at gpu scope) and
// claims the next entry with a compare-and-swap on a device counter.  A CTA
// has kSrvSmallWarps warps with small shared-memory slices and one with a
// large slice: ring 0 holds chunks whose tiles fit a small slice (planned
// for 8 warps per CTA), ring 1 the larger tiles, which only the large-slice
// warp takes (it serves ring 0 too when ring 1 is empty).  After
// its chunk a warp bumps the job's completed-chunk counter; the warp that
// completes a job adds the job's chunk partials in chunk order and posts the
// result and a flag to host memory (release store at system scope).  A warp
// with no work sleeps between polls with exponential back-off; when no warp
// has claimed anything for idle_ns the first warp to notice raises the stop
// flag and every warp leaves, and the host relaunches the kernel when new
// work arrives.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned int ld_relaxed_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(unsigned int* p, unsigned int v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_sys(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ long long globaltimer() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <class T>
__global__ void __launch_bounds__(32 * kSrvWarps, 1) server_kernel(ServerArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // warps 0..kSrvSmallWarps-1 own small slices; the last warp owns the large
  // one and serves the large-tile ring first, then the small-tile ring
  const bool big = warp == kSrvSmallWarps;
  unsigned char* wbase = smem + warp * kSrvSmallBytes;
  volatile long long* const last_claim = reinterpret_cast<volatile long long*>(a.head + kSrvHeadLast);
  const long long started = globaltimer();
  unsigned long long t_seen[2] = {0, 0};  // published counts this warp has acquired, per ring
  for (;;) {
    unsigned long long idx = 0;
    int status = 0;  // 1: claimed an entry, 2: leave
    int rsel = 0;
    if (lane == 0) {
      unsigned int nap = 256;
      for (;;) {
        // once the stop flag is up no warp claims anything more, so the
        // kernel ends when the chunks already claimed are done
        if (ld_relaxed_gpu(a.stop) != 0u) {
          status = 2;
          break;
        }
        // try the rings this warp serves, in order
        for (int q = big ? 0 : 1; q < 2 && status == 0; ++q) {
          const int rg = big ? 1 - q : 0;  // big warp: ring 1, then ring 0
          unsigned long long* const claims = a.head + (rg ? kSrvHeadClaim1 : kSrvHeadClaim0);
          unsigned long long h = atomicAdd(claims, 0ull);
          for (;;) {
            if (h < t_seen[rg]) {
              // entries below t_seen are published; take entry h unless another
              // warp got there first (then retry with the value it left)
              const unsigned long long prev = atomicCAS(claims, h, h + 1);
              if (prev == h) {
                idx = h;
                rsel = rg;
                status = 1;
                *last_claim = globaltimer();
                break;
              }
              h = prev;
              continue;
            }
            const unsigned long long t = ld_acquire_gpu(a.tail[rg]);
            if (t == t_seen[rg]) break;  // nothing new on this ring
            t_seen[rg] = t;
          }
        }
        if (status) break;
        atomicAdd(a.head + 2, 1ull);  // diagnostic: idle polls
        const long long quiet = globaltimer() - max(started, *last_claim);
        if (quiet > a.idle_ns) {
          // idle: no claim for idle_ns, and every claimed chunk finished (the
          // finished count is read first, so a zero difference means none was
          // in flight when it was read and none claimed since).  While a warp
          // still works on a long chunk the others keep polling: a stop then
          // would strand the published entries behind a kernel that runs on
          // with only the busy warps.
          const unsigned long long fin = atomicAdd(a.head + kSrvHeadDone, 0ull);
          const unsigned long long cl =
              atomicAdd(a.head + kSrvHeadClaim0, 0ull) + atomicAdd(a.head + kSrvHeadClaim1, 0ull);
          if (cl == fin || quiet / kSrvQuietCap > a.idle_ns) {
            atomicExch(a.stop, 1u);
            status = 2;
            break;
          }
        }
        __nanosleep(nap);
        nap = min(nap * 2u, 32768u);
      }
    }
    status = __shfl_sync(kFull, status, 0);
    if (status == 2) break;
    idx = __shfl_sync(kFull, idx, 0);
    rsel = __shfl_sync(kFull, rsel, 0);
    // lane 0 reads the descriptor and the job entry (device memory, through
    // L2) and hands them to the warp
    Chunk ch;
    SrvJob sj;
    {
      unsigned long long cw[sizeof(Chunk) / 8], jw[sizeof(SrvJob) / 8];
      if (lane == 0) {
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(a.ring[rsel] + idx % a.cap[rsel]);
#pragma unroll
        for (int k = 0; k < (int)(sizeof(Chunk) / 8); ++k) cw[k] = __ldcg(src + k);
        const Chunk* cp = reinterpret_cast<const Chunk*>(cw);
        const unsigned long long* js = reinterpret_cast<const unsigned long long*>(a.jobs + cp->job);
#pragma unroll
        for (int k = 0; k < (int)(sizeof(SrvJob) / 8); ++k) jw[k] = __ldcg(js + k);
      }
#pragma unroll
      for (int k = 0; k < (int)(sizeof(Chunk) / 8); ++k) cw[k] = __shfl_sync(kFull, cw[k], 0);
#pragma unroll
      for (int k = 0; k < (int)(sizeof(SrvJob) / 8); ++k) jw[k] = __shfl_sync(kFull, jw[k], 0);
      memcpy(&ch, cw, sizeof(Chunk));
      memcpy(&sj, jw, sizeof(SrvJob));
    }
    if (ch.tag != (uint16_t)(sj.gen & 0xffffu)) {
      // a descriptor that does not belong to the job now in its slot: count
      // it and leave the job's counters alone (diagnostic; never expected)
      if (lane == 0) {
        st_relaxed_sys(a.stats + 3, atomicAdd(a.head + 5, 1ull) + 1);
        atomicAdd(a.head + kSrvHeadDone, 1ull);
      }
      continue;
    }
    const long long tc0 = globaltimer();
    process_chunk<T, T>(sj.job, ch, sj.partials + 5 * (size_t)ch.aux, a.tables, nullptr, nullptr, wbase, lane);
    __threadfence();
    unsigned int prev = 0;
    if (lane == 0) {
      prev = atomicAdd(sj.done, 1u);
      // diagnostics: chunks done, total chunk time
      const unsigned long long c = atomicAdd(a.head + 3, 1ull) + 1;
      const unsigned long long tt = atomicAdd(a.head + 4, (unsigned long long)(globaltimer() - tc0));
      if ((c & 255ull) == 0) {
        st_relaxed_sys(a.stats, c);
        st_relaxed_sys(a.stats + 1, tt);
        st_relaxed_sys(a.stats + 2, *reinterpret_cast<volatile unsigned long long*>(a.head + 2));
      }
    }
    prev = __shfl_sync(kFull, prev, 0);
    if (prev >= sj.nchunks && lane == 0) st_relaxed_sys(a.stats + 4, atomicAdd(a.head + 6, 1ull) + 1);
    if (prev + 1 == sj.nchunks) {
      __threadfence();
      // fixed-order sum of the job's partials: lane l takes chunks l, l+32, ...
      double rh = 0, rl = 0, ih = 0, il = 0, ab = 0;
      unsigned int unwritten = 0;
      for (unsigned int c = lane; c < sj.nchunks; c += 32) {
        const double* p = sj.partials + 5 * (size_t)c;
        if (__ldcg(p) != __ldcg(p)) ++unwritten;  // diagnostic fill seen: chunk c never wrote
        dd_add_dd(rh, rl, __ldcg(p), __ldcg(p + 1));
        dd_add_dd(ih, il, __ldcg(p + 2), __ldcg(p + 3));
        ab += __ldcg(p + 4);
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double a0 = __shfl_xor_sync(kFull, rh, o), a1 = __shfl_xor_sync(kFull, rl, o);
        const double b0 = __shfl_xor_sync(kFull, ih, o), b1 = __shfl_xor_sync(kFull, il, o);
        const double c0 = __shfl_xor_sync(kFull, ab, o);
        dd_add_dd(rh, rl, a0, a1);
        dd_add_dd(ih, il, b0, b1);
        ab += c0;
      }
      for (int o = 16; o > 0; o >>= 1) unwritten += __shfl_xor_sync(kFull, unwritten, o);
      if (lane == 0 && unwritten) st_relaxed_sys(a.stats + 5, atomicAdd(a.head + 9, (unsigned long long)unwritten) + unwritten);
      if (lane == 0) {
        volatile double* r = sj.result;
        r[0] = rh;
        r[1] = ih;
        r[2] = rl;
        r[3] = il;
        r[4] = ab;
        __threadfence_system();
        st_release_sys(sj.flag, sj.gen);
      }
    }
    if (lane == 0) atomicAdd(a.head + kSrvHeadDone, 1ull);  // this claim is finished
  }
}

// Symmetrised, pair-swapped copy of A: At[i][j] = A[i^1][j] off the
// diagonal of A (upper triangle read), 0 where j == i^1; diag = diag(A).
template <class T>
__global__ void prep_kernel(const double* __restrict__ A, int n, double* __restrict__ At,
                            double* __restrict__ diag) {
  const int total = n * n;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int i = e / n, j = e - (e / n) * n;
    const int ii = i ^ 1;
    const int r = min(ii, j), c = max(ii, j);
    if (sizeof(T) == 16) {
      double2 v = make_double2(0.0, 0.0);
      if (ii != j) v = reinterpret_cast<const double2*>(A)[(size_t)r * n + c];
      reinterpret_cast<double2*>(At)[e] = v;
      if (j == i) reinterpret_cast<double2*>(diag)[i] = reinterpret_cast<const double2*>(A)[(size_t)i * n + i];
    } else {
      At[e] = (ii != j) ? A[(size_t)r * n + c] : 0.0;
      if (j == i) diag[i] = A[(size_t)i * n + i];
    }
  }
}

// Batched form of prep_kernel: block b prepares job b from srcs[b].
template <class T>
__global__ void prep_batch_kernel(const double* const* __restrict__ srcs, const Job* __restrict__ jobs) {
  const Job jb = jobs[blockIdx.x];
  const double* A = srcs[blockIdx.x];
  const int n = jb.n, total = n * n;
  double* At = const_cast<double*>(jb.At);
  double* diag = const_cast<double*>(jb.diag);
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int i = e / n, j = e - (e / n) * n;
    const int ii = i ^ 1;
    const int r = min(ii, j), c = max(ii, j);
    if (sizeof(T) == 16) {
      double2 v = make_double2(0.0, 0.0);
      if (ii != j) v = reinterpret_cast<const double2*>(A)[(size_t)r * n + c];
      reinterpret_cast<double2*>(At)[e] = v;
      if (j == i) reinterpret_cast<double2*>(diag)[i] = reinterpret_cast<const double2*>(A)[(size_t)i * n + i];
    } else {
      At[e] = (ii != j) ? A[(size_t)r * n + c] : 0.0;
      if (j == i) diag[i] = A[(size_t)i * n + i];
    }
  }
}

// Fixed-order double-double reduction of one job's chunk partials.
__global__ void finalize_kernel(const double* __restrict__ partials, const int* __restrict__ job_begin,
                                double* __restrict__ out) {
  __shared__ double sh[5][256];
  const int job = blockIdx.x;
  const int b = job_begin[job], e = job_begin[job + 1];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int len = e - b;
  const int per = (len + nt - 1) / nt;
  const int lo = b + tid * per, hi = min(e, lo + per);
  double rh = 0, rl = 0, ih = 0, il = 0, ab = 0;
  for (int c = lo; c < hi; ++c) {
    const double* p = partials + 5 * (size_t)c;
    dd_add_dd(rh, rl, p[0], p[1]);
    dd_add_dd(ih, il, p[2], p[3]);
    ab += p[4];
  }
  sh[0][tid] = rh;
  sh[1][tid] = rl;
  sh[2][tid] = ih;
  sh[3][tid] = il;
  sh[4][tid] = ab;
  __syncthreads();
  for (int st = 1; st < nt; st <<= 1) {
    if ((tid & (2 * st - 1)) == 0 && tid + st < nt) {
      double a = sh[0][tid], bl = sh[1][tid], c = sh[2][tid], d = sh[3][tid];
      dd_add_dd(a, bl, sh[0][tid + st], sh[1][tid + st]);
      dd_add_dd(c, d, sh[2][tid + st], sh[3][tid + st]);
      sh[0][tid] = a;
      sh[1][tid] = bl;
      sh[2][tid] = c;
      sh[3][tid] = d;
      sh[4][tid] += sh[4][tid + st];
    }
    __syncthreads();
  }
  if (tid == 0) {
    double* o = out + 5 * (size_t)job;
    o[0] = sh[0][0];
    o[1] = sh[2][0];
    o[2] = sh[1][0];
    o[3] = sh[3][0];
    o[4] = sh[4][0];
  }
}

// Dependent DFMA chains over every SM: the FP64 roofline denominator.
// Eight independent chains per thread with operands in registers (b and c
// arrive as kernel arguments), 16 warps per SM.
__global__ void __launch_bounds__(512) fp64_probe_kernel(double* sink, int iters, double b, double c) {
  double a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = 1.0 + 1e-3 * (threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = ::fma(a[i], b, c);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

namespace {

template <class TB, class TS, int WPB>
cudaError_t set_smem_attr() {
  return cudaFuncSetAttribute(subset_kernel<TB, TS, WPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kMaxSmemPerBlock);
}

template <class TB, class TS>
cudaError_t set_smem_attrs() {
  cudaError_t e = set_smem_attr<TB, TS, 4>();
  if (e == cudaSuccess) e = set_smem_attr<TB, TS, 8>();
  if (e == cudaSuccess) e = set_smem_attr<TB, TS, 16>();
  return e;
}

template <class TB, class TS>
cudaError_t launch_kind(const KernelArgs& a, int wpb, int grid, cudaStream_t st) {
  const int smem = a.warp_bytes * wpb;
  switch (wpb) {
    case 4: subset_kernel<TB, TS, 4><<<grid, 32 * 4, smem, st>>>(a); break;
    case 8: subset_kernel<TB, TS, 8><<<grid, 32 * 8, smem, st>>>(a); break;
    case 16: subset_kernel<TB, TS, 16><<<grid, 32 * 16, smem, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t configure_kernels() {
  cudaError_t e = set_smem_attrs<cplx, cplx>();
  if (e == cudaSuccess) e = set_smem_attrs<double, double>();
  if (e == cudaSuccess) e = set_smem_attrs<cplxf, cplx>();
  if (e == cudaSuccess) e = set_smem_attrs<float, double>();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(server_kernel<cplx>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSrvSmemBytes);
  return e;
}

cudaError_t launch_prep(const double* A, int n, int is_real, double* At, double* diag,
                        cudaStream_t st) {
  const int total = n * n;
  const int threads = 256, blocks = (total + threads - 1) / threads;
  if (is_real)
    prep_kernel<double><<<blocks, threads, 0, st>>>(A, n, At, diag);
  else
    prep_kernel<cplx><<<blocks, threads, 0, st>>>(A, n, At, diag);
  return cudaGetLastError();
}

cudaError_t launch_prep_batch(const double* const* srcs, const Job* jobs, int njobs, int is_real,
                              cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  if (is_real)
    prep_batch_kernel<double><<<njobs, 256, 0, st>>>(srcs, jobs);
  else
    prep_batch_kernel<cplx><<<njobs, 256, 0, st>>>(srcs, jobs);
  return cudaGetLastError();
}

cudaError_t launch_subsets(const KernelArgs& a, int kind, int wpb, int grid, cudaStream_t st) {
  switch (kind) {
    case kKindC128: return launch_kind<cplx, cplx>(a, wpb, grid, st);
    case kKindF64: return launch_kind<double, double>(a, wpb, grid, st);
    case kKindC64: return launch_kind<cplxf, cplx>(a, wpb, grid, st);
    case kKindF32: return launch_kind<float, double>(a, wpb, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_server(const ServerArgs& a, int grid, cudaStream_t st) {
  server_kernel<cplx><<<grid, 32 * kSrvWarps, kSrvSmemBytes, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const double* partials, const int* job_begin, int njobs, double* out,
                            cudaStream_t st) {
  finalize_kernel<<<njobs, 256, 0, st>>>(partials, job_begin, out);
  return cudaGetLastError();
}

cudaError_t launch_fp64_probe(double* sink, int iters, int blocks, cudaStream_t st) {
  fp64_probe_kernel<<<blocks, 512, 0, st>>>(sink, iters, 0.9999999, 1e-7);
  return cudaGetLastError();
}

}  // namespace hafgb
