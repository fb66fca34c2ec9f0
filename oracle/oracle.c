/*
 * oracle.c -- CPU oracle for the hafnian and the loop hafnian.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library calls, links or loads
 * this file: only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code with the CUDA path.
 *
 * Everything is computed in IEEE binary128 ("quad"): __float128 on x86-64,
 * long double on AArch64 (which is binary128 there).  Both are software
 * implementations with correctly rounded basic operations, so the two
 * machines give the same numbers for the same inputs.
 *
 * Contents (each function cites the passage it restates):
 *   oracle_haf_brute      -- the definition: sum over perfect matchings
 *                            (Sec. 2, eq. hafA) or over single-pair
 *                            matchings with loops (Sec. 2, lhaf definition).
 *   oracle_term           -- one summand f(Z) of the inclusion-exclusion
 *                            sum, by the literal trace generating function
 *                            p(lambda, B) of Sec. 3.3 (eq. poly) and its
 *                            loop counterpart q(lambda, B, v), with traces
 *                            taken from explicit matrix powers.
 *   oracle_haf_formula    -- the full signed subset sum of Sec. 3.2
 *                            (eq. main / Pset) over those summands, i.e.
 *                            eq. haffinal and its loop-hafnian analogue.
 *   oracle_ryser          -- Ryser's inclusion-exclusion permanent (cited
 *                            in Sec. 1), used to pin the bipartite identity
 *                            haf([[0,W],[W^T,0]]) = per(W) (eq. bipartite).
 *
 * Input convention (shared with the library): A is n x n, row-major,
 * complex values interleaved (re, im).  Off-diagonal entries are read
 * from the upper triangle only (i < j); the hafnian depends on nothing
 * else (App. C: haf(A) = haf(A + L) for lower-triangular L).  The loop
 * hafnian also reads the diagonal.
 *
 * Reading of the loop term (Sec. 3.3): the printed vector term
 * v (X B)^{k-1} v^T / 2 fails already at n = 2.  The oracle uses
 * u_k = v B^{k-1} X v^T with B = X A^{(Z)} (A's diagonal removed) and
 * v = diag(A^{(Z)}); the test-suite checks this reading against brute
 * force and checks that the printed form disagrees (variant flag below).
 *
 * Output convention: a quad value q is returned as a double-double
 * (hi = (double)q, lo = (double)(q - hi)).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#if defined(__x86_64__) || defined(__i386__)
typedef __float128 quad;
#elif defined(__aarch64__)
typedef long double quad;
#else
#error "the oracle needs an IEEE binary128 type"
#endif

typedef struct {
  quad re, im;
} cq;

static inline cq cq_mk(quad re, quad im) {
  cq z;
  z.re = re;
  z.im = im;
  return z;
}
static inline cq cq_add(cq a, cq b) { return cq_mk(a.re + b.re, a.im + b.im); }
static inline cq cq_sub(cq a, cq b) { return cq_mk(a.re - b.re, a.im - b.im); }
static inline cq cq_mul(cq a, cq b) {
  return cq_mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
static inline cq cq_scale(cq a, quad s) { return cq_mk(a.re * s, a.im * s); }

static void q_to_dd(quad q, double* hi, double* lo) {
  double h = (double)q;
  *hi = h;
  *lo = (double)(q - (quad)h);
}

static void cq_out(cq z, double* out4) {
  /* out4 = {re_hi, im_hi, re_lo, im_lo} */
  q_to_dd(z.re, &out4[0], &out4[2]);
  q_to_dd(z.im, &out4[1], &out4[3]);
}

/* Entry (i, j) of the symmetric matrix defined by the upper triangle. */
static cq entry(const double* A, int n, int i, int j) {
  int r = i < j ? i : j, c = i < j ? j : i;
  return cq_mk((quad)A[2 * ((size_t)r * n + c)], (quad)A[2 * ((size_t)r * n + c) + 1]);
}

/* ------------------------------------------------------------------ */
/* Brute force over matchings (Sec. 2).                                */
/* ------------------------------------------------------------------ */

typedef struct {
  const double* A;
  int n;
  int loops;
  uint64_t full;
} bf_ctx;

/* Match the lowest unmatched vertex i with every unmatched j > i (and,
 * for the loop hafnian, with itself), multiplying the edge weight into
 * the running product.  Each perfect (resp. single-pair) matching is
 * reached exactly once. */
static void bf_rec(const bf_ctx* ctx, uint64_t used, cq prod, cq* acc) {
  if (used == ctx->full) {
    *acc = cq_add(*acc, prod);
    return;
  }
  int i = 0;
  while ((used >> i) & 1u) i++;
  uint64_t u2 = used | ((uint64_t)1 << i);
  if (ctx->loops) bf_rec(ctx, u2, cq_mul(prod, entry(ctx->A, ctx->n, i, i)), acc);
  for (int j = i + 1; j < ctx->n; j++) {
    if ((u2 >> j) & 1u) continue;
    bf_rec(ctx, u2 | ((uint64_t)1 << j), cq_mul(prod, entry(ctx->A, ctx->n, i, j)), acc);
  }
}

/* haf(A) (loops = 0) or lhaf(A) (loops = 1) by enumeration; n <= 24.
 * Returns 0, or -1 on a bad argument. */
int oracle_haf_brute(const double* A, int n, int loops, double* out4) {
  if (n < 0 || n > 24 || !out4 || (n > 0 && !A)) return -1;
  bf_ctx ctx;
  ctx.A = A;
  ctx.n = n;
  ctx.loops = loops;
  ctx.full = (n == 64) ? ~(uint64_t)0 : (((uint64_t)1 << n) - 1);
  cq acc = cq_mk(0, 0);
  bf_rec(&ctx, 0, cq_mk(1, 0), &acc);
  cq_out(acc, out4);
  return 0;
}

/* ------------------------------------------------------------------ */
/* One summand f(Z) by the trace generating function (Sec. 3.3).       */
/* ------------------------------------------------------------------ */

/* variant 0: loop term u_k = v B^{k-1} X v^T (the reading the tests pin)
 * variant 1: loop term as printed, u_k = v (X B)^{k-1} v^T            */
static cq term_formula(const double* A, int n, uint64_t mask, int loops, int variant) {
  const int h = n / 2;
  int idx[128];
  int N = 0;
  for (int i = 0; i < h; i++)
    if ((mask >> i) & 1u) {
      idx[N++] = 2 * i;
      idx[N++] = 2 * i + 1;
    }
  /* Empty Z: the generating function has no lambda^h term for h >= 1. */
  if (N == 0) return cq_mk(0, 0);

  cq* B = (cq*)malloc(sizeof(cq) * N * N);
  cq* P = (cq*)malloc(sizeof(cq) * N * N);
  cq* T = (cq*)malloc(sizeof(cq) * N * N);
  cq* c = (cq*)calloc((size_t)h + 1, sizeof(cq));
  /* B = (X A)^{(Z)}: row r of X A is row (idx[r] ^ 1) of A, i.e. the two
   * rows of each kept pair are swapped (eq. matA).  The diagonal of A
   * is a loop weight, not an edge, so it is left out of B. */
  for (int r = 0; r < N; r++)
    for (int s = 0; s < N; s++) {
      int i = idx[r] ^ 1, j = idx[s];
      B[r * N + s] = (i == j) ? cq_mk(0, 0) : entry(A, n, i, j);
    }
  /* Power traces tr(B^k), k = 1..h, from explicit powers P = B^k. */
  memcpy(P, B, sizeof(cq) * N * N);
  for (int k = 1; k <= h; k++) {
    cq t = cq_mk(0, 0);
    for (int r = 0; r < N; r++) t = cq_add(t, P[r * N + r]);
    c[k] = cq_scale(t, (quad)1 / (quad)(2 * k));
    if (k < h) {
      for (int r = 0; r < N; r++)
        for (int s = 0; s < N; s++) {
          cq acc = cq_mk(0, 0);
          for (int l = 0; l < N; l++) acc = cq_add(acc, cq_mul(P[r * N + l], B[l * N + s]));
          T[r * N + s] = acc;
        }
      memcpy(P, T, sizeof(cq) * N * N);
    }
  }
  if (loops) {
    /* v = diag(A^{(Z)}) as a row vector. */
    cq* v = (cq*)malloc(sizeof(cq) * N);
    cq* y = (cq*)malloc(sizeof(cq) * N);
    cq* y2 = (cq*)malloc(sizeof(cq) * N);
    for (int r = 0; r < N; r++) v[r] = entry(A, n, idx[r], idx[r]);
    if (variant == 0) {
      /* y = X v^T (X swaps the two members of each kept pair), then
       * u_k = v . (B^{k-1} y). */
      for (int r = 0; r < N; r++) y[r] = v[r ^ 1];
    } else {
      /* printed form: u_k = v . ((X B)^{k-1} v^T) */
      for (int r = 0; r < N; r++) y[r] = v[r];
    }
    for (int k = 1; k <= h; k++) {
      cq u = cq_mk(0, 0);
      for (int r = 0; r < N; r++) u = cq_add(u, cq_mul(v[r], y[r]));
      c[k] = cq_add(c[k], cq_scale(u, (quad)0.5));
      if (k < h) {
        for (int r = 0; r < N; r++) {
          cq acc = cq_mk(0, 0);
          for (int l = 0; l < N; l++) {
            cq b = (variant == 0) ? B[r * N + l] : B[(r ^ 1) * N + l]; /* (XB)_{rl} */
            acc = cq_add(acc, cq_mul(b, y[l]));
          }
          y2[r] = acc;
        }
        memcpy(y, y2, sizeof(cq) * N);
      }
    }
    free(v);
    free(y);
    free(y2);
  }
  /* Generating function: sum_{j=1}^{h} (1/j!) (sum_k c_k lambda^k)^j,
   * truncated at lambda^h; the summand is its lambda^h coefficient. */
  cq* Q = (cq*)calloc((size_t)h + 1, sizeof(cq)); /* running Q^j / j! */
  cq* Q2 = (cq*)calloc((size_t)h + 1, sizeof(cq));
  cq* E = (cq*)calloc((size_t)h + 1, sizeof(cq));
  for (int k = 1; k <= h; k++) Q[k] = c[k];
  for (int k = 0; k <= h; k++) E[k] = Q[k];
  for (int j = 2; j <= h; j++) {
    for (int k = 0; k <= h; k++) {
      cq acc = cq_mk(0, 0);
      for (int a = 1; a < k; a++) acc = cq_add(acc, cq_mul(Q[a], c[k - a]));
      Q2[k] = cq_scale(acc, (quad)1 / (quad)j);
    }
    memcpy(Q, Q2, sizeof(cq) * (h + 1));
    for (int k = 0; k <= h; k++) E[k] = cq_add(E[k], Q[k]);
  }
  cq f = E[h];
  free(Q);
  free(Q2);
  free(E);
  free(B);
  free(P);
  free(T);
  free(c);
  return f;
}

/* f(Z) for each mask in masks[0..count): out has 4 doubles per term
 * (re_hi, im_hi, re_lo, im_lo).  The sign (-1)^{h-|Z|} is NOT applied.
 * n must be even, 2 <= n <= 128.  Returns 0 or -1. */
int oracle_terms(const double* A, int n, int loops, int variant, const uint64_t* masks,
                 int64_t count, int nthreads, double* out) {
  if (n < 2 || n > 128 || (n & 1) || !A || !masks || !out || count < 0) return -1;
  const int h = n / 2;
  for (int64_t t = 0; t < count; t++)
    if (h < 64 && (masks[t] >> h) != 0) return -1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
  for (int64_t t = 0; t < count; t++) {
    cq f = term_formula(A, n, masks[t], loops, variant);
    cq_out(f, out + 4 * t);
  }
  return 0;
}

/* Full signed sum over all 2^{n/2} subsets (eq. main, eq. haffinal).
 * out4 receives the value, abs_sum receives sum_Z |f(Z)| (double).
 * n must be even and <= 48 (the loop over 2^{n/2} masks is the caller's
 * time budget).  n = 0 gives 1.  Returns 0 or -1. */
int oracle_haf_formula(const double* A, int n, int loops, int variant, int nthreads,
                       double* out4, double* abs_sum) {
  if (n < 0 || n > 48 || (n & 1) || !out4 || (n > 0 && !A)) return -1;
  if (n == 0) {
    cq_out(cq_mk(1, 0), out4);
    if (abs_sum) *abs_sum = 1.0;
    return 0;
  }
  const int h = n / 2;
  const int64_t count = (int64_t)1 << h;
  cq* terms = (cq*)malloc(sizeof(cq) * (size_t)count);
  if (!terms) return -1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
  for (int64_t z = 0; z < count; z++) terms[z] = term_formula(A, n, (uint64_t)z, loops, variant);
  /* Fixed-order signed sum in quad. */
  cq s = cq_mk(0, 0);
  double t_abs = 0.0;
  for (int64_t z = 0; z < count; z++) {
    int m = __builtin_popcountll((unsigned long long)z);
    cq f = terms[z];
    if ((h - m) & 1)
      s = cq_sub(s, f);
    else
      s = cq_add(s, f);
    t_abs += hypot((double)f.re, (double)f.im);
  }
  free(terms);
  cq_out(s, out4);
  if (abs_sum) *abs_sum = t_abs;
  return 0;
}

/* ------------------------------------------------------------------ */
/* Ryser's permanent (cited in Sec. 1; used for eq. bipartite).        */
/* ------------------------------------------------------------------ */

/* per(W) = (-1)^k sum_{S subset [k]} (-1)^{|S|} prod_i sum_{j in S} W_ij,
 * W k x k row-major interleaved complex, k <= 20. */
int oracle_ryser(const double* W, int k, double* out4) {
  if (k < 0 || k > 20 || !out4 || (k > 0 && !W)) return -1;
  if (k == 0) {
    cq_out(cq_mk(1, 0), out4);
    return 0;
  }
  cq total = cq_mk(0, 0);
  for (uint64_t S = 1; S < ((uint64_t)1 << k); S++) {
    cq prod = cq_mk(1, 0);
    for (int i = 0; i < k; i++) {
      cq rs = cq_mk(0, 0);
      for (int j = 0; j < k; j++)
        if ((S >> j) & 1u)
          rs = cq_add(rs, cq_mk((quad)W[2 * (i * k + j)], (quad)W[2 * (i * k + j) + 1]));
      prod = cq_mul(prod, rs);
    }
    int sz = __builtin_popcountll((unsigned long long)S);
    if ((k - sz) & 1)
      total = cq_sub(total, prod);
    else
      total = cq_add(total, prod);
  }
  cq_out(total, out4);
  return 0;
}
