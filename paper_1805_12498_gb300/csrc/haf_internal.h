// haf_internal.h -- structures shared by the host planner (haf_capi.cu) and
// the device kernels (haf_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace hafgb {

// One matrix of a launch.
struct Job {
  const double* At;    // device, n*n scalars: At[i*n+j] = A[i^1][j] (X A), 0 where j == i^1
  const double* diag;  // device, n scalars: diag(A) (loop weights)
  int n;               // even, >= 2
  int loops;           // 1: loop hafnian summand
};

// A contiguous range of colex-ordered subsets of one size m of one job.
// Subsets are bitmasks over the h = n/2 pairs; `mask0` is the first one
// (or, in per-term mode, `rank0` indexes the caller's mask list).
struct Chunk {
  uint64_t mask0;
  uint64_t rank0;
  uint32_t count;  // subsets in the chunk
  uint16_t job;
  uint8_t m;       // |Z|; the tile is N = 2m square
  uint8_t G;       // lanes per subset (1,2,4,8,16,32); 32/G subsets per warp
  uint8_t ld;      // tile leading dimension (N or N+1)
  uint8_t pad;
  uint16_t tag;    // server: low 16 bits of the job's generation
  uint32_t aux;    // server: index of the chunk within its job
};
static_assert(sizeof(Chunk) == 32, "Chunk layout");

struct KernelArgs {
  const Job* jobs;
  const Chunk* chunks;
  const int* order;        // scheduling order (LPT): chunk ids
  int nchunks;
  int* counter;            // work counter, zeroed before the launch
  double* partials;        // 5 doubles per chunk: re_hi, re_lo, im_hi, im_lo, abs
  const double* tables;    // [0..127] k/2, [128..255] 1/k (1/0 := 0)
  const uint64_t* masks;   // per-term mode: subset list (else null)
  double* terms_out;       // per-term mode: 2 doubles per subset (else null)
  int warp_bytes;          // shared-memory bytes owned by each warp
};

#ifndef HAF_WARPS_PER_BLOCK
#define HAF_WARPS_PER_BLOCK 4
#endif
// Warps per CTA of the FP64 default plan and of the server kernel.
constexpr int kWarpsPerBlock = HAF_WARPS_PER_BLOCK;

// Server: one admitted job as the device sees it (slot-indexed table in
// device memory, written by the host before the job's chunks are published).
struct SrvJob {
  Job job;
  double* partials;     // device, 5 doubles per chunk
  unsigned int* done;   // device, completed-chunk counter (zeroed at admission)
  double* result;       // device view of mapped host memory, 5 doubles
  unsigned int* flag;   // device view of mapped host memory, set to `gen` when done
  unsigned int nchunks;
  unsigned int gen;
};

static_assert(sizeof(SrvJob) % 8 == 0, "SrvJob is moved as 64-bit words");

struct ServerArgs {
  const Chunk* ring[2];               // device: chunk descriptors (written by the host's copies);
                                      // [0] tiles that fit a small slice, [1] larger tiles
  unsigned long long cap[2];          // ring entries
  const unsigned long long* tail[2];  // device: chunks published so far (host copy, after the entries)
  unsigned long long* head;           // device: [kSrvHeadClaim0/1] chunks claimed per ring,
                                      // [kSrvHeadLast] time of the latest claim, [kSrvHeadDone]
                                      // claimed chunks finished, the rest diagnostics
  unsigned int* stop;                 // device: nonzero makes every warp leave (set by the host's
                                      // copy at shutdown, or by the first warp that finds the
                                      // kernel idle)
  unsigned long long* stats;          // mapped host, diagnostic words (see the server's log)
  const SrvJob* jobs;                 // device job table
  const double* tables;
  long long idle_ns;                  // the kernel leaves after this long without a claim and
                                      // with no claimed chunk unfinished
};
constexpr int kMaxSmemPerBlock = 232448;  // 227 KiB opt-in on sm_100/sm_103
// Shared memory owned by each warp when a CTA has `wpb` warps.
constexpr int warp_bytes_for(int wpb) { return (kMaxSmemPerBlock / wpb) / 16 * 16; }
constexpr int kWarpBytes = warp_bytes_for(kWarpsPerBlock);
constexpr int kMaxN = 56;

// Server kernel CTA: kSrvSmallWarps warps with the 8-warps-per-CTA slice and
// one warp with the 4-warps-per-CTA slice (232,448 B in all).
constexpr int kSrvSmallWarps = 6;
constexpr int kSrvWarps = kSrvSmallWarps + 1;
constexpr int kSrvSmallBytes = warp_bytes_for(8);
constexpr int kSrvBigBytes = warp_bytes_for(4);
constexpr int kSrvSmemBytes = kSrvSmallWarps * kSrvSmallBytes + kSrvBigBytes;
static_assert(kSrvSmemBytes <= kMaxSmemPerBlock, "server CTA shared memory");
constexpr int kSrvHeadClaim0 = 0, kSrvHeadLast = 1, kSrvHeadDone = 7, kSrvHeadClaim1 = 10;
// A quiet spell this many times idle_ns ends the kernel even with chunks
// still counted in flight (a bound on the idle wait; the warps then finish
// what they hold, claim nothing more, and the host relaunches).
constexpr long long kSrvQuietCap = 3000;

// Precision of the bulk steps (gather, Householder, loop moments, La Budde).
// The power series, f(Z) and the subset sum are FP64 in both modes.
enum { kPrecF64 = 0, kPrecF32 = 1 };

// Kernel kinds: complex128, real float64, complex64 bulk, float32 bulk.
enum { kKindC128 = 0, kKindF64 = 1, kKindC64 = 2, kKindF32 = 3 };
inline int kernel_kind(int is_real, int prec) { return (is_real ? 1 : 0) + (prec == kPrecF32 ? 2 : 0); }
// Bytes of the bulk element (TB) and of the series element (TS) of a kind.
inline int bulk_elem_bytes(int kind) {
  static const int b[4] = {16, 8, 8, 4};
  return b[kind];
}
inline int series_elem_bytes(int kind) { return (kind & 1) ? 8 : 16; }
inline bool kind_mixed(int kind) { return kind >= kKindC64; }

// Shared-memory layout of one subset (byte offsets from the subset's base).
// sb / ss: bytes of the bulk element (gather, Householder, loop moments, La
// Budde) and of the series element (power series, f(Z)); equal in FP64.
//   tile : N x ld bulk elements; after La Budde its first 4 (h+1) series
//          elements hold the power-series arrays (GS, AC, ES, AC2), so it is
//          at least that large
//   vec  : W, P, TV (and VA for the loop hafnian), N bulk elements each; the
//          loop hafnian's b = X v^T is gathered into P, which the Krylov
//          start reads before its first pass writes P
//   dnb  : La Budde's output, h+1 bulk elements (ub: loop moments, h+1);
//          for the loop hafnian with N >= h+1 they take W and P, free by
//          the time the moments and La Budde run
//   dn   : h+1 series elements (u: loop moments), equal to dnb / ub in FP64
//   pos  : h ints, the pair list of the subset (dead after the gather; the
//          loop hafnian then keeps b's first entry, beta, in its first 16
//          bytes)
struct SubsetLayout {
  int vec, dnb, ub, dn, u, pos, total;
};
inline __host__ __device__ int round16(int b) { return (b + 15) & ~15; }

// Walk of lane g over the elements g, g + G, g + 2G, ... of a row-major
// block with L columns: (i, j) = (e / L, e % L) for element e, stepped with
// two divisions per walk instead of one per element (G / L and G % L are
// fixed; one carry per step since j + G % L < 2 L).
struct BlockWalk {
  int i, j, di, dj, L;
  __host__ __device__ __forceinline__ BlockWalk(int g, int G, int cols) : L(cols) {
    i = g / L;
    j = g - i * L;
    di = G / L;
    dj = G - di * L;
  }
  __host__ __device__ __forceinline__ void next() {
    i += di;
    j += dj;
    if (j >= L) {
      j -= L;
      ++i;
    }
  }
};
inline __host__ __device__ SubsetLayout subset_layout(int N, int ld, int h, int sb, int ss, bool mixed,
                                                      bool loops) {
  SubsetLayout L;
  const int tile = N * ld * sb, ser = 4 * (h + 1) * ss;
  L.vec = round16(tile > ser ? tile : ser);
  int end;
  if (!loops) {  // W, P, TV; La Budde's output
    L.dnb = L.vec + 3 * N * sb;
    L.ub = L.dnb;
    end = L.dnb + (h + 1) * sb;
  } else if (N >= h + 1) {  // W, P, TV, VA; La Budde's output in W, the moments in P
    L.dnb = L.vec;
    L.ub = L.vec + N * sb;
    end = L.vec + 4 * N * sb;
  } else {  // W, P, TV, VA; La Budde's output; the moments
    L.dnb = L.vec + 4 * N * sb;
    L.ub = L.dnb + (h + 1) * sb;
    end = L.ub + (h + 1) * sb;
  }
  if (mixed) {
    L.dn = round16(end);
    L.u = L.dn + (h + 1) * ss;
    end = L.u + (loops ? (h + 1) * ss : 0);
  } else {
    L.dn = L.dnb;
    L.u = L.ub;
  }
  L.pos = round16(end);
  L.total = round16(L.pos + 4 * h);
  return L;
}
inline __host__ __device__ int subset_bytes(int N, int ld, int h, int sb, int ss, bool mixed, bool loops) {
  return subset_layout(N, ld, h, sb, ss, mixed, loops).total;
}

// Host planner (haf_capi.cu).
struct JobSpec {
  int n;
  int loops;
  int is_real;
  int64_t part = 0;  // this job covers part `part` of `nparts` of every size class
  int64_t nparts = 1;
  double max_chunk_units = 0;  // cap on a chunk's work in N^3 units (0: none) ...
  double max_chunks = 65536;   // ... but never more chunks than this per job (part)
  int prec = kPrecF64;         // all jobs of one plan share is_real and prec
};
// Launch shape of a plan: warps per CTA (4, 8 or 16; size classes whose
// tiles do not fit that warp slice run in a second launch with fewer warps
// per CTA) and the chunk granularity (about chunks_per_warp chunks per
// resident warp, per launch).
struct PlanCfg {
  int wpb = kWarpsPerBlock;
  int chunks_per_warp = 8;
};
// One launch of a plan: order[begin, end) run with `wpb` warps per CTA.
struct PlanSeg {
  int begin = 0, end = 0;
  int wpb = kWarpsPerBlock;
  int warp_bytes = kWarpBytes;
};
struct Plan {
  std::vector<Chunk> chunks;   // grouped by job (job_begin), then by size
  std::vector<int> order;      // launch order: segment by segment, largest chunks first
  std::vector<PlanSeg> segs;   // most warps per CTA first
  std::vector<int> job_begin;  // njobs + 1
  int64_t subsets = 0;
  int kind = kKindC128;
  int wpb = kWarpsPerBlock;    // first segment's (a one-segment plan's) shape
  int warp_bytes = kWarpBytes;
};
uint64_t binom(int a, int b);
uint64_t unrank_colex(uint64_t rank, int m, int h);
int build_plan(const std::vector<JobSpec>& jobs, int sms, const PlanCfg& cfg, Plan* plan);
int set_error(int code, const std::string& msg);

// Launchers (haf_kernels.cu).
cudaError_t launch_prep(const double* A, int n, int is_real, double* At, double* diag,
                        cudaStream_t st);
// kind: kKind*; wpb: 4, 8 or 16 warps per CTA (a.warp_bytes = warp_bytes_for(wpb)).
cudaError_t launch_subsets(const KernelArgs& a, int kind, int wpb, int grid, cudaStream_t st);
cudaError_t launch_prep_batch(const double* const* srcs, const Job* jobs, int njobs, int is_real,
                              cudaStream_t st);
cudaError_t launch_finalize(const double* partials, const int* job_begin, int njobs, double* out,
                            cudaStream_t st);
cudaError_t launch_fp64_probe(double* sink, int iters, int blocks, cudaStream_t st);
cudaError_t configure_kernels();
cudaError_t launch_server(const ServerArgs& a, int grid, cudaStream_t st);

}  // namespace hafgb
