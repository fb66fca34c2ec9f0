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
  const Chunk* ring;                  // device: chunk descriptors (written by the host's copies)
  unsigned long long cap;             // ring entries
  const unsigned long long* tail;     // device: chunks published so far (host copy, after the entries)
  unsigned long long* head;           // device: [0] chunks claimed, [1] time of the latest claim,
                                      // [2..] diagnostic counters
  unsigned int* stop;                 // device: nonzero makes every warp leave (set by the host's
                                      // copy at shutdown, or by the first warp that finds the
                                      // kernel idle)
  unsigned long long* stats;          // mapped host, diagnostic words (see the server's log)
  const SrvJob* jobs;                 // device job table
  const double* tables;
  long long idle_ns;                  // the kernel leaves after this long without a claim
  int warp_bytes;
};
constexpr int kMaxSmemPerBlock = 232448;  // 227 KiB opt-in on sm_100/sm_103
constexpr int kWarpBytes = (kMaxSmemPerBlock / kWarpsPerBlock) / 16 * 16;
constexpr int kMaxN = 56;

// Shared-memory bytes one subset needs: tile N x ld, five length-N vectors,
// six length-(h+1) series and h pair indices.
inline __host__ __device__ int subset_bytes(int N, int ld, int h, int elem_bytes) {
  int elems = N * ld + 5 * N + 6 * (h + 1);
  int b = elems * elem_bytes + 4 * h;
  return (b + 15) & ~15;
}

// Host planner (haf_capi.cu).
struct JobSpec {
  int n;
  int loops;
  int is_real;
  int64_t part = 0;  // this job covers part `part` of `nparts` of every size class
  int64_t nparts = 1;
  double max_chunk_units = 0;  // cap on a chunk's work in N^3 units (0: none)
};
struct Plan {
  std::vector<Chunk> chunks;
  std::vector<int> order;
  std::vector<int> job_begin;  // njobs + 1
  int64_t subsets = 0;
};
uint64_t binom(int a, int b);
uint64_t unrank_colex(uint64_t rank, int m, int h);
int build_plan(const std::vector<JobSpec>& jobs, int num_warps, Plan* plan);
int set_error(int code, const std::string& msg);

// Launchers (haf_kernels.cu).
cudaError_t launch_prep(const double* A, int n, int is_real, double* At, double* diag,
                        cudaStream_t st);
cudaError_t launch_subsets(const KernelArgs& a, int is_real, int grid, cudaStream_t st);
cudaError_t launch_prep_batch(const double* const* srcs, const Job* jobs, int njobs, int is_real,
                              cudaStream_t st);
cudaError_t launch_finalize(const double* partials, const int* job_begin, int njobs, double* out,
                            cudaStream_t st);
cudaError_t launch_fp64_probe(double* sink, int iters, int blocks, cudaStream_t st);
cudaError_t configure_kernels();
cudaError_t launch_server(const ServerArgs& a, int grid, cudaStream_t st);

}  // namespace hafgb
