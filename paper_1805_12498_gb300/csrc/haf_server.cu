// haf_server.cu -- continuous-batching hafnian server: the host scheduler
// around server_kernel (haf_kernels.cu).
//
// Requests (haf or lhaf of one matrix) are queued on submit.  A scheduler
// thread admits them while job slots and device memory allow, prepares each
// admitted matrix on the host (pair swap X A, upper-triangle symmetrisation,
// diagonal, Sec. 3.3 eq. matA), copies it into the job's region of a device
// arena on a copy stream, and then publishes the job's subset chunks into
// descriptor rings in device memory that the resident kernel's warps drain
// (the host stages new descriptors in pinned memory and copies them, then
// the new published count, on one stream, so a warp that sees the count
// sees the descriptors below it).  A job is planned for the kernel's CTA of
// six small-slice warps and one large-slice warp: chunks whose tiles fit a
// small slice go to ring 0, which every warp serves; the larger tiles go to
// ring 1, which the large-slice warp serves first.  Chunks of
// all admitted jobs are published round robin with a bounded queue depth,
// so a large-n job is split into chunks that interleave with small jobs
// that arrive while it runs.  The warp that finishes a job's last chunk
// reduces the job's chunk partials in chunk order and posts the result and
// a flag to host memory; the scheduler sees the flag, frees the job's slot
// and memory and wakes the caller waiting in haf_server_poll.  Because each
// job's chunking and reduction order depend only on the job, a result is
// the same whether the job ran alone or among others.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/hafnian_gb300.h"
#include "haf_internal.h"
#include "haf_nvtx.h"

using namespace hafgb;

namespace {

int sfail(int code, const std::string& msg) { return set_error(code, msg); }

#define SRV_CUDA(call)                                                                    \
  do {                                                                                    \
    cudaError_t _e = (call);                                                              \
    if (_e != cudaSuccess) return sfail(HAF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
  } while (0)

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

enum JobStateKind { kPending = 0, kUploading = 1, kReady = 2, kDone = 3 };

struct JobRec {
  uint64_t ticket = 0;
  int loops = 0;
  int n = 0;                 // after padding (even, >= 2), or 0 for trivial jobs
  std::vector<double> A;     // host copy, complex interleaved
  double submit_t = 0, done_t = 0;
  int state = kPending;
  int slot = -1;
  unsigned int gen = 0;
  size_t off = 0, bytes = 0;  // arena region
  std::vector<Chunk> chunks[2];  // per ring (0: small tiles, 1: large), publication order
  size_t next_pub[2] = {0, 0};
  double pub_units = 0;      // work published so far (both rings), for the publication order
  int64_t subsets = 0;
  bool all_published() const { return next_pub[0] >= chunks[0].size() && next_pub[1] >= chunks[1].size(); }
  cudaEvent_t uploaded = nullptr;
  double result[5] = {0, 0, 0, 0, 0};
};

// First-fit allocator over the device arena (256-byte granules).
struct Arena {
  std::map<size_t, size_t> free_;  // offset -> size
  size_t total = 0;
  void init(size_t bytes) {
    total = bytes;
    free_.clear();
    free_[0] = bytes;
  }
  bool alloc(size_t bytes, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t roff = it->first + bytes;
        free_.erase(it);
        if (rest) free_[roff] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

}  // namespace

struct haf_server {
  haf_server_cfg cfg{};
  int dev = 0, sms = 0;
  cudaStream_t comp = nullptr, copy = nullptr;
  char* arena = nullptr;
  char* stage = nullptr;  // pinned mirror of the arena layout (upload staging)
  Arena alloc;
  SrvJob* jobs_dev = nullptr;
  SrvJob* jobs_stage = nullptr;  // pinned
  unsigned int* zeros = nullptr;  // pinned, 256 zero bytes
  double* nan_src = nullptr;      // pinned NaNs (diagnostic fill of partial slots)
  size_t nan_len = 0;
  unsigned long long* head_dev = nullptr;  // claims per ring, last claim time, diagnostics (kSrvHead*)
  unsigned int* stop_dev = nullptr;
  double* tables = nullptr;
  // publication: descriptors and the published counts reach the device by
  // copies.  Ring 0 holds chunks whose tiles fit the small warp slices, ring 1
  // the larger ones (served by the one large-slice warp of each CTA).
  struct Ring {
    Chunk* dev = nullptr;
    Chunk* stage = nullptr;  // pinned, same indexing as dev
    uint64_t cap = 0;
    uint64_t published = 0;
    uint64_t claimed = 0;    // a lower bound, from the read-back
    std::vector<double> cum; // cum[i % cap] = work of entries 0..i (N^3 units)
    double pub_units = 0;    // work of all published entries
    double queued_units() const {  // published, not (known to be) claimed
      const uint64_t c = std::min(claimed, published);
      return pub_units - (c ? cum[(c - 1) % cap] : 0.0);
    }
  } ring[2];
  unsigned long long* tail_dev = nullptr;  // ring r's count at tail_dev[16 r]
  unsigned long long* tail_src = nullptr;  // pinned rotating sources of the count copies
  unsigned int tail_k = 0;
  unsigned int* flag_src = nullptr;        // pinned: {0, 1} for the stop-flag copies
  unsigned long long* claimed_h = nullptr; // pinned: read-back of head_dev[0..kSrvHeadClaim1]
  cudaEvent_t claimed_ev = nullptr;
  bool claimed_pending = false;
  cudaStream_t pub = nullptr, status = nullptr;
  // mapped host memory written by the kernel
  unsigned long long* stats_h = nullptr;
  unsigned long long* stats_d = nullptr;
  double* results_h = nullptr;
  unsigned int* flags_h = nullptr;
  unsigned int* flags_d = nullptr;
  double* results_d = nullptr;
  // scheduler
  std::thread thr;
  std::mutex mu;
  std::condition_variable wake, done_cv;
  std::deque<uint64_t> pending;
  std::map<uint64_t, std::unique_ptr<JobRec>> jobs;
  std::vector<int> free_slots;
  std::vector<unsigned int> slot_gen;
  std::vector<JobRec*> pub_order;  // scheduler scratch: ready jobs in publication order
  uint64_t next_ticket = 1;
  cudaEvent_t kernel_done = nullptr;
  bool kernel_launched = false;
  bool quit = false;
  int fatal = 0;
  std::string fatal_msg;
  int64_t launches = 0;
};

namespace {

// Host preparation of one admitted job into the staging mirror:
// At[i][j] = A[i^1][j] from the upper triangle (0 where j == i^1), diag(A).
void prep_host(const JobRec& j, char* dst_at, char* dst_diag) {
  const int n = j.n;
  double* At = reinterpret_cast<double*>(dst_at);
  double* dg = reinterpret_cast<double*>(dst_diag);
  for (int i = 0; i < n; ++i) {
    const int ii = i ^ 1;
    for (int c = 0; c < n; ++c) {
      double re = 0.0, im = 0.0;
      if (ii != c) {
        const int r0 = std::min(ii, c), c0 = std::max(ii, c);
        re = j.A[2 * ((size_t)r0 * n + c0)];
        im = j.A[2 * ((size_t)r0 * n + c0) + 1];
      }
      At[2 * ((size_t)i * n + c)] = re;
      At[2 * ((size_t)i * n + c) + 1] = im;
    }
    dg[2 * i] = j.A[2 * ((size_t)i * n + i)];
    dg[2 * i + 1] = j.A[2 * ((size_t)i * n + i) + 1];
  }
}

// Server jobs are cut into chunks of about cfg.chunk_us of one warp's time
// (a warp retires roughly 75 N^3 units per microsecond at the FP64 rate), so
// a newly admitted small job waits at most about one chunk for a warp.  Up
// to kSrvMaxChunks chunks per job: at n = 52 that keeps a chunk near 60 ms
// of a warp (40-byte partial per chunk, 10 MB for such a job).
constexpr double kSrvUnitsPerUs = 75.0;
constexpr double kSrvMaxChunks = 262144.0;
JobSpec server_spec(const haf_server* s, int n, int loops) {
  JobSpec js{n, loops, 0};
  js.max_chunk_units = kSrvUnitsPerUs * (double)s->cfg.chunk_us;
  js.max_chunks = kSrvMaxChunks;
  return js;
}

// Work of a chunk in N^3 units (the planner's measure).
double chunk_units(const Chunk& c) {
  const double N = 2.0 * c.m;
  return (double)c.count * N * N * N;
}

// Server plans: 8 warps per CTA for the tiles that fit the small slices,
// the rest at 4 (the large-slice warp), matching the server kernel's CTA.
PlanCfg server_cfg() {
  PlanCfg c;
  c.wpb = 8;
  c.chunks_per_warp = 8;
  return c;
}

size_t job_bytes(int n, size_t nchunks) {
  return al256((size_t)n * n * 16) + al256((size_t)n * 16) + al256(nchunks * 5 * sizeof(double)) + 256;
}

// Try to admit the oldest pending job (FIFO: a large job at the head is not
// overtaken, so it cannot starve).  Called with the lock held.
bool admit_one(haf_server* s) {
  if (s->pending.empty() || s->free_slots.empty()) return false;
  JobRec& j = *s->jobs[s->pending.front()];
  Plan p;
  if (build_plan({server_spec(s, j.n, j.loops)}, s->sms, server_cfg(), &p) != HAF_OK) {
    s->fatal = HAF_EINVAL;
    s->fatal_msg = "server: planning failed";
    return false;
  }
  const size_t bytes = job_bytes(j.n, p.chunks.size());
  size_t off;
  if (!s->alloc.alloc(bytes, &off)) return false;  // wait for memory to free up
  s->pending.pop_front();
  j.slot = s->free_slots.back();
  s->free_slots.pop_back();
  j.gen = ++s->slot_gen[j.slot];
  j.off = off;
  j.bytes = bytes;
  j.subsets = p.subsets;
  for (int r = 0; r < 2; ++r) {
    j.chunks[r].clear();
    j.next_pub[r] = 0;
  }
  j.pub_units = 0;
  for (const PlanSeg& sg : p.segs) {
    const int r = sg.wpb == 8 ? 0 : 1;  // 8-warp slices: small ring; 4-warp slices: large ring
    for (int q = sg.begin; q < sg.end; ++q) {
      Chunk c = p.chunks[p.order[q]];
      c.job = (uint16_t)j.slot;
      c.tag = (uint16_t)(j.gen & 0xffffu);
      c.aux = (uint32_t)p.order[q];  // partial slot = index in the job's plan
      j.chunks[r].push_back(c);
    }
  }
  char* st = s->stage + off;
  const size_t at_b = al256((size_t)j.n * j.n * 16), dg_b = al256((size_t)j.n * 16);
  prep_host(j, st, st + at_b);
  std::vector<double>().swap(j.A);  // the staged copy is all that is needed now
  const size_t part_b = al256(p.chunks.size() * 5 * sizeof(double));
  char* dbase = s->arena + off;
  SrvJob& sj = s->jobs_stage[j.slot];
  sj.job = Job{reinterpret_cast<double*>(dbase), reinterpret_cast<double*>(dbase + at_b), j.n, j.loops};
  sj.partials = reinterpret_cast<double*>(dbase + at_b + dg_b);
  sj.done = reinterpret_cast<unsigned int*>(dbase + at_b + dg_b + part_b);
  sj.result = s->results_d + 5 * j.slot;
  sj.flag = s->flags_d + j.slot;
  sj.nchunks = (unsigned int)p.chunks.size();
  sj.gen = j.gen;
  cudaError_t e = cudaMemcpyAsync(dbase, st, (size_t)j.n * j.n * 16, cudaMemcpyHostToDevice, s->copy);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dbase + at_b, st + at_b, (size_t)j.n * 16, cudaMemcpyHostToDevice, s->copy);
  // a DMA copy, not cudaMemsetAsync: a memset is a kernel and could not
  // start while the resident kernel holds every SM
  if (e == cudaSuccess) e = cudaMemcpyAsync(sj.done, s->zeros, sizeof(unsigned int), cudaMemcpyHostToDevice, s->copy);
  if (e == cudaSuccess && s->nan_src && p.chunks.size() * 5 <= s->nan_len)
    e = cudaMemcpyAsync(sj.partials, s->nan_src, p.chunks.size() * 5 * sizeof(double), cudaMemcpyHostToDevice, s->copy);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->jobs_dev + j.slot, &sj, sizeof(SrvJob), cudaMemcpyHostToDevice, s->copy);
  if (e == cudaSuccess && !j.uploaded) e = cudaEventCreateWithFlags(&j.uploaded, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(j.uploaded, s->copy);
  if (e != cudaSuccess) {
    s->fatal = HAF_ECUDA;
    s->fatal_msg = std::string("server upload: ") + cudaGetErrorString(e);
    return false;
  }
  j.state = kUploading;
  return true;
}

void scheduler(haf_server* s) {
  cudaSetDevice(s->dev);
  // warps that take chunks from each ring: every warp serves ring 0, the
  // large-slice warp of each CTA ring 1
  const uint64_t ring_warps[2] = {(uint64_t)s->sms * kSrvWarps, (uint64_t)s->sms};
  const char* env = std::getenv("HAF_SERVER_LOG");
  const bool log = env && env[0] == '1';
  double last_log = now_s();
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->quit) {
    if (log && now_s() - last_log > 1.0) {
      // diagnostic: one line per second with the scheduler's state
      int st[4] = {0, 0, 0, 0};
      for (auto& kv : s->jobs) st[kv.second->state]++;
      const bool up = s->kernel_launched && cudaEventQuery(s->kernel_done) == cudaErrorNotReady;
      std::fprintf(stderr,
                   "[haf_server] pending=%zu uploading=%d ready=%d done=%d published=%llu/%llu claimed>=%llu/%llu "
                   "kernel=%d launches=%lld free_slots=%zu chunks_done=%llu chunk_ns=%llu idle_polls=%llu "
                   "stale=%llu over=%llu unwritten=%llu\n",
                   s->pending.size(), st[kUploading], st[kReady], st[kDone],
                   (unsigned long long)s->ring[0].published, (unsigned long long)s->ring[1].published,
                   (unsigned long long)s->ring[0].claimed, (unsigned long long)s->ring[1].claimed, up ? 1 : 0,
                   (long long)s->launches, s->free_slots.size(),
                   (unsigned long long)__atomic_load_n(s->stats_h, __ATOMIC_RELAXED),
                   (unsigned long long)__atomic_load_n(s->stats_h + 1, __ATOMIC_RELAXED),
                   (unsigned long long)__atomic_load_n(s->stats_h + 2, __ATOMIC_RELAXED),
                   (unsigned long long)__atomic_load_n(s->stats_h + 3, __ATOMIC_RELAXED),
                   (unsigned long long)__atomic_load_n(s->stats_h + 4, __ATOMIC_RELAXED),
                   (unsigned long long)__atomic_load_n(s->stats_h + 5, __ATOMIC_RELAXED));
      last_log = now_s();
    }
    bool active = false;
    // 1. completions
    for (auto& kv : s->jobs) {
      JobRec& j = *kv.second;
      if (j.state != kReady || !j.all_published()) continue;
      if (__atomic_load_n(&s->flags_h[j.slot], __ATOMIC_ACQUIRE) == j.gen) {
        volatile double* r = s->results_h + 5 * j.slot;
        for (int k = 0; k < 5; ++k) j.result[k] = r[k];
        j.done_t = now_s();
        j.state = kDone;
        s->alloc.release(j.off, j.bytes);
        s->free_slots.push_back(j.slot);
        j.slot = -1;
        s->done_cv.notify_all();
      }
    }
    // 2. admission (FIFO)
    while (admit_one(s)) {
    }
    // 3. uploads that have landed
    for (auto& kv : s->jobs) {
      JobRec& j = *kv.second;
      if (j.state == kUploading && cudaEventQuery(j.uploaded) == cudaSuccess) j.state = kReady;
    }
    // 4. publish, least published work first, with bounded depth and ring
    //    space.  The count of claimed chunks comes from a copy of the device
    //    counter (a lower bound, refreshed every pass).  A ring slot may be
    //    rewritten once its entry has been claimed and read: a warp reads the
    //    entry it claimed before it claims another, so at most one
    //    claimed-but-unread entry per warp exists, which the margin covers.
    //    Order: the jobs with the least work published so far go first, a
    //    burst of chunks each in turn, so a new job's chunks enter the ring
    //    ahead of the rest of a long job's.  Depth: at most one queued
    //    (published, unclaimed) chunk per warp that serves the ring, and at
    //    most about two target-sized chunks of work per such warp, so a new
    //    entry waits behind little work even when a long job's chunks are
    //    large.
    if (s->claimed_pending && cudaEventQuery(s->claimed_ev) == cudaSuccess) {
      s->ring[0].claimed = std::max<uint64_t>(s->ring[0].claimed, s->claimed_h[kSrvHeadClaim0]);
      s->ring[1].claimed = std::max<uint64_t>(s->ring[1].claimed, s->claimed_h[kSrvHeadClaim1]);
      s->claimed_pending = false;
    }
    if (!s->claimed_pending) {
      if (cudaMemcpyAsync(s->claimed_h, s->head_dev, (kSrvHeadClaim1 + 1) * sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, s->status) == cudaSuccess &&
          cudaEventRecord(s->claimed_ev, s->status) == cudaSuccess)
        s->claimed_pending = true;
    }
    std::vector<JobRec*>& order = s->pub_order;  // reused: no allocation per pass
    order.clear();
    for (auto& kv : s->jobs)
      if (kv.second->state == kReady && !kv.second->all_published()) order.push_back(kv.second.get());
    std::stable_sort(order.begin(), order.end(),
                     [](const JobRec* a, const JobRec* b) { return a->pub_units < b->pub_units; });
    for (int r = 0; r < 2; ++r) {
      haf_server::Ring& R = s->ring[r];
      const uint64_t claimed = std::min<uint64_t>(R.claimed, R.published);
      const uint64_t margin = 4ull * ring_warps[r];
      const uint64_t lim = (claimed > margin ? claimed - margin : 0) + R.cap;
      const double work_cap = 2.0 * kSrvUnitsPerUs * (double)s->cfg.chunk_us * (double)ring_warps[r];
      double queued = R.queued_units();
      bool progress = true;
      const uint64_t before = R.published;
      while (progress) {
        progress = false;
        for (JobRec* jp : order) {
          JobRec& j = *jp;
          if (j.next_pub[r] >= j.chunks[r].size()) continue;
          if (R.published - claimed >= ring_warps[r] || R.published >= lim || queued >= work_cap) break;
          const size_t burst = 4;
          for (size_t q = 0; q < burst && j.next_pub[r] < j.chunks[r].size() && R.published < lim; ++q) {
            const Chunk& c = j.chunks[r][j.next_pub[r]++];
            const double u = chunk_units(c);
            R.stage[R.published % R.cap] = c;
            R.pub_units += u;
            R.cum[R.published % R.cap] = R.pub_units;
            ++R.published;
            queued += u;
            j.pub_units += u;
            progress = true;
          }
        }
      }
      if (R.published != before) {
        // copy the new entries (one or two contiguous pieces), then the count
        cudaError_t e = cudaSuccess;
        uint64_t p0 = before;
        while (e == cudaSuccess && p0 < R.published) {
          const uint64_t i0 = p0 % R.cap;
          const uint64_t len = std::min<uint64_t>(R.published - p0, R.cap - i0);
          e = cudaMemcpyAsync(R.dev + i0, R.stage + i0, len * sizeof(Chunk), cudaMemcpyHostToDevice, s->pub);
          p0 += len;
        }
        unsigned long long* src = s->tail_src + (s->tail_k++ & 4095u);
        *src = R.published;
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(s->tail_dev + 16 * r, src, sizeof(unsigned long long), cudaMemcpyHostToDevice, s->pub);
        if (e != cudaSuccess) {
          s->fatal = HAF_ECUDA;
          s->fatal_msg = std::string("server publish: ") + cudaGetErrorString(e);
        }
      }
    }
    // 5. keep the resident kernel running while any admitted job is unfinished
    for (auto& kv : s->jobs)
      if (kv.second->state == kReady || kv.second->state == kUploading) active = true;
    if (active && s->ring[0].published + s->ring[1].published > 0) {
      bool running = s->kernel_launched && cudaEventQuery(s->kernel_done) == cudaErrorNotReady;
      if (!running) {
        // the previous instance has ended (its warps raised the stop flag
        // together when idle): clear the flag, in stream order, for the new one
        ServerArgs a;
        for (int r = 0; r < 2; ++r) {
          a.ring[r] = s->ring[r].dev;
          a.cap[r] = s->ring[r].cap;
          a.tail[r] = s->tail_dev + 16 * r;
        }
        a.head = s->head_dev;
        a.stop = s->stop_dev;
        a.stats = s->stats_d;
        a.jobs = s->jobs_dev;
        a.tables = s->tables;
        a.idle_ns = (long long)s->cfg.idle_us * 1000LL;
        cudaError_t e = cudaMemcpyAsync(s->stop_dev, s->flag_src, sizeof(unsigned int), cudaMemcpyHostToDevice,
                                        s->comp);
        if (e == cudaSuccess) e = launch_server(a, s->sms, s->comp);
        if (e == cudaSuccess) e = cudaEventRecord(s->kernel_done, s->comp);
        if (e != cudaSuccess) {
          s->fatal = HAF_ECUDA;
          s->fatal_msg = std::string("server kernel: ") + cudaGetErrorString(e);
        } else {
          s->kernel_launched = true;
          ++s->launches;
        }
      }
    }
    if (s->fatal) {
      s->done_cv.notify_all();
      s->wake.wait_for(lk, std::chrono::milliseconds(10));
      continue;
    }
    s->wake.wait_for(lk, active ? std::chrono::microseconds(50) : std::chrono::milliseconds(5));
  }
}

}  // namespace

extern "C" {

int haf_server_create(const haf_server_cfg* cfg, haf_server** out) {
  if (!out) return sfail(HAF_EINVAL, "haf_server_create: null pointer");
  std::unique_ptr<haf_server> s(new haf_server());
  if (cfg) s->cfg = *cfg;
  if (s->cfg.max_jobs <= 0) s->cfg.max_jobs = 256;
  if (s->cfg.max_jobs > 65535) return sfail(HAF_EINVAL, "haf_server_create: max_jobs > 65535");
  if (s->cfg.max_bytes <= 0) s->cfg.max_bytes = (int64_t)256 << 20;
  if (s->cfg.ring_entries <= 0) s->cfg.ring_entries = (int64_t)1 << 20;
  if (s->cfg.ring_entries < (int64_t)1 << 16) return sfail(HAF_EINVAL, "haf_server_create: ring_entries < 65536");
  if (s->cfg.idle_us <= 0) s->cfg.idle_us = 20000;
  if (s->cfg.chunk_us <= 0) s->cfg.chunk_us = 4000;
  SRV_CUDA(cudaGetDevice(&s->dev));
  SRV_CUDA(cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->dev));
  SRV_CUDA(configure_kernels());
  SRV_CUDA(cudaStreamCreateWithFlags(&s->comp, cudaStreamNonBlocking));
  SRV_CUDA(cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking));
  SRV_CUDA(cudaEventCreateWithFlags(&s->kernel_done, cudaEventDisableTiming));
  const size_t ab = al256((size_t)s->cfg.max_bytes);
  if (cudaMalloc(&s->arena, ab) != cudaSuccess) return sfail(HAF_ENOMEM, "haf_server_create: device arena");
  SRV_CUDA(cudaMallocHost(&s->stage, ab));
  s->alloc.init(ab);
  const int mj = (int)s->cfg.max_jobs;
  SRV_CUDA(cudaMalloc(&s->jobs_dev, sizeof(SrvJob) * mj));
  SRV_CUDA(cudaMallocHost(&s->jobs_stage, sizeof(SrvJob) * mj));
  SRV_CUDA(cudaMallocHost(&s->zeros, 256));
  if (std::getenv("HAF_SERVER_LOG") && std::getenv("HAF_SERVER_LOG")[0] == '1') {
    s->nan_len = (size_t)5 * 65536;
    SRV_CUDA(cudaMallocHost(&s->nan_src, s->nan_len * sizeof(double)));
    for (size_t k = 0; k < s->nan_len; ++k) s->nan_src[k] = std::nan("");
  }
  std::memset(s->zeros, 0, 256);
  SRV_CUDA(cudaMalloc(&s->head_dev, 256));
  SRV_CUDA(cudaMemset(s->head_dev, 0, 256));
  std::vector<double> tab(256, 0.0);
  for (int k = 0; k < 128; ++k) tab[k] = 0.5 * k;
  for (int k = 1; k < 128; ++k) tab[128 + k] = 1.0 / k;
  SRV_CUDA(cudaMalloc(&s->tables, 256 * sizeof(double)));
  SRV_CUDA(cudaMemcpy(s->tables, tab.data(), 256 * sizeof(double), cudaMemcpyHostToDevice));
  for (int r = 0; r < 2; ++r) {
    s->ring[r].cap = (uint64_t)s->cfg.ring_entries;
    s->ring[r].cum.assign(s->ring[r].cap, 0.0);
  }
  SRV_CUDA(cudaStreamCreateWithFlags(&s->pub, cudaStreamNonBlocking));
  SRV_CUDA(cudaStreamCreateWithFlags(&s->status, cudaStreamNonBlocking));
  SRV_CUDA(cudaEventCreateWithFlags(&s->claimed_ev, cudaEventDisableTiming));
  for (int r = 0; r < 2; ++r) {
    SRV_CUDA(cudaMalloc(&s->ring[r].dev, sizeof(Chunk) * s->ring[r].cap));
    SRV_CUDA(cudaMallocHost(&s->ring[r].stage, sizeof(Chunk) * s->ring[r].cap));
  }
  SRV_CUDA(cudaMalloc(&s->tail_dev, 256));
  SRV_CUDA(cudaMemset(s->tail_dev, 0, 256));
  SRV_CUDA(cudaMalloc(&s->stop_dev, 256));
  SRV_CUDA(cudaMemset(s->stop_dev, 0, 256));
  SRV_CUDA(cudaMallocHost(&s->tail_src, 4096 * sizeof(unsigned long long)));
  SRV_CUDA(cudaMallocHost(&s->flag_src, 2 * sizeof(unsigned int)));
  s->flag_src[0] = 0u;
  s->flag_src[1] = 1u;
  SRV_CUDA(cudaMallocHost(&s->claimed_h, (kSrvHeadClaim1 + 1) * sizeof(unsigned long long)));
  std::memset(s->claimed_h, 0, (kSrvHeadClaim1 + 1) * sizeof(unsigned long long));
  SRV_CUDA(cudaHostAlloc(&s->stats_h, 256, cudaHostAllocMapped));
  std::memset(s->stats_h, 0, 256);
  SRV_CUDA(cudaHostAlloc(&s->results_h, sizeof(double) * 5 * mj, cudaHostAllocMapped));
  SRV_CUDA(cudaHostAlloc(&s->flags_h, sizeof(unsigned int) * mj, cudaHostAllocMapped));
  std::memset(s->flags_h, 0, sizeof(unsigned int) * mj);
  SRV_CUDA(cudaHostGetDevicePointer((void**)&s->stats_d, s->stats_h, 0));
  SRV_CUDA(cudaHostGetDevicePointer((void**)&s->results_d, s->results_h, 0));
  SRV_CUDA(cudaHostGetDevicePointer((void**)&s->flags_d, s->flags_h, 0));
  SRV_CUDA(cudaDeviceSynchronize());
  for (int k = mj - 1; k >= 0; --k) s->free_slots.push_back(k);
  s->slot_gen.assign(mj, 0u);
  haf_server* raw = s.release();
  raw->thr = std::thread(scheduler, raw);
  *out = raw;
  return HAF_OK;
}

int haf_server_submit(haf_server* s, int kind, const double* A, int64_t n, uint64_t* ticket) {
  const NvtxRange nvtx_range("haf_server_submit");
  if (!s || !ticket || (kind != 0 && kind != 1)) return sfail(HAF_EINVAL, "haf_server_submit: bad arguments");
  if (n < 0 || n > kMaxN || (n > 0 && !A)) return sfail(HAF_EINVAL, "haf_server_submit: n out of range or null A");
  std::unique_ptr<JobRec> j(new JobRec());
  j->loops = kind;
  j->submit_t = now_s();
  const int ni = (int)n;
  if (ni == 0 || ((ni & 1) && !kind)) {
    j->result[0] = ni == 0 ? 1.0 : 0.0;
    j->result[4] = std::fabs(j->result[0]);
    j->state = kDone;
    j->done_t = j->submit_t;
  } else {
    const int np = ni + (ni & 1);
    if (np > kMaxN) return sfail(HAF_EINVAL, "haf_server_submit: n out of range");
    j->n = np;
    j->A.assign((size_t)np * np * 2, 0.0);
    for (int i = 0; i < ni; ++i) std::memcpy(&j->A[(size_t)i * np * 2], A + (size_t)i * ni * 2, (size_t)ni * 16);
    if (np != ni) j->A[((size_t)ni * np + ni) * 2] = 1.0;
    // a job larger than the whole arena could never be admitted
    Plan p;
    if (build_plan({server_spec(s, np, kind)}, s->sms, server_cfg(), &p) != HAF_OK)
      return sfail(HAF_EINVAL, "haf_server_submit: cannot plan this size");
    if (job_bytes(np, p.chunks.size()) > s->alloc.total)
      return sfail(HAF_ENOMEM, "haf_server_submit: job exceeds the server's device memory");
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->fatal) return sfail(s->fatal, s->fatal_msg);
  if ((int64_t)s->pending.size() >= std::max<int64_t>(s->cfg.max_jobs * 64, 4096))
    return sfail(HAF_EBUSY, "haf_server_submit: queue full");
  j->ticket = s->next_ticket++;
  *ticket = j->ticket;
  const bool trivial = j->state == kDone;
  s->jobs[j->ticket] = std::move(j);
  if (!trivial) s->pending.push_back(*ticket);
  s->wake.notify_all();
  return HAF_OK;
}

int haf_server_poll(haf_server* s, uint64_t ticket, double* out, haf_info* info, int64_t timeout_us) {
  const NvtxRange nvtx_range("haf_server_poll");
  if (!s || !out) return sfail(HAF_EINVAL, "haf_server_poll: bad arguments");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return sfail(HAF_ENOTFOUND, "haf_server_poll: unknown ticket");
  auto ready = [&] { return it->second->state == kDone || s->fatal != 0; };
  if (timeout_us < 0)
    s->done_cv.wait(lk, ready);
  else if (!s->done_cv.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
    return sfail(HAF_ETIMEDOUT, "haf_server_poll: not finished");
  if (it->second->state != kDone) return sfail(s->fatal, s->fatal_msg);
  const JobRec& j = *it->second;
  out[0] = j.result[0] + j.result[2];
  out[1] = j.result[1] + j.result[3];
  if (info) {
    info->abs_sum = j.result[4];
    info->value_lo[0] = j.result[2];
    info->value_lo[1] = j.result[3];
    info->subsets = j.subsets;
    info->seconds = j.done_t - j.submit_t;
    info->launches = s->launches;
    {
      const double v = std::hypot(out[0], out[1]);
      const double a = j.result[4];
      info->rel_err_bound = a == 0.0 ? 0.0 : (v == 0.0 ? HUGE_VAL : HAF_FP64_REL_TOL * a / v);
    }
    info->precision_mode = 0;
    info->reserved = 0;
  }
  if (j.uploaded) cudaEventDestroy(j.uploaded);
  s->jobs.erase(it);
  return HAF_OK;
}

int haf_server_destroy(haf_server* s) {
  if (!s) return HAF_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->quit = true;
    s->wake.notify_all();
  }
  if (s->thr.joinable()) s->thr.join();
  cudaMemcpyAsync(s->stop_dev, s->flag_src + 1, sizeof(unsigned int), cudaMemcpyHostToDevice, s->pub);
  cudaStreamSynchronize(s->pub);
  cudaStreamSynchronize(s->comp);
  cudaStreamSynchronize(s->copy);
  cudaStreamSynchronize(s->status);
  for (auto& kv : s->jobs)
    if (kv.second->uploaded) cudaEventDestroy(kv.second->uploaded);
  cudaEventDestroy(s->kernel_done);
  cudaEventDestroy(s->claimed_ev);
  cudaFree(s->arena);
  cudaFreeHost(s->stage);
  cudaFree(s->jobs_dev);
  cudaFreeHost(s->jobs_stage);
  cudaFreeHost(s->zeros);
  if (s->nan_src) cudaFreeHost(s->nan_src);
  cudaFree(s->head_dev);
  cudaFree(s->stop_dev);
  cudaFree(s->tables);
  for (int r = 0; r < 2; ++r) {
    cudaFree(s->ring[r].dev);
    cudaFreeHost(s->ring[r].stage);
  }
  cudaFree(s->tail_dev);
  cudaFreeHost(s->tail_src);
  cudaFreeHost(s->flag_src);
  cudaFreeHost(s->claimed_h);
  cudaFreeHost(s->stats_h);
  cudaFreeHost(s->results_h);
  cudaFreeHost(s->flags_h);
  cudaStreamDestroy(s->pub);
  cudaStreamDestroy(s->status);
  cudaStreamDestroy(s->comp);
  cudaStreamDestroy(s->copy);
  delete s;
  return HAF_OK;
}

}  // extern "C"
