// haf_server.cu -- continuous-batching hafnian server: the host scheduler
// around server_kernel (haf_kernels.cu).
//
// Requests (haf or lhaf of one matrix) are queued on submit.  A scheduler
// thread admits them while job slots and device memory allow, prepares each
// admitted matrix on the host (pair swap X A, upper-triangle symmetrisation,
// diagonal, Sec. 3.3 eq. matA), copies it into the job's region of a device
// arena on a copy stream, and then publishes the job's subset chunks into a
// ring in host memory that the resident kernel's warps drain.  Chunks of
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
  std::vector<Chunk> chunks;  // publication order
  size_t next_pub = 0;
  uint64_t first_pub = UINT64_MAX;
  int64_t subsets = 0;
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
  unsigned long long* head_dev = nullptr;
  double* tables = nullptr;
  // mapped host memory
  Chunk* ring_h = nullptr;
  Chunk* ring_d = nullptr;
  unsigned long long cap = 0;
  unsigned long long* tail_h = nullptr;
  unsigned long long* mirror_h = nullptr;
  unsigned int* stop_h = nullptr;
  double* results_h = nullptr;
  unsigned int* flags_h = nullptr;
  unsigned long long *tail_d = nullptr, *mirror_d = nullptr;
  unsigned int *stop_d = nullptr, *flags_d = nullptr;
  double* results_d = nullptr;
  // scheduler
  std::thread thr;
  std::mutex mu;
  std::condition_variable wake, done_cv;
  std::deque<uint64_t> pending;
  std::map<uint64_t, std::unique_ptr<JobRec>> jobs;
  std::vector<int> free_slots;
  std::vector<unsigned int> slot_gen;
  uint64_t next_ticket = 1;
  uint64_t published = 0;
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

size_t job_bytes(int n, size_t nchunks) {
  return al256((size_t)n * n * 16) + al256((size_t)n * 16) + al256(nchunks * 5 * sizeof(double)) + 256;
}

// Try to admit the oldest pending job (FIFO: a large job at the head is not
// overtaken, so it cannot starve).  Called with the lock held.
bool admit_one(haf_server* s) {
  if (s->pending.empty() || s->free_slots.empty()) return false;
  JobRec& j = *s->jobs[s->pending.front()];
  Plan p;
  if (build_plan({JobSpec{j.n, j.loops, 0}}, s->sms * kWarpsPerBlock, &p) != HAF_OK) {
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
  j.chunks.resize(p.chunks.size());
  for (size_t q = 0; q < p.order.size(); ++q) {
    Chunk c = p.chunks[p.order[q]];
    c.job = (uint16_t)j.slot;
    c.aux = (uint32_t)p.order[q];  // partial slot = index in the job's plan
    j.chunks[q] = c;
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
  if (e == cudaSuccess) e = cudaMemsetAsync(sj.done, 0, sizeof(unsigned int), s->copy);
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
  const uint64_t depth_target = (uint64_t)s->sms * kWarpsPerBlock * 2;
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->quit) {
    bool active = false;
    // 1. completions
    for (auto& kv : s->jobs) {
      JobRec& j = *kv.second;
      if (j.state != kReady || j.next_pub < j.chunks.size()) continue;
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
    // 4. publish round robin, bounded depth and ring space
    uint64_t oldest = UINT64_MAX;
    for (auto& kv : s->jobs)
      if (kv.second->state == kReady) oldest = std::min(oldest, kv.second->first_pub);
    const uint64_t claimed = __atomic_load_n(s->mirror_h, __ATOMIC_RELAXED);
    bool progress = true;
    const uint64_t before = s->published;
    while (progress) {
      progress = false;
      for (auto& kv : s->jobs) {
        JobRec& j = *kv.second;
        if (j.state != kReady || j.next_pub >= j.chunks.size()) continue;
        if (s->published - std::min(claimed, s->published) >= depth_target) break;
        const uint64_t lim = (oldest == UINT64_MAX ? s->published : oldest) + s->cap;
        if (s->published >= lim) break;
        const size_t burst = 4;
        for (size_t q = 0; q < burst && j.next_pub < j.chunks.size() && s->published < lim; ++q) {
          if (j.first_pub == UINT64_MAX) {
            j.first_pub = s->published;
            oldest = std::min(oldest, j.first_pub);
          }
          s->ring_h[s->published % s->cap] = j.chunks[j.next_pub++];
          ++s->published;
          progress = true;
        }
      }
    }
    if (s->published != before) __atomic_store_n(s->tail_h, (unsigned long long)s->published, __ATOMIC_RELEASE);
    // 5. keep the resident kernel running while any admitted job is unfinished
    for (auto& kv : s->jobs)
      if (kv.second->state == kReady || kv.second->state == kUploading) active = true;
    if (active && s->published > 0) {
      bool running = s->kernel_launched && cudaEventQuery(s->kernel_done) == cudaErrorNotReady;
      if (!running) {
        ServerArgs a;
        a.ring = s->ring_d;
        a.cap = s->cap;
        a.tail = s->tail_d;
        a.head = s->head_dev;
        a.head_mirror = s->mirror_d;
        a.stop = s->stop_d;
        a.jobs = s->jobs_dev;
        a.tables = s->tables;
        a.idle_ns = (long long)s->cfg.idle_us * 1000LL;
        a.warp_bytes = kWarpBytes;
        cudaError_t e = launch_server(a, s->sms, s->comp);
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
  if (s->cfg.idle_us <= 0) s->cfg.idle_us = 20000;
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
  SRV_CUDA(cudaMalloc(&s->head_dev, 256));
  SRV_CUDA(cudaMemset(s->head_dev, 0, 256));
  std::vector<double> tab(256, 0.0);
  for (int k = 0; k < 128; ++k) tab[k] = 0.5 * k;
  for (int k = 1; k < 128; ++k) tab[128 + k] = 1.0 / k;
  SRV_CUDA(cudaMalloc(&s->tables, 256 * sizeof(double)));
  SRV_CUDA(cudaMemcpy(s->tables, tab.data(), 256 * sizeof(double), cudaMemcpyHostToDevice));
  s->cap = (unsigned long long)s->cfg.ring_entries;
  SRV_CUDA(cudaHostAlloc(&s->ring_h, sizeof(Chunk) * s->cap, cudaHostAllocMapped));
  SRV_CUDA(cudaHostAlloc(&s->tail_h, 256, cudaHostAllocMapped));
  SRV_CUDA(cudaHostAlloc(&s->mirror_h, 256, cudaHostAllocMapped));
  SRV_CUDA(cudaHostAlloc(&s->stop_h, 256, cudaHostAllocMapped));
  SRV_CUDA(cudaHostAlloc(&s->results_h, sizeof(double) * 5 * mj, cudaHostAllocMapped));
  SRV_CUDA(cudaHostAlloc(&s->flags_h, sizeof(unsigned int) * mj, cudaHostAllocMapped));
  *s->tail_h = 0;
  *s->mirror_h = 0;
  *s->stop_h = 0;
  std::memset(s->flags_h, 0, sizeof(unsigned int) * mj);
  SRV_CUDA(cudaHostGetDevicePointer((void**)&s->ring_d, s->ring_h, 0));
  SRV_CUDA(cudaHostGetDevicePointer((void**)&s->tail_d, s->tail_h, 0));
  SRV_CUDA(cudaHostGetDevicePointer((void**)&s->mirror_d, s->mirror_h, 0));
  SRV_CUDA(cudaHostGetDevicePointer((void**)&s->stop_d, s->stop_h, 0));
  SRV_CUDA(cudaHostGetDevicePointer((void**)&s->results_d, s->results_h, 0));
  SRV_CUDA(cudaHostGetDevicePointer((void**)&s->flags_d, s->flags_h, 0));
  for (int k = mj - 1; k >= 0; --k) s->free_slots.push_back(k);
  s->slot_gen.assign(mj, 0u);
  haf_server* raw = s.release();
  raw->thr = std::thread(scheduler, raw);
  *out = raw;
  return HAF_OK;
}

int haf_server_submit(haf_server* s, int kind, const double* A, int64_t n, uint64_t* ticket) {
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
    if (build_plan({JobSpec{np, kind, 0}}, s->sms * kWarpsPerBlock, &p) != HAF_OK)
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
  __atomic_store_n(s->stop_h, 1u, __ATOMIC_RELEASE);
  cudaStreamSynchronize(s->comp);
  cudaStreamSynchronize(s->copy);
  for (auto& kv : s->jobs)
    if (kv.second->uploaded) cudaEventDestroy(kv.second->uploaded);
  cudaEventDestroy(s->kernel_done);
  cudaFree(s->arena);
  cudaFreeHost(s->stage);
  cudaFree(s->jobs_dev);
  cudaFreeHost(s->jobs_stage);
  cudaFree(s->head_dev);
  cudaFree(s->tables);
  cudaFreeHost(s->ring_h);
  cudaFreeHost(s->tail_h);
  cudaFreeHost(s->mirror_h);
  cudaFreeHost(s->stop_h);
  cudaFreeHost(s->results_h);
  cudaFreeHost(s->flags_h);
  cudaStreamDestroy(s->comp);
  cudaStreamDestroy(s->copy);
  delete s;
  return HAF_OK;
}

}  // extern "C"
