// haf_capi.cu -- host side of the C ABI declared in include/hafnian_gb300.h:
// argument checks, the work plan (subset chunks per size |Z|), device
// buffers, launches and the read-back of results.
//
// Plan.  For a matrix of size n (h = n/2 pairs), subsets of size m = 1..h
// (the empty subset contributes 0 for h >= 1) are grouped into chunks of
// consecutive colex ranks.  A plan has a launch shape (warps per CTA, chunk
// granularity; tuned per size by haf_tune, else a default).  Each size gets
// a lane-group width G (1..32 lanes per subset, 32/G subsets per warp), the
// smallest that fits the warp's shared-memory slice; sizes whose tiles do
// not fit at the plan's warps per CTA run in a second launch with fewer.
// Within a launch chunks are ordered largest-work-first so the persistent
// warps finish together.  Each chunk writes one partial; partials are
// reduced in chunk order, independent of scheduling.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/hafnian_gb300.h"
#include "haf_internal.h"
#include "haf_nvtx.h"

using namespace hafgb;

namespace hafgb {
thread_local std::string g_last_error;
int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
}  // namespace hafgb

namespace {

int fail(int code, const std::string& msg) { return hafgb::set_error(code, msg); }

#define HAF_CUDA(call)                                                                    \
  do {                                                                                    \
    cudaError_t _e = (call);                                                              \
    if (_e != cudaSuccess)                                                                \
      return fail(HAF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e));         \
  } while (0)

}  // namespace

namespace hafgb {

uint64_t binom(int a, int b) {
  if (b < 0 || b > a) return 0;
  uint64_t r = 1;
  for (int i = 1; i <= b; ++i) r = r * (uint64_t)(a - b + i) / (uint64_t)i;
  return r;
}

// Colex unranking: the rank-th m-subset of {0..h-1} (combinatorial number system).
uint64_t unrank_colex(uint64_t rank, int m, int h) {
  uint64_t mask = 0;
  int c = h - 1;
  for (int i = m; i >= 1; --i) {
    while (binom(c, i) > rank) --c;
    mask |= 1ull << c;
    rank -= binom(c, i);
    --c;
  }
  return mask;
}

struct SizeCfg {
  int G;
  int ld;
};

// Smallest lane-group width whose S = 32/G subsets fit the warp slice
// (kernel kind `kind`, `warp_bytes` of shared memory per warp); at equal
// width an odd leading dimension (column walks on distinct banks) is
// preferred to ld = N.
bool choose_cfg(int N, int h, int kind, int loops, int warp_bytes, SizeCfg* out) {
  const int sb = bulk_elem_bytes(kind), ss = series_elem_bytes(kind);
  const bool mixed = kind_mixed(kind);
  for (int G = 1; G <= 32; G *= 2) {
    for (int ld : {N + 1, N}) {
      const int S = 32 / G;
      if ((long)S * subset_bytes(N, ld, h, sb, ss, mixed, loops != 0) <= warp_bytes) {
        out->G = G;
        out->ld = ld;
        return true;
      }
    }
  }
  return false;
}

// Colex rank range [lo, hi) of the m-subsets that part p of P covers: each
// size class is cut into P contiguous, nearly equal pieces, so the parts
// are balanced and depend on nothing but (h, m, p, P).
void part_range(uint64_t cnt, int64_t p, int64_t P, uint64_t* lo, uint64_t* hi) {
  const unsigned __int128 c = cnt;
  *lo = (uint64_t)(c * (unsigned __int128)p / (unsigned __int128)P);
  *hi = (uint64_t)(c * (unsigned __int128)(p + 1) / (unsigned __int128)P);
}

int build_plan(const std::vector<JobSpec>& jobs, int sms, const PlanCfg& pc, Plan* plan) {
  plan->chunks.clear();
  plan->order.clear();
  plan->segs.clear();
  plan->job_begin.assign(1, 0);
  plan->subsets = 0;
  if (pc.wpb != 4 && pc.wpb != 8 && pc.wpb != 16) return fail(HAF_EINVAL, "warps per CTA must be 4, 8 or 16");
  if (pc.chunks_per_warp < 1 || pc.chunks_per_warp > 64) return fail(HAF_EINVAL, "chunks per warp out of range");
  const int kind = jobs.empty() ? kKindC128 : kernel_kind(jobs[0].is_real, jobs[0].prec);
  for (const JobSpec& js : jobs)
    if (kernel_kind(js.is_real, js.prec) != kind) return fail(HAF_EINVAL, "jobs of one plan differ in type");
  plan->kind = kind;
  // Every size class (job, m) runs with the requested warps per CTA, or
  // fewer where its tile does not fit one warp's slice of shared memory;
  // each warps-per-CTA value present becomes one launch (segment).
  struct Cls {
    int job, m, wpb;
    SizeCfg cfg;
    uint64_t rlo, cnt;
  };
  std::vector<Cls> cls;
  double work[17] = {0};  // N^3 units per warps-per-CTA value
  for (size_t jb = 0; jb < jobs.size(); ++jb) {
    const JobSpec& js = jobs[jb];
    const int h = js.n / 2;
    for (int m = 1; m <= h; ++m) {
      Cls c;
      c.job = (int)jb;
      c.m = m;
      c.wpb = pc.wpb;
      while (!choose_cfg(2 * m, h, kind, js.loops, warp_bytes_for(c.wpb), &c.cfg)) {
        if (c.wpb == 4) return fail(HAF_EINVAL, "matrix too large for the shared-memory plan");
        c.wpb /= 2;
      }
      uint64_t rhi;
      part_range(binom(h, m), js.part, js.nparts, &c.rlo, &rhi);
      c.cnt = rhi - c.rlo;
      work[c.wpb] += (double)c.cnt * std::pow(2.0 * m, 3);
      cls.push_back(c);
    }
  }
  // Chunks in (job, m) order, so each job's chunk ids are contiguous (the
  // finalize sums them in id order); each segment sized for its own work.
  std::vector<double> cost;
  std::vector<int> seg_of;
  size_t ci = 0;
  for (size_t jb = 0; jb < jobs.size(); ++jb) {
    const JobSpec& js = jobs[jb];
    const int h = js.n / 2;
    double job_total = 0.0;
    for (int mm = 1; mm <= h; ++mm) job_total += (double)binom(h, mm) * std::pow(2.0 * mm, 3);
    for (; ci < cls.size() && cls[ci].job == (int)jb; ++ci) {
      const Cls& c = cls[ci];
      const int N = 2 * c.m, S = 32 / c.cfg.G;
      const double per = std::pow((double)N, 3);
      const double target = std::max(1.0, work[c.wpb] / ((double)sms * c.wpb * pc.chunks_per_warp));
      // a cap on chunk work, but never more than js.max_chunks chunks per job
      double tj = target;
      if (js.max_chunk_units > 0)
        tj = std::max(std::min(target, js.max_chunk_units), job_total / (double)js.nparts / js.max_chunks);
      uint64_t csz = (uint64_t)std::ceil(tj / per / S) * S;
      csz = std::max<uint64_t>(csz, (uint64_t)S);
      csz = std::min<uint64_t>(csz, (uint64_t)1 << 30);
      for (uint64_t r0 = 0; r0 < c.cnt; r0 += csz) {
        Chunk k;
        std::memset(&k, 0, sizeof(k));
        k.rank0 = c.rlo + r0;
        k.mask0 = unrank_colex(c.rlo + r0, c.m, h);
        k.count = (uint32_t)std::min<uint64_t>(csz, c.cnt - r0);
        k.job = (uint16_t)jb;
        k.m = (uint8_t)c.m;
        k.G = (uint8_t)c.cfg.G;
        k.ld = (uint8_t)c.cfg.ld;
        plan->chunks.push_back(k);
        cost.push_back((double)k.count * per * (js.loops ? 1.3 : 1.0) / (js.is_real ? 4.0 : 1.0));
        seg_of.push_back(c.wpb);
      }
      plan->subsets += (int64_t)c.cnt;
    }
    plan->job_begin.push_back((int)plan->chunks.size());
  }
  // segments, most warps per CTA first; inside each, largest chunks first
  for (int w : {16, 8, 4}) {
    PlanSeg sg;
    sg.begin = (int)plan->order.size();
    for (size_t i = 0; i < plan->chunks.size(); ++i)
      if (seg_of[i] == w) plan->order.push_back((int)i);
    sg.end = (int)plan->order.size();
    if (sg.end == sg.begin) continue;
    std::stable_sort(plan->order.begin() + sg.begin, plan->order.end(),
                     [&](int a, int b) { return cost[a] > cost[b]; });
    sg.wpb = w;
    sg.warp_bytes = warp_bytes_for(w);
    plan->segs.push_back(sg);
  }
  plan->wpb = plan->segs.empty() ? pc.wpb : plan->segs[0].wpb;
  plan->warp_bytes = warp_bytes_for(plan->wpb);
  return HAF_OK;
}

}  // namespace hafgb

namespace {

// Device-resident copy of a plan.
struct DevPlan {
  Chunk* chunks = nullptr;
  int* order = nullptr;
  int* job_begin = nullptr;
  int nchunks = 0;
  int njobs = 0;
  int64_t subsets = 0;
  int kind = kKindC128;
  int wpb = kWarpsPerBlock;  // first segment's
  int warp_bytes = kWarpBytes;
  std::vector<PlanSeg> segs;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Device {
  int id = -1;
  int sms = 0;
  bool configured = false;
  cudaStream_t stream = nullptr;
  double* tables = nullptr;
  // growable scratch for the host-pointer entry points
  void* work = nullptr;
  size_t work_bytes = 0;
  double* host_out = nullptr;  // pinned, grows
  size_t host_out_n = 0;
  // (n, loops, real, prec, part, nparts, warps per CTA, chunks per warp)
  std::map<std::tuple<int, int, int, int, int64_t, int64_t, int, int>, DevPlan> plans;
  std::map<std::tuple<int, int, int, int>, PlanCfg> tuned;  // (n, loops, real, prec) -> launch shape
};

std::mutex g_mu;
std::map<int, std::unique_ptr<Device>> g_devices;

int get_device(Device** out) {
  int id = 0;
  HAF_CUDA(cudaGetDevice(&id));
  auto it = g_devices.find(id);
  if (it != g_devices.end()) {
    *out = it->second.get();
    return HAF_OK;
  }
  std::unique_ptr<Device> d(new Device());
  d->id = id;
  HAF_CUDA(cudaDeviceGetAttribute(&d->sms, cudaDevAttrMultiProcessorCount, id));
  HAF_CUDA(configure_kernels());
  HAF_CUDA(cudaStreamCreateWithFlags(&d->stream, cudaStreamNonBlocking));
  std::vector<double> tab(256, 0.0);
  for (int k = 0; k < 128; ++k) tab[k] = 0.5 * k;
  for (int k = 1; k < 128; ++k) tab[128 + k] = 1.0 / k;
  HAF_CUDA(cudaMalloc(&d->tables, 256 * sizeof(double)));
  HAF_CUDA(cudaMemcpy(d->tables, tab.data(), 256 * sizeof(double), cudaMemcpyHostToDevice));
  *out = d.get();
  g_devices[id] = std::move(d);
  return HAF_OK;
}

int upload_plan(const Plan& p, cudaStream_t st, DevPlan* dp) {
  dp->nchunks = (int)p.chunks.size();
  dp->njobs = (int)p.job_begin.size() - 1;
  dp->subsets = p.subsets;
  dp->kind = p.kind;
  dp->wpb = p.wpb;
  dp->warp_bytes = p.warp_bytes;
  dp->segs = p.segs;
  HAF_CUDA(cudaMalloc(&dp->chunks, std::max<size_t>(1, p.chunks.size()) * sizeof(Chunk)));
  HAF_CUDA(cudaMalloc(&dp->order, std::max<size_t>(1, p.order.size()) * sizeof(int)));
  HAF_CUDA(cudaMalloc(&dp->job_begin, p.job_begin.size() * sizeof(int)));
  HAF_CUDA(cudaMemcpyAsync(dp->chunks, p.chunks.data(), p.chunks.size() * sizeof(Chunk),
                           cudaMemcpyHostToDevice, st));
  HAF_CUDA(cudaMemcpyAsync(dp->order, p.order.data(), p.order.size() * sizeof(int),
                           cudaMemcpyHostToDevice, st));
  HAF_CUDA(cudaMemcpyAsync(dp->job_begin, p.job_begin.data(), p.job_begin.size() * sizeof(int),
                           cudaMemcpyHostToDevice, st));
  HAF_CUDA(cudaStreamSynchronize(st));
  return HAF_OK;
}

// Launch shape for one matrix: the tuned one if haf_tune (or haf_tune_set)
// recorded one for this (n, kind), else the default: 4 warps per CTA for
// FP64 (one warp per SM sub-partition saturates the DFMA pipe), 8 for the
// FP32 mode (more warps hide shared-memory latency), 8 chunks per warp.
PlanCfg plan_cfg(Device* d, int n, int loops, int is_real, int prec) {
  auto it = d->tuned.find(std::make_tuple(n, loops, is_real, prec));
  if (it != d->tuned.end()) return it->second;
  PlanCfg c;
  c.wpb = (prec == kPrecF32) ? 8 : kWarpsPerBlock;
  return c;
}

int cached_plan(Device* d, int n, int loops, int is_real, int prec, DevPlan** out, int64_t part = 0,
                int64_t nparts = 1, const PlanCfg* force = nullptr) {
  const PlanCfg pc = force ? *force : plan_cfg(d, n, loops, is_real, prec);
  auto key = std::make_tuple(n, loops, is_real, prec, part, nparts, pc.wpb, pc.chunks_per_warp);
  auto it = d->plans.find(key);
  if (it != d->plans.end()) {
    *out = &it->second;
    return HAF_OK;
  }
  Plan p;
  JobSpec js{n, loops, is_real};
  js.part = part;
  js.nparts = nparts;
  js.prec = prec;
  int rc = build_plan({js}, d->sms, pc, &p);
  if (rc) return rc;
  DevPlan dp;
  rc = upload_plan(p, d->stream, &dp);
  if (rc) return rc;
  d->plans[key] = dp;
  *out = &d->plans[key];
  return HAF_OK;
}

// Workspace layout for one single-matrix launch.
struct WsLayout {
  size_t at, diag, partials, counter, total;
};
WsLayout ws_layout(int n, int nchunks) {
  WsLayout w;
  size_t off = 0;
  w.at = off;
  off += align256((size_t)n * n * 16);
  w.diag = off;
  off += align256((size_t)n * 16);
  w.partials = off;
  off += align256((size_t)std::max(1, nchunks) * 5 * sizeof(double));
  w.counter = off;
  off += 256;
  w.total = off;
  return w;
}

int ensure_work(Device* d, size_t bytes) {
  if (d->work_bytes >= bytes) return HAF_OK;
  if (d->work) cudaFree(d->work);
  d->work = nullptr;
  d->work_bytes = 0;
  cudaError_t e = cudaMalloc(&d->work, bytes);
  if (e != cudaSuccess) return fail(HAF_ENOMEM, std::string("cudaMalloc workspace: ") + cudaGetErrorString(e));
  d->work_bytes = bytes;
  return HAF_OK;
}

int ensure_host_out(Device* d, size_t ndoubles) {
  if (d->host_out_n >= ndoubles) return HAF_OK;
  if (d->host_out) cudaFreeHost(d->host_out);
  d->host_out = nullptr;
  d->host_out_n = 0;
  HAF_CUDA(cudaMallocHost(&d->host_out, ndoubles * sizeof(double)));
  d->host_out_n = ndoubles;
  return HAF_OK;
}

// Enqueue prep + subset kernel + finalize for a plan whose jobs' At/diag
// already sit in device memory.
int enqueue(Device* d, const DevPlan& dp, const std::vector<Job>& jobs_host, Job* jobs_dev,
            double* partials, int* counter, double* d_out, cudaStream_t st,
            const uint64_t* masks = nullptr, double* terms_out = nullptr) {
  HAF_CUDA(cudaMemcpyAsync(jobs_dev, jobs_host.data(), jobs_host.size() * sizeof(Job),
                           cudaMemcpyHostToDevice, st));
  HAF_CUDA(cudaMemsetAsync(counter, 0, sizeof(int) * std::max<size_t>(1, dp.segs.size()), st));
  // one launch per segment (counter si for segment si)
  for (size_t si = 0; si < dp.segs.size(); ++si) {
    const PlanSeg& sg = dp.segs[si];
    KernelArgs a;
    a.jobs = jobs_dev;
    a.chunks = dp.chunks;
    a.order = dp.order + sg.begin;
    a.nchunks = sg.end - sg.begin;
    a.counter = counter + si;
    a.partials = partials;
    a.tables = d->tables;
    a.masks = masks;
    a.terms_out = terms_out;
    a.warp_bytes = sg.warp_bytes;
    const int grid = std::max(1, std::min(d->sms, (a.nchunks + sg.wpb - 1) / sg.wpb));
    HAF_CUDA(launch_subsets(a, dp.kind, sg.wpb, grid, st));
  }
  if (!terms_out) HAF_CUDA(launch_finalize(partials, dp.job_begin, dp.njobs, d_out, st));
  return HAF_OK;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Estimated |error| / |value| of a whole-matrix result (the Accuracy
// paragraph of the header): the measured error per unit of abs_sum, scaled
// by abs_sum / |value|.
double rel_err_bound(double re, double im, double abs_sum, int prec) {
  const double tol = prec == kPrecF32 ? HAF_FP32_REL_TOL : HAF_FP64_REL_TOL;
  const double v = std::hypot(re, im);
  if (abs_sum == 0.0) return 0.0;
  if (v == 0.0) return HUGE_VAL;
  return tol * abs_sum / v;
}

// The FP32-bulk gate: HAF_EACCURACY when the estimated relative error of an
// FP32-bulk result exceeds HAF_FP32_MAX_REL_ERR.
int accuracy_gate(double rel, int prec, const char* where) {
  if (prec != kPrecF32 || rel <= HAF_FP32_MAX_REL_ERR) return HAF_OK;
  char msg[200];
  std::snprintf(msg, sizeof(msg),
                "%s: FP32-bulk result's estimated relative error %.3g exceeds HAF_FP32_MAX_REL_ERR (%.0e); "
                "recompute in FP64", where, rel, (double)HAF_FP32_MAX_REL_ERR);
  return fail(HAF_EACCURACY, msg);
}

// Synchronous single matrix from host memory.
int run_single(const double* A, int64_t n64, int loops, int is_real, int prec, double* out, haf_info* info) {
  const NvtxRange nvtx_range("haf_single");
  const double t0 = now_s();
  if (n64 < 0 || n64 > kMaxN) return fail(HAF_EINVAL, "n out of range");
  if (prec == kPrecF32 && n64 > HAF_FP32_MAX_N) return fail(HAF_EINVAL, "FP32 mode: n above HAF_FP32_MAX_N");
  if (!out || (n64 > 0 && !A)) return fail(HAF_EINVAL, "null pointer");
  int n = (int)n64;
  const int elem = is_real ? 1 : 2;
  double rel = 0.0;
  auto write = [&](double re, double im, double lre, double lim, double abs_sum, int64_t subsets,
                   int64_t launches) {
    out[0] = re;
    if (!is_real) out[1] = im;
    rel = rel_err_bound(re, is_real ? 0.0 : im, abs_sum, prec);
    if (info) {
      info->abs_sum = abs_sum;
      info->value_lo[0] = lre;
      info->value_lo[1] = lim;
      info->subsets = subsets;
      info->seconds = now_s() - t0;
      info->launches = launches;
      info->rel_err_bound = rel;
      info->precision_mode = prec == kPrecF32 ? 1 : 0;
      info->reserved = 0;
    }
  };
  if (n == 0) {
    write(1.0, 0.0, 0.0, 0.0, 1.0, 0, 0);
    return HAF_OK;
  }
  std::vector<double> padded;
  if (n & 1) {
    if (!loops) {
      write(0.0, 0.0, 0.0, 0.0, 0.0, 0, 0);
      return HAF_OK;
    }
    // lhaf: append an isolated vertex with loop weight 1.
    const int np = n + 1;
    padded.assign((size_t)np * np * elem, 0.0);
    for (int i = 0; i < n; ++i)
      std::memcpy(&padded[(size_t)i * np * elem], A + (size_t)i * n * elem, (size_t)n * elem * sizeof(double));
    padded[((size_t)n * np + n) * elem] = 1.0;
    A = padded.data();
    n = np;
    if (n > kMaxN) return fail(HAF_EINVAL, "n out of range");
  }
  std::lock_guard<std::mutex> lk(g_mu);
  Device* d;
  int rc = get_device(&d);
  if (rc) return rc;
  DevPlan* dp;
  rc = cached_plan(d, n, loops, is_real, prec, &dp);
  if (rc) return rc;
  WsLayout w = ws_layout(n, dp->nchunks);
  const size_t jobs_off = w.total;
  const size_t out_off = jobs_off + 256;
  const size_t stage_off = out_off + 256;
  const size_t abytes = (size_t)n * n * elem * sizeof(double);
  rc = ensure_work(d, stage_off + align256(abytes));
  if (rc) return rc;
  rc = ensure_host_out(d, 5);
  if (rc) return rc;
  char* base = (char*)d->work;
  double* At = (double*)(base + w.at);
  double* diag = (double*)(base + w.diag);
  double* Ad = (double*)(base + stage_off);
  cudaStream_t st = d->stream;
  HAF_CUDA(cudaMemcpyAsync(Ad, A, abytes, cudaMemcpyHostToDevice, st));
  HAF_CUDA(launch_prep(Ad, n, is_real, At, diag, st));
  std::vector<Job> jobs{Job{At, diag, n, loops}};
  rc = enqueue(d, *dp, jobs, (Job*)(base + jobs_off), (double*)(base + w.partials),
               (int*)(base + w.counter), (double*)(base + out_off), st);
  if (rc) return rc;
  HAF_CUDA(cudaMemcpyAsync(d->host_out, base + out_off, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
  HAF_CUDA(cudaStreamSynchronize(st));
  const double* o = d->host_out;
  write(o[0] + o[2], o[1] + o[3], o[2], o[3], o[4], dp->subsets, 2 + (int64_t)dp->segs.size());
  return accuracy_gate(rel, prec, "haf_eval");
}

// Part `part` of `nparts` of the subset sum of one matrix (host pointers,
// synchronous): writes the raw record {re_hi, im_hi, re_lo, im_lo, abs_sum}
// of that part's signed terms.  n = 0 and odd n follow the conventions of
// the whole-matrix entry points (the value goes to part 0).
int run_part(const double* A, int64_t n64, int loops, int is_real, int prec, int64_t part, int64_t nparts,
             double* rec, haf_info* info) {
  const NvtxRange nvtx_range("haf_part");
  const double t0 = now_s();
  if (n64 < 0 || n64 > kMaxN) return fail(HAF_EINVAL, "n out of range");
  if (prec == kPrecF32 && n64 > HAF_FP32_MAX_N) return fail(HAF_EINVAL, "FP32 mode: n above HAF_FP32_MAX_N");
  if (nparts < 1 || part < 0 || part >= nparts) return fail(HAF_EINVAL, "part must satisfy 0 <= part < nparts");
  if (!rec || (n64 > 0 && !A)) return fail(HAF_EINVAL, "null pointer");
  int n = (int)n64;
  const int elem = is_real ? 1 : 2;
  auto trivial = [&](double v) {
    rec[0] = (part == 0) ? v : 0.0;
    rec[1] = rec[2] = rec[3] = 0.0;
    rec[4] = (part == 0) ? std::fabs(v) : 0.0;
    if (info) *info = haf_info{rec[4], {0.0, 0.0}, 0, now_s() - t0, 0, 0.0, prec == kPrecF32 ? 1 : 0, 0};
    return HAF_OK;
  };
  if (n == 0) return trivial(1.0);
  std::vector<double> padded;
  if (n & 1) {
    if (!loops) return trivial(0.0);
    const int np = n + 1;
    if (np > kMaxN) return fail(HAF_EINVAL, "n out of range");
    padded.assign((size_t)np * np * elem, 0.0);
    for (int i = 0; i < n; ++i)
      std::memcpy(&padded[(size_t)i * np * elem], A + (size_t)i * n * elem, (size_t)n * elem * sizeof(double));
    padded[((size_t)n * np + n) * elem] = 1.0;
    A = padded.data();
    n = np;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  Device* d;
  int rc = get_device(&d);
  if (rc) return rc;
  DevPlan* dp;
  rc = cached_plan(d, n, loops, is_real, prec, &dp, part, nparts);
  if (rc) return rc;
  WsLayout w = ws_layout(n, dp->nchunks);
  const size_t jobs_off = w.total, out_off = jobs_off + 256, stage_off = out_off + 256;
  const size_t abytes = (size_t)n * n * elem * sizeof(double);
  rc = ensure_work(d, stage_off + align256(abytes));
  if (rc) return rc;
  rc = ensure_host_out(d, 5);
  if (rc) return rc;
  char* base = (char*)d->work;
  double* At = (double*)(base + w.at);
  double* diag = (double*)(base + w.diag);
  double* Ad = (double*)(base + stage_off);
  cudaStream_t st = d->stream;
  HAF_CUDA(cudaMemcpyAsync(Ad, A, abytes, cudaMemcpyHostToDevice, st));
  HAF_CUDA(launch_prep(Ad, n, is_real, At, diag, st));
  if (dp->nchunks == 0) {
    rec[0] = rec[1] = rec[2] = rec[3] = rec[4] = 0.0;
  } else {
    std::vector<Job> jobs{Job{At, diag, n, loops}};
    rc = enqueue(d, *dp, jobs, (Job*)(base + jobs_off), (double*)(base + w.partials), (int*)(base + w.counter),
                 (double*)(base + out_off), st);
    if (rc) return rc;
    HAF_CUDA(cudaMemcpyAsync(d->host_out, base + out_off, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
    HAF_CUDA(cudaStreamSynchronize(st));
    std::memcpy(rec, d->host_out, 5 * sizeof(double));
  }
  if (info)
    *info = haf_info{rec[4], {rec[2], rec[3]}, dp->subsets, now_s() - t0, dp->nchunks ? 2 + (int64_t)dp->segs.size() : 1,
                     0.0, prec == kPrecF32 ? 1 : 0, 0};
  return HAF_OK;
}

// ---------------------------------------------------------------------------
// Batch engine: many matrices of mixed sizes in one persistent launch.
// A batch's plan (chunks of every matrix, largest tiles first), its device
// buffers and a CUDA graph of the whole sequence -- one host-to-device copy
// from pinned staging, one prep launch for all matrices, the subset kernel,
// the finalize kernel and one device-to-host copy -- are built once per
// list of sizes and replayed while the sizes repeat.
// ---------------------------------------------------------------------------
struct BatchPlan {
  std::vector<int> ns;  // sizes after padding (all even, >= 2)
  int loops = -1;
  int is_real = 0;
  int prec = kPrecF64;
  PlanCfg cfg;      // requested launch shape
  int wpb = kWarpsPerBlock;  // planned warps per CTA (first launch)
  int nsegs = 1;             // subset-kernel launches per replay
  char* dbuf = nullptr;
  double* h_in = nullptr;   // pinned staging of the inputs
  double* h_out = nullptr;  // pinned results, 5 per job
  std::vector<size_t> in_off;  // per job offset in h_in (doubles)
  size_t in_doubles = 0;
  int64_t subsets = 0;
  int nchunks = 0;
  cudaGraphExec_t exec = nullptr;
};

void free_batch(BatchPlan* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->dbuf) cudaFree(b->dbuf);
  if (b->h_in) cudaFreeHost(b->h_in);
  if (b->h_out) cudaFreeHost(b->h_out);
  *b = BatchPlan();
}

std::map<int, BatchPlan> g_batch;  // device -> last batch plan

int build_batch(Device* d, const std::vector<int>& ns, int loops, int is_real, int prec, const PlanCfg& pc,
                BatchPlan* b) {
  free_batch(b);
  b->ns = ns;
  b->loops = loops;
  b->is_real = is_real;
  b->prec = prec;
  b->cfg = pc;
  const int njobs = (int)ns.size();
  std::vector<JobSpec> specs;
  for (int n : ns) {
    JobSpec js{n, loops, is_real};
    js.prec = prec;
    specs.push_back(js);
  }
  Plan p;
  int rc = build_plan(specs, d->sms, pc, &p);
  if (rc) return rc;
  b->wpb = p.wpb;
  b->nsegs = (int)p.segs.size();
  b->subsets = p.subsets;
  b->nchunks = (int)p.chunks.size();
  const size_t elem = is_real ? 8 : 16;
  // device layout
  size_t off = 0;
  std::vector<size_t> in_off(njobs), at_off(njobs), dg_off(njobs);
  size_t in_doubles = 0;
  for (int j = 0; j < njobs; ++j) {
    const size_t nn = (size_t)ns[j] * ns[j];
    in_off[j] = in_doubles;
    in_doubles += (nn * elem / 8 + 31) / 32 * 32;  // 256-byte aligned per job
  }
  const size_t din_off = off;
  off += align256(in_doubles * 8);
  for (int j = 0; j < njobs; ++j) {
    at_off[j] = off;
    off += align256((size_t)ns[j] * ns[j] * elem);
    dg_off[j] = off;
    off += align256((size_t)ns[j] * elem);
  }
  const size_t jobs_off = off;
  off += align256((size_t)njobs * sizeof(Job));
  const size_t srcs_off = off;
  off += align256((size_t)njobs * sizeof(double*));
  const size_t part_off = off;
  off += align256((size_t)std::max(1, b->nchunks) * 5 * sizeof(double));
  const size_t cnt_off = off;
  off += 256;
  const size_t out_off = off;
  off += align256((size_t)njobs * 5 * sizeof(double));
  const size_t ch_off = off;
  off += align256(p.chunks.size() * sizeof(Chunk));
  const size_t ord_off = off;
  off += align256(p.order.size() * sizeof(int));
  const size_t jb_off = off;
  off += align256(p.job_begin.size() * sizeof(int));
  cudaError_t e = cudaMalloc(&b->dbuf, off);
  if (e != cudaSuccess) return fail(HAF_ENOMEM, std::string("batch buffers: ") + cudaGetErrorString(e));
  HAF_CUDA(cudaMallocHost(&b->h_in, std::max<size_t>(1, in_doubles) * 8));
  HAF_CUDA(cudaMallocHost(&b->h_out, (size_t)njobs * 5 * sizeof(double)));
  b->in_off = in_off;
  b->in_doubles = in_doubles;
  char* base = b->dbuf;
  std::vector<Job> jobs(njobs);
  std::vector<const double*> srcs(njobs);
  for (int j = 0; j < njobs; ++j) {
    jobs[j] = Job{(double*)(base + at_off[j]), (double*)(base + dg_off[j]), ns[j], loops};
    srcs[j] = (const double*)(base + din_off) + in_off[j];
  }
  cudaStream_t st = d->stream;
  HAF_CUDA(cudaMemcpyAsync(base + jobs_off, jobs.data(), njobs * sizeof(Job), cudaMemcpyHostToDevice, st));
  HAF_CUDA(cudaMemcpyAsync(base + srcs_off, srcs.data(), njobs * sizeof(double*), cudaMemcpyHostToDevice, st));
  HAF_CUDA(cudaMemcpyAsync(base + ch_off, p.chunks.data(), p.chunks.size() * sizeof(Chunk), cudaMemcpyHostToDevice, st));
  HAF_CUDA(cudaMemcpyAsync(base + ord_off, p.order.data(), p.order.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  HAF_CUDA(cudaMemcpyAsync(base + jb_off, p.job_begin.data(), p.job_begin.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  HAF_CUDA(cudaStreamSynchronize(st));
  // capture the per-batch sequence once
  KernelArgs a;
  a.jobs = (const Job*)(base + jobs_off);
  a.chunks = (const Chunk*)(base + ch_off);
  a.counter = (int*)(base + cnt_off);
  a.partials = (double*)(base + part_off);
  a.tables = d->tables;
  a.masks = nullptr;
  a.terms_out = nullptr;
  cudaGraph_t graph;
  HAF_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  cudaError_t ce = cudaMemcpyAsync(base + din_off, b->h_in, in_doubles * 8, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = launch_prep_batch((const double* const*)(base + srcs_off), a.jobs, njobs, is_real, st);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(a.counter, 0, sizeof(int) * std::max<size_t>(1, p.segs.size()), st);
  for (size_t si = 0; si < p.segs.size() && ce == cudaSuccess; ++si) {
    const PlanSeg& sg = p.segs[si];
    KernelArgs as = a;
    as.order = (const int*)(base + ord_off) + sg.begin;
    as.nchunks = sg.end - sg.begin;
    as.counter = a.counter + si;
    as.warp_bytes = sg.warp_bytes;
    const int grid = std::max(1, std::min(d->sms, (as.nchunks + sg.wpb - 1) / sg.wpb));
    ce = launch_subsets(as, p.kind, sg.wpb, grid, st);
  }
  if (ce == cudaSuccess) ce = launch_finalize(a.partials, (const int*)(base + jb_off), njobs, (double*)(base + out_off), st);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(b->h_out, base + out_off, (size_t)njobs * 5 * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaError_t ee = cudaStreamEndCapture(st, &graph);
  if (ce != cudaSuccess) return fail(HAF_ECUDA, std::string("batch capture: ") + cudaGetErrorString(ce));
  if (ee != cudaSuccess) return fail(HAF_ECUDA, std::string("batch capture end: ") + cudaGetErrorString(ee));
  ee = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ee != cudaSuccess) return fail(HAF_ECUDA, std::string("batch graph: ") + cudaGetErrorString(ee));
  return HAF_OK;
}

// Launch shape of a batch: the tuned one for this size list if
// haf_batched_tune recorded one; else the single-matrix shape recorded for
// the batch's largest size (its tiles dominate the shared-memory plan);
// else 4 warps per CTA (FP64) / 8 (FP32) and 8 chunks per warp.
std::map<std::tuple<std::vector<int>, int, int>, PlanCfg> g_batch_tuned;  // (sizes, loops, prec)

PlanCfg batch_cfg(Device* d, const std::vector<int>& sizes, int loops, int prec) {
  auto it = g_batch_tuned.find(std::make_tuple(sizes, loops, prec));
  if (it != g_batch_tuned.end()) return it->second;
  const int nmax = sizes.empty() ? 2 : *std::max_element(sizes.begin(), sizes.end());
  return plan_cfg(d, nmax, loops, 0, prec);
}

// Sizes after the odd-n convention; trivial entries (n = 0, odd haf) are
// written to outs/infos directly and left out of `sizes`/`idx`.
int batch_sizes(const double* const* As, const int64_t* ns, int64_t count, int loops, int prec, double* outs,
                haf_info* infos, std::vector<int>* sizes, std::vector<int64_t>* idx) {
  if (count < 0 || (count > 0 && (!As || !ns || !outs))) return fail(HAF_EINVAL, "null pointer");
  if (count > 65535) return fail(HAF_EINVAL, "batch too large (max 65535 matrices per call)");
  for (int64_t b = 0; b < count; ++b)
    if (ns[b] < 0 || ns[b] > kMaxN || (ns[b] > 0 && !As[b])) return fail(HAF_EINVAL, "bad matrix in batch");
  for (int64_t b = 0; b < count; ++b) {
    const int n = (int)ns[b];
    if (n == 0 || ((n & 1) && !loops)) {
      const double v = (n == 0) ? 1.0 : 0.0;
      if (outs) {
        outs[2 * b] = v;
        outs[2 * b + 1] = 0.0;
      }
      if (infos) infos[b] = haf_info{v, {0.0, 0.0}, 0, 0.0, 0, 0.0, prec == kPrecF32 ? 1 : 0, 0};
      continue;
    }
    if (n + (n & 1) > kMaxN) return fail(HAF_EINVAL, "n out of range");
    if (prec == kPrecF32 && n + (n & 1) > HAF_FP32_MAX_N) return fail(HAF_EINVAL, "FP32 mode: n above HAF_FP32_MAX_N");
    sizes->push_back(n + (n & 1));
    idx->push_back(b);
  }
  return HAF_OK;
}

// Copy the inputs into the batch's pinned staging (odd lhaf matrices padded
// with an isolated looped vertex).
void stage_batch(const BatchPlan& bp, const double* const* As, const int64_t* ns, const std::vector<int64_t>& idx) {
  for (size_t j = 0; j < bp.ns.size(); ++j) {
    const int64_t b = idx[j];
    const int n = (int)ns[b], np = bp.ns[j];
    double* dst = bp.h_in + bp.in_off[j];
    if (np == n) {
      std::memcpy(dst, As[b], (size_t)n * n * 16);
    } else {
      std::memset(dst, 0, (size_t)np * np * 16);
      for (int i = 0; i < n; ++i) std::memcpy(dst + (size_t)i * np * 2, As[b] + (size_t)i * n * 2, (size_t)n * 16);
      dst[((size_t)n * np + n) * 2] = 1.0;
    }
  }
}

int run_batched(const double* const* As, const int64_t* ns, int64_t count, int loops, int prec, double* outs,
                haf_info* infos) {
  const NvtxRange nvtx_range("haf_batched");
  const double t0 = now_s();
  if (count > 0 && !outs) return fail(HAF_EINVAL, "null pointer");
  std::vector<int> sizes;
  std::vector<int64_t> idx;  // job -> batch index
  int rc = batch_sizes(As, ns, count, loops, prec, outs, infos, &sizes, &idx);
  if (rc) return rc;
  if (sizes.empty()) return HAF_OK;
  std::lock_guard<std::mutex> lk(g_mu);
  Device* d;
  rc = get_device(&d);
  if (rc) return rc;
  BatchPlan& bp = g_batch[d->id];
  const PlanCfg pc = batch_cfg(d, sizes, loops, prec);
  if (bp.ns != sizes || bp.loops != loops || bp.is_real != 0 || bp.prec != prec || bp.cfg.wpb != pc.wpb ||
      bp.cfg.chunks_per_warp != pc.chunks_per_warp || !bp.exec) {
    rc = build_batch(d, sizes, loops, 0, prec, pc, &bp);
    if (rc) {
      free_batch(&bp);
      return rc;
    }
  }
  stage_batch(bp, As, ns, idx);
  HAF_CUDA(cudaGraphLaunch(bp.exec, d->stream));
  HAF_CUDA(cudaStreamSynchronize(d->stream));
  const double secs = now_s() - t0;
  double worst = 0.0;
  int64_t worst_b = -1;
  for (size_t j = 0; j < sizes.size(); ++j) {
    const double* o = bp.h_out + 5 * j;
    const int64_t b = idx[j];
    outs[2 * b] = o[0] + o[2];
    outs[2 * b + 1] = o[1] + o[3];
    const double rel = rel_err_bound(o[0] + o[2], o[1] + o[3], o[4], prec);
    if (rel > worst || worst_b < 0) {
      worst = rel;
      worst_b = b;
    }
    if (infos) {
      const int h = sizes[j] / 2;
      infos[b] = haf_info{o[4], {o[2], o[3]}, (int64_t)((1ull << h) - 1), secs, 2 + (int64_t)bp.nsegs,
                          rel, prec == kPrecF32 ? 1 : 0, 0};
    }
  }
  if (prec == kPrecF32 && worst > HAF_FP32_MAX_REL_ERR) {
    char where[64];
    std::snprintf(where, sizeof(where), "haf_batched (matrix %lld)", (long long)worst_b);
    return accuracy_gate(worst, prec, where);
  }
  return HAF_OK;
}

}  // namespace

extern "C" {

int haf_c128(const double* A, int64_t n, double* out, haf_info* info) {
  return run_single(A, n, 0, 0, kPrecF64, out, info);
}
int lhaf_c128(const double* A, int64_t n, double* out, haf_info* info) {
  return run_single(A, n, 1, 0, kPrecF64, out, info);
}
int haf_f64(const double* A, int64_t n, double* out, haf_info* info) {
  return run_single(A, n, 0, 1, kPrecF64, out, info);
}
int lhaf_f64(const double* A, int64_t n, double* out, haf_info* info) {
  return run_single(A, n, 1, 1, kPrecF64, out, info);
}

int haf_eval(const double* A, int64_t n, uint32_t flags, double* out, haf_info* info) {
  if (flags & ~(HAF_FLAG_LOOPS | HAF_FLAG_REAL | HAF_FLAG_FP32)) return fail(HAF_EINVAL, "haf_eval: unknown flags");
  return run_single(A, n, (flags & HAF_FLAG_LOOPS) ? 1 : 0, (flags & HAF_FLAG_REAL) ? 1 : 0,
                    (flags & HAF_FLAG_FP32) ? kPrecF32 : kPrecF64, out, info);
}

int haf_c128_batched(const double* const* As, const int64_t* ns, int64_t count, double* outs, haf_info* infos) {
  return run_batched(As, ns, count, 0, kPrecF64, outs, infos);
}
int lhaf_c128_batched(const double* const* As, const int64_t* ns, int64_t count, double* outs, haf_info* infos) {
  return run_batched(As, ns, count, 1, kPrecF64, outs, infos);
}
int haf_batched(const double* const* As, const int64_t* ns, int64_t count, uint32_t flags, double* outs,
                haf_info* infos) {
  if (flags & ~(HAF_FLAG_LOOPS | HAF_FLAG_FP32)) return fail(HAF_EINVAL, "haf_batched: unknown flags");
  return run_batched(As, ns, count, (flags & HAF_FLAG_LOOPS) ? 1 : 0, (flags & HAF_FLAG_FP32) ? kPrecF32 : kPrecF64,
                     outs, infos);
}

int haf_part(const double* A, int64_t n, uint32_t flags, int64_t part, int64_t nparts, double* rec,
             haf_info* info) {
  if (flags & ~(HAF_FLAG_LOOPS | HAF_FLAG_REAL | HAF_FLAG_FP32)) return fail(HAF_EINVAL, "haf_part: unknown flags");
  return run_part(A, n, (flags & HAF_FLAG_LOOPS) ? 1 : 0, (flags & HAF_FLAG_REAL) ? 1 : 0,
                  (flags & HAF_FLAG_FP32) ? kPrecF32 : kPrecF64, part, nparts, rec, info);
}

int haf_part_subsets(int64_t n, int64_t part, int64_t nparts, int64_t* subsets) {
  if (n < 0 || n > kMaxN || nparts < 1 || part < 0 || part >= nparts || !subsets)
    return fail(HAF_EINVAL, "haf_part_subsets: bad arguments");
  const int h = (int)(n / 2);
  int64_t total = 0;
  for (int m = 1; m <= h; ++m) {
    uint64_t lo, hi;
    part_range(binom(h, m), part, nparts, &lo, &hi);
    total += (int64_t)(hi - lo);
  }
  *subsets = total;
  return HAF_OK;
}

int haf_plan_stats(int64_t n, uint32_t flags, int32_t warps_per_block, int32_t chunks_per_warp, int32_t sms,
                   int64_t* out) {
  if (n < 2 || n > kMaxN || (n & 1) || !out || sms < 1 || sms > 1024)
    return fail(HAF_EINVAL, "haf_plan_stats: bad arguments");
  if (flags & ~(HAF_FLAG_LOOPS | HAF_FLAG_REAL | HAF_FLAG_FP32)) return fail(HAF_EINVAL, "haf_plan_stats: unknown flags");
  JobSpec js{(int)n, (flags & HAF_FLAG_LOOPS) ? 1 : 0, (flags & HAF_FLAG_REAL) ? 1 : 0};
  js.prec = (flags & HAF_FLAG_FP32) ? kPrecF32 : kPrecF64;
  PlanCfg pc;
  pc.wpb = warps_per_block;
  pc.chunks_per_warp = chunks_per_warp;
  Plan p;
  const int rc = build_plan({js}, sms, pc, &p);
  if (rc) return rc;
  for (int k = 0; k < 8; ++k) out[k] = 0;
  out[0] = (int64_t)p.chunks.size();
  out[1] = (int64_t)p.segs.size();
  for (size_t si = 0; si < p.segs.size() && si < 3; ++si) {
    out[2 + si] = p.segs[si].wpb;
    for (int q = p.segs[si].begin; q < p.segs[si].end; ++q) out[5 + si] += p.chunks[p.order[q]].count;
  }
  return HAF_OK;
}

int haf_combine(const double* recs, int64_t nparts, double* out) {
  if (nparts < 1 || !recs || !out) return fail(HAF_EINVAL, "haf_combine: bad arguments");
  // Fixed-order double-double sum (Knuth's TwoSum, then a fast renormalisation).
  double rh = 0.0, rl = 0.0, ih = 0.0, il = 0.0, ab = 0.0;
  auto add = [](double& hi, double& lo, double xh, double xl) {
    const double s = hi + xh;
    const double bb = s - hi;
    double e = (hi - (s - bb)) + (xh - bb);
    e += lo + xl;
    hi = s + e;
    lo = e - (hi - s);
  };
  for (int64_t p = 0; p < nparts; ++p) {
    const double* r = recs + 5 * p;
    add(rh, rl, r[0], r[2]);
    add(ih, il, r[1], r[3]);
    ab += r[4];
  }
  out[0] = rh;
  out[1] = ih;
  out[2] = rl;
  out[3] = il;
  out[4] = ab;
  return HAF_OK;
}

size_t haf_workspace_bytes(int64_t n, uint32_t flags) {
  if (n < 2 || n > kMaxN || (n & 1)) return 0;
  if (flags & ~(HAF_FLAG_LOOPS | HAF_FLAG_REAL | HAF_FLAG_FP32)) return 0;
  const int prec = (flags & HAF_FLAG_FP32) ? kPrecF32 : kPrecF64;
  if (prec == kPrecF32 && n > HAF_FP32_MAX_N) return 0;
  std::lock_guard<std::mutex> lk(g_mu);
  Device* d;
  if (get_device(&d)) return 0;
  DevPlan* dp;
  if (cached_plan(d, (int)n, (flags & HAF_FLAG_LOOPS) ? 1 : 0, (flags & HAF_FLAG_REAL) ? 1 : 0, prec, &dp)) return 0;
  return ws_layout((int)n, dp->nchunks).total + 256;
}

int haf_launch(const double* dA, int64_t n, uint32_t flags, double* d_out, void* d_work, size_t ws_bytes,
               void* stream) {
  const NvtxRange nvtx_range("haf_launch");
  if (n < 2 || n > kMaxN || (n & 1)) return fail(HAF_EINVAL, "haf_launch: n must be even, 2..HAF_MAX_N");
  if (!dA || !d_out || !d_work) return fail(HAF_EINVAL, "haf_launch: null pointer");
  if (((uintptr_t)d_work & 255) != 0) return fail(HAF_EINVAL, "haf_launch: workspace not 256-byte aligned");
  if (flags & ~(HAF_FLAG_LOOPS | HAF_FLAG_REAL | HAF_FLAG_FP32)) return fail(HAF_EINVAL, "haf_launch: unknown flags");
  const int loops = (flags & HAF_FLAG_LOOPS) ? 1 : 0, is_real = (flags & HAF_FLAG_REAL) ? 1 : 0;
  const int prec = (flags & HAF_FLAG_FP32) ? kPrecF32 : kPrecF64;
  if (prec == kPrecF32 && n > HAF_FP32_MAX_N) return fail(HAF_EINVAL, "FP32 mode: n above HAF_FP32_MAX_N");
  std::lock_guard<std::mutex> lk(g_mu);
  Device* d;
  int rc = get_device(&d);
  if (rc) return rc;
  DevPlan* dp;
  rc = cached_plan(d, (int)n, loops, is_real, prec, &dp);
  if (rc) return rc;
  WsLayout w = ws_layout((int)n, dp->nchunks);
  if (ws_bytes < w.total + 256) return fail(HAF_ESMALL, "haf_launch: workspace too small");
  char* base = (char*)d_work;
  cudaStream_t st = (cudaStream_t)stream;
  double* At = (double*)(base + w.at);
  double* diag = (double*)(base + w.diag);
  HAF_CUDA(launch_prep(dA, (int)n, is_real, At, diag, st));
  std::vector<Job> jobs{Job{At, diag, (int)n, loops}};
  return enqueue(d, *dp, jobs, (Job*)(base + w.total), (double*)(base + w.partials), (int*)(base + w.counter),
                 d_out, st);
}

int haf_terms_c128(const double* A, int64_t n64, int loops, const uint64_t* masks, int64_t count, double* terms) {
  return haf_terms(A, n64, loops ? HAF_FLAG_LOOPS : 0u, masks, count, terms);
}

int haf_terms(const double* A, int64_t n64, uint32_t flags, const uint64_t* masks, int64_t count, double* terms) {
  const NvtxRange nvtx_range("haf_terms");
  if (n64 < 2 || n64 > kMaxN || (n64 & 1)) return fail(HAF_EINVAL, "haf_terms: n must be even, 2..HAF_MAX_N");
  if (!A || (count > 0 && (!masks || !terms)) || count < 0) return fail(HAF_EINVAL, "haf_terms: bad arguments");
  if (flags & ~(HAF_FLAG_LOOPS | HAF_FLAG_FP32)) return fail(HAF_EINVAL, "haf_terms: unknown flags");
  const int loops = (flags & HAF_FLAG_LOOPS) ? 1 : 0;
  const int prec = (flags & HAF_FLAG_FP32) ? kPrecF32 : kPrecF64;
  if (prec == kPrecF32 && n64 > HAF_FP32_MAX_N) return fail(HAF_EINVAL, "FP32 mode: n above HAF_FP32_MAX_N");
  const int kind = kernel_kind(0, prec);
  const int n = (int)n64, h = n / 2;
  for (int64_t i = 0; i < count; ++i)
    if (masks[i] >> h) return fail(HAF_EINVAL, "haf_terms: mask has bits beyond n/2");
  if (count == 0) return HAF_OK;
  // The device and its launch shape for (n, flags): the summands are
  // computed by the same kernel instantiations, with the same lanes per
  // subset for each size, as a whole-matrix call of this size.
  std::lock_guard<std::mutex> lk(g_mu);
  Device* d;
  int rc = get_device(&d);
  if (rc) return rc;
  const PlanCfg pc = plan_cfg(d, n, loops, 0, prec);
  // sort subsets by size; each size becomes chunks of four group-rounds
  std::vector<int64_t> perm(count);
  for (int64_t i = 0; i < count; ++i) perm[i] = i;
  std::stable_sort(perm.begin(), perm.end(), [&](int64_t a, int64_t b) {
    return __builtin_popcountll(masks[a]) < __builtin_popcountll(masks[b]);
  });
  std::vector<uint64_t> sorted(count);
  for (int64_t i = 0; i < count; ++i) sorted[i] = masks[perm[i]];
  Plan p;
  p.job_begin = {0};
  std::vector<int> seg_of;
  int64_t i = 0;
  while (i < count) {
    const int m = __builtin_popcountll(sorted[i]);
    int64_t e = i;
    while (e < count && __builtin_popcountll(sorted[e]) == m) ++e;
    if (m == 0) {  // empty subset: f = 0 for h >= 1
      i = e;
      continue;
    }
    int wpb = pc.wpb;
    SizeCfg cfg;
    while (!choose_cfg(2 * m, h, kind, loops, warp_bytes_for(wpb), &cfg)) {
      if (wpb == 4) return fail(HAF_EINVAL, "haf_terms: size too large");
      wpb /= 2;
    }
    const int S = 32 / cfg.G;
    for (int64_t r = i; r < e; r += 4 * S) {
      Chunk c;
      std::memset(&c, 0, sizeof(c));
      c.rank0 = (uint64_t)r;
      c.count = (uint32_t)std::min<int64_t>(4 * S, e - r);
      c.m = (uint8_t)m;
      c.G = (uint8_t)cfg.G;
      c.ld = (uint8_t)cfg.ld;
      p.chunks.push_back(c);
      seg_of.push_back(wpb);
    }
    i = e;
  }
  p.job_begin.push_back((int)p.chunks.size());
  p.kind = kind;
  for (int w : {16, 8, 4}) {
    PlanSeg sg;
    sg.begin = (int)p.order.size();
    for (size_t q = 0; q < p.chunks.size(); ++q)
      if (seg_of[q] == w) p.order.push_back((int)q);
    sg.end = (int)p.order.size();
    if (sg.end == sg.begin) continue;
    sg.wpb = w;
    sg.warp_bytes = warp_bytes_for(w);
    p.segs.push_back(sg);
  }
  p.wpb = p.segs.empty() ? kWarpsPerBlock : p.segs[0].wpb;
  p.warp_bytes = warp_bytes_for(p.wpb);
  std::vector<double> res((size_t)count * 2, 0.0);
  if (!p.chunks.empty()) {
    const size_t nn = (size_t)n * n * 16;
    size_t off = 0;
    const size_t a_off = off; off += align256(nn);
    const size_t at_off = off; off += align256(nn);
    const size_t dg_off = off; off += align256((size_t)n * 16);
    const size_t mk_off = off; off += align256((size_t)count * 8);
    const size_t tm_off = off; off += align256((size_t)count * 16);
    const size_t ch_off = off; off += align256(p.chunks.size() * sizeof(Chunk));
    const size_t ord_off = off; off += align256(p.order.size() * sizeof(int));
    const size_t jb_off = off; off += 256;
    const size_t job_off = off; off += 256;
    const size_t cnt_off = off; off += 256;
    rc = ensure_work(d, off);
    if (rc) return rc;
    char* base = (char*)d->work;
    cudaStream_t st = d->stream;
    HAF_CUDA(cudaMemcpyAsync(base + a_off, A, nn, cudaMemcpyHostToDevice, st));
    HAF_CUDA(launch_prep((double*)(base + a_off), n, 0, (double*)(base + at_off), (double*)(base + dg_off), st));
    HAF_CUDA(cudaMemcpyAsync(base + mk_off, sorted.data(), (size_t)count * 8, cudaMemcpyHostToDevice, st));
    HAF_CUDA(cudaMemsetAsync(base + tm_off, 0, (size_t)count * 16, st));
    DevPlan dp;
    dp.chunks = (Chunk*)(base + ch_off);
    dp.order = (int*)(base + ord_off);
    dp.job_begin = (int*)(base + jb_off);
    dp.nchunks = (int)p.chunks.size();
    dp.njobs = 1;
    dp.kind = p.kind;
    dp.wpb = p.wpb;
    dp.warp_bytes = p.warp_bytes;
    dp.segs = p.segs;
    HAF_CUDA(cudaMemcpyAsync(dp.chunks, p.chunks.data(), p.chunks.size() * sizeof(Chunk), cudaMemcpyHostToDevice, st));
    HAF_CUDA(cudaMemcpyAsync(dp.order, p.order.data(), p.order.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    std::vector<Job> jobs{Job{(double*)(base + at_off), (double*)(base + dg_off), n, loops ? 1 : 0}};
    rc = enqueue(d, dp, jobs, (Job*)(base + job_off), nullptr, (int*)(base + cnt_off), nullptr, st,
                 (const uint64_t*)(base + mk_off), (double*)(base + tm_off));
    if (rc) return rc;
    std::vector<double> tmp((size_t)count * 2);
    HAF_CUDA(cudaMemcpyAsync(tmp.data(), base + tm_off, (size_t)count * 16, cudaMemcpyDeviceToHost, st));
    HAF_CUDA(cudaStreamSynchronize(st));
    for (int64_t q = 0; q < count; ++q) {
      res[2 * perm[q]] = tmp[2 * q];
      res[2 * perm[q] + 1] = tmp[2 * q + 1];
    }
  }
  std::memcpy(terms, res.data(), res.size() * sizeof(double));
  return HAF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner.  The launch shape of a plan -- warps per CTA (which sets the
// shared-memory slice per warp, hence the lanes per subset G and the
// subsets per CTA) and the chunk granularity -- is picked by timing every
// candidate on the device and keeping the fastest.  Inputs are synthetic
// (the work does not depend on the matrix entries); results are recorded
// per device and used by every later call with the same key.
// ---------------------------------------------------------------------------
namespace {

const int kTuneWpb[3] = {4, 8, 16};
const int kTuneCpw[4] = {2, 4, 8, 16};

// Deterministic symmetric test matrix for timing (entries in [-1, 1)).
std::vector<double> tune_matrix(int n, int is_real) {
  const int elem = is_real ? 1 : 2;
  std::vector<double> A((size_t)n * n * elem);
  uint64_t x = 0x9e3779b97f4a7c15ull;
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j)
      for (int c = 0; c < elem; ++c) {
        x ^= x << 13;
        x ^= x >> 7;
        x ^= x << 17;
        const double v = (double)(x >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
        A[((size_t)i * n + j) * elem + c] = v;
        A[((size_t)j * n + i) * elem + c] = v;
      }
  return A;
}

// Mean milliseconds of `reps` launches of one plan (after one warm-up).
int time_plan(Device* d, const DevPlan& dp, int n, int loops, const double* Ad, int is_real, char* base, int reps,
              double* ms_out) {
  WsLayout w = ws_layout(n, dp.nchunks);
  cudaStream_t st = d->stream;
  double* At = (double*)(base + w.at);
  double* diag = (double*)(base + w.diag);
  HAF_CUDA(launch_prep(Ad, n, is_real, At, diag, st));
  std::vector<Job> jobs{Job{At, diag, n, loops}};
  cudaEvent_t e0, e1;
  HAF_CUDA(cudaEventCreate(&e0));
  HAF_CUDA(cudaEventCreate(&e1));
  int rc = HAF_OK;
  for (int r = 0; r <= reps && rc == HAF_OK; ++r) {
    if (r == 1) cudaEventRecord(e0, st);
    rc = enqueue(d, dp, jobs, (Job*)(base + w.total), (double*)(base + w.partials), (int*)(base + w.counter),
                 (double*)(base + w.total + 256), st);
  }
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (rc == HAF_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (e != cudaSuccess) return fail(HAF_ECUDA, std::string("tune timing: ") + cudaGetErrorString(e));
  *ms_out = ms / reps;
  return HAF_OK;
}

bool same_cfg(const PlanCfg& a, const PlanCfg& b) {
  return a.wpb == b.wpb && a.chunks_per_warp == b.chunks_per_warp;
}

}  // namespace

extern "C" {

int haf_tune(int64_t n64, uint32_t flags, int32_t reps, haf_tune_result* out) {
  const NvtxRange nvtx_range("haf_tune");
  if (n64 < 2 || n64 > kMaxN || (n64 & 1)) return fail(HAF_EINVAL, "haf_tune: n must be even, 2..HAF_MAX_N");
  if (flags & ~(HAF_FLAG_LOOPS | HAF_FLAG_REAL | HAF_FLAG_FP32)) return fail(HAF_EINVAL, "haf_tune: unknown flags");
  if (reps < 1 || reps > 100 || !out) return fail(HAF_EINVAL, "haf_tune: reps must be 1..100, out non-null");
  const int n = (int)n64, loops = (flags & HAF_FLAG_LOOPS) ? 1 : 0, is_real = (flags & HAF_FLAG_REAL) ? 1 : 0;
  const int prec = (flags & HAF_FLAG_FP32) ? kPrecF32 : kPrecF64;
  if (prec == kPrecF32 && n > HAF_FP32_MAX_N) return fail(HAF_EINVAL, "FP32 mode: n above HAF_FP32_MAX_N");
  std::lock_guard<std::mutex> lk(g_mu);
  Device* d;
  int rc = get_device(&d);
  if (rc) return rc;
  const auto key = std::make_tuple(n, loops, is_real, prec);
  d->tuned.erase(key);
  const PlanCfg def = plan_cfg(d, n, loops, is_real, prec);
  // plans of every feasible candidate (a shape the planner had to lower is skipped)
  std::vector<std::pair<PlanCfg, DevPlan*>> cands;
  size_t ws = 0;
  for (int wpb : kTuneWpb)
    for (int cpw : kTuneCpw) {
      PlanCfg c;
      c.wpb = wpb;
      c.chunks_per_warp = cpw;
      DevPlan* dp;
      rc = cached_plan(d, n, loops, is_real, prec, &dp, 0, 1, &c);
      if (rc) return rc;
      if (dp->wpb != wpb) continue;
      cands.push_back({c, dp});
      ws = std::max(ws, ws_layout(n, dp->nchunks).total + 512);
    }
  const size_t abytes = (size_t)n * n * (is_real ? 8 : 16);
  rc = ensure_work(d, ws + align256(abytes));
  if (rc) return rc;
  char* base = (char*)d->work;
  double* Ad = (double*)(base + ws);
  const std::vector<double> A = tune_matrix(n, is_real);
  HAF_CUDA(cudaMemcpyAsync(Ad, A.data(), abytes, cudaMemcpyHostToDevice, d->stream));
  double best = 1e300, ms_def = -1.0;
  PlanCfg best_cfg = def;
  for (auto& c : cands) {
    double ms;
    rc = time_plan(d, *c.second, n, loops, Ad, is_real, base, reps, &ms);
    if (rc) return rc;
    if (same_cfg(c.first, def)) ms_def = ms;
    if (ms < best) {
      best = ms;
      best_cfg = c.first;
    }
  }
  d->tuned[key] = best_cfg;
  out->warps_per_block = best_cfg.wpb;
  out->chunks_per_warp = best_cfg.chunks_per_warp;
  out->ms = best;
  out->ms_default = ms_def;
  out->candidates = (int32_t)cands.size();
  return HAF_OK;
}

int haf_tune_set(int64_t n64, uint32_t flags, int32_t warps_per_block, int32_t chunks_per_warp) {
  if (n64 < 2 || n64 > kMaxN || (n64 & 1)) return fail(HAF_EINVAL, "haf_tune_set: n must be even, 2..HAF_MAX_N");
  if (flags & ~(HAF_FLAG_LOOPS | HAF_FLAG_REAL | HAF_FLAG_FP32)) return fail(HAF_EINVAL, "haf_tune_set: unknown flags");
  if ((warps_per_block != 4 && warps_per_block != 8 && warps_per_block != 16) || chunks_per_warp < 1 ||
      chunks_per_warp > 64)
    return fail(HAF_EINVAL, "haf_tune_set: warps per CTA must be 4, 8 or 16 and chunks per warp 1..64");
  std::lock_guard<std::mutex> lk(g_mu);
  Device* d;
  int rc = get_device(&d);
  if (rc) return rc;
  PlanCfg c;
  c.wpb = warps_per_block;
  c.chunks_per_warp = chunks_per_warp;
  d->tuned[std::make_tuple((int)n64, (flags & HAF_FLAG_LOOPS) ? 1 : 0, (flags & HAF_FLAG_REAL) ? 1 : 0,
                           (flags & HAF_FLAG_FP32) ? kPrecF32 : kPrecF64)] = c;
  return HAF_OK;
}

int haf_batched_tune(const double* const* As, const int64_t* ns, int64_t count, uint32_t flags, int32_t reps,
                     haf_tune_result* out) {
  const NvtxRange nvtx_range("haf_batched_tune");
  if (flags & ~(HAF_FLAG_LOOPS | HAF_FLAG_FP32)) return fail(HAF_EINVAL, "haf_batched_tune: unknown flags");
  if (reps < 1 || reps > 100 || !out) return fail(HAF_EINVAL, "haf_batched_tune: reps must be 1..100, out non-null");
  const int loops = (flags & HAF_FLAG_LOOPS) ? 1 : 0, prec = (flags & HAF_FLAG_FP32) ? kPrecF32 : kPrecF64;
  std::vector<double> scratch((size_t)std::max<int64_t>(count, 1) * 2);
  std::vector<int> sizes;
  std::vector<int64_t> idx;
  int rc = batch_sizes(As, ns, count, loops, prec, scratch.data(), nullptr, &sizes, &idx);
  if (rc) return rc;
  if (sizes.empty()) return fail(HAF_EINVAL, "haf_batched_tune: no non-trivial matrix in the batch");
  std::lock_guard<std::mutex> lk(g_mu);
  Device* d;
  rc = get_device(&d);
  if (rc) return rc;
  const auto key = std::make_tuple(sizes, loops, prec);
  g_batch_tuned.erase(key);
  const PlanCfg def = batch_cfg(d, sizes, loops, prec);
  cudaEvent_t e0, e1;
  HAF_CUDA(cudaEventCreate(&e0));
  HAF_CUDA(cudaEventCreate(&e1));
  double best = 1e300, ms_def = -1.0;
  PlanCfg best_cfg = def;
  int ncand = 0;
  for (int wpb : kTuneWpb)
    for (int cpw : kTuneCpw) {
      PlanCfg c;
      c.wpb = wpb;
      c.chunks_per_warp = cpw;
      BatchPlan bp;
      rc = build_batch(d, sizes, loops, 0, prec, c, &bp);
      if (rc == HAF_OK && bp.wpb == wpb) {
        ++ncand;
        stage_batch(bp, As, ns, idx);
        cudaError_t e = cudaGraphLaunch(bp.exec, d->stream);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, d->stream);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(bp.exec, d->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, d->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) rc = fail(HAF_ECUDA, std::string("haf_batched_tune: ") + cudaGetErrorString(e));
        const double m = ms / reps;
        if (rc == HAF_OK) {
          if (same_cfg(c, def)) ms_def = m;
          if (m < best) {
            best = m;
            best_cfg = c;
          }
        }
      }
      free_batch(&bp);
      if (rc) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return rc;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g_batch_tuned[key] = best_cfg;
  out->warps_per_block = best_cfg.wpb;
  out->chunks_per_warp = best_cfg.chunks_per_warp;
  out->ms = best;
  out->ms_default = ms_def;
  out->candidates = ncand;
  return HAF_OK;
}

int haf_fp64_peak(double* tflops, double* ms_out) {
  if (!tflops) return fail(HAF_EINVAL, "haf_fp64_peak: null pointer");
  std::lock_guard<std::mutex> lk(g_mu);
  Device* d;
  int rc = get_device(&d);
  if (rc) return rc;
  const int blocks = d->sms, threads = 512, iters = 2000;
  double* sink = nullptr;
  HAF_CUDA(cudaMalloc(&sink, (size_t)blocks * threads * sizeof(double)));
  cudaEvent_t e0, e1;
  HAF_CUDA(cudaEventCreate(&e0));
  HAF_CUDA(cudaEventCreate(&e1));
  HAF_CUDA(launch_fp64_probe(sink, 10, blocks, d->stream));
  HAF_CUDA(cudaEventRecord(e0, d->stream));
  HAF_CUDA(launch_fp64_probe(sink, iters, blocks, d->stream));
  HAF_CUDA(cudaEventRecord(e1, d->stream));
  HAF_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  HAF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  const double flops = 2.0 * 8.0 * 16.0 * iters * (double)blocks * threads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return HAF_OK;
}

const char* haf_last_error(void) { return hafgb::g_last_error.c_str(); }
const char* haf_version(void) { return "hafnian_gb300 0.1 (sm_103a)"; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free entry point (haf_launch_noalloc).
//
// Some callers cannot allocate device memory at the moment they want a
// hafnian: code that runs under a caching allocator or memory pool that
// owns every byte of the device, plug-ins and callbacks that may not call
// cudaMalloc/cudaFree (which synchronise the device), and services that
// must not grow their footprint after start-up.  This path therefore keeps
// all of its scratch -- the pair-swapped copy of A, the work plan, the
// per-chunk partial sums and the work counter -- in one file-scope device
// array of fixed size, reserved when the library is loaded and held by every
// GPU that loads it until the process exits.
//
// The array is shared by every call: a call overwrites what the previous one
// left, and clears the work counter itself before its kernels run.  Two calls
// that overlap on the GPU (different streams without ordering between them)
// race on the array and give wrong results; serialise them.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocBytes = HAF_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[HAF_NOALLOC_SCRATCH_BYTES];

// Fixed layout inside the array.
constexpr size_t kNaCounter = 0;                                // 3 work counters
constexpr size_t kNaTables = 256;                               // 256 doubles
constexpr size_t kNaJobs = kNaTables + 256 * sizeof(double);    // one Job
constexpr size_t kNaAt = kNaJobs + 256;                         // n*n*16 <= 56*56*16
constexpr size_t kNaDiag = kNaAt + (size_t)kMaxN * kMaxN * 16;  // n*16
constexpr size_t kNaJobBegin = kNaDiag + 1024;                 // 2 ints (diag: n*16 <= 896)
constexpr size_t kNaChunks = kNaJobBegin + 256;
constexpr size_t kNaPerChunk = sizeof(Chunk) + sizeof(int) + 5 * sizeof(double);
constexpr int kNaMaxChunks = (int)((kNoAllocBytes - kNaChunks) / kNaPerChunk) / 8 * 8;
static_assert(kNaChunks % 256 == 0, "no-alloc layout alignment");
static_assert(kNaMaxChunks >= 4096, "no-alloc scratch too small for the chunk budget");

struct NoAllocDevice {
  bool ready = false;
  unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch
  int sms = 0;
};
std::mutex g_na_mu;
NoAllocDevice g_na_dev[64];

// Host-side plan storage (static: this path allocates nothing, host or device).
Chunk g_na_chunks[kNaMaxChunks];
int g_na_order[kNaMaxChunks];
PlanSeg g_na_segs[3];
int g_na_nsegs = 0;
double g_na_tables[256];

// Per-device set-up: the device address of the array (the host-side name
// g_noalloc_scratch is only a stand-in for it) and the kernel attributes.
int noalloc_setup(int dev, NoAllocDevice** out) {
  if (dev < 0 || dev >= 64) return fail(HAF_EINVAL, "haf_launch_noalloc: device ordinal out of range");
  NoAllocDevice& d = g_na_dev[dev];
  if (!d.ready) {
    void* ptr = nullptr;
    HAF_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    HAF_CUDA(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
    // with one chunk per warp every plan has at most sms * (16 + 8 + 4)
    // chunks plus one partial chunk per size class and launch
    if ((long)d.sms * 28 + 3 * (kMaxN / 2) > kNaMaxChunks)
      return fail(HAF_EINVAL, "haf_launch_noalloc: the scratch array is too small for this GPU's SM count");
    HAF_CUDA(configure_kernels());
    for (int k = 0; k < 128; ++k) g_na_tables[k] = 0.5 * k;
    g_na_tables[128] = 0.0;
    for (int k = 1; k < 128; ++k) g_na_tables[128 + k] = 1.0 / k;
    d.scratch = (unsigned char*)ptr;
    d.ready = true;
  }
  *out = &d;
  return HAF_OK;
}

// Work plan for one matrix written into the static host arrays, in the
// launch shape `pc` (the one haf_launch uses for this n and kind): size
// classes whose tiles do not fit pc.wpb warps per CTA drop to fewer; one
// segment (launch) per warps-per-CTA value, most warps first, largest tiles
// first inside each.  If the chunks exceed kNaMaxChunks the chunk
// granularity is halved until they fit.  Returns the chunk count or < 0.
int noalloc_plan(int n, int is_real, int loops, PlanCfg pc, int sms) {
  const int h = n / 2, kind = kernel_kind(is_real, kPrecF64);
  int wpb_of[kMaxN / 2 + 1];
  SizeCfg cfg_of[kMaxN / 2 + 1];
  double work[17] = {0};
  for (int m = 1; m <= h; ++m) {
    int w = pc.wpb;
    while (!choose_cfg(2 * m, h, kind, loops, warp_bytes_for(w), &cfg_of[m])) {
      if (w == 4) return fail(HAF_EINVAL, "haf_launch_noalloc: n too large");
      w /= 2;
    }
    wpb_of[m] = w;
    work[w] += (double)binom(h, m) * std::pow(2.0 * m, 3);
  }
  for (int per_warp = pc.chunks_per_warp;; per_warp = std::max(1, per_warp / 2)) {
    int nc = 0;
    bool over = false;
    g_na_nsegs = 0;
    for (int w : {16, 8, 4}) {
      const int begin = nc;
      const double target = std::max(1.0, work[w] / ((double)sms * w * per_warp));
      for (int m = h; m >= 1 && !over; --m) {
        if (wpb_of[m] != w) continue;
        const int N = 2 * m, S = 32 / cfg_of[m].G;
        const uint64_t cnt = binom(h, m);
        uint64_t csz = (uint64_t)std::ceil(target / std::pow((double)N, 3) / S) * S;
        csz = std::min<uint64_t>(std::max<uint64_t>(csz, (uint64_t)S), (uint64_t)1 << 30);
        for (uint64_t r0 = 0; r0 < cnt; r0 += csz) {
          if (nc >= kNaMaxChunks) {
            over = true;
            break;
          }
          Chunk& c = g_na_chunks[nc];
          std::memset(&c, 0, sizeof(c));
          c.rank0 = r0;
          c.mask0 = unrank_colex(r0, m, h);
          c.count = (uint32_t)std::min<uint64_t>(csz, cnt - r0);
          c.m = (uint8_t)m;
          c.G = (uint8_t)cfg_of[m].G;
          c.ld = (uint8_t)cfg_of[m].ld;
          g_na_order[nc] = nc;
          ++nc;
        }
      }
      if (over) break;
      if (nc > begin) {
        PlanSeg& sg = g_na_segs[g_na_nsegs++];
        sg.begin = begin;
        sg.end = nc;
        sg.wpb = w;
        sg.warp_bytes = warp_bytes_for(w);
      }
    }
    if (!over) return nc;
    if (per_warp == 1) return fail(HAF_EINVAL, "haf_launch_noalloc: plan exceeds the scratch array");
  }
}

}  // namespace

extern "C" int haf_launch_noalloc(const double* dA, int64_t n, uint32_t flags, double* d_out, void* stream) {
  if (n < 2 || n > kMaxN || (n & 1))
    return fail(HAF_EINVAL, "haf_launch_noalloc: n must be even and 2 <= n <= HAF_MAX_N (56)");
  if (!dA || !d_out) return fail(HAF_EINVAL, "haf_launch_noalloc: null pointer");
  if (flags & ~(HAF_FLAG_LOOPS | HAF_FLAG_REAL)) return fail(HAF_EINVAL, "haf_launch_noalloc: unknown flags");
  const int loops = (flags & HAF_FLAG_LOOPS) ? 1 : 0, is_real = (flags & HAF_FLAG_REAL) ? 1 : 0;
  int dev = 0;
  HAF_CUDA(cudaGetDevice(&dev));
  // the launch shape haf_launch would use (tuned by haf_tune / haf_tune_set,
  // else the default); a look-up only, nothing is created
  PlanCfg pc;
  pc.wpb = kWarpsPerBlock;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_devices.find(dev);
    if (it != g_devices.end()) {
      auto t = it->second->tuned.find(std::make_tuple((int)n, loops, is_real, (int)kPrecF64));
      if (t != it->second->tuned.end()) pc = t->second;
    }
  }
  std::lock_guard<std::mutex> lk(g_na_mu);
  NoAllocDevice* d;
  int rc = noalloc_setup(dev, &d);
  if (rc) return rc;
  const int nc = noalloc_plan((int)n, is_real, loops, pc, d->sms);
  if (nc < 0) return nc;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* s = d->scratch;
  Chunk* chunks = (Chunk*)(s + kNaChunks);
  int* order = (int*)(s + kNaChunks + (size_t)kNaMaxChunks * sizeof(Chunk));
  double* partials = (double*)(s + kNaChunks + (size_t)kNaMaxChunks * (sizeof(Chunk) + sizeof(int)));
  int* job_begin = (int*)(s + kNaJobBegin);
  int* counters = (int*)(s + kNaCounter);  // one per launch
  const int jb[2] = {0, nc};
  double* At = (double*)(s + kNaAt);
  double* diag = (double*)(s + kNaDiag);
  const Job job{At, diag, (int)n, loops};
  HAF_CUDA(cudaMemcpyAsync(s + kNaTables, g_na_tables, sizeof(g_na_tables), cudaMemcpyHostToDevice, st));
  HAF_CUDA(cudaMemcpyAsync(s + kNaJobs, &job, sizeof(Job), cudaMemcpyHostToDevice, st));
  HAF_CUDA(cudaMemcpyAsync(job_begin, jb, sizeof(jb), cudaMemcpyHostToDevice, st));
  HAF_CUDA(cudaMemcpyAsync(chunks, g_na_chunks, (size_t)nc * sizeof(Chunk), cudaMemcpyHostToDevice, st));
  HAF_CUDA(cudaMemcpyAsync(order, g_na_order, (size_t)nc * sizeof(int), cudaMemcpyHostToDevice, st));
  HAF_CUDA(cudaMemsetAsync(counters, 0, 3 * sizeof(int), st));
  HAF_CUDA(launch_prep(dA, (int)n, is_real, At, diag, st));
  for (int si = 0; si < g_na_nsegs; ++si) {
    const PlanSeg& sg = g_na_segs[si];
    KernelArgs a;
    a.jobs = (const Job*)(s + kNaJobs);
    a.chunks = chunks;
    a.order = order + sg.begin;
    a.nchunks = sg.end - sg.begin;
    a.counter = counters + si;
    a.partials = partials;
    a.tables = (const double*)(s + kNaTables);
    a.masks = nullptr;
    a.terms_out = nullptr;
    a.warp_bytes = sg.warp_bytes;
    const int grid = std::max(1, std::min(d->sms, (a.nchunks + sg.wpb - 1) / sg.wpb));
    HAF_CUDA(launch_subsets(a, kernel_kind(is_real, kPrecF64), sg.wpb, grid, st));
  }
  HAF_CUDA(launch_finalize(partials, job_begin, 1, d_out, st));
  return HAF_OK;
}
