"""Benchmark: hafnian subset-terms/s at n = 48 (complex128) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--n 48] [--impl reference]

One step is one complete hafnian of a seeded complex Gaussian symmetric
48 x 48 matrix: all 2^24 subset terms of the signed sum (Sec. 3.2, eq. main),
each by Householder-Hessenberg + La Budde + power series on the GPU.

Printed (rank 0, one JSON line):
  value   subset-terms/s over all ranks, device-resident input, CUDA-event
          timed on the launching stream (L2 flushed between steps);
  e2e     the same metric through the host-pointer C entry point haf_c128,
          pinned host input copied in and the result read back every step;
  roofline  FP64 pipe: algorithmic flops of the step (44/3) 2^h h^2 (h+3)
          over the measured step time, against the FP64 DFMA rate measured
          live on the same GPU by the library's probe kernel;
  cpu_baseline  the binary128 CPU oracle on a bounded sample of the same
          workload's subsets, on the host's cores;
  batched  4096 GBS-shaped submatrices (n even in [8, 32]) in one
          graph-captured launch sequence, against one call per matrix;
  serving  a Poisson stream of haf/lhaf GBS requests through the
          continuous-batching server (capacity, p50/p99), against one
          synchronous call per request (capacity and FIFO latency);
  precision  the FP32-bulk mode against FP64 at n = 40 and 48 (error
          relative to sum |f(Z)| and to |haf|, speed-up);
  lowrank  the App. C expansion at n = 56, r = 4, 6, 8;
  sweep  complex and real haf and lhaf at n = 24, 28, ..., 52, one call each.
The last six legs run at N = 1 only; --no-<leg> flags skip them.
Multi-GPU (torchrun): each rank computes its own hafnian (independent
problems, no collective on the data path): weak scaling.
``--impl reference``: the oracle itself, timed on the host cores (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# DRAM bytes (read + write) of one launch of the dominant subset kernel at
# n = 48, from the one-pass ncu capture of this workload kept under
# profiles/; re-captured whenever the kernel changes.
TRAFFIC_BYTES = {48: 1152000 + 0}


def metric_name(n: int) -> str:
    return f"subset-terms/s (haf, n={n}, complex128)"
UNIT = "subset-terms/s"


def alg_flops(n: int) -> float:
    """Algorithmic FP64 flops of one hafnian: sum over subsets of the
    Householder-Hessenberg (40/3 N^3) + La Budde (4/3 N^3) counts, N = 2|Z|:
    (44/3) sum_m C(h,m) (2m)^3 = (44/3) 2^h h^2 (h+3)."""
    h = n // 2
    return (44.0 / 3.0) * (2 ** h) * h * h * (h + 3)


def lhaf_extra_flops(N: int, h: int) -> float:
    """FP64 flops that a loop-hafnian summand adds to the hafnian's for one
    subset of size N = 2|Z| (Sec. 3.3, q(lambda, B, v)), as the kernels do
    it (a complex multiply-add is 8 flops):
      - the Krylov-start reflector of length N applied to B from both sides:
        4 N^2 multiply-adds;
      - every reflector applied to the vector a: about N^2 multiply-adds;
      - the moments u_k = a H^(k-1) b for k = 2..K, K = min(N, h): the
        Hessenberg product on a vector supported on its first k-1 entries,
        (k-1)(k+2)/2 multiply-adds, and the dot with a, k more;
      - for N < h, Cayley-Hamilton's continuation to u_h: N per moment."""
    K = min(N, h)
    mom = sum((k - 1) * (k + 2) / 2.0 + k for k in range(2, K + 1))
    tail = (h - N) * N if N < h else 0
    return 8.0 * (4 * N * N + N * N + mom + tail)


def alg_flops_lhaf(n: int) -> float:
    """Algorithmic FP64 flops of one loop hafnian: the hafnian's count plus
    lhaf_extra_flops summed over the subsets."""
    from math import comb
    h = n // 2
    return alg_flops(n) + sum(comb(h, m) * lhaf_extra_flops(2 * m, h) for m in range(1, h + 1))


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        sm = [float(s[0]) for s in self.samples if s and s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if len(s) > 1 and s[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            for k, name in enumerate(names):
                if len(s) > 4 + k and s[4 + k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def cpu_baseline(n: int, seed: int, budget_s: float = 12.0):
    """The oracle (binary128, as it stands) on a bounded random sample of
    the workload's subsets; subset-terms/s on the host cores."""
    import oracle
    from paper_1805_12498_gb300 import inputs

    A = inputs.complex_gaussian_symmetric(n, seed)
    h = n // 2
    cores = oracle.default_threads()
    masks = inputs.random_masks(h, cores, seed + 7)
    t = time.perf_counter()
    oracle.terms(A, False, masks, nthreads=cores)
    dt = time.perf_counter() - t
    count = max(cores, int(cores * max(1.0, (budget_s - dt) / max(dt, 1e-3))))
    masks = inputs.random_masks(h, count, seed + 8)
    t = time.perf_counter()
    oracle.terms(A, False, masks, nthreads=cores)
    dt = time.perf_counter() - t
    return {"value": count / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{count} uniformly random subsets of the n={n} seeded complex Gaussian "
                      f"matrix, binary128 trace-power summands, {dt:.1f} s"}


def sweep_leg(seed: int, sizes=(24, 28, 32, 36, 40, 44, 48, 52)):
    """The single-hafnian size sweep: one seeded matrix per size, complex
    (A = (G + G^T)/2, re, im ~ N(0, 1/2)) and real (N(0, 1) entries), haf
    and lhaf, each timed once with CUDA events on the launching stream
    through haf_launch (device-resident input; one untimed warm-up call
    below n = 40, where plan building would show).  The FP64 fraction uses
    the hafnian's and loop hafnian's flop counts, a quarter of them for real
    input (a real multiply-add is 2 flops, a complex one 8)."""
    import torch

    import paper_1805_12498_gb300 as hg
    from paper_1805_12498_gb300 import inputs

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    peak, _ = hg.fp64_peak()
    rows = []
    for n in sizes:
        for real in (False, True):
            A = inputs.real_gaussian_symmetric(n, seed + n) if real else inputs.complex_gaussian_symmetric(n, seed + n)
            dA = torch.from_numpy(np.ascontiguousarray(A).view(np.float64).copy()).to(dev)
            for loops in (False, True):
                ws = hg.workspace_bytes(n, loops=loops, real=real)
                work = torch.empty(ws // 8 + 64, dtype=torch.float64, device=dev)
                wptr = (work.data_ptr() + 255) // 256 * 256
                out = torch.zeros(5, dtype=torch.float64, device=dev)

                def launch():
                    hg.haf_launch(dA.data_ptr(), n, out.data_ptr(), wptr, ws, stream.cuda_stream, loops=loops,
                                  real=real)

                if n < 40:
                    launch()
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                launch()
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ms = e0.elapsed_time(e1)
                flops = (alg_flops_lhaf(n) if loops else alg_flops(n)) / (4.0 if real else 1.0)
                rec = out.cpu().numpy()
                rows.append({"n": n, "dtype": "f64" if real else "c128", "loops": loops, "ms": ms,
                             "subset_terms_per_s": 2 ** (n // 2) / (ms * 1e-3),
                             "fp64_frac": flops / (ms * 1e-3) / 1e12 / peak, "abs_sum": float(rec[4])})
                del work
    return {"workload": "one seeded complex and one real Gaussian symmetric matrix per size n = "
                        + ",".join(str(n) for n in sizes) + "; haf and lhaf; haf_launch, CUDA events, one call each",
            "peak_tflops": peak, "rows": rows}


def batched_leg(count: int, seed: int, reps: int = 3):
    """GBS-shaped batch: ``count`` submatrices of a 32-mode kernel
    B = U diag(tanh 0.88) U^T with total photons uniform on even n in
    [8, 32], in one graph-captured persistent launch, against one launch per
    hafnian through the host entry point; both on this GPU."""
    import paper_1805_12498_gb300 as hg
    from paper_1805_12498_gb300 import inputs

    _, mats = inputs.gbs_batch(count, seed)
    sizes = [M.shape[0] for M in mats]
    hg.haf_batched(mats)  # plan + graph
    t = time.perf_counter()
    for _ in range(reps):
        vals, infos = hg.haf_batched(mats, with_info=True)
    t_b = (time.perf_counter() - t) / reps
    singles = [hg.haf_info(M) for M in mats[:8]]  # warm the per-size plans
    for nn in sorted(set(sizes)):
        hg.haf_info(mats[sizes.index(nn)])
    t = time.perf_counter()
    singles = [hg.haf_info(M) for M in mats]
    t_s = time.perf_counter() - t
    worst = max(abs(v - s.value) / max(s.abs_sum, 1e-300) for v, s in zip(vals, singles))
    subsets = sum(2 ** (nn // 2) for nn in sizes)
    flops = sum(alg_flops(nn) for nn in sizes)
    peak, _ = hg.fp64_peak()
    return {"workload": f"{count} GBS submatrices (32 modes, r=0.88, n uniform on even 8..32), complex128",
            "haf_per_s": count / t_b, "subset_terms_per_s": subsets / t_b, "s_per_batch": t_b,
            "one_launch_per_haf_per_s": count / t_s, "speedup_vs_one_launch_per_haf": t_s / t_b,
            "max_abs_diff_over_abs_sum_vs_single": worst, "timing": "host clock, synchronous calls",
            "roofline": {"bound": "alu", "achieved": flops / t_b / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops / t_b / 1e12 / peak,
                         "note": "(44/3) 2^h h^2 (h+3) flops summed over the batch / host-clock batch time "
                                 "(includes the H2D/D2H copies of the graph); peak = DFMA probe (of measured)"}}


def precision_leg(seed: int, value48=None):
    """Precision study: FP32-bulk mode against FP64 at n = 16, 40 and 48 on a
    complex Gaussian matrix and on a GBS submatrix (haf).  Errors of the
    values relative to abs_sum = sum_Z |f(Z)| (the stated per-unit error) and
    to |haf|; the accuracy gate's decision (admitted when the estimate
    HAF_FP32_REL_TOL * abs_sum / |value| <= HAF_FP32_MAX_REL_ERR, else
    refused with HAF_EACCURACY); sampled summands of the two modes against
    each other (the tests pin both to the binary128 oracle)."""
    import paper_1805_12498_gb300 as hg
    from paper_1805_12498_gb300 import inputs

    def fp32(A):
        try:
            return hg.haf_info(A, precision="fp32"), True
        except hg.HafAccuracyError as e:
            return e.result, False

    rows = []
    for kind in ("gauss", "gbs"):
        for n in (16, 40, 48):
            if kind == "gauss":
                A = inputs.complex_gaussian_symmetric(n, seed if n == 48 else seed + n)
            else:
                B = inputs.gbs_kernel(32, 0.88, seed + n)
                A = inputs.repeat_submatrix(B, inputs.click_pattern(n, 32, inputs.rng(seed + n + 7)))
            if kind == "gauss" and n == 48 and value48 is not None:
                v64, a64, t64 = value48
            else:
                t = time.perf_counter()
                r = hg.haf_info(A)
                v64, a64, t64 = r.value, r.abs_sum, time.perf_counter() - t
            fp32(A)
            t = time.perf_counter()
            r32, admitted = fp32(A)
            t32 = time.perf_counter() - t
            d = abs(r32.value - v64)
            masks = inputs.random_masks(n // 2, 1024, seed=seed + n)
            masks = masks[masks != 0]  # the empty subset's term is 0
            f64 = hg.haf_terms(A, masks)
            rel = np.abs(hg.haf_terms(A, masks, precision="fp32") - f64) / np.abs(f64)
            rows.append({"input": kind, "n": n, "err_over_abs_sum": d / a64,
                         "err_over_abs_value": d / max(abs(v64), 1e-300), "abs_value_over_abs_sum": abs(v64) / a64,
                         "rel_err_bound": r32.rel_err_bound, "admitted": admitted,
                         "s_fp64": t64, "s_fp32": t32, "speedup": t64 / t32,
                         "term_rel_err_median": float(np.median(rel)), "term_rel_err_max": float(rel.max())})
    return {"workload": "haf, n = 16, 40 and 48, complex Gaussian symmetric and GBS submatrix of a 32-mode kernel "
                        "(r = 0.88); FP32 bulk (single-precision Householder + La Budde) vs FP64; 1024 sampled "
                        "summands per case",
            "stated_tol_over_abs_sum": hg.HAF_FP32_REL_TOL, "max_rel_err": hg.HAF_FP32_MAX_REL_ERR, "rows": rows}


def lowrank_leg(seed: int):
    """Low-rank hafnian (App. C expansion) at n = 56 for ranks 4, 6, 8.  The
    step kernels are bound by the FP64 pipe (5 DFMA per term), so the
    roofline is against the DFMA probe.  The device leg times
    haf_lowrank_launch (G, workspace and result in device
    memory; the n + 3 launches of one expansion) with CUDA events on the
    launching stream; the host leg times the synchronous haf_lowrank call
    (G from host memory, the result read back, the workspace allocated and
    freed inside the call above 256 MB).  The expansion processes
    C(k+r-1, r-1) monomials at each degree k = 1..n."""
    import math

    import torch

    import paper_1805_12498_gb300 as hg
    from paper_1805_12498_gb300 import inputs

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    peak_tflops, _ = hg.fp64_peak()
    rows = []
    for n, r in ((56, 4), (56, 6), (56, 8)):
        g = inputs.rng(seed + 100 * r + n)
        G = (g.normal(size=(n, r)) + 1j * g.normal(size=(n, r))) / np.sqrt(2 * r)
        ws = hg.lowrank_workspace_bytes(n, r)
        work = torch.empty(ws // 8 + 64, dtype=torch.float64, device=dev)
        wptr = (work.data_ptr() + 255) // 256 * 256
        dG = torch.from_numpy(G.view(np.float64).copy()).to(dev)
        out = torch.zeros(5, dtype=torch.float64, device=dev)

        def launch():
            hg.haf_lowrank_launch(dG.data_ptr(), n, r, out.data_ptr(), wptr, ws, stream.cuda_stream)

        launch()
        torch.cuda.synchronize(dev)
        reps = 3
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            a.record(stream)
            launch()
            b.record(stream)
        torch.cuda.synchronize(dev)
        ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
        rec = out.cpu().numpy()
        del work
        torch.cuda.empty_cache()
        t = time.perf_counter()
        a = hg.haf_lowrank(G)
        dt = time.perf_counter() - t
        same = complex(rec[0] + rec[2], rec[1] + rec[3]) == a.value
        mono = sum(math.comb(k + r - 1, r - 1) for k in range(1, n + 1))
        # algorithmic work: at degree k every monomial e takes one term per
        # j with e_j >= 1, i.e. r * C(k-1+r-1, r-1) terms in all; a term is a
        # complex multiply-add and a real one (|g| recurrence): 10 flops
        flops = 10.0 * r * math.comb(n - 1 + r, r)
        # minimal traffic: every degree-k array (24 B per monomial: value + abs) written once, read once
        traffic = 2 * 24 * mono
        tf = flops / (ms / 1e3) / 1e12
        rows.append({"n": n, "r": r, "ms_device": ms, "monomials_per_s": mono / (ms / 1e3),
                     "s_host_call": dt, "host_equals_device": bool(same), "abs_sum": a.abs_sum,
                     "hbm_alg_gbs": traffic / (ms / 1e3) / 1e9,
                     "roofline": {"bound": "alu", "achieved": tf, "peak": peak_tflops, "unit": "TFLOP/s",
                                  "frac": tf / peak_tflops,
                                  "note": "FP64 pipe: 10 flops (5 DFMA) per term, r * C(n-1+r, r) terms per "
                                          "expansion, / CUDA-event time of the n + 3 launches; peak = DFMA probe "
                                          "measured in this run (of measured). hbm_alg_gbs = 48 B per monomial "
                                          "(each degree array written once, read once) over the same time"}})
    return {"workload": "haf(G G^T), G complex Gaussian n x r, App. C expansion on the GPU", "rows": rows}


def hbm_peak_gbs() -> float:
    """Measured HBM copy bandwidth of this machine's GB300 (MEASURED_PEAKS.json),
    else the recipe's fallback figure."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def serving_leg(requests: int, n_max: int, seed: int, load: float = 0.7, rate: float = 0.0):
    """Serving: haf/lhaf requests (50/50) on GBS
    submatrices, n even in [8, n_max] with P(n) proportional to 2^(-n/8),
    through the continuous-batching server.  The capacity is measured first
    with all requests submitted at once; the open-loop run then offers
    Poisson arrivals at `load` x capacity and reports throughput and the
    p50/p99 of the submit-to-result latency the server records.  With
    rate > 0 (requests/s) the open-loop run alone is made at that rate:
    no capacity run and no one-launch comparison, for long streams."""
    import threading as th

    import paper_1805_12498_gb300 as hg
    from paper_1805_12498_gb300 import inputs

    B = inputs.gbs_kernel(32, 0.88, seed)
    g = inputs.rng(seed + 3)
    ns = np.arange(8, n_max + 1, 2)
    w = 2.0 ** (-ns / 8.0)
    reqs = []
    for _ in range(requests):
        n = int(g.choice(ns, p=w / w.sum()))
        reqs.append((inputs.repeat_submatrix(B, inputs.click_pattern(n, 32, g)), bool(g.integers(0, 2))))
    with hg.Server() as srv:
        for M, loops in reqs[:16]:  # warm the resident kernel and the plans
            srv.poll(srv.submit(M, loops), timeout_s=3600)
        capacity = None
        if rate <= 0:
            t = time.perf_counter()
            tickets = [srv.submit(M, loops) for M, loops in reqs]
            for tk in tickets:
                srv.poll(tk, timeout_s=3600)
            capacity = requests / (time.perf_counter() - t)
            rate = load * capacity
        gaps = g.exponential(1.0 / rate, size=requests)
        submitted = []
        lock = th.Lock()

        def submitter():
            t_next = time.perf_counter()
            for (M, loops), gap in zip(reqs, gaps):
                t_next += gap
                d = t_next - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                tk = srv.submit(M, loops)
                with lock:
                    submitted.append(tk)

        thr = th.Thread(target=submitter)
        t0 = time.perf_counter()
        thr.start()
        lat = []
        k = 0
        while k < requests:
            with lock:
                ready = k < len(submitted)
                tk = submitted[k] if ready else None
            if not ready:
                time.sleep(0.0005)
                continue
            lat.append(srv.poll(tk, timeout_s=3600).seconds)
            k += 1
        thr.join()
        wall = time.perf_counter() - t0
    lat = np.array(lat) * 1e3
    if capacity is None:
        return {"workload": f"{requests} requests, haf/lhaf 50/50, GBS submatrices of a 32-mode kernel (r=0.88), "
                            f"n even in [8,{n_max}], P(n) ~ 2^(-n/8), Poisson arrivals at {rate:g} req/s",
                "offered_req_per_s": rate, "throughput_req_per_s": requests / wall,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "max_ms": float(lat.max()), "jobs_by_n": {int(k): int(v) for k, v in
                                                         zip(*np.unique([M.shape[0] for M, _ in reqs],
                                                                        return_counts=True))}}
    # the same requests, one synchronous single-matrix call each (the plain
    # one-launch-per-hafnian form) on the same GPU: its capacity, and its
    # latency under the same Poisson arrivals with one FIFO worker
    t = time.perf_counter()
    for M, loops in reqs:
        hg.haf_info(M, loops)
    single = requests / (time.perf_counter() - t)
    import queue
    q: "queue.Queue" = queue.Queue()

    def arrivals():
        t_next = time.perf_counter()
        for (M, loops), gap in zip(reqs, gaps):
            t_next += gap
            d = t_next - time.perf_counter()
            if d > 0:
                time.sleep(d)
            q.put((time.perf_counter(), M, loops))

    thr = th.Thread(target=arrivals)
    thr.start()
    fifo = []
    for _ in range(requests):
        t_arr, M, loops = q.get()
        hg.haf_info(M, loops)
        fifo.append(time.perf_counter() - t_arr)
    thr.join()
    fifo = np.array(fifo) * 1e3
    return {"workload": f"{requests} requests, haf/lhaf 50/50, GBS submatrices of a 32-mode kernel (r=0.88), "
                        f"n even in [8,{n_max}], P(n) ~ 2^(-n/8), Poisson arrivals at {load:g} x capacity",
            "capacity_req_per_s": capacity, "offered_req_per_s": rate, "throughput_req_per_s": requests / wall,
            "one_launch_per_request_req_per_s": single, "capacity_vs_one_launch": capacity / single,
            "one_launch_fifo_p50_ms": float(np.percentile(fifo, 50)),
            "one_launch_fifo_p99_ms": float(np.percentile(fifo, 99)),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max())}


def lhaf_leg(hg, torch, dA, n, stream, flush, steps: int, peak: float):
    """Loop hafnian of the same matrix (its diagonal kept), device-resident
    and CUDA-event timed on the launching stream like the headline (L2 flushed
    between steps); roofline against the lhaf algorithmic flop count."""
    dev = dA.device
    ws = hg.workspace_bytes(n, loops=True)
    work = torch.empty(ws // 8 + 64, dtype=torch.float64, device=dev)
    wptr = (work.data_ptr() + 255) // 256 * 256
    out = torch.zeros(5, dtype=torch.float64, device=dev)

    def step():
        hg.haf_launch(dA.data_ptr(), n, out.data_ptr(), wptr, ws, stream.cuda_stream, loops=True)

    step()
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    achieved = alg_flops_lhaf(n) / (ms * 1e-3) / 1e12
    return {"workload": f"lhaf of the same {n}x{n} matrix (diagonal kept), 2^{n // 2} subset terms",
            "ms_per_step": ms, "steps": steps, "subset_terms_per_s": 2 ** (n // 2) / (ms * 1e-3),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "note": "haf flops + per subset the Krylov-start reflector, the reflectors on a, "
                                 "the sparse moments and the Cayley-Hamilton tail (lhaf_extra_flops); "
                                 "CUDA-event time; peak = DFMA probe (of measured)"}}


def summary_fields(line: dict) -> dict:
    """Short top-level scalars of the side legs, so that a record that keeps
    only the line's first keys still has them."""
    out = {}
    if "lhaf" in line:
        out["lhaf_ms_per_step"] = line["lhaf"]["ms_per_step"]
        out["lhaf_over_haf"] = line["lhaf"]["ms_per_step"] / line["ms_per_step"]
        out["lhaf_roofline_frac"] = line["lhaf"]["roofline"]["frac"]
    if "batched" in line:
        out["batched_haf_per_s"] = line["batched"]["haf_per_s"]
        out["batched_speedup_vs_one_launch_per_haf"] = line["batched"]["speedup_vs_one_launch_per_haf"]
    if "serving" in line:
        sv = line["serving"]
        if "capacity_vs_one_launch" in sv:
            out["serving_capacity_vs_one_launch"] = sv["capacity_vs_one_launch"]
        out["serving_p50_ms"] = sv["p50_ms"]
        out["serving_p99_ms"] = sv["p99_ms"]
        if "one_launch_fifo_p50_ms" in sv:
            out["one_launch_fifo_p50_ms"] = sv["one_launch_fifo_p50_ms"]
            out["one_launch_fifo_p99_ms"] = sv["one_launch_fifo_p99_ms"]
    if "sweep" in line:
        for row in line["sweep"]["rows"]:
            if row["n"] == max(r["n"] for r in line["sweep"]["rows"]) and row["dtype"] == "c128":
                out[f"sweep_c128_n{row['n']}_{'lhaf' if row['loops'] else 'haf'}_s"] = row["ms"] / 1e3
    if "lowrank" in line:
        last = line["lowrank"]["rows"][-1]
        out[f"lowrank_r{last['r']}_ms"] = last["ms_device"]
        out[f"lowrank_r{last['r']}_fp64_frac"] = last["roofline"]["frac"]
    return out


def run_shard(args, hg, inputs, torch, dist, world: int, rank: int, dev):
    """One hafnian split over the ranks: rank p evaluates part p of `world`
    of every size class of the subset sum (haf_part, host pointers), the
    40-byte part records are gathered and combined in part order on rank 0
    (haf_combine).  Strong scaling: the work per step is one hafnian."""
    n, h = args.n, args.n // 2
    A = inputs.complex_gaussian_symmetric(n, args.seed)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(max(1, args.warmup)):
        hg.haf_part(A, rank, world)
    times, value, abs_sum, launches = [], None, None, 0
    for _ in range(args.steps):
        barrier()
        t0 = time.perf_counter()
        rec, info = hg.haf_part(A, rank, world, with_info=True)
        launches += int(info.launches)
        t = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device=dev)
        recs = torch.tensor(rec, dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            gathered = [torch.zeros_like(recs) for _ in range(world)]
            dist.all_gather(gathered, recs)
            allrec = torch.stack(gathered).cpu().numpy()
        else:
            allrec = recs.cpu().numpy()[None, :]
        value, abs_sum = hg.combine(allrec)
        times.append(float(t[0]))
    barrier()
    s_step = statistics.mean(times)
    if rank == 0:
        achieved = alg_flops(n) / s_step / 1e12
        peak, _ = hg.fp64_peak()
        line = {"metric": f"subset-terms/s (one haf sharded over ranks, n={n}, complex128)",
                "value": 2 ** h / s_step, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": s_step * 1e3, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                "dtype": "f64 (complex128, double-double subset sum)", "data": "synthetic",
                "config": {"workload": f"haf of one seeded complex Gaussian symmetric {n}x{n} matrix split into "
                                       f"{world} subset-range parts (one per rank), part records combined on rank 0",
                           "n": n, "l2": "inputs far below L2; each step is seconds of FP64 work",
                           "parallelism": f"subset-range shards x{world}"},
                "result": {"re": value.real, "im": value.imag, "abs_sum": abs_sum},
                "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak / world,
                             "note": "per-GPU fraction: (44/3) 2^h h^2 (h+3) flops / (host-clock step time x ranks); "
                                     "peak = DFMA probe of rank 0 (of measured)"},
                "e2e": {"value": 2 ** h / s_step, "unit": UNIT, "h2d_bytes_per_step": world * n * n * 16,
                        "d2h_bytes_per_step": world * 40},
                "gpu_launches": launches}
        print(json.dumps(line), flush=True)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    base = cpu_baseline(args.n, args.seed, budget_s=max(5.0, 20.0 / max(1, args.steps + args.warmup)))
    vals = []
    for _ in range(args.steps):
        b = cpu_baseline(args.n, args.seed, budget_s=max(5.0, 60.0 / max(1, args.steps)))
        vals.append(b["value"])
    value = statistics.mean(vals) if vals else base["value"]
    line = {"impl": "reference", "metric": metric_name(args.n), "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f128 (binary128, CPU oracle)", "data": "synthetic",
            "config": {"workload": f"haf of one seeded complex Gaussian symmetric {args.n}x{args.n} matrix "
                                   f"(2^{args.n // 2} subset terms); bounded subset sample on the host"},
            "cpu_baseline": {**base, "value": value},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--n", type=int, default=48)
    ap.add_argument("--seed", type=int, default=48)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--gbs-batch", type=int, default=4096,
                    help="GBS-shaped batch size for the batched leg (0 skips it)")
    ap.add_argument("--serve-requests", type=int, default=300,
                    help="requests in the serving leg (0 skips it)")
    ap.add_argument("--serve-nmax", type=int, default=52,
                    help="largest n of the serving mix (n even in [8, nmax], P(n) ~ 2^(-n/8))")
    ap.add_argument("--no-precision", action="store_true", help="skip the FP32-vs-FP64 precision leg")
    ap.add_argument("--no-lhaf", action="store_true", help="skip the loop-hafnian leg")
    ap.add_argument("--no-lowrank", action="store_true", help="skip the low-rank (App. C) leg")
    ap.add_argument("--serve-rate", type=float, default=0.0,
                    help="serving leg: offer this many requests/s and skip the capacity and one-launch runs")
    ap.add_argument("--no-sweep", action="store_true", help="skip the n = 24..52 size sweep")
    ap.add_argument("--sweep-sizes", default="24,28,32,36,40,44,48,52",
                    help="sizes of the sweep leg (n = 56 adds about six minutes)")
    ap.add_argument("--shard", action="store_true",
                    help="split ONE hafnian of size --n over the ranks (strong scaling) instead of one per rank")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import paper_1805_12498_gb300 as hg
    from paper_1805_12498_gb300 import inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    if args.shard:
        run_shard(args, hg, inputs, torch, dist, world, rank, dev)
        if world > 1:
            dist.destroy_process_group()
        return

    n, h = args.n, args.n // 2
    A = inputs.complex_gaussian_symmetric(n, args.seed + rank)
    dA = torch.from_numpy(A.view(np.float64).copy()).to(dev)
    ws = hg.workspace_bytes(n)
    work = torch.empty(ws // 8 + 64, dtype=torch.float64, device=dev)
    wptr = (work.data_ptr() + 255) // 256 * 256
    out = torch.zeros(5, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)

    def step():
        hg.haf_launch(dA.data_ptr(), n, out.data_ptr(), wptr, ws, stream.cuda_stream)

    peak_tflops, _ = hg.fp64_peak()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # device-resident timed region: one event pair per step on the launching stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clocks:
        barrier()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    ms_step = statistics.mean(ms)
    res = out.cpu().numpy()

    # end to end through the host-pointer entry point (pinned input, result read back)
    pinned = torch.from_numpy(A.view(np.float64).copy()).pin_memory()
    import ctypes
    from paper_1805_12498_gb300 import _native
    L = _native.lib()
    host_out = np.zeros(2)
    info = _native.HafInfo()
    L.haf_c128(ctypes.cast(pinned.data_ptr(), _native._DP), n, host_out.ctypes.data_as(_native._DP),
               ctypes.byref(info))
    launches_per_step = int(info.launches)  # prep + subset-kernel launches + finalize
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _native.check(L.haf_c128(ctypes.cast(pinned.data_ptr(), _native._DP), n,
                                 host_out.ctypes.data_as(_native._DP), ctypes.byref(info)))
    t_e2e = (time.perf_counter() - t0) / args.steps
    barrier()

    # max over ranks
    t_dev = torch.tensor([ms_step, t_e2e], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_dev, op=dist.ReduceOp.MAX)
    ms_step, t_e2e = float(t_dev[0]), float(t_dev[1])
    subsets = 2 ** h
    value = world * subsets / (ms_step * 1e-3)
    e2e = world * subsets / t_e2e
    achieved = alg_flops(n) / (ms_step * 1e-3) / 1e12
    if rank == 0:
        line = {
            "metric": metric_name(n), "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (complex128, double-double subset sum)", "data": "synthetic",
            "config": {"workload": f"haf of one seeded complex Gaussian symmetric {n}x{n} matrix per GPU "
                                   f"(A=(G+G^T)/2, re,im ~ N(0,1/2)); 2^{h} subset terms per step",
                       "n": n, "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": f"independent problems x{world}"},
            "result": {"re": float(res[0] + res[2]), "im": float(res[1] + res[3]), "abs_sum": float(res[4])},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                         "frac": achieved / peak_tflops, "traffic": TRAFFIC_BYTES.get(n),
                         "note": "FP64 pipe; peak = DFMA probe measured in this run (of measured); achieved = "
                                 "(44/3) 2^h h^2 (h+3) flops per step / CUDA-event step time; a step is the "
                                 f"{launches_per_step} launches of one haf_launch (prep, subset-kernel launches, "
                                 "finalize), the subset kernel >99.9% of it; traffic = ncu DRAM bytes of "
                                 "one launch of the dominant subset kernel (profiles/)"},
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": n * n * 16,
                    "d2h_bytes_per_step": 5 * 8},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks.summary(),
        }
        # the single-GPU legs run at N = 1 only (a scaling run reports the
        # headline metric alone)
        if not args.no_lhaf and world == 1:
            line["lhaf"] = lhaf_leg(hg, torch, dA, n, stream, flush, max(2, min(args.steps, 5)), peak_tflops)
        if args.gbs_batch > 0 and world == 1:
            line["batched"] = batched_leg(args.gbs_batch, args.seed)
        if args.serve_requests > 0 and world == 1:
            line["serving"] = serving_leg(args.serve_requests, args.serve_nmax, args.seed, rate=args.serve_rate)
        if not args.no_lowrank and world == 1:
            line["lowrank"] = lowrank_leg(args.seed)
        if not args.no_sweep and world == 1:
            line["sweep"] = sweep_leg(args.seed, tuple(int(x) for x in args.sweep_sizes.split(",")))
        if not args.no_precision and world == 1:
            line["precision"] = precision_leg(args.seed, (complex(res[0] + res[2], res[1] + res[3]), float(res[4]),
                                                          ms_step * 1e-3))
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(n, args.seed)
        summary = summary_fields(line)
        # scalars first, after the contract's keys; the large leg objects last
        legs = {k: line.pop(k) for k in ("lhaf", "batched", "serving", "lowrank", "sweep", "precision") if k in line}
        line.update(summary)
        line.update(legs)
        print(json.dumps(line), flush=True)
        sys.stderr.write("summary: " + json.dumps({"value": value, "ms_per_step": ms_step,
                                                   "roofline_frac": line["roofline"]["frac"], **summary}) + "\n")
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
