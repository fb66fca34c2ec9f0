"""Host-side logic of bench.py, on the CPU: the algorithmic flop count the
roofline divides by, the clock-record summary, the HBM peak lookup, and the
reference arm's JSON line (the oracle timed on the host cores)."""
import json
import os
import subprocess
import sys
from math import comb

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("n", list(range(2, 58, 2)))
def test_alg_flops_is_the_sum_over_subset_sizes(n):
    """(40/3 + 4/3) N^3 real flops per subset of N = 2m rows, summed over
    the C(h, m) subsets of each size, against the closed form."""
    h = n // 2
    direct = sum(comb(h, m) * (44 * (2 * m) ** 3) for m in range(h + 1)) / 3
    assert bench.alg_flops(n) == pytest.approx(direct, rel=1e-15)


def test_alg_flops_at_the_benchmark_size():
    # 2^24 subsets, (44/3) 2^24 24^2 27 = 3.826e12 flops
    assert bench.alg_flops(48) == pytest.approx(3.8268e12, rel=1e-4)


@pytest.mark.parametrize("N,h", [(2, 1), (4, 6), (10, 8), (24, 24), (48, 24)])
def test_lhaf_extra_flops_counts_the_kernels_loops(N, h):
    """The moments' count, by walking the loop structure the kernel runs:
    at step k the rows 0..k-1 of H times a vector supported on its first
    k-1 entries (row 0: k-1 entries, row i >= 1: k-i), then the dot with a;
    Cayley-Hamilton past N; the Krylov-start reflector both sides (4 N^2)
    and the reflectors on a (N^2)."""
    K = min(N, h)
    macs = 4 * N * N + N * N
    for k in range(2, K + 1):
        macs += sum(k - 1 if i == 0 else k - i for i in range(k)) + k
    for k in range(N + 1, h + 1):
        macs += N
    assert bench.lhaf_extra_flops(N, h) == pytest.approx(8 * macs, rel=1e-15)


def test_alg_flops_lhaf_sums_the_subsets():
    n, h = 12, 6
    want = bench.alg_flops(n) + sum(comb(h, m) * bench.lhaf_extra_flops(2 * m, h) for m in range(1, h + 1))
    assert bench.alg_flops_lhaf(n) == pytest.approx(want, rel=1e-15)
    assert 1.15 < bench.alg_flops_lhaf(48) / bench.alg_flops(48) < 1.25


def test_clock_summary():
    s = bench.ClockSampler(0)
    s.samples = [["2070", "2070", "900.1", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
                 ["2055", "2070", "1300.0", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
                 ["1980", "2070", "1390.5", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
                 ["[N/A]"]]
    out = s.summary()
    assert out["sm_mhz"] == 2055 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 4


def test_hbm_peak_is_a_positive_figure():
    assert bench.hbm_peak_gbs() > 1000


def test_reference_arm_prints_the_contract_line():
    env = dict(os.environ, RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "16",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unit"] == "subset-terms/s" and line["higher_is_better"]
    assert line["value"] > 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["metric"] == bench.metric_name(16)


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "16",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=120, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_summary_fields_with_a_fixed_rate_serving_leg():
    """--serve-rate runs the open-loop stream alone: the summary keeps its
    latencies and leaves out the capacity and one-launch fields."""
    line = {"ms_per_step": 1000.0,
            "serving": {"offered_req_per_s": 3.0, "throughput_req_per_s": 2.9, "p50_ms": 12.0, "p99_ms": 900.0,
                        "max_ms": 5000.0}}
    out = bench.summary_fields(line)
    assert out == {"serving_p50_ms": 12.0, "serving_p99_ms": 900.0}
    line["serving"].update({"capacity_vs_one_launch": 1.01, "one_launch_fifo_p50_ms": 100.0,
                            "one_launch_fifo_p99_ms": 2000.0})
    out = bench.summary_fields(line)
    assert out["serving_capacity_vs_one_launch"] == 1.01 and out["one_launch_fifo_p99_ms"] == 2000.0


class _FakeResult:
    def __init__(self, seconds):
        self.seconds = seconds
        self.value = 0j


class _FakeServer:
    """Stands in for hg.Server on the CPU: every request finishes at once
    with a latency of 1 ms."""

    def __init__(self, *a, **k):
        self.n = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def submit(self, M, loops=False):
        self.n += 1
        return self.n

    def poll(self, ticket, timeout_s=None):
        return _FakeResult(0.001)


@pytest.mark.parametrize("rate", [0.0, 500.0])
def test_serving_leg_logic_on_a_fake_server(monkeypatch, rate):
    """Both forms of the serving leg (with the capacity and one-launch runs,
    and the fixed-rate stream alone) run through and report their fields."""
    import paper_1805_12498_gb300 as hg
    monkeypatch.setattr(hg, "Server", _FakeServer)
    monkeypatch.setattr(hg, "haf_info", lambda M, loops=False: _FakeResult(0.0))
    out = bench.serving_leg(24, 12, seed=3, rate=rate)
    assert out["p50_ms"] == pytest.approx(1.0) and out["p99_ms"] == pytest.approx(1.0)
    assert out["throughput_req_per_s"] > 0
    if rate > 0:
        assert out["offered_req_per_s"] == rate and "capacity_req_per_s" not in out
        assert sum(out["jobs_by_n"].values()) == 24
    else:
        assert out["capacity_req_per_s"] > 0 and out["capacity_vs_one_launch"] > 0
        assert out["one_launch_fifo_p99_ms"] >= 0
    json.dumps(out)  # the record is plain JSON
