"""Continuous-batching server (haf_server_*): results are the same alone
and in the mix, large-n jobs interleave with small ones, the resident
kernel idles out and is relaunched, and bad calls fail cleanly."""
import time

import numpy as np
import pytest

import oracle
import paper_1805_12498_gb300 as hg
from paper_1805_12498_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _mix(seed=11):
    B = inputs.gbs_kernel(32, 0.88, seed)
    g = inputs.rng(seed + 1)
    reqs = []
    for k in range(36):
        n = int(g.choice([2, 6, 8, 10, 12, 16, 20, 24, 28])) + (1 if k % 9 == 4 else 0)  # a few odd n
        M = inputs.repeat_submatrix(B, inputs.click_pattern(n, 32, g))
        reqs.append((M, bool(k % 2)))
    reqs.append((inputs.complex_gaussian_symmetric(34, seed + 2), False))
    return reqs


def test_results_same_alone_and_in_the_mix():
    reqs = _mix()
    with hg.Server() as srv:
        alone = []
        for M, loops in reqs:
            t = srv.submit(M, loops)
            alone.append(srv.poll(t, timeout_s=120))
        tickets = [srv.submit(M, loops) for M, loops in reqs]
        mixed = [srv.poll(t, timeout_s=120) for t in tickets]
    for k, ((M, loops), a, b) in enumerate(zip(reqs, alone, mixed)):
        ref = hg.haf_info(M, loops)
        scale = max(ref.abs_sum, 1e-300)
        assert abs(a.value - ref.value) <= TOL * scale, ("alone", k, M.shape[0], loops, a.value, ref.value)
        assert abs(b.value - ref.value) <= TOL * scale, ("mixed", k, M.shape[0], loops, b.value, ref.value)
        assert a.value == b.value and a.abs_sum == b.abs_sum  # bit-identical
    # a sample against the oracle
    for (M, loops), b in list(zip(reqs, mixed))[:8]:
        if M.shape[0] <= 16 and M.shape[0] % 2 == 0:
            want, scale = oracle.haf_formula(M, loops)
            assert abs(b.value - want) <= TOL * max(scale, 1e-300)


def test_small_jobs_overtake_a_large_one():
    """Small requests that arrive while a large one runs are admitted at
    once and finish long before it (its chunks interleave with theirs)."""
    big = inputs.complex_gaussian_symmetric(44, 3)  # about a second of GPU time
    smalls = [inputs.complex_gaussian_symmetric(12, 100 + k) for k in range(16)]
    with hg.Server() as srv:
        tb = srv.submit(big)
        time.sleep(0.05)
        ts = [srv.submit(M) for M in smalls]
        rs = [srv.poll(t, timeout_s=60) for t in ts]
        rb = srv.poll(tb, timeout_s=120)
    assert max(r.seconds for r in rs) < 0.25 * rb.seconds, ([r.seconds for r in rs], rb.seconds)
    ref = hg.haf_info(big)
    assert abs(rb.value - ref.value) <= TOL * ref.abs_sum


def test_idle_exit_and_relaunch():
    A = inputs.complex_gaussian_symmetric(16, 9)
    ref = hg.haf_info(A)
    with hg.Server(idle_us=2000) as srv:
        for _ in range(3):
            r = srv.poll(srv.submit(A), timeout_s=30)
            assert r.value == pytest.approx(ref.value, abs=TOL * ref.abs_sum)
            time.sleep(0.02)  # the resident kernel idles out in between
        assert r.launches >= 2


def test_errors_and_timeouts():
    with hg.Server() as srv:
        with pytest.raises(hg.HafError) as e:
            srv.poll(12345, timeout_s=0)
        assert e.value.code == -6  # unknown ticket
        big = inputs.complex_gaussian_symmetric(40, 4)
        t = srv.submit(big)
        with pytest.raises(hg.HafError) as e:
            srv.poll(t, timeout_s=0)
        assert e.value.code == -4  # not finished yet
        r = srv.poll(t, timeout_s=120)
        assert r.abs_sum > 0
        with pytest.raises(hg.HafError):
            srv.poll(t, timeout_s=0)  # collected already
        assert srv.poll(srv.submit(np.zeros((0, 0))), 1).value == 1
        assert srv.poll(srv.submit(inputs.complex_gaussian_symmetric(5, 1)), 1).value == 0


def test_ring_wraps_around_with_many_chunks():
    """More chunks than ring entries: slots are reused once claimed, and
    jobs whose chunks are published over several wraps still finish."""
    mats = [inputs.complex_gaussian_symmetric(40, 20 + k) for k in range(3)]
    with hg.Server(ring_entries=65536, chunk_us=1000) as srv:
        ts = [srv.submit(M) for M in mats]
        ts += [srv.submit(inputs.complex_gaussian_symmetric(10, 30 + k), True) for k in range(20)]
        rs = [srv.poll(t, timeout_s=120) for t in ts]
    for M, r in zip(mats, rs[:3]):
        ref = hg.haf_info(M)
        assert abs(r.value - ref.value) <= TOL * ref.abs_sum
