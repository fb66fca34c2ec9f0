"""Continuous-batching server (haf_server_*): results are the same alone
and in the mix, large-n jobs interleave with small ones, the resident
kernel idles out and is relaunched, and bad calls fail cleanly."""
import time

import numpy as np
import pytest

import oracle
import paper_1805_12498_gb300 as hg
from paper_1805_12498_gb300 import inputs

from golden import cases as golden_cases

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _mix(seed=11):
    """36 GBS requests with n in {2, ..., 28} (a few odd), haf/lhaf
    alternating, and one complex Gaussian n = 34 haf (tests/golden/cases.py)."""
    return golden_cases.server_mix(seed)


def _oracle_values(reqs, seed=11):
    """Oracle (value, sum |f|) of every request: at test time up to the
    evaluated size 24, the stored binary128 sums above it."""
    stored = {k for k, _, _ in golden_cases.server_mix_stored(seed)}
    out = []
    for k, (M, loops) in enumerate(reqs):
        n = M.shape[0]
        if golden_cases.evaluated_size(n, loops) == 0:
            out.append((0j if n else 1 + 0j, 0.0 if n else 1.0))
        elif k in stored:
            out.append(golden_cases.stored(f"server{seed}_req{k}"))
        else:
            out.append(oracle.haf_formula(golden_cases.pad_odd(M), loops))
    return out


def test_results_same_alone_and_in_the_mix():
    """Every request of the mix, served alone and in the mix, against the
    oracle (1e-10 sum |f|); the two results bit-identical."""
    reqs = _mix()
    with hg.Server() as srv:
        alone = []
        for M, loops in reqs:
            t = srv.submit(M, loops)
            alone.append(srv.poll(t, timeout_s=120))
        tickets = [srv.submit(M, loops) for M, loops in reqs]
        mixed = [srv.poll(t, timeout_s=120) for t in tickets]
    for k, ((M, loops), a, b, (want, scale)) in enumerate(zip(reqs, alone, mixed, _oracle_values(reqs))):
        scale = max(scale, 1e-300)
        assert abs(a.value - want) <= TOL * scale, ("alone", k, M.shape[0], loops, a.value, want)
        assert abs(b.value - want) <= TOL * scale, ("mixed", k, M.shape[0], loops, b.value, want)
        assert a.value == b.value and a.abs_sum == b.abs_sum  # bit-identical


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
    for M, r in zip(smalls, rs):
        want, scale = oracle.haf_formula(M)
        assert abs(r.value - want) <= TOL * scale


def test_idle_exit_and_relaunch():
    A = inputs.complex_gaussian_symmetric(16, 9)
    want, scale = oracle.haf_formula(A)
    with hg.Server(idle_us=2000) as srv:
        for _ in range(3):
            r = srv.poll(srv.submit(A), timeout_s=30)
            assert abs(r.value - want) <= TOL * scale
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
    # the first n = 40 matrix is the stored oracle case cgauss40_haf
    mats = [inputs.complex_gaussian_symmetric(40, 40)] + [inputs.complex_gaussian_symmetric(40, 20 + k)
                                                          for k in range(2)]
    smalls = [inputs.complex_gaussian_symmetric(10, 30 + k) for k in range(20)]
    with hg.Server(ring_entries=65536, chunk_us=1000) as srv:
        ts = [srv.submit(M) for M in mats]
        ts += [srv.submit(M, True) for M in smalls]
        rs = [srv.poll(t, timeout_s=120) for t in ts]
    want, scale = golden_cases.stored("cgauss40_haf")
    assert abs(rs[0].value - want) <= TOL * scale, (rs[0].value, want, scale)
    for M, r in zip(mats[1:], rs[1:3]):
        ref = hg.haf_info(M)
        assert abs(r.value - ref.value) <= TOL * ref.abs_sum
    for M, r in zip(smalls, rs[3:]):
        want, scale = oracle.haf_formula(M, True)
        assert abs(r.value - want) <= TOL * scale
