"""Host-side work plan (haf_plan_stats, no GPU): every subset is planned
exactly once, and size classes whose tiles do not fit a warp's
shared-memory slice at the requested warps per CTA run in a later launch
with fewer warps per CTA."""
from math import comb

import numpy as np
import pytest

from paper_1805_12498_gb300 import _native

FP32 = _native.HAF_FLAG_FP32
REAL = _native.HAF_FLAG_REAL


def stats(n, flags=0, wpb=4, cpw=8, sms=152):
    out = np.zeros(8, dtype=np.int64)
    _native.check(_native.lib().haf_plan_stats(n, flags, wpb, cpw, sms, out.ctypes.data_as(_native._I64P)))
    return out


@pytest.mark.parametrize("n", [2, 4, 10, 24, 36, 48, 56])
@pytest.mark.parametrize("flags", [0, REAL, FP32, FP32 | REAL, _native.HAF_FLAG_LOOPS])
@pytest.mark.parametrize("wpb", [4, 8, 16])
def test_every_subset_planned_once(n, flags, wpb):
    s = stats(n, flags, wpb)
    nseg = int(s[1])
    assert 1 <= nseg <= 3
    assert s[5:5 + nseg].sum() == 2 ** (n // 2) - 1
    w = list(s[2:2 + nseg])
    assert w == sorted(w, reverse=True) and w[0] <= wpb and all(x in (4, 8, 16) for x in w)


def _r16(b):
    return (b + 15) // 16 * 16


def _fits(N, h, sb, ss, mixed, warp_bytes, loops=False):
    """One subset fits a warp slice (mirror of the planner's rule, written
    from the layout the kernel documents: the N x ld tile, which also holds
    the four power-series arrays once La Budde is done; W, P, TV and, for
    lhaf, VA (b is gathered into P); La Budde's output and, for lhaf, the
    loop moments, which for N >= h + 1 reuse W and P; in the FP32 mode
    their FP64 copies; the pair list)."""
    for ld in (N + 1, N):
        b = _r16(max(N * ld * sb, 4 * (h + 1) * ss))
        if not loops:
            b += 3 * N * sb + (h + 1) * sb
        else:
            b += 4 * N * sb + (0 if N >= h + 1 else 2 * (h + 1) * sb)
        if mixed:
            b = _r16(b) + (2 if loops else 1) * (h + 1) * ss
        b = _r16(_r16(b) + 4 * h)
        if b <= warp_bytes:
            return True
    return False


def test_large_tiles_fall_back_to_fewer_warps():
    # complex128 at n = 48: with 8 warps per CTA (29,056 B per warp) the tiles
    # of |Z| >= 21 (N >= 42) do not fit, so they form a 4-warp launch
    h = 24
    s = stats(48, 0, 8)
    assert int(s[1]) == 2 and list(s[2:4]) == [8, 4]
    big = sum(comb(h, m) for m in range(1, h + 1) if not _fits(2 * m, h, 16, 16, False, 29056))
    assert big == sum(comb(h, m) for m in range(21, h + 1))
    assert s[6] == big and s[5] == 2 ** h - 1 - big
    # the loop hafnian's extra vector (VA) still fits |Z| = 20, because its
    # moments and La Budde's output reuse W and P
    s = stats(48, _native.HAF_FLAG_LOOPS, 8)
    big = sum(comb(h, m) for m in range(1, h + 1) if not _fits(2 * m, h, 16, 16, False, 29056, True))
    assert big == sum(comb(h, m) for m in range(21, h + 1))
    assert s[6] == big
    # with 4 warps per CTA everything fits one launch
    s = stats(48, 0, 4)
    assert int(s[1]) == 1 and s[2] == 4


def test_chunk_granularity_scales_chunk_count():
    a = stats(40, 0, 4, 2)[0]
    b = stats(40, 0, 4, 16)[0]
    assert b > 4 * a


def test_bad_shapes_rejected():
    out = np.zeros(8, dtype=np.int64)
    L = _native.lib()
    assert L.haf_plan_stats(40, 0, 6, 8, 152, out.ctypes.data_as(_native._I64P)) == _native.HAF_EINVAL
    assert L.haf_plan_stats(40, 0, 8, 0, 152, out.ctypes.data_as(_native._I64P)) == _native.HAF_EINVAL
    assert L.haf_plan_stats(41, 0, 8, 8, 152, out.ctypes.data_as(_native._I64P)) == _native.HAF_EINVAL
