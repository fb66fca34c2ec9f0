"""Sharding one hafnian over several processes (Sec. 4.1: independent
ranges, one final sum).  Host logic on CPU: the part slices cover every
subset exactly once, and the double-double combine of per-part records is
exact enough; then two gloo ranks each sum their part's oracle terms and
combine.  The GPU test runs every part on one GPU."""
import itertools
import os
import socket
from math import comb

import numpy as np
import pytest

import oracle
import paper_1805_12498_gb300 as hg
from paper_1805_12498_gb300 import inputs


def colex_subsets(h, m):
    """m-subsets of range(h) in colex order, as bitmasks."""
    combs = sorted(itertools.combinations(range(h), m), key=lambda c: tuple(reversed(c)))
    return [sum(1 << i for i in c) for c in combs]


def part_masks(h, part, nparts):
    masks = []
    for m in range(1, h + 1):
        cnt = comb(h, m)
        lo, hi = cnt * part // nparts, cnt * (part + 1) // nparts
        masks.extend(colex_subsets(h, m)[lo:hi])
    return masks


@pytest.mark.parametrize("n", [0, 2, 10, 24, 48, 56])
@pytest.mark.parametrize("nparts", [1, 2, 3, 7, 8])
def test_parts_cover_all_subsets(n, nparts):
    h = n // 2
    total = sum(hg.part_subsets(n, p, nparts) for p in range(nparts))
    assert total == 2 ** h - 1  # every non-empty subset once
    sizes = [hg.part_subsets(n, p, nparts) for p in range(nparts)]
    assert max(sizes) - min(sizes) <= h  # at most one per size class apart


def test_part_slices_match_colex_enumeration():
    h = 7
    for nparts in (2, 3, 5):
        seen = []
        for p in range(nparts):
            masks = part_masks(h, p, nparts)
            assert len(masks) == hg.part_subsets(2 * h, p, nparts)
            seen.extend(masks)
        assert sorted(seen) == list(range(1, 1 << h))


def test_combine_is_fixed_order_double_double():
    """Records whose values cancel: the double-double combine keeps the
    small remainder that a plain double sum loses."""
    from fractions import Fraction
    big = 2.0 ** 60
    recs = np.array([[big, 0, 0, 0, big], [1.0, 0, 0, 0, 1.0], [-big, 0, 0, 0, big]])
    v, s = hg.combine(recs)
    assert v == 1.0  # a plain left-to-right double sum gives 0
    assert s == 2 * big + 1.0
    g = np.random.default_rng(3)
    recs = np.zeros((6, 5))
    recs[:, 0] = g.standard_normal(6) * 1e16
    recs[:, 2] = g.standard_normal(6)  # low parts
    v, _ = hg.combine(recs)
    want = sum(Fraction(float(x)) for x in recs[:, 0]) + sum(Fraction(float(x)) for x in recs[:, 2])
    assert abs(Fraction(v.real) - want) <= abs(want) * Fraction(1, 2 ** 50)
    with pytest.raises(hg.HafError):
        hg.combine(np.zeros((0, 5)))


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, n, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    h = n // 2
    A = inputs.complex_gaussian_symmetric(n, 77)
    masks = np.array(part_masks(h, rank, world), dtype=np.uint64)
    f = oracle.terms(A, False, masks, nthreads=2)
    signs = np.array([(-1) ** (h - bin(int(z)).count("1")) for z in masks])
    t = signs * f
    # this rank's record: value split into double-double (hi, lo) parts
    re, im = float(np.sum(t.real)), float(np.sum(t.imag))
    rec = torch.tensor([re, im, 0.0, 0.0, float(np.sum(np.abs(f)))], dtype=torch.float64)
    out = [torch.zeros(5, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(out, rec)
    recs = torch.stack(out).numpy()
    v, s = hg.combine(recs)
    q.put((rank, v, s, recs))
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_to_the_whole_sum():
    import torch.multiprocessing as mp
    n, world = 14, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want, scale = oracle.haf_formula(inputs.complex_gaussian_symmetric(n, 77))
    for rank, v, s, recs in res:
        assert abs(v - want) <= 1e-12 * scale
        assert s == pytest.approx(scale, rel=1e-12)
    # every rank combines the same records in part order: bit-identical
    # results, equal to a single process combining them in part order
    assert res[0][1] == res[1][1] and res[0][2] == res[1][2]
    v_local, s_local = hg.combine(res[0][3])
    assert v_local == res[0][1] and s_local == res[0][2]


@pytest.mark.gpu
@pytest.mark.parametrize("n,loops", [(24, False), (22, True)])
def test_parts_on_one_gpu_combine_to_single_call(n, loops):
    A = inputs.complex_gaussian_symmetric(n, 88)
    whole = hg.haf_info(A, loops)
    for nparts in (2, 3, 5):
        recs = [hg.haf_part(A, p, nparts, loops) for p in range(nparts)]
        v, s = hg.combine(recs)
        assert abs(v - whole.value) <= 1e-10 * whole.abs_sum
        assert s == pytest.approx(whole.abs_sum, rel=1e-9)


@pytest.mark.gpu
def test_bench_shard_path_matches_single_call(capsys):
    """bench.py --shard at one rank: the sharded path (part records and the
    combine) gives the single call's value."""
    import argparse
    import json
    import sys

    import torch
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    args = argparse.Namespace(n=24, seed=5, steps=1, warmup=1)
    bench.run_shard(args, hg, inputs, torch, None, 1, 0, torch.device("cuda", 0))
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    whole = hg.haf_info(inputs.complex_gaussian_symmetric(24, 5))
    got = complex(line["result"]["re"], line["result"]["im"])
    assert abs(got - whole.value) <= 1e-10 * whole.abs_sum
    assert line["scaling"] == "strong" and line["n_gpus"] == 1
