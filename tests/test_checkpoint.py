"""Checkpoint/resume of a hafnian evaluated part by part.  The CPU tests
replace the GPU part evaluator with a fake (a worker that returns fixed
records, raises, or returns garbage); the host-only combine and subset
counts are the library's own.  The GPU test resumes a real run."""
import json
import os
import shutil

import numpy as np
import pytest

import paper_1805_12498_gb300 as hg
from paper_1805_12498_gb300 import checkpoint, inputs


SCRATCH = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_build", "test_checkpoint")


@pytest.fixture
def scratch(request):
    """A scratch directory inside the repository's git-ignored build folder
    (removed afterwards), so the tests write nothing outside the tree."""
    d = os.path.join(SCRATCH, request.node.name.replace("[", "_").replace("]", ""))
    shutil.rmtree(d, ignore_errors=True)
    os.makedirs(d)

    class _P(str):
        def __truediv__(self, name):
            return os.path.join(self, name)

    yield _P(d)
    shutil.rmtree(d, ignore_errors=True)


def _fake_rec(p):
    return np.array([p + 1.0, -0.5 * (p + 1), 1e-17 * p, -3e-18 * p, p + 2.0])


class FakeParts:
    def __init__(self, fail_at=None, bad_at=None):
        self.calls = []
        self.fail_at, self.bad_at = fail_at, bad_at

    def __call__(self, A, part, nparts, loops=False, real=None, precision="fp64"):
        self.calls.append(part)
        if part == self.fail_at:
            raise RuntimeError("worker lost")
        if part == self.bad_at:
            return np.array([np.nan, 0, 0, 0, 1.0])
        return _fake_rec(part)


@pytest.fixture
def fake(monkeypatch):
    f = FakeParts()
    monkeypatch.setattr(hg, "haf_part", f)
    return f


def _A(n=12, seed=3):
    return inputs.complex_gaussian_symmetric(n, seed)


def test_full_run_then_nothing_to_do(scratch, fake):
    path = str(scratch / "h.json")
    prog = checkpoint.run(_A(), path, nparts=4)
    assert prog.complete and prog.computed == [0, 1, 2, 3] and fake.calls == [0, 1, 2, 3]
    want = hg.combine([_fake_rec(p) for p in range(4)])
    assert prog.value == want[0] and prog.abs_sum == want[1]
    prog2 = checkpoint.run(_A(), path, nparts=4)
    assert prog2.computed == [] and fake.calls == [0, 1, 2, 3] and prog2.value == prog.value


def test_resume_runs_only_the_missing_parts(scratch, fake):
    path = str(scratch / "h.json")
    prog = checkpoint.run(_A(), path, nparts=5, parts=[3, 0])
    assert not prog.complete and prog.value is None and prog.done == [0, 3]
    prog = checkpoint.run(_A(), path, nparts=5)
    assert prog.computed == [1, 2, 4] and fake.calls == [0, 3, 1, 2, 4] and prog.complete


def test_records_round_trip_bit_exactly(scratch, fake):
    path = str(scratch / "h.json")
    checkpoint.run(_A(), path, nparts=3)
    with open(path) as f:
        state = json.load(f)
    for p in range(3):
        got = [float.fromhex(x) for x in state["records"][str(p)]["rec"]]
        assert got == list(_fake_rec(p))


def test_another_matrix_or_split_is_refused(scratch, fake):
    path = str(scratch / "h.json")
    checkpoint.run(_A(), path, nparts=4, parts=[0])
    B = _A()
    B[0, 1] += 1e-15
    with pytest.raises(ValueError):
        checkpoint.run(B, path, nparts=4)
    with pytest.raises(ValueError):
        checkpoint.run(_A(), path, nparts=5)
    with pytest.raises(ValueError):
        checkpoint.run(_A(), path, nparts=4, loops=True)


def test_corrupted_record_is_dropped_and_recomputed(scratch, fake):
    path = str(scratch / "h.json")
    checkpoint.run(_A(), path, nparts=4)
    with open(path) as f:
        state = json.load(f)
    state["records"]["2"]["rec"][0] = (3.5).hex()  # value changed, checksum not
    del state["records"]["1"]["sha256"]
    with open(path, "w") as f:
        json.dump(state, f)
    prog = checkpoint.run(_A(), path, nparts=4)
    assert prog.dropped == [1, 2] and prog.computed == [1, 2] and prog.complete
    assert prog.value == hg.combine([_fake_rec(p) for p in range(4)])[0]


def test_a_failing_worker_keeps_the_finished_parts(scratch, monkeypatch):
    path = str(scratch / "h.json")
    monkeypatch.setattr(hg, "haf_part", FakeParts(fail_at=2))
    with pytest.raises(RuntimeError, match="worker lost"):
        checkpoint.run(_A(), path, nparts=4)
    monkeypatch.setattr(hg, "haf_part", FakeParts(bad_at=3))
    with pytest.raises(RuntimeError, match="invalid record"):
        checkpoint.run(_A(), path, nparts=4)
    good = FakeParts()
    monkeypatch.setattr(hg, "haf_part", good)
    prog = checkpoint.run(_A(), path, nparts=4)
    assert good.calls == [3] and prog.complete  # parts 0, 1 from the first run, 2 from the second


def test_coverage_is_checked(scratch, fake, monkeypatch):
    monkeypatch.setattr(hg, "part_subsets", lambda n, p, P: 1)
    with pytest.raises(RuntimeError, match="cover"):
        checkpoint.run(_A(), str(scratch / "h.json"), nparts=4)


def test_odd_loop_case_counts_the_padded_size(scratch, fake):
    prog = checkpoint.run(_A(11), str(scratch / "h.json"), nparts=3, loops=True)
    assert prog.complete


def test_bad_arguments(scratch, fake):
    with pytest.raises(ValueError):
        checkpoint.run(np.zeros((3, 4)), str(scratch / "h.json"))
    with pytest.raises(ValueError):
        checkpoint.run(_A(), str(scratch / "h.json"), nparts=0)
    with pytest.raises(ValueError):
        checkpoint.run(_A(), str(scratch / "h.json"), nparts=2, parts=[2])


@pytest.mark.gpu
@pytest.mark.parametrize("loops", [False, True])
def test_resumed_run_on_the_gpu(scratch, loops):
    A = inputs.complex_gaussian_symmetric(24, 77)
    path = str(scratch / "h.json")
    first = checkpoint.run(A, path, nparts=4, loops=loops, parts=[1, 2])
    assert not first.complete
    prog = checkpoint.run(A, path, nparts=4, loops=loops)
    assert prog.computed == [0, 3] and prog.complete
    direct = hg.combine([hg.haf_part(A, p, 4, loops=loops) for p in range(4)])
    assert prog.value == direct[0] and prog.abs_sum == direct[1]
    single = hg.haf_info(A, loops=loops)
    assert abs(prog.value - single.value) <= 1e-10 * single.abs_sum
