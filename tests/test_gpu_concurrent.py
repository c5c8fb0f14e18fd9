"""Independent problems solved at once, each handle on its own stream (the
bench's concurrent schedule): one by mg_solve, the others by mg_solve_async,
or every one by mg_solve in its own host thread with host buffers.  Each
result and its statistics must equal those of the problems solved one after
the other on one stream, bit for bit, in both precisions, and stay so over
repeated steps (the set-up of one problem overlapping the solve of another)."""
import os
import sys

import numpy as np
import pytest

from paper_2206_11294_gb300 import inputs as I

pytestmark = pytest.mark.gpu

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_11294_gb300 import binding
    binding.load()
    return torch


def _problems():
    return [I.bubble_2d(256, seed=91, n_bubbles=4, rmin=0.04, rmax=0.1, centred=False),
            I.bubble_axi(nr=128, nz=256, seed=92),
            I.stiff(I.bubble_2d, 192, seed=93, n_bubbles=2, rmin=0.05, rmax=0.12, centred=False)]


PROBS = _problems()


def _data(torch, probs):
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return [dict(lam=T(p.lam), fa=[T(f) for f in p.fa], fk=[T(f) for f in p.fk], b=T(p.b), x0=T(p.x0),
                 x=T(p.x0)) for p in probs]


def _stats_equal(a, b):
    return (a["cycles"] == b["cycles"] and a["outer"] == b["outer"] and a["status"] == b["status"]
            and list(a["rfinal"]) == list(b["rfinal"]) and list(a["r0"]) == list(b["r0"]))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_concurrent_step_equals_serial(torch_cuda, precision):
    torch = torch_cuda
    import bench
    from paper_2206_11294_gb300.binding import Solver
    main = torch.cuda.current_stream()
    ref_d = _data(torch, PROBS)
    ref_s = [Solver(p.grid, precision=precision, rtol=1e-10, max_cycles=200, stream=main) for p in PROBS]
    ref = bench.solve_serially(ref_s, ref_d, allow=True)
    ref_x = [d["x"].cpu().numpy() for d in ref_d]
    d = _data(torch, PROBS)
    s = [Solver(p.grid, precision=precision, rtol=1e-10, max_cycles=200, stream=torch.cuda.Stream())
         for p in PROBS]
    s[0].set_timing(True)                   # problem 0 carries the hooks, as in the bench
    for step in range(3):
        for q in d:
            q["x"].copy_(q["x0"])
        sts = bench.solve_concurrently(s, d, main, allow=True)
        torch.cuda.synchronize()
        for q in range(len(PROBS)):
            assert np.array_equal(d[q]["x"].cpu().numpy(), ref_x[q]), (step, q)
            assert _stats_equal(sts[q], ref[q]), (step, q, sts[q], ref[q])
    assert s[0].counters()["smooth_launches"] > 0


def test_threads_with_host_buffers_equal_serial(torch_cuda):
    torch = torch_cuda
    import bench
    from paper_2206_11294_gb300.binding import Solver
    probs = PROBS[:2]
    ref_d = _data(torch, probs)
    ref_s = [Solver(p.grid, precision="fp64", rtol=1e-10, max_cycles=200) for p in probs]
    ref = bench.solve_serially(ref_s, ref_d)
    s = [Solver(p.grid, precision="fp64", rtol=1e-10, max_cycles=200, stream=torch.cuda.Stream()) for p in probs]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    host = [dict(lam=pin(p.lam), fa=[pin(f) for f in p.fa], fk=[pin(f) for f in p.fk], b=pin(p.b)) for p in probs]
    for _ in range(2):
        xs = [p.x0.copy() for p in probs]

        def one(q):
            s[q].set_coeffs(host[q]["lam"], host[q]["fa"], host[q]["fk"])
            return s[q].solve(host[q]["b"], xs[q])
        sts = bench.in_threads([lambda q=q: one(q) for q in range(len(probs))])
        for q in range(len(probs)):
            assert np.array_equal(xs[q], ref_d[q]["x"].cpu().numpy()), q
            assert _stats_equal(sts[q], ref[q]), q

