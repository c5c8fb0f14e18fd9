"""mg_solve_async: the whole solve as one graph with the stop test on the
device.  Its result and statistics must equal mg_solve's bit for bit (the same
kernels in the same order), in both precisions, with both smoothers, for 2D,
axisymmetric and 3D grids; its event must let work on another stream wait for
the result without a host synchronisation; the degenerate stops (nothing to
do, no cycle allowed, not converged) must report as mg_solve does."""
import numpy as np
import pytest

from paper_2206_11294_gb300 import inputs as I

pytestmark = pytest.mark.gpu

W, D, A = I.BC_WALL, I.BC_DIRICHLET, I.BC_AXIS


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_11294_gb300 import binding
    binding.load()
    return torch


def _cases():
    g2 = I.Grid(dim=2, axisym=0, n=(96, 40, 1), h=1e-4, bc=((D, W), (W, D), (0, 0)),
                bcT=((310, 0), (0, 290), (0, 0)), bcp=((1.1e5, 0), (0, 0.9e5), (0, 0)))
    ga = I.Grid(dim=2, axisym=1, n=(48, 104, 1), h=1e-4, bc=((A, D), (W, W), (0, 0)),
                bcT=((0, 300), (0, 0), (0, 0)), bcp=((0, 1e5), (0, 0), (0, 0)))
    g3 = I.Grid(dim=3, axisym=0, n=(40, 24, 16), h=1e-4, bc=((D, D), (D, D), (W, D)),
                bcT=((300, 300), (300, 300), (0, 300)), bcp=((1e5, 1e5), (1e5, 1e5), (0, 1e5)))
    return {"2d_stiff": I.random_coeff_problem(g2, seed=81, dt=1e-5),
            "axi_stiff": I.random_coeff_problem(ga, seed=82, dt=1e-5),
            "3d_stiff": I.random_coeff_problem(g3, seed=83, dt=1e-5),
            "2d_literal": I.bubble_2d(128, seed=84, n_bubbles=3, rmin=0.05, rmax=0.15, centred=False)}


CASES = _cases()


def _dev(torch, p):
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return dict(lam=T(p.lam), fa=[T(f) for f in p.fa], fk=[T(f) for f in p.fk], b=T(p.b), x0=T(p.x0))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision,smoother", [("fp64", "rbgs"), ("mixed", "rbgs"), ("fp64", "wjac")])
def test_async_equals_sync(torch_cuda, orc, name, precision, smoother):
    torch = torch_cuda
    from paper_2206_11294_gb300.binding import Solver
    p = CASES[name]
    d = _dev(torch, p)
    s = Solver(p.grid, precision=precision, rtol=1e-10, max_cycles=120, smoother=smoother)
    s.set_coeffs(d["lam"], d["fa"], d["fk"])
    xs = d["x0"].clone()
    st = s.solve(d["b"], xs)
    for _ in range(2):                      # twice: the captured graph is replayed
        xa = d["x0"].clone()
        s.solve_async(d["b"], xa)
        sa = s.async_stats()
        assert torch.equal(xa, xs)
        for k in ("cycles", "outer", "r0", "rfinal", "status", "levels"):
            assert sa[k] == st[k], k
        assert sa["seconds"] > 0.0
    if precision == "fp64":                 # and the oracle's solve with the same rule
        ref, cyc, _ = orc.mg_solve(p.grid.as_dict(), p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=120, rtol=1e-10,
                                   smoother=smoother)
        assert sa["cycles"] == cyc
        x = xa.cpu().numpy()
        for f in range(2):
            dev = np.linalg.norm(ref[:, f] - p.x0[:, f])
            assert np.linalg.norm(x[:, f] - ref[:, f]) <= 1e-9 * dev
    s.close()


def test_event_orders_other_streams(torch_cuda):
    """Work on another stream that waits for the event sees the result, with
    no host synchronisation between the enqueue and that work."""
    torch = torch_cuda
    from paper_2206_11294_gb300.binding import Solver
    p = CASES["2d_stiff"]
    d = _dev(torch, p)
    s = Solver(p.grid, rtol=1e-10, max_cycles=120)
    s.set_coeffs(d["lam"], d["fa"], d["fk"])
    xs = d["x0"].clone()
    s.solve(d["b"], xs)
    other = torch.cuda.Stream()
    for _ in range(3):
        xa = d["x0"].clone()
        y = torch.zeros_like(xa)
        torch.cuda.synchronize()
        ev = torch.cuda.Event()
        s.solve_async(d["b"], xa, event=ev)
        other.wait_event(ev)
        with torch.cuda.stream(other):
            y.copy_(xa)
        other.synchronize()
        assert torch.equal(y, xs)
        s.async_stats()
    s.close()


def test_many_handles_in_flight(torch_cuda):
    """Several handles, each on its own stream, enqueue their solves before any
    statistics are read; each result equals its synchronous solve."""
    torch = torch_cuda
    from paper_2206_11294_gb300.binding import Solver
    hs = []
    for name, p in CASES.items():
        st = torch.cuda.Stream()
        d = _dev(torch, p)
        s = Solver(p.grid, precision="mixed" if name.startswith("3d") else "fp64", rtol=1e-10, max_cycles=120,
                   stream=st)
        s.set_coeffs(d["lam"], d["fa"], d["fk"])
        xs = d["x0"].clone()
        ref = s.solve(d["b"], xs)
        hs.append((s, d, xs, ref))
    outs = []
    for s, d, xs, ref in hs:
        xa = d["x0"].clone()
        s.solve_async(d["b"], xa)
        outs.append(xa)
    for (s, d, xs, ref), xa in zip(hs, outs):
        sa = s.async_stats()
        assert sa["cycles"] == ref["cycles"]
        assert torch.equal(xa, xs)
        s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_degenerate_stops(torch_cuda, precision):
    """Nothing to do (zero right-hand side and guess), rtol >= 1, no cycle
    allowed, and a cap reached: the same statistics and x as mg_solve."""
    torch = torch_cuda
    from paper_2206_11294_gb300.binding import MgError, Solver, MG_ERR_NOT_CONVERGED, MG_ERR_STATE
    p = I.bubble_2d(64)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    for kw, b, x0 in [(dict(), np.zeros_like(p.b), np.zeros_like(p.x0)), (dict(rtol=2.0), p.b, p.x0),
                      (dict(max_cycles=0), p.b, p.x0), (dict(rtol=1e-14, max_cycles=1), p.b, p.x0)]:
        s = Solver(p.grid, precision=precision, **kw)
        s.set_coeffs(p.lam, p.fa, p.fk)
        with pytest.raises(MgError) as e:
            s.async_stats()
        assert e.value.status == MG_ERR_STATE
        xs = T(x0)
        st = s.solve(T(b), xs, allow_not_converged=True)
        xa = T(x0)
        s.solve_async(T(b), xa)
        if st["status"] == "MG_ERR_NOT_CONVERGED":
            with pytest.raises(MgError) as e:
                s.async_stats()
            assert e.value.status == MG_ERR_NOT_CONVERGED
            s.solve_async(T(b), xa.copy_(T(x0)))
        sa = s.async_stats(allow_not_converged=True)
        for k in ("cycles", "outer", "r0", "rfinal", "status"):
            assert sa[k] == st[k], (kw, k)
        assert torch.equal(xa, xs), kw
        s.close()


def test_set_stream_orders_after_the_running_set_up(torch_cuda):
    """mg_set_coeffs returns with its set-up still running; mg_set_stream then
    makes the new stream wait for it on the device, not for the old stream's
    later work and not on the host.  The old stream is held back by a bounded
    spin kernel enqueued before the set-up, so a solve on the new stream that
    did not wait would read the previous coefficients (a different problem's)
    and give another result."""
    torch = torch_cuda
    from paper_2206_11294_gb300.binding import Solver
    p, q = CASES["2d_stiff"], I.random_coeff_problem(CASES["2d_stiff"].grid, seed=91, dt=1e-5)
    d, e = _dev(torch, p), _dev(torch, q)
    ref = Solver(p.grid, precision="fp64", rtol=1e-10, max_cycles=120)
    ref.set_coeffs(d["lam"], d["fa"], d["fk"])
    x_ref = d["x0"].clone()
    st_ref = ref.solve(d["b"], x_ref)
    ref.close()
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    s = Solver(p.grid, precision="fp64", rtol=1e-10, max_cycles=120, stream=sa)
    x = d["x0"].clone()
    s.set_coeffs(e["lam"], e["fa"], e["fk"])         # another problem's coefficients first
    torch.cuda.synchronize()
    with torch.cuda.stream(sa):
        torch.cuda._sleep(20_000_000)                # about 10 ms of spinning on sa
    s.set_coeffs(d["lam"], d["fa"], d["fk"])         # on sa, queued behind the spin
    s.set_stream(sb)
    st = s.solve(d["b"], x)                          # on sb, at once
    assert st["cycles"] == st_ref["cycles"]
    assert np.array_equal(x.cpu().numpy(), x_ref.cpu().numpy())
    s.close()
