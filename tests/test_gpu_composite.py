"""Refined-patch (adaptive) grids on the GPU (mg_composite_*) against the
oracle of composite_oracle.c: the composite operator element by element, the
FAC defect-correction loop after fixed numbers of steps (same residual
history), and the converged result against the dense solution of the
composite system.  Tolerance 1e-12 of the deviation from the initial guess
(the composite residual takes neighbour differences first on both sides, so
no background cancels)."""
import numpy as np
import pytest

from paper_2206_11294_gb300 import inputs as I

pytestmark = pytest.mark.gpu

W, D = I.BC_WALL, I.BC_DIRICHLET


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_11294_gb300 import binding
    binding.load()
    return torch


def _cases():
    dbc = ((D, W), (W, D), (0, 0))
    dT = ((305.0, 0.0), (0.0, 295.0), (0.0, 0.0))
    dP = ((1.05e5, 0.0), (0.0, 0.97e5), (0.0, 0.0))
    return {
        "literal_bubbles_64": I.composite_bubble(64, seed=21, n_bubbles=2),
        "stiff_bubbles_64": I.composite_bubble(64, seed=22, n_bubbles=2, length=6.4e-3, dt=1e-5),
        "stiff_dirichlet_corner": I.composite_bubble(48, box=((0, 20), (0, 24)), seed=23, n_bubbles=1, rmin=0.08,
                                                     rmax=0.12, length=6.4e-3, dt=1e-5, bc=dbc, bcT=dT, bcp=dP),
        "literal_edge_box": I.composite_bubble(64, box=((40, 64), (10, 30)), seed=24, n_bubbles=1, rmin=0.05,
                                               rmax=0.08, bc=dbc, bcT=dT, bcp=dP),
    }


CASES = _cases()


def _dev(b, p, box):
    from oracle import composite as cf
    return b.grid.as_dict(), cf


def _rel(x, ref, x0):
    return max(float(np.abs(x[:, f] - ref[:, f]).max() / max(np.abs(ref[:, f] - x0[:, f]).max(), 1e-300))
               for f in range(2))


def _composite(b, p, box):
    from paper_2206_11294_gb300.binding import Composite
    c = Composite(b.grid, box)
    c.set_coeffs(b.lam, b.fa, b.fk, p.lam, p.fa, p.fk)
    return c


@pytest.mark.parametrize("name", list(CASES))
def test_composite_apply(torch_cuda, name):
    from oracle import composite as cf
    b, p, box = CASES[name]
    rng = np.random.default_rng(5)
    xb = b.x0 * (1 + 1e-2 * rng.standard_normal(b.x0.shape))
    xf = p.x0 * (1 + 1e-2 * rng.standard_normal(p.x0.shape))
    c = _composite(b, p, box)
    yb, yf = c.apply(xb, xf)
    rb, rf = cf.apply(b.grid.as_dict(), box, b.lam, b.fa, b.fk, p.lam, p.fa, p.fk, xb, xf)
    for f in range(2):
        scale = max(np.abs(rb[:, f]).max(), np.abs(rf[:, f]).max())
        assert np.abs(yb.cpu().numpy()[:, f] - rb[:, f]).max() <= 1e-12 * scale
        assert np.abs(yf.cpu().numpy()[:, f] - rf[:, f]).max() <= 1e-12 * scale
    c.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("cycles", [1, 3])
def test_composite_fac_fixed_cycles(torch_cuda, name, cycles):
    from oracle import composite as cf
    b, p, box = CASES[name]
    c = _composite(b, p, box)
    xb, xf, hist = c.solve(b.b, p.b, b.x0.copy(), p.x0.copy(), cycles)
    ob, of_, ohist = cf.fac_solve(b.grid.as_dict(), box, b.lam, b.fa, b.fk, p.lam, p.fa, p.fk, b.b, p.b, b.x0,
                                  p.x0, cycles)
    xb, xf = xb.cpu().numpy(), xf.cpu().numpy()
    assert _rel(xf, of_, p.x0) <= 1e-12
    assert _rel(xb, ob, b.x0) <= 1e-12
    for q in range(4):                         # residual norms where well above rounding noise
        for k in range(cycles + 1):
            if ohist[k, q] > 1e-6 * ohist[0, q]:
                assert abs(hist[k, q] - ohist[k, q]) <= 1e-6 * ohist[k, q]
    c.close()


def test_composite_autotune_keeps_results(torch_cuda):
    """The base hierarchy's kernel choices change no arithmetic: after
    mg_composite_autotune (which also drops the captured FAC-cycle graph) the
    same solve gives the same result bit for bit."""
    b, p, box = CASES["stiff_bubbles_64"]
    c = _composite(b, p, box)
    xb0, xf0, h0 = c.solve(b.b, p.b, b.x0.copy(), p.x0.copy(), 4)
    assert c.autotune(reps=2) > 0
    xb1, xf1, h1 = c.solve(b.b, p.b, b.x0.copy(), p.x0.copy(), 4)
    assert np.array_equal(xb0.cpu().numpy(), xb1.cpu().numpy())
    assert np.array_equal(xf0.cpu().numpy(), xf1.cpu().numpy())
    assert np.array_equal(h0, h1)
    c.close()


def test_composite_converges_to_the_dense_solution(torch_cuda):
    from oracle import composite as cf
    b, p, box = I.composite_bubble(16, seed=25, n_bubbles=1, rmin=0.15, rmax=0.2, length=6.4e-3, dt=1e-5)
    xd_b, xd_f = cf.dense_solve(b.grid.as_dict(), box, b.lam, b.fa, b.fk, p.lam, p.fa, p.fk, b.b, p.b)
    c = _composite(b, p, box)
    xb, xf, hist = c.solve(b.b, p.b, b.x0.copy(), p.x0.copy(), 40)
    assert _rel(xf.cpu().numpy(), xd_f, p.x0) <= 1e-9
    c.close()


@pytest.mark.parametrize("name", ["stiff_bubbles_64", "stiff_dirichlet_corner", "literal_edge_box"])
def test_composite_mixed_base_correction(torch_cuda, name):
    """MG_MIXED: the base correction's V-cycle in FP32, the composite
    residual, the patch sweeps and the update in FP64.  The defect
    correction reaches the FP64 composite solve's fixed point: against the
    FP64 solve run to its rounding floor, 1e-8 of the deviation, in at most a
    few more steps."""
    from paper_2206_11294_gb300.binding import Composite
    b, p, box = CASES[name]
    ref = _composite(b, p, box)
    xb64, xf64, h64 = ref.solve(b.b, p.b, b.x0.copy(), p.x0.copy(), 40)
    ref.close()
    c = Composite(b.grid, box, precision="mixed")
    c.set_coeffs(b.lam, b.fa, b.fk, p.lam, p.fa, p.fk)
    xb, xf, h = c.solve(b.b, p.b, b.x0.copy(), p.x0.copy(), 40)
    xb, xf = xb.cpu().numpy(), xf.cpu().numpy()
    assert _rel(xf, xf64.cpu().numpy(), p.x0) <= 1e-8
    assert _rel(xb, xb64.cpu().numpy(), b.x0) <= 1e-8
    # the same contraction until the floors: within a factor 2 after 3 steps
    for q in range(4):
        if h64[3, q] > 1e-6 * h64[0, q]:
            assert h[3, q] <= 2.0 * h64[3, q] + 1e-30
    c.close()


def test_composite_rejects_bad_arguments(torch_cuda):
    from paper_2206_11294_gb300.binding import Composite, MgError, MG_ERR_INVALID_ARG
    b, p, box = CASES["literal_bubbles_64"]
    for bad in (((10, 10), (0, 4)), ((0, 70), (0, 4)), ((-1, 4), (0, 4))):
        with pytest.raises(MgError) as e:
            Composite(b.grid, bad)
        assert e.value.status == MG_ERR_INVALID_ARG
    ax = I.Grid(dim=2, axisym=1, n=(32, 32, 1), h=0.1, bc=((I.BC_AXIS, W), (W, W), (0, 0)))
    with pytest.raises(MgError):
        Composite(ax, ((0, 8), (0, 8)))
