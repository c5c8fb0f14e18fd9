"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Element-by-element comparisons on the same seeded inputs, at sizes that span
several thread blocks and leave ragged tails, for every geometry and boundary
mix, in two regimes:

  literal   the workloads' own units (unit domain, dt = 1e-7): the local 2x2
            blocks dominate the Laplacians;
  stiff     the paper's bubble scale (h = 1e-4 m, dt = 1e-5 s): the p-row is
            Laplacian-dominated with a density jump of 1000.

Tolerances (relative L2 of the deviation from the initial guess, per field):
  - operator application, one or three sweeps, norms: 1e-12 (FP64 rounding;
    the GPU contracts to FMA, the oracle does not);
  - FP64 solves after the same number of cycles, literal regime: 1e-12;
  - FP64 solves, stiff regime: 1e-9.  Both sides carry a 1e5 Pa background
    through rows whose diagonal nearly cancels the face sums (sum_f G_f up to
    ~1e8 against a Helmholtz term ~5), so each side's rounding alone moves the
    solution by up to eps * 2 sum_f G_f |p| / (|l3| dev) ~ 3e-9 of the deviation;
  - mixed precision at 1e-10 residual reduction: 1e-8 against the converged oracle.
"""
import numpy as np
import pytest

from paper_2206_11294_gb300 import inputs as I

pytestmark = pytest.mark.gpu

W, D, A = I.BC_WALL, I.BC_DIRICHLET, I.BC_AXIS


def rel_dev(x, ref, x0):
    out = 0.0
    for f in range(2):
        d = ref[:, f] - x0[:, f]
        out = max(out, np.linalg.norm(x[:, f] - ref[:, f]) / max(np.linalg.norm(d), 1e-300))
    return out


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_11294_gb300 import binding
    binding.load()
    return torch


def _solver(p, **kw):
    from paper_2206_11294_gb300.binding import Solver
    s = Solver(p.grid, **kw)
    s.set_coeffs(p.lam, p.fa, p.fk)
    return s


# grids: several blocks of 32 x 8 threads, ragged tails, every boundary mix
def _grids(h):
    return {
        "2d_ragged_walls": I.Grid(dim=2, axisym=0, n=(200, 72, 1), h=h, bc=((W, W), (W, W), (0, 0))),
        "2d_dirichlet_mix": I.Grid(dim=2, axisym=0, n=(96, 40, 1), h=h, bc=((D, W), (W, D), (0, 0)),
                                   bcT=((310, 0), (0, 290), (0, 0)), bcp=((1.1e5, 0), (0, 0.9e5), (0, 0))),
        "axi_axis": I.Grid(dim=2, axisym=1, n=(48, 104, 1), h=h, bc=((A, D), (W, W), (0, 0)),
                           bcT=((0, 300), (0, 0), (0, 0)), bcp=((0, 1e5), (0, 0), (0, 0))),
        "axi_annulus": I.Grid(dim=2, axisym=1, n=(40, 64, 1), h=h, r0=2 * h, bc=((W, D), (D, W), (0, 0)),
                              bcT=((0, 300), (305, 0), (0, 0)), bcp=((0, 1e5), (1.2e5, 0), (0, 0))),
        "3d_wall_dirichlet": I.Grid(dim=3, axisym=0, n=(40, 24, 16), h=h, bc=((D, D), (D, D), (W, D)),
                                    bcT=((300, 300), (300, 300), (0, 300)),
                                    bcp=((1e5, 1e5), (1e5, 1e5), (0, 1e5))),
        "3d_walls_odd": I.Grid(dim=3, axisym=0, n=(56, 24, 16), h=h, bc=((W, W), (W, W), (W, W))),
    }


def _cases():
    out = {}
    for q, (name, g) in enumerate(_grids(1.0 / 200).items()):
        out["literal_" + name] = (I.random_coeff_problem(g, seed=20 + q, dt=1e-7), 1e-12)
    for q, (name, g) in enumerate(_grids(1e-4).items()):
        out["stiff_" + name] = (I.random_coeff_problem(g, seed=40 + q, dt=1e-5), 1e-9)
    return out


CASES = _cases()


@pytest.mark.parametrize("name", list(CASES))
def test_apply(torch_cuda, orc, name):
    p, _ = CASES[name]
    s = _solver(p)
    rng = np.random.default_rng(1)
    x = p.x0 * (1 + 1e-2 * rng.standard_normal(p.x0.shape))
    y = s.apply(x)
    ref = orc.apply_paper(p.grid.as_dict(), p.lam, p.fa, p.fk, x)
    for f in range(2):
        assert np.abs(y[:, f] - ref[:, f]).max() <= 1e-12 * np.abs(ref[:, f]).max()
    s.close()


@pytest.mark.parametrize("smoother", ["rbgs", "wjac"])
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("sweeps", [1, 3])
def test_smooth(torch_cuda, orc, name, sweeps, smoother):
    """One and three sweeps of either smoother: red-black block Gauss-Seidel,
    or weighted block Jacobi (omega 0.8; three sweeps end in the ping-pong
    partner and are copied back)."""
    p, _ = CASES[name]
    s = _solver(p, smoother=smoother, omega=0.8)
    x = p.x0.copy()
    s.smooth(p.b, x, sweeps)
    if smoother == "rbgs":
        ref = orc.rbgs_sweeps(p.grid.as_dict(), p.lam, p.fa, p.fk, p.b, p.x0, sweeps)
    else:
        ref = orc.wjac_sweeps(p.grid.as_dict(), p.lam, p.fa, p.fk, p.b, p.x0, sweeps, omega=0.8)
    assert rel_dev(x, ref, p.x0) <= 1e-12
    s.close()


@pytest.mark.parametrize("name", list(CASES))
def test_residual_norms(torch_cuda, orc, name):
    p, _ = CASES[name]
    s = _solver(p)
    got = s.residual_norms(p.b, p.x0)
    ref = orc.residual_norms(p.grid.as_dict(), p.lam, p.fa, p.fk, p.b, p.x0)
    assert np.allclose(got, ref, rtol=1e-12, atol=0)
    s.close()


@pytest.mark.parametrize("smoother", ["rbgs", "wjac"])
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("cycles", [1, 4])
def test_fixed_cycles_fp64(torch_cuda, orc, name, cycles, smoother):
    p, tol = CASES[name]
    s = _solver(p, rtol=0.0, max_cycles=cycles, smoother=smoother)
    x = p.x0.copy()
    st = s.solve(p.b, x)
    ref, cyc, _ = orc.mg_solve(p.grid.as_dict(), p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=cycles, rtol=0.0,
                               smoother=smoother)
    assert st["cycles"] == cycles == cyc
    assert rel_dev(x, ref, p.x0) <= tol
    assert st["levels"] == orc.num_levels(p.grid.as_dict())
    s.close()


@pytest.mark.parametrize("tile", [0, 2])
@pytest.mark.parametrize("name", [n for n in CASES if CASES[n][0].grid.dim == 2])
def test_fixed_cycles_fused_pairs_vs_oracle(torch_cuda, orc, name, tile):
    """Two sweeps per launch on tiles with a 4-cell halo (MG_SWEEP_FUSED2) on
    every smoothed level, no tail: 1 and 3 fixed V(2,2) cycles against the
    oracle's, at the tolerance of the plain kernels, and the colour sweeps'
    results bit for bit."""
    p, tol = CASES[name]
    for cycles in (1, 3):
        s = _solver(p, rtol=0.0, max_cycles=cycles)
        n = s.tuning()["levels"]
        s.set_tuning(dict(s.tuning(), sweep=["fused2"] * n, tile=[tile] * n, tail_level=n))
        x = p.x0.copy()
        st = s.solve(p.b, x)
        ref, cyc, _ = orc.mg_solve(p.grid.as_dict(), p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=cycles, rtol=0.0)
        assert st["cycles"] == cycles == cyc
        assert rel_dev(x, ref, p.x0) <= tol
        c = _solver(p, rtol=0.0, max_cycles=cycles)
        c.set_tuning(dict(c.tuning(), sweep=["colour"] * n, tile=[0] * n, tail_level=n))
        xc = p.x0.copy()
        c.solve(p.b, xc)
        assert np.array_equal(x, xc)
        s.close()
        c.close()


@pytest.mark.parametrize("name", list(CASES))
def test_converged_fp64_same_cycles_as_oracle(torch_cuda, orc, name):
    p, tol = CASES[name]
    s = _solver(p, rtol=1e-10, max_cycles=60)
    x = p.x0.copy()
    st = s.solve(p.b, x)
    ref, cyc, hist = orc.mg_solve(p.grid.as_dict(), p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=60, rtol=1e-10)
    assert st["cycles"] == cyc
    assert np.allclose(st["r0"], hist[0], rtol=1e-12)
    assert rel_dev(x, ref, p.x0) <= tol
    s.close()


def _background_free(orc, p):
    """The problem restated for its deviation from the initial guess: x0 = 0,
    homogeneous Dirichlet values, and b the residual of the original initial
    guess (evaluated by the oracle).  Its solution is the original solution
    minus the background, so no 1e5 Pa offset enters the rounding."""
    import dataclasses
    b = p.b - orc.apply_paper(p.grid.as_dict(), p.lam, p.fa, p.fk, p.x0)
    g = dataclasses.replace(p.grid, bcT=((0.0, 0.0),) * 3, bcp=((0.0, 0.0),) * 3)
    return dataclasses.replace(p, grid=g, b=b, x0=np.zeros_like(p.x0))


@pytest.mark.parametrize("name", [n for n in CASES if n.startswith("stiff")])
@pytest.mark.parametrize("cycles", [1, 4])
def test_fixed_cycles_fp64_stiff_background_free(torch_cuda, orc, name, cycles):
    """Stiff regime with the background removed: where the coarse levels carry
    the convergence, the FP64 path matches the oracle after the same number of
    cycles to 1e-12, as in the literal regime.  (With the background, each
    side's rounding of terms of size sum_f G_f |p| ~ 1e13 bounds the agreement;
    without it, the same rounding is relative to the deviation itself.)"""
    p = _background_free(orc, CASES[name][0])
    s = _solver(p, rtol=0.0, max_cycles=cycles)
    x = p.x0.copy()
    st = s.solve(p.b, x)
    ref, cyc, _ = orc.mg_solve(p.grid.as_dict(), p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=cycles, rtol=0.0)
    assert st["cycles"] == cycles == cyc
    assert rel_dev(x, ref, p.x0) <= 1e-12
    s.close()


@pytest.mark.parametrize("cycle", ["W", "F"])
@pytest.mark.parametrize("name", ["literal_2d_ragged_walls", "stiff_axi_axis", "literal_3d_wall_dirichlet",
                                  "stiff_3d_walls_odd"])
def test_w_f_cycles_vs_oracle(torch_cuda, orc, name, cycle):
    """W- and F-cycles: fixed cycles against the oracle's, and converged solves
    with the oracle's cycle count; mixed precision converges to the oracle's
    solution."""
    p, tol = CASES[name]
    g = p.grid.as_dict()
    s = _solver(p, rtol=0.0, max_cycles=2, cycle=cycle)
    x = p.x0.copy()
    st = s.solve(p.b, x)
    ref, cyc, _ = orc.mg_solve(g, p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=2, rtol=0.0, cycle=cycle)
    assert st["cycles"] == 2 == cyc
    assert rel_dev(x, ref, p.x0) <= tol
    s.close()
    s = _solver(p, rtol=1e-10, max_cycles=60, cycle=cycle)
    x = p.x0.copy()
    st = s.solve(p.b, x)
    ref, cyc, _ = orc.mg_solve(g, p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=60, rtol=1e-10, cycle=cycle)
    assert st["cycles"] == cyc
    assert rel_dev(x, ref, p.x0) <= tol
    s.close()
    s = _solver(p, rtol=1e-10, max_cycles=60, cycle=cycle, precision="mixed")
    xm = p.x0.copy()
    st = s.solve(p.b, xm)
    assert st["status"] == "MG_OK"
    assert rel_dev(xm, ref, p.x0) <= 1e-8
    s.close()


@pytest.mark.parametrize("name", ["literal_2d_dirichlet_mix", "stiff_axi_axis", "stiff_3d_wall_dirichlet",
                                  "stiff_2d_ragged_walls"])
def test_wjac_converged_and_mixed_vs_oracle(torch_cuda, orc, name):
    """Weighted block Jacobi (omega 0.8 and 0.6): converged FP64 solves take
    the oracle's cycle count and match its result; mixed precision with the
    same smoother reaches the converged oracle to 1e-8 (stiff cases run to
    1e-12, as in test_mixed_precision); background-free stiff cases match after
    fixed cycles to 1e-12."""
    p, tol = CASES[name]
    g = p.grid.as_dict()
    for omega in (0.8, 0.6):
        s = _solver(p, rtol=1e-10, max_cycles=120, smoother="wjac", omega=omega)
        x = p.x0.copy()
        st = s.solve(p.b, x)
        ref, cyc, _ = orc.mg_solve(g, p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=120, rtol=1e-10,
                                   smoother="wjac", omega=omega)
        assert st["cycles"] == cyc
        assert rel_dev(x, ref, p.x0) <= tol
        s.close()
    rtol = 1e-10 if name.startswith("literal") else 1e-12
    s = _solver(p, precision="mixed", rtol=rtol, max_cycles=120, smoother="wjac")
    xm = p.x0.copy()
    st = s.solve(p.b, xm)
    conv, _, _ = orc.mg_solve(g, p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=80, rtol=1e-13)
    assert st["status"] == "MG_OK"
    assert rel_dev(xm, conv, p.x0) <= 1e-8
    s.close()
    if name.startswith("stiff"):
        q = _background_free(orc, p)
        s = _solver(q, rtol=0.0, max_cycles=3, smoother="wjac")
        x = q.x0.copy()
        s.solve(q.b, x)
        ref, _, _ = orc.mg_solve(q.grid.as_dict(), q.lam, q.fa, q.fk, q.b, q.x0, max_cycles=3, rtol=0.0,
                                 smoother="wjac")
        assert rel_dev(x, ref, q.x0) <= 1e-12
        s.close()


def test_wjac_refused_by_batches_and_validated(torch_cuda):
    from paper_2206_11294_gb300.binding import Batch, MgError, MG_ERR_INVALID_ARG
    p, _ = CASES["literal_2d_ragged_walls"]
    s = _solver(p, smoother="wjac")
    with pytest.raises(MgError) as e:
        Batch([s])
    assert e.value.status == MG_ERR_INVALID_ARG and "Gauss-Seidel" in str(e.value)
    s.close()
    for omega in (0.0, 1.5, float("nan")):
        with pytest.raises(MgError) as e:
            _solver(p, smoother="wjac", omega=omega)
        assert e.value.status == MG_ERR_INVALID_ARG


def test_w_f_cycles_refused_by_batches(torch_cuda):
    from paper_2206_11294_gb300.binding import Batch, MgError, MG_ERR_INVALID_ARG
    p, _ = CASES["literal_2d_ragged_walls"]
    s = _solver(p, cycle="W")
    with pytest.raises(MgError) as e:
        Batch([s])
    assert e.value.status == MG_ERR_INVALID_ARG and "V-cycles" in str(e.value)
    s.close()


SHAPE_CASES = ["literal_2d_ragged_walls", "stiff_axi_axis", "literal_3d_wall_dirichlet", "stiff_3d_walls_odd"]


@pytest.mark.parametrize("name", SHAPE_CASES)
@pytest.mark.parametrize("nu1,nu2", [(0, 2), (2, 0), (1, 1), (3, 1)])
def test_cycle_shapes_fp64(torch_cuda, orc, name, nu1, nu2):
    """V(nu1, nu2) shapes: with nu1 = 0 the restriction evaluates every child
    (no sweep has zeroed the black residuals) and with nu2 = 0 the stopping
    norm visits every cell; both against the oracle, fixed and converged."""
    p, tol = CASES[name]
    g = p.grid.as_dict()
    # one cycle: the stopping norm against the oracle's, per field where it is
    # still well above rounding noise (a field whose 2x2 blocks dominate is
    # solved to noise level by one cycle)
    s = _solver(p, rtol=0.0, max_cycles=1, nu1=nu1, nu2=nu2)
    x = p.x0.copy()
    st = s.solve(p.b, x)
    _, _, hist = orc.mg_solve(g, p.lam, p.fa, p.fk, p.b, p.x0, nu1=nu1, nu2=nu2, max_cycles=1, rtol=0.0)
    checked = 0
    for f in range(2):
        if hist[-1][f] > 1e-6 * hist[0][f]:
            assert abs(st["rfinal"][f] - hist[-1][f]) <= 1e-6 * hist[-1][f], f
            checked += 1
    assert checked > 0 or name.startswith("literal")   # literal cases: noise level after one cycle
    s.close()
    s = _solver(p, rtol=0.0, max_cycles=3, nu1=nu1, nu2=nu2)
    x = p.x0.copy()
    st = s.solve(p.b, x)
    ref, cyc, hist = orc.mg_solve(g, p.lam, p.fa, p.fk, p.b, p.x0, nu1=nu1, nu2=nu2, max_cycles=3, rtol=0.0)
    assert st["cycles"] == 3 == cyc
    assert rel_dev(x, ref, p.x0) <= tol
    s.close()
    s = _solver(p, rtol=1e-10, max_cycles=80, nu1=nu1, nu2=nu2)
    x = p.x0.copy()
    st = s.solve(p.b, x)
    ref, cyc, hist = orc.mg_solve(g, p.lam, p.fa, p.fk, p.b, p.x0, nu1=nu1, nu2=nu2, max_cycles=80, rtol=1e-10)
    assert st["cycles"] == cyc
    assert rel_dev(x, ref, p.x0) <= tol
    s.close()


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_precision(torch_cuda, orc, name):
    """FP32 cycles inside FP64 refinement against the converged FP64 oracle.
    Literal regime: the workloads' stopping rule (1e-10 reduction) must give
    1e-8.  Stiff regime: at 1e-10 the algebraic error of ANY solver is up to
    cond(D^-1 A) * 1e-10 (~1e-7 here), so the solve runs to 1e-12 and must then
    reach the same 1e-8, i.e. FP32 cycles lose nothing the FP64 loop needs."""
    p, _ = CASES[name]
    rtol = 1e-10 if name.startswith("literal") else 1e-12
    s = _solver(p, precision="mixed", rtol=rtol, max_cycles=60)
    x = p.x0.copy()
    st = s.solve(p.b, x)
    ref, cyc, hist = orc.mg_solve(p.grid.as_dict(), p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=80, rtol=1e-13)
    assert max(st["rfinal"][f] / st["r0"][f] for f in range(2)) <= rtol
    assert rel_dev(x, ref, p.x0) <= 1e-8
    s.close()


def test_device_pointers_and_workspace(torch_cuda, orc):
    """Device-side inputs (torch tensors) give the same result as host inputs."""
    torch = torch_cuda
    p, _ = CASES["stiff_2d_dirichlet_mix"]
    s = _solver(p, rtol=0.0, max_cycles=2)
    x_h = p.x0.copy()
    s.solve(p.b, x_h)
    s2 = _solver(p, rtol=0.0, max_cycles=2)
    s2.set_coeffs(torch.from_numpy(p.lam).cuda(), [torch.from_numpy(f).cuda() for f in p.fa],
                  [torch.from_numpy(f).cuda() for f in p.fk])
    x_d = torch.from_numpy(p.x0.copy()).cuda()
    s2.solve(torch.from_numpy(p.b).cuda(), x_d)
    assert np.array_equal(x_d.cpu().numpy(), x_h)
    s.close()
    s2.close()


def test_repeat_solves_are_bitwise_identical(torch_cuda):
    p, _ = CASES["stiff_3d_walls_odd"]
    s = _solver(p, rtol=1e-10, max_cycles=60)
    xs = []
    for _ in range(3):
        x = p.x0.copy()
        s.solve(p.b, x)
        xs.append(x)
    assert np.array_equal(xs[0], xs[1]) and np.array_equal(xs[1], xs[2])
    s.close()


def test_invalid_coefficients_rejected(torch_cuda):
    from paper_2206_11294_gb300.binding import MgError, Solver, MG_ERR_INVALID_COEFF, MG_ERR_STATE
    p, _ = CASES["literal_2d_ragged_walls"]
    s = Solver(p.grid)
    with pytest.raises(MgError) as e:
        s.solve(p.b, p.x0.copy())
    assert e.value.status == MG_ERR_STATE
    lam = p.lam.copy()
    lam[5, 0] = np.nan
    with pytest.raises(MgError) as e:
        s.set_coeffs(lam, p.fa, p.fk)
    assert e.value.status == MG_ERR_INVALID_COEFF
    # the rejected set-up (whose coarsest inverse ran on non-finite values)
    # leaves nothing behind: valid coefficients then solve as on a new handle
    s.set_coeffs(p.lam, p.fa, p.fk)
    x = p.x0.copy()
    st = s.solve(p.b, x)
    fresh = Solver(p.grid)
    fresh.set_coeffs(p.lam, p.fa, p.fk)
    xf = p.x0.copy()
    stf = fresh.solve(p.b, xf)
    assert st["cycles"] == stf["cycles"] and np.array_equal(x, xf)
    # a rejected set-up after a valid one: no solve until coefficients are set again
    with pytest.raises(MgError) as e:
        s.set_coeffs(lam, p.fa, p.fk)
    assert e.value.status == MG_ERR_INVALID_COEFF
    with pytest.raises(MgError) as e:
        s.solve(p.b, p.x0.copy())
    assert e.value.status == MG_ERR_STATE
    s.close()
    fresh.close()


def test_not_converged_status(torch_cuda):
    from paper_2206_11294_gb300.binding import MgError, MG_ERR_NOT_CONVERGED
    p = I.stiff(I.bubble_2d, 64)
    s = _solver(p, rtol=1e-14, max_cycles=2)
    x = p.x0.copy()
    with pytest.raises(MgError) as e:
        s.solve(p.b, x)
    assert e.value.status == MG_ERR_NOT_CONVERGED
    st = s.solve(p.b, p.x0.copy(), allow_not_converged=True)
    assert st["cycles"] == 2 and st["status"] == "MG_ERR_NOT_CONVERGED"
    s.close()


# ------------------------------------------------------------- full sizes
def _full_case(name):
    if name == "bubbles_1024":
        return I.bubbles_1024()
    if name == "axi_512x1024":
        return I.bubble_axi()
    return I.bubble_wall_3d(256)


@pytest.mark.parametrize("name", ["bubbles_1024", "axi_512x1024"])
def test_full_size_2d_vs_oracle(torch_cuda, orc, name):
    """The benchmark's 2D workloads at full size, in the launch configuration
    the benchmark times: whole-field comparison with the oracle's solve."""
    p = _full_case(name)
    s = _solver(p, rtol=1e-10, max_cycles=50)
    x = p.x0.copy()
    st = s.solve(p.b, x)
    ref, cyc, hist = orc.mg_solve(p.grid.as_dict(), p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=50, rtol=1e-10)
    assert st["cycles"] == cyc
    assert rel_dev(x, ref, p.x0) <= 1e-12
    s.close()


@pytest.fixture(scope="module")
def wall3d_oracle(orc):
    """The 256^3 bubble near a wall (Dirichlet on five faces, a wall at z = 0)
    and the oracle's solve of it to 1e-10 (about 20 s on one host core)."""
    p = _full_case("wall3d")
    ref, cyc, hist = orc.mg_solve(p.grid.as_dict(), p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=50, rtol=1e-10)
    return p, ref, cyc, hist


def test_full_size_3d_fp64_vs_oracle(torch_cuda, wall3d_oracle):
    """256^3, FP64, in the benchmark's launch configuration: the oracle's cycle
    count and the whole field to 1e-12."""
    p, ref, cyc, hist = wall3d_oracle
    s = _solver(p, rtol=1e-10, max_cycles=50)
    x = p.x0.copy()
    st = s.solve(p.b, x)
    assert st["cycles"] == cyc
    assert np.allclose(st["r0"], hist[0], rtol=1e-12)
    assert rel_dev(x, ref, p.x0) <= 1e-12
    s.close()


def test_full_size_3d_mixed_vs_oracle(torch_cuda, wall3d_oracle):
    """256^3, mixed precision stopped at the same 1e-10 reduction: the whole
    field against the FP64 oracle's solution to 1e-8."""
    p, ref, cyc, hist = wall3d_oracle
    s = _solver(p, precision="mixed", rtol=1e-10, max_cycles=50)
    x = p.x0.copy()
    st = s.solve(p.b, x)
    assert st["status"] == "MG_OK"
    assert max(st["rfinal"][f] / st["r0"][f] for f in range(2)) <= 1e-10
    assert rel_dev(x, ref, p.x0) <= 1e-8
    s.close()


@pytest.mark.parametrize("nu1,nu2", [(2, 2), (0, 3), (3, 1)])
def test_timing_counters(torch_cuda, nu1, nu2):
    """mg_set_timing brackets one finest-level smoothing pass per cycle (the
    pre-smoothing, or the post-smoothing when nu1 = 0); the counters say how
    many launches and sweeps that time covers, and timing does not change the
    result."""
    p = I.bubble_2d(128)
    s = _solver(p, rtol=0.0, max_cycles=3, nu1=nu1, nu2=nu2)
    s.set_tuning(dict(s.tuning(), sweep=["colour"] * len(s.levels())))
    x0 = p.x0.copy()
    s.solve(p.b, x0)
    s.set_timing(True)
    x = p.x0.copy()
    st = s.solve(p.b, x)
    c = s.counters()
    per = nu1 if nu1 > 0 else nu2
    assert st["cycles"] == 3
    assert c["smooth_sweeps"] == 3 * per and c["smooth_launches"] == 3 * 2 * per   # two colour launches a sweep
    assert c["smooth_ms"] > 0.0 and c["smooth_cells"] == p.grid.N and c["launches"] > c["smooth_launches"]
    assert np.array_equal(x, x0)
    s.set_timing(True)                  # unchanged setting: counters reset, graphs kept
    assert s.counters()["launches"] == 0 and s.counters()["smooth_ms"] == 0.0
    s.set_timing(False)
    x = p.x0.copy()
    s.solve(p.b, x)
    c = s.counters()
    assert c["smooth_launches"] == 0 and c["launches"] > 0 and np.array_equal(x, x0)
    s.close()


def test_setup_graph_follows_inputs(torch_cuda):
    """The set-up of the levels is a captured graph keyed by the input
    pointers: new values behind the same pointers (host staging, or the same
    device tensors refilled) and new pointers both give the result of a fresh
    handle, bit for bit."""
    torch = torch_cuda
    from paper_2206_11294_gb300.binding import Solver
    pa = I.bubble_2d(96, seed=3)
    pb = I.bubble_2d(96, seed=4, n_bubbles=3, rmin=0.08, rmax=0.15)

    def fresh(p):
        s = _solver(p)
        x = p.x0.copy()
        st = s.solve(p.b, x)
        s.close()
        return x, st["cycles"]

    ref = {"a": fresh(pa), "b": fresh(pb)}
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    dev = {n: dict(lam=T(p.lam), fa=[T(f) for f in p.fa], fk=[T(f) for f in p.fk]) for n, p in (("a", pa), ("b", pb))}
    s = Solver(pa.grid)
    # more distinct pointer sets than the handle keeps graphs for (4): replaced ones are captured again
    extra = [(n, dict(lam=T(p.lam), fa=[T(f) for f in p.fa], fk=[T(f) for f in p.fk]))
             for n, p in (("a", pa), ("b", pb), ("a", pa), ("b", pb))]
    for n, d in extra + extra:
        p = pa if n == "a" else pb
        s.set_coeffs(d["lam"], d["fa"], d["fk"])
        x = p.x0.copy()
        st = s.solve(p.b, x)
        assert st["cycles"] == ref[n][1] and np.array_equal(x, ref[n][0]), n
    for name, how in [("a", "host"), ("b", "host"), ("a", "dev"), ("b", "dev"), ("a", "dev"), ("b", "refill")]:
        p = pa if name == "a" else pb
        if how == "host":
            s.set_coeffs(p.lam, p.fa, p.fk)
        elif how == "dev":
            d = dev[name]
            s.set_coeffs(d["lam"], d["fa"], d["fk"])
        else:                                   # the tensors of "a", refilled with the values of "b"
            d = dev["a"]
            d["lam"].copy_(T(p.lam))
            for dst, src in zip(d["fa"] + d["fk"], p.fa + p.fk):
                dst.copy_(T(src))
            s.set_coeffs(d["lam"], d["fa"], d["fk"])
        x = p.x0.copy()
        st = s.solve(p.b, x)
        assert st["cycles"] == ref[name][1], (name, how)
        assert np.array_equal(x, ref[name][0]), (name, how)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("on_device", [False, True])
def test_no_cycle_when_stop_test_met_at_start(torch_cuda, precision, on_device):
    """The first iteration is launched before the initial norms are read; when
    they already meet the stop test (exactly zero here, or rtol >= 1), or no
    cycle is allowed, the solve reports zero cycles and x is left as given, bit
    for bit, from host and from device arrays."""
    torch = torch_cuda
    p = I.bubble_2d(64)                              # walls: no boundary data
    zero_b = np.zeros_like(p.b)
    zero_x = np.zeros_like(p.x0)
    cases = [(dict(), zero_b, zero_x), (dict(rtol=2.0), p.b, p.x0), (dict(max_cycles=0), p.b, p.x0)]
    for kw, b, x0 in cases:
        s = _solver(p, precision=precision, **kw)
        if on_device:
            bd = torch.from_numpy(np.ascontiguousarray(b)).cuda()
            xd = torch.from_numpy(np.ascontiguousarray(x0)).cuda()
            st = s.solve(bd, xd, allow_not_converged=True)
            x = xd.cpu().numpy()
        else:
            x = x0.copy()
            st = s.solve(b, x, allow_not_converged=True)
        assert st["cycles"] == 0 and st["outer"] == 0, kw
        assert np.array_equal(x, x0), kw
        assert list(st["rfinal"]) == list(st["r0"])
        if "max_cycles" in kw:
            assert st["status"] == "MG_ERR_NOT_CONVERGED"
        else:
            assert st["status"] == "MG_OK"
        # the handle stays usable: a normal solve afterwards matches a fresh handle
        x = p.x0.copy()
        st = s.solve(p.b, x, allow_not_converged=True)
        f = _solver(p, precision=precision, **kw)
        xf = p.x0.copy()
        stf = f.solve(p.b, xf, allow_not_converged=True)
        assert st["cycles"] == stf["cycles"] and np.array_equal(x, xf)
        s.close()
        f.close()


def _large_coarse_cases():
    return {
        # 736 = 23 x 32: the coarsest level is 23 x 23 cells (1058 unknowns)
        "2d_736_bubbles": I.bubble_2d(736, seed=95, n_bubbles=5, rmin=0.03, rmax=0.1, centred=False),
        # coarsest 9 x 13 (234 unknowns), stiff, Dirichlet and wall sides
        "2d_stiff_9x13": I.random_coeff_problem(I.Grid(dim=2, axisym=0, n=(144, 208, 1), h=1e-4,
                                                       bc=((D, W), (W, D), (0, 0)), bcT=((310, 0), (0, 290), (0, 0)),
                                                       bcp=((1.1e5, 0), (0, 0.9e5), (0, 0))), seed=96, dt=1e-5),
        # coarsest 5 x 7 x 3 (210 unknowns, band 71): too wide for the windowed LU
        "3d_5x7x3": I.random_coeff_problem(I.Grid(dim=3, axisym=0, n=(40, 56, 24), h=1e-4, bc=((W, D), (W, W), (D, W)),
                                                  bcT=((0, 300), (0, 0), (300, 0)), bcp=((0, 1e5), (0, 0), (1e5, 0))),
                                           seed=97, dt=1e-5),
        # coarsest 6 x 6 x 6 (432 unknowns, band 73): the LU blocked over a cluster, 3D
        "3d_6x6x6": I.random_coeff_problem(I.Grid(dim=3, axisym=0, n=(48, 48, 48), h=1e-4, bc=((D, W), (W, W), (W, D)),
                                                  bcT=((300, 0), (0, 0), (0, 300)), bcp=((1e5, 0), (0, 0), (0, 1e5))),
                                           seed=98, dt=1e-5),
    }


@pytest.mark.parametrize("coarse", ["auto", "inverse"])
@pytest.mark.parametrize("name", ["2d_736_bubbles", "2d_stiff_9x13", "3d_5x7x3", "3d_6x6x6"])
def test_large_coarsest_levels_vs_oracle(torch_cuda, orc, name, coarse):
    """Coarsest levels above 128 unknowns take the windowed banded LU; each
    cycle then solves from the factors (auto) or multiplies by the
    block-column inverse (inverse): FP64 solves after fixed cycles match the
    oracle (whose coarsest solve is Gaussian elimination) at the usual
    tolerance, and mixed precision reaches the converged oracle."""
    p = _large_coarse_cases()[name]
    g = p.grid.as_dict()
    tol = 1e-9 if "stiff" in name or "3d" in name else 1e-12
    s = _solver(p, rtol=0.0, max_cycles=2, coarse=coarse)
    lv = s.levels()
    assert 2 * int(np.prod(lv[-1])) > 128
    x = p.x0.copy()
    st = s.solve(p.b, x)
    ref, cyc, _ = orc.mg_solve(g, p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=2, rtol=0.0)
    assert st["cycles"] == 2 == cyc
    assert rel_dev(x, ref, p.x0) <= tol
    s.close()
    s = _solver(p, precision="mixed", rtol=1e-12 if tol > 1e-12 else 1e-10, max_cycles=80, coarse=coarse)
    xm = p.x0.copy()
    s.solve(p.b, xm)
    conv, _, _ = orc.mg_solve(g, p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=80, rtol=1e-13)
    assert rel_dev(xm, conv, p.x0) <= 1e-8
    s.close()


@pytest.mark.parametrize("name", ["2d_736_bubbles", "2d_stiff_9x13", "3d_5x7x3", "3d_6x6x6"])
def test_factored_coarse_solve_equals_inverse(torch_cuda, name):
    """The two coarsest solves are exact up to rounding: the same cycle count
    and results within 1e-13 of the deviation, FP64 and mixed (1e-11 on the
    stiff and 3D cases, whose rows carry the 1e5 Pa background: a rounding
    difference anywhere is amplified there as in the oracle comparisons).
    The factored one forms no inverse (smaller workspace) and refuses the
    tail kernel, which multiplies by the inverse; its autotuner picks no
    tail.  The 5 x 7 x 3 coarsest level (210 unknowns, band 71) is too wide
    for the windowed LU and keeps the inverse either way."""
    from paper_2206_11294_gb300.binding import MgError, MG_ERR_INVALID_ARG
    p = _large_coarse_cases()[name]
    tol = 1e-11 if "stiff" in name or "3d" in name else 1e-13
    factored = name != "3d_5x7x3"
    for prec, rtol in (("fp64", 1e-10), ("mixed", 1e-10)):
        a = _solver(p, precision=prec, rtol=rtol, max_cycles=80)
        b = _solver(p, precision=prec, rtol=rtol, max_cycles=80, coarse="inverse")
        assert (a.workspace_bytes < b.workspace_bytes) if factored else (a.workspace_bytes == b.workspace_bytes)
        xa, xb = p.x0.copy(), p.x0.copy()
        sa, sb = a.solve(p.b, xa), b.solve(p.b, xb)
        assert sa["cycles"] == sb["cycles"] and sa["outer"] == sb["outer"]
        assert rel_dev(xa, xb, p.x0) <= tol
        if factored:
            t = a.tuning()
            n = t["levels"]
            assert t["tail_level"] >= n
            for lvl in range(1, n - 1):
                with pytest.raises(MgError) as e:
                    a.set_tuning(dict(t, tail_level=lvl))
                assert e.value.status == MG_ERR_INVALID_ARG
            tuned, _ = a.autotune(reps=1)
            assert tuned["tail_level"] >= n
            x2 = p.x0.copy()
            assert a.solve(p.b, x2)["cycles"] == sa["cycles"] and np.array_equal(x2, xa)
        a.close()
        b.close()
