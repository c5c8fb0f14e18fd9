"""The momentum predictor (mg_momentum_*) against the FP64 oracle (oracle/momentum.py).

apply(): element by element.  The GPU forms the same face stresses with 1/h
and 1/dt taken once and the tangential derivatives from the same cells; the
results differ by rounding, bounded by 1e-12 of the largest term of the row
(rho u/dt, the stress differences over h, the hoop term).
solve(): R is the oracle's A(u_true), so u_true is the discrete solution (the
oracle's direct solve of such systems is pinned on the CPU); the device
solution must match it to the accuracy the stopping tolerance gives (rtol
1e-12 on ||dt r/rho||: 1e-9 relative to u).
"""
import numpy as np
import pytest

from paper_2206_11294_gb300 import inputs as I

pytestmark = pytest.mark.gpu

W, D, AX = I.BC_WALL, I.BC_DIRICHLET, I.BC_AXIS


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_11294_gb300 import binding
    binding.load()
    return torch


@pytest.fixture(scope="module")
def orc():
    from oracle import momentum
    return momentum


GRIDS = {
    "2d": I.Grid(dim=2, axisym=0, n=(64, 48, 1), h=1e-2, bc=((W, D), (W, W), (0, 0))),
    "2d_ragged": I.Grid(dim=2, axisym=0, n=(40, 36, 1), h=1e-2, bc=((D, W), (W, D), (0, 0))),
    "axi": I.Grid(dim=2, axisym=1, n=(32, 64, 1), h=1e-2, r0=0.0, bc=((AX, W), (W, D), (0, 0))),
    "3d": I.Grid(dim=3, axisym=0, n=(40, 16, 16), h=1e-2, bc=((W, D), (W, W), (D, W))),
}


def _fields(g, seed, viscous=1.0):
    """rho in [1, 1000], mu in [1e-3, 1] x viscous, a smooth velocity plus noise, dt 1e-2."""
    rng = np.random.default_rng(seed)
    shape = (g.n[2], g.n[1], g.n[0])
    rho = rng.uniform(1.0, 1000.0, shape)
    mu = viscous * rng.uniform(1e-3, 1.0, shape)
    X = np.meshgrid(*[(np.arange(g.n[a]) + 0.5) * g.h for a in (2, 1, 0)], indexing="ij")[::-1]
    u = [np.sin(3.0 * X[0] + c) * np.cos(2.0 * X[1] - c) + 0.1 * rng.normal(size=shape) for c in range(g.dim)]
    return rho, mu, 1e-2, u


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _row_scale(g, rho, mu, dt, u):
    U = max(np.abs(v).max() for v in u)
    return rho / dt * U + 16 * g.dim * np.abs(mu).max() * U / g.h ** 2 * (4 if g.axisym else 1)


@pytest.mark.parametrize("no_slip", [False, True])
@pytest.mark.parametrize("name", list(GRIDS))
def test_apply_matches_oracle(torch_cuda, orc, name, no_slip):
    from paper_2206_11294_gb300.binding import Momentum
    torch = torch_cuda
    g = GRIDS[name]
    rho, mu, dt, u = _fields(g, 40 + len(name))
    m = Momentum(g, no_slip=no_slip)
    m.set_coeffs(dt, _dev(torch, rho), _dev(torch, mu))
    ud = [_dev(torch, v) for v in u]
    yd = [torch.empty_like(v) for v in ud]
    m.apply(ud, yd)
    ref = orc.apply(g, rho, mu, dt, u, no_slip=no_slip)
    scale = _row_scale(g, rho, mu, dt, u)
    for c in range(g.dim):
        err = np.abs(yd[c].cpu().numpy() - ref[c])
        assert np.all(err <= 1e-12 * scale), (c, float((err / scale).max()))
    m.close()


@pytest.mark.parametrize("krylov", [False, True])
@pytest.mark.parametrize("no_slip", [False, True])
@pytest.mark.parametrize("name", list(GRIDS))
def test_solve_recovers_discrete_solution(torch_cuda, orc, name, no_slip, krylov):
    from paper_2206_11294_gb300.binding import Momentum
    torch = torch_cuda
    g = GRIDS[name]
    rho, mu, dt, exact = _fields(g, 50 + len(name))
    R = orc.apply(g, rho, mu, dt, exact, no_slip=no_slip)
    m = Momentum(g, no_slip=no_slip, krylov=krylov)
    m.set_coeffs(dt, _dev(torch, rho), _dev(torch, mu))
    ud = [torch.zeros(rho.shape, dtype=torch.float64, device="cuda") for _ in range(g.dim)]
    st = m.solve([_dev(torch, r) for r in R], ud, rtol=1e-12, max_iters=300)
    assert st["status"] == "MG_OK" and st["rfinal"] <= 1e-12 * st["r0"], st
    for c in range(g.dim):
        got = ud[c].cpu().numpy()
        err = np.linalg.norm(got - exact[c]) / np.linalg.norm(exact[c])
        assert err <= 1e-9, (c, err, st)
    m.close()


def test_viscous_dominated_converges(torch_cuda, orc):
    """mu dt / (rho h^2) up to ~1e4: the cross terms are as large as the diagonal stresses.  With exact
    correction solves the outer iteration contracts by ~0.64 per step here (the spectrum of A_diag^-1 A lies in
    [0.36, 1.64] for this kind of field); two V-cycles per correction must stay close to that."""
    from paper_2206_11294_gb300.binding import Momentum
    torch = torch_cuda
    g = GRIDS["2d"]
    rho, mu, dt, u_true = _fields(g, 61, viscous=1.0)
    rho = np.ones_like(rho)
    dt = 1.0
    R = orc.apply(g, rho, mu, dt, u_true)
    m = Momentum(g, inner_cycles_per_step=2)
    m.set_coeffs(dt, _dev(torch, rho), _dev(torch, mu))
    ud = [torch.zeros(rho.shape, dtype=torch.float64, device="cuda") for _ in range(g.dim)]
    st = m.solve([_dev(torch, r) for r in R], ud, rtol=1e-10, max_iters=300)
    assert st["status"] == "MG_OK", st
    assert st["iterations"] <= 90, st
    for c in range(g.dim):
        err = np.linalg.norm(ud[c].cpu().numpy() - u_true[c]) / np.linalg.norm(u_true[c])
        assert err <= 1e-6, (c, err, st)
    m.close()
    # GMRES right-preconditioned by the same correction: far fewer steps (~20-25 with exact corrections)
    k = Momentum(g, inner_cycles_per_step=2, krylov=True)
    k.set_coeffs(dt, _dev(torch, rho), _dev(torch, mu))
    uk = [torch.zeros(rho.shape, dtype=torch.float64, device="cuda") for _ in range(g.dim)]
    sk = k.solve([_dev(torch, r) for r in R], uk, rtol=1e-10, max_iters=300)
    assert sk["status"] == "MG_OK" and sk["iterations"] <= 30 and sk["iterations"] < st["iterations"], (sk, st)
    for c in range(g.dim):
        err = np.linalg.norm(uk[c].cpu().numpy() - u_true[c]) / np.linalg.norm(u_true[c])
        assert err <= 1e-6, (c, err, sk)
    k.close()


def test_full_size_bubbles_state(torch_cuda, orc):
    """The 16-bubble 1024^2 state, rho = m1 + m2, mu = C mu_1 + (1 - C) mu_2, R = (rho u)^(adv) / dt, at dt = 1e-7
    and at dt = 1e-3 (viscous-dominated in the gas): the device solution's residual by the oracle's operator.  At
    dt = 1e-7 the start is within ~1e-7 of the solution relative to rho u / dt, so the library iterates on the
    correction (r0 - A delta) rather than on R - A(u)."""
    from paper_2206_11294_gb300.binding import Momentum
    torch = torch_cuda
    s = I.bubbles_state_1024()
    g = s.grid
    rho = s.m1 + s.m2
    mu = s.C * s.ph1.mu + (1 - s.C) * s.ph2.mu
    m = Momentum(g)
    for dt in (1e-7, 1e-3):
        R = [mom / dt for mom in s.mom]
        m.set_coeffs(dt, _dev(torch, rho), _dev(torch, mu))
        u0 = [mom / rho for mom in s.mom]
        ud = [_dev(torch, v) for v in u0]
        st = m.solve([_dev(torch, r) for r in R], ud, rtol=1e-10, max_iters=200)
        assert st["status"] == "MG_OK", (dt, st)
        u = [v.cpu().numpy() for v in ud]
        res = [R[c] - a for c, a in enumerate(orc.apply(g, rho, mu, dt, u))]
        num = np.sqrt(sum(np.sum((dt * r / rho) ** 2) for r in res))
        res0 = [R[c] - a for c, a in enumerate(orc.apply(g, rho, mu, dt, u0))]
        den = np.sqrt(sum(np.sum((dt * r / rho) ** 2) for r in res0))
        # R - A(u) is formed from terms of size rho u / dt: below a few ulps of those no check can see further
        floor = 16 * np.finfo(float).eps * np.sqrt(sum(np.sum((dt * r / rho) ** 2) for r in R))
        assert num <= 2e-10 * den + floor, (dt, num, den, floor, st)
        # the diffusion number picks the corrections: point-Jacobi at the time step's dt, multigrid at 1e-3
        assert st["jacobi"] == (dt == 1e-7), st
        if dt == 1e-7:
            mg = Momentum(g, multigrid_only=True)
            mg.set_coeffs(dt, _dev(torch, rho), _dev(torch, mu))
            um = [_dev(torch, v) for v in u0]
            sm = mg.solve([_dev(torch, r) for r in R], um, rtol=1e-10, max_iters=200)
            assert not sm["jacobi"] and sm["nu"] == st["nu"], (sm, st)
            for c in range(g.dim):
                d_j = u[c] - u0[c]
                d_m = um[c].cpu().numpy() - u0[c]
                assert np.linalg.norm(d_j - d_m) <= 1e-8 * np.linalg.norm(d_j), c
            mg.close()
    m.close()


@pytest.mark.parametrize("name", list(GRIDS))
def test_jacobi_corrections_recover_discrete_solution(torch_cuda, orc, name):
    """A small diffusion number (mu dt / (rho h^2) <= 1e-5, Jacobi bound <= 2e-3 in 3D): point-Jacobi corrections,
    no hierarchy."""
    from paper_2206_11294_gb300.binding import Momentum
    torch = torch_cuda
    g = GRIDS[name]
    rho, mu, _, exact = _fields(g, 95 + len(name))
    mu = mu * 1e-4
    dt = 1e-4
    R = orc.apply(g, rho, mu, dt, exact)
    m = Momentum(g)
    m.set_coeffs(dt, _dev(torch, rho), _dev(torch, mu))
    ud = [torch.zeros(rho.shape, dtype=torch.float64, device="cuda") for _ in range(g.dim)]
    st = m.solve([_dev(torch, r) for r in R], ud, rtol=1e-12, max_iters=50)
    assert st["jacobi"] and st["cycles"] == 0 and st["iterations"] <= 6, st
    for c in range(g.dim):
        err = np.linalg.norm(ud[c].cpu().numpy() - exact[c]) / np.linalg.norm(exact[c])
        assert err <= 1e-11, (c, err, st)
    m.close()


def test_invalid_use_rejected(torch_cuda):
    from paper_2206_11294_gb300 import binding as B
    from paper_2206_11294_gb300.binding import Momentum, MgError, MG_ERR_INVALID_ARG, MG_ERR_STATE
    torch = torch_cuda
    g = GRIDS["2d"]
    rho, mu, dt, u = _fields(g, 70)
    m = Momentum(g)
    ud = [_dev(torch, v) for v in u]
    with pytest.raises(MgError) as e:
        m.solve(ud, [torch.empty_like(v) for v in ud])
    assert e.value.status == MG_ERR_STATE
    with pytest.raises(MgError) as e:
        m.set_coeffs(0.0, _dev(torch, rho), _dev(torch, mu))
    assert e.value.status == MG_ERR_INVALID_ARG
    m.set_coeffs(dt, _dev(torch, rho), _dev(torch, mu))
    with pytest.raises(MgError) as e:
        m.solve(ud, ud)                                   # R aliases u
    assert e.value.status == MG_ERR_INVALID_ARG
    with pytest.raises(MgError) as e:
        m.apply(ud, ud)
    assert e.value.status == MG_ERR_INVALID_ARG
    import ctypes as C
    h = C.c_void_p()
    with pytest.raises(MgError) as e:
        B.check(B.load().mg_momentum_create(C.byref(B.make_grid(g)), 8, None, None, C.byref(h)))
    assert e.value.status == MG_ERR_INVALID_ARG
    o = B.make_options("mixed", 0.0, 1)                  # the correction solves run in FP64
    with pytest.raises(MgError) as e:
        B.check(B.load().mg_momentum_create(C.byref(B.make_grid(g)), 0, C.byref(o), None, C.byref(h)))
    assert e.value.status == MG_ERR_INVALID_ARG
    m.close()


def _side_inputs(g, seed):
    rng = np.random.default_rng(seed)
    shape = (g.n[2], g.n[1], g.n[0])
    mom = [rng.normal(0.0, 50.0, shape) for _ in range(g.dim)]
    p = 1e5 + rng.normal(0.0, 300.0, shape)
    kappa = rng.normal(0.0, 100.0, shape)
    C = rng.uniform(0.0, 1.0, shape)
    rho = rng.uniform(1.0, 1000.0, shape)
    u = [rng.normal(size=shape) for _ in range(g.dim)]
    return mom, p, kappa, C, rho, u


def _with_pressure_values(g):
    import dataclasses
    return dataclasses.replace(g, bcp=((1.01e5, 0.99e5), (1.0e5, 1.02e5), (0.98e5, 1.0e5)))


@pytest.mark.parametrize("name", list(GRIDS))
def test_rhs_and_provisional_match_oracle(torch_cuda, orc, name):
    from paper_2206_11294_gb300 import binding as B
    torch = torch_cuda
    g = _with_pressure_values(GRIDS[name])
    mom, p, kappa, C, rho, u = _side_inputs(g, 80 + len(name))
    dt, sigma = 1e-4, 0.072
    R = [torch.empty(p.shape, dtype=torch.float64, device="cuda") for _ in range(g.dim)]
    B.momentum_rhs(g, dt, sigma, [_dev(torch, m_) for m_ in mom], _dev(torch, p), _dev(torch, kappa), _dev(torch, C), R)
    uf = [torch.empty(g.face_shape(a), dtype=torch.float64, device="cuda") for a in range(g.dim)]
    B.provisional(g, dt, _dev(torch, rho), _dev(torch, p), [_dev(torch, v) for v in u], uf)
    torch.cuda.synchronize()
    ref_R = orc.rhs(g, dt, sigma, mom, p, kappa, C)
    gp = orc.cell_gradient(g, p, g.bcp)
    gC = orc.cell_gradient(g, C)
    for c in range(g.dim):
        scale = np.abs(mom[c] / dt) + np.abs(gp[c]) + np.abs(sigma * kappa * gC[c]) + 1e-300
        err = np.abs(R[c].cpu().numpy() - ref_R[c])
        assert np.all(err <= 1e-13 * scale), (c, float((err / scale).max()))
    ref_f = orc.provisional_faces(g, dt, rho, p, u)
    for a in range(g.dim):
        ustar = np.abs(u[a]) + np.abs(dt / rho * gp[a])
        s = np.zeros(g.face_shape(a))
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[2 - a] = slice(0, -1)
        hi[2 - a] = slice(1, None)
        s[tuple(lo)] += ustar
        s[tuple(hi)] += ustar
        err = np.abs(uf[a].cpu().numpy() - ref_f[a])
        assert np.all(err <= 1e-13 * s + 1e-300), (a, float((err / (s + 1e-300)).max()))


def test_predictor_chain_matches_oracle(torch_cuda, orc):
    """R, the predictor solve and Eq. provel on the device against the oracle's R, its direct solve and its
    face velocities (the solve converged to rtol 1e-12)."""
    from paper_2206_11294_gb300 import binding as B
    from paper_2206_11294_gb300.binding import Momentum
    torch = torch_cuda
    g = _with_pressure_values(GRIDS["2d_ragged"])
    mom, p, kappa, C, rho, _ = _side_inputs(g, 90)
    mu = np.random.default_rng(91).uniform(1e-3, 1.0, rho.shape)
    dt, sigma = 1e-3, 0.072
    R = [torch.empty(p.shape, dtype=torch.float64, device="cuda") for _ in range(g.dim)]
    B.momentum_rhs(g, dt, sigma, [_dev(torch, m_) for m_ in mom], _dev(torch, p), _dev(torch, kappa), _dev(torch, C), R)
    m = Momentum(g)
    m.set_coeffs(dt, _dev(torch, rho), _dev(torch, mu))
    u = [_dev(torch, m_ / rho) for m_ in mom]
    st = m.solve(R, u, rtol=1e-12, max_iters=300)
    assert st["status"] == "MG_OK", st
    uf = [torch.empty(g.face_shape(a), dtype=torch.float64, device="cuda") for a in range(g.dim)]
    B.provisional(g, dt, _dev(torch, rho), _dev(torch, p), u, uf)
    torch.cuda.synchronize()
    ref_R = orc.rhs(g, dt, sigma, mom, p, kappa, C)
    u_ref = orc.solve(g, rho, mu, dt, ref_R)
    ref_f = orc.provisional_faces(g, dt, rho, p, u_ref)
    for a in range(g.dim):
        got = uf[a].cpu().numpy()
        err = np.linalg.norm(got - ref_f[a]) / np.linalg.norm(ref_f[a])
        assert err <= 1e-9, (a, err, st)
    m.close()


@pytest.mark.parametrize("name", ["2d", "axi", "3d"])
def test_inviscid_predictor_is_one_jacobi_step(torch_cuda, name):
    """mu = 0 (the paper's inviscid water): A = (rho/dt) I, the Jacobi bound is 0 and one step gives u = dt R / rho."""
    from paper_2206_11294_gb300.binding import Momentum
    torch = torch_cuda
    g = GRIDS[name]
    rho, _, dt, _ = _fields(g, 101)
    rng = np.random.default_rng(102)
    R = [rng.normal(0.0, 1e6, rho.shape) for _ in range(g.dim)]
    m = Momentum(g)
    m.set_coeffs(dt, _dev(torch, rho), _dev(torch, np.zeros_like(rho)))
    ud = [torch.zeros(rho.shape, dtype=torch.float64, device="cuda") for _ in range(g.dim)]
    st = m.solve([_dev(torch, r) for r in R], ud, rtol=1e-12, max_iters=10)
    assert st["jacobi"] and st["nu"] == 0.0 and st["iterations"] == 1 and st["rfinal"] <= 1e-15 * st["r0"], st
    for c in range(g.dim):
        np.testing.assert_allclose(ud[c].cpu().numpy(), dt * R[c] / rho, rtol=1e-15, atol=0)
    m.close()


def test_uniform_provisional_velocity(torch_cuda, orc):
    """Uniform u_pred and a uniform pressure equal to the boundary values: interior faces carry u exactly, walls 0."""
    from paper_2206_11294_gb300 import binding as B
    import dataclasses
    torch = torch_cuda
    g = dataclasses.replace(GRIDS["2d"], bcp=((1e5, 1e5), (1e5, 1e5), (0.0, 0.0)))
    shape = (1, g.n[1], g.n[0])
    u = [np.full(shape, 0.3), np.full(shape, -0.7)]
    uf = [torch.empty(g.face_shape(a), dtype=torch.float64, device="cuda") for a in range(2)]
    B.provisional(g, 1e-3, _dev(torch, np.full(shape, 2.0)), _dev(torch, np.full(shape, 1e5)), [_dev(torch, v) for v in u], uf)
    torch.cuda.synchronize()
    for a in range(2):
        got = uf[a].cpu().numpy()
        ref = orc.provisional_faces(g, 1e-3, np.full(shape, 2.0), np.full(shape, 1e5), u)[a]
        np.testing.assert_array_equal(got, ref)
        inner = [slice(None)] * 3
        inner[2 - a] = slice(1, -1)
        np.testing.assert_array_equal(got[tuple(inner)], u[a][0, 0, 0])
