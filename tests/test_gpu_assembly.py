"""Coefficient assembly (mg_assemble_async) and the update after the solve
(mg_correct_async) against the FP64 oracle, element by element.

Tolerances follow the arithmetic: the GPU evaluates the same formulas with
reciprocals taken once (1/dt, 1/h, 1/(Gamma - 1), 1/c_p) and the per-phase
terms arranged to need three divisions, so results differ by rounding only.
p^(adv) is a difference of terms of size Gamma Pi / (Gamma - 1) ~ 4e9 (liquid):
its bound is 64 ulps of that.  The bracket of lambda_3 cancels two terms of
similar size: 1e-10 relative.  lambda_p adds lambda_3 p and div(u*)/dt, which
can cancel: its bound is relative to the larger term.  Everything else: 1e-12
relative.
"""
import numpy as np
import pytest

from paper_2206_11294_gb300 import inputs as I

pytestmark = pytest.mark.gpu

W, D, AX = I.BC_WALL, I.BC_DIRICHLET, I.BC_AXIS
EPS = np.finfo(float).eps


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
    from oracle import assembly
    return assembly


GRIDS = {
    "2d_walls": I.Grid(dim=2, axisym=0, n=(200, 72, 1), h=1e-3, bc=((W, W), (W, W), (0, 0))),
    "2d_dirichlet": I.Grid(dim=2, axisym=0, n=(33, 70, 1), h=1e-3, bc=((D, W), (W, D), (0, 0)),
                           bcT=((300.0, 0.0), (0.0, 305.0), (0, 0)), bcp=((1.02e5, 0.0), (0.0, 0.99e5), (0, 0))),
    "axi": I.Grid(dim=2, axisym=1, n=(96, 160, 1), h=1e-3, r0=0.0, bc=((AX, W), (W, D), (0, 0)),
                  bcp=((0, 0), (0.0, 1.01e5), (0, 0))),
    "3d": I.Grid(dim=3, axisym=0, n=(40, 24, 20), h=1e-3, bc=((W, D), (W, W), (D, W)),
                 bcp=((0.0, 1e5), (0, 0), (1.01e5, 0.0))),
}


def _state(g, seed=21):
    X = I._centres(g)
    c = [X[a].mean() for a in range(g.dim)]
    R = 0.3 * min(g.n[a] * g.h for a in range(g.dim))
    return I.advected_state(g, I.volume_fraction(g, [c], [R]), seed)


def _dev(torch, s):
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    return dict(C=T(s.C), m1=T(s.m1), m2=T(s.m2), E=T(s.E), mom=[T(m) for m in s.mom], uf=[T(u) for u in s.uf],
                kappa=T(s.kappa))


def _gpu_assemble(torch, s, lambda4_printed=False, with_x0=True, harmonic_k=False):
    from paper_2206_11294_gb300 import binding as B
    g = s.grid
    d = _dev(torch, s)
    N = g.N
    z = lambda *shape: torch.zeros(*shape, dtype=torch.float64, device="cuda")
    out = dict(lam=z(N, 4), b=z(N, 2), x0=z(N, 2) if with_x0 else None,
               fa=[z(*g.face_shape(a)) for a in range(g.dim)], fk=[z(*g.face_shape(a)) for a in range(g.dim)])
    B.assemble(g, (s.ph1, s.ph2), s.dt, d["C"], d["m1"], d["m2"], d["E"], d["mom"], d["uf"], out,
               lambda4_printed=lambda4_printed, harmonic_k=harmonic_k)
    torch.cuda.synchronize()
    host = {k: (v.cpu().numpy() if v is not None and not isinstance(v, list) else
                ([t.cpu().numpy() for t in v] if isinstance(v, list) else None)) for k, v in out.items()}
    return host, d, out


def _close(got, ref, tol, scale=None, what=""):
    scale = np.abs(ref) if scale is None else scale
    err = np.abs(got - ref)
    bad = err > tol * scale
    assert not np.any(bad), f"{what}: {int(bad.sum())} elements, worst {np.max(err / np.maximum(scale, 1e-300)):.3e}"


def _compare(g, s, got, ref):
    p_scale = 64 * EPS * s.ph1.Gamma * s.ph1.Pi / (s.ph1.Gamma - 1.0)
    _close(got["x0"][:, 1], ref["x0"][:, 1], 1.0, scale=np.full(g.N, p_scale), what="p_adv")
    _close(got["x0"][:, 0], ref["x0"][:, 0], 1e-12, what="T_adv")
    _close(got["lam"][:, 0], ref["lam"][:, 0], 1e-12, what="lambda_1")
    _close(got["lam"][:, 1], ref["lam"][:, 1], 1e-12, what="lambda_2")
    _close(got["lam"][:, 2], ref["lam"][:, 2], 1e-10, what="lambda_3")
    _close(got["lam"][:, 3], ref["lam"][:, 3], 1e-12, what="lambda_4")
    _close(got["b"][:, 0], ref["b"][:, 0], 1e-12, what="lambda_T")
    lp_scale = np.abs(ref["lam"][:, 2] * ref["x0"][:, 1]) + np.abs(ref["div"].reshape(-1) / s.dt)
    _close(got["b"][:, 1], ref["b"][:, 1], 1e-10, scale=lp_scale, what="lambda_p")
    for a in range(g.dim):
        _close(got["fa"][a], ref["fa"][a], 1e-14, what=f"1/rho faces {a}")
        _close(got["fk"][a], ref["fk"][a], 1e-14, what=f"k faces {a}")


@pytest.mark.parametrize("name", list(GRIDS))
@pytest.mark.parametrize("lambda4", ["restored", "printed"])
def test_assemble_matches_oracle(torch_cuda, orc, name, lambda4):
    g = GRIDS[name]
    s = _state(g)
    got, _, _ = _gpu_assemble(torch_cuda, s, lambda4_printed=lambda4 == "printed")
    ref = orc.assemble(g, s.ph1, s.ph2, s.dt, s.C, s.m1, s.m2, s.E, s.mom, s.uf, lambda4=lambda4)
    _compare(g, s, got, ref)


@pytest.mark.parametrize("name", list(GRIDS))
def test_assemble_harmonic_face_k(torch_cuda, orc, name):
    g = GRIDS[name]
    s = _state(g, seed=25)
    got, _, _ = _gpu_assemble(torch_cuda, s, harmonic_k=True)
    ref = orc.assemble(g, s.ph1, s.ph2, s.dt, s.C, s.m1, s.m2, s.E, s.mom, s.uf, face_k="harmonic")
    _compare(g, s, got, ref)


def test_assemble_pure_cells_and_no_x0(torch_cuda, orc):
    """Cells of one phase only (C exactly 0 or 1 in blocks, so a phase is absent there), at rest."""
    g = GRIDS["2d_walls"]
    s = _state(g, seed=22)
    C = np.zeros_like(s.C)
    C[:, :, : g.n[0] // 2] = 1.0
    r1, r2 = I.phase_density(s.T, s.p, s.ph1), I.phase_density(s.T, s.p, s.ph2)
    s.C, s.m1, s.m2 = C, C * r1, (1 - C) * r2
    s.mom = [np.zeros_like(C) for _ in range(g.dim)]
    s.E = C * I.phase_energy(s.p, r1, s.ph1) + (1 - C) * I.phase_energy(s.p, r2, s.ph2)
    got, _, _ = _gpu_assemble(torch_cuda, s)
    ref = orc.assemble(g, s.ph1, s.ph2, s.dt, s.C, s.m1, s.m2, s.E, s.mom, s.uf)
    _compare(g, s, got, ref)
    got2, _, _ = _gpu_assemble(torch_cuda, s, with_x0=False)
    assert got2["x0"] is None
    np.testing.assert_array_equal(got2["lam"], got["lam"])


@pytest.mark.parametrize("name", list(GRIDS))
def test_correct_matches_oracle(torch_cuda, orc, name):
    from paper_2206_11294_gb300 import binding as B
    torch = torch_cuda
    g = GRIDS[name]
    s = _state(g, seed=23)
    got, d, out = _gpu_assemble(torch, s)
    ref = orc.assemble(g, s.ph1, s.ph2, s.dt, s.C, s.m1, s.m2, s.E, s.mom, s.uf)
    rng = np.random.default_rng(4)
    x = ref["x0"] + rng.normal(0, 1.0, ref["x0"].shape) * np.array([1.0, 300.0])
    xd = torch.from_numpy(x).cuda()
    uo = [torch.empty_like(u) for u in d["uf"]]
    p1 = torch.empty_like(d["C"])
    p2 = torch.empty_like(d["C"])
    B.correct(g, s.dt, s.sigma, xd, d["C"], d["kappa"], out["fa"], d["uf"], uo, p1, p2)
    torch.cuda.synchronize()
    rc = orc.correct(g, s.dt, s.sigma, x, s.C, s.kappa, ref["fa"], s.uf)
    for a in range(g.dim):
        scale = np.abs(rc["uf"][a]) + np.abs(s.uf[a]) + 1e-30
        _close(uo[a].cpu().numpy(), rc["uf"][a], 1e-12, scale=scale, what=f"u^(n+1) faces {a}")
    _close(p1.cpu().numpy(), rc["p1"], 1e-14, what="p1")
    _close(p2.cpu().numpy(), rc["p2"], 1e-14, what="p2")
    # in place: uf_out = uf_star
    B.correct(g, s.dt, s.sigma, xd, d["C"], d["kappa"], out["fa"], d["uf"], d["uf"], p1, p2)
    torch.cuda.synchronize()
    for a in range(g.dim):
        np.testing.assert_array_equal(d["uf"][a].cpu().numpy(), uo[a].cpu().numpy())


def test_full_size_step_matches_oracle(torch_cuda, orc):
    """The 16-bubble 1024^2 state: assembly over every cell against the oracle,
    then the set-up and solve on those device arrays from (T^(adv), p^(adv)),
    and the corrected velocity's divergence against div u* - dt L_alpha p."""
    from paper_2206_11294_gb300 import binding as B
    from paper_2206_11294_gb300.binding import Solver
    torch = torch_cuda
    s = I.bubbles_state_1024()
    g = s.grid
    got, d, out = _gpu_assemble(torch, s)
    ref = orc.assemble(g, s.ph1, s.ph2, s.dt, s.C, s.m1, s.m2, s.E, s.mom, s.uf)
    _compare(g, s, got, ref)
    solver = Solver(g, rtol=1e-10)
    solver.set_coeffs(out["lam"], out["fa"], out["fk"])
    x = out["x0"].clone()
    st = solver.solve(out["b"], x)
    assert st["status"] == "MG_OK" and 1 <= st["cycles"] <= 10
    uo = [torch.empty_like(u) for u in d["uf"]]
    p1, p2 = torch.empty_like(d["C"]), torch.empty_like(d["C"])
    B.correct(g, s.dt, s.sigma, x, d["C"], d["kappa"], out["fa"], d["uf"], uo, p1, p2)
    torch.cuda.synchronize()
    # the correction removes dt div((1/rho) grad p) from div u*: check it against the independent sparse
    # assembly of that operator (tests/fv_matrix.py) on the solved p
    from fv_matrix import laplacian
    div_new = orc.div_faces(g, [u.cpu().numpy() for u in uo]).reshape(-1)
    div_old = ref["div"].reshape(-1)
    La, _ = laplacian(g, [f.reshape(-1) for f in got["fa"]])      # walls only: no boundary-value part
    Lp = La @ x.cpu().numpy()[:, 1]
    expect = div_old - s.dt * Lp
    scale = np.abs(div_old) + s.dt * np.abs(Lp) + 1.0
    _close(div_new, expect, 1e-10, scale=scale, what="div u^(n+1)")
    solver.close()


def test_invalid_arguments_rejected(torch_cuda):
    from paper_2206_11294_gb300 import binding as B
    from paper_2206_11294_gb300.binding import MgError, MG_ERR_INVALID_ARG
    torch = torch_cuda
    g = GRIDS["2d_walls"]
    s = _state(g, seed=24)
    d = _dev(torch, s)
    N = g.N
    z = lambda *shape: torch.zeros(*shape, dtype=torch.float64, device="cuda")
    out = dict(lam=z(N, 4), b=z(N, 2), x0=None, fa=[z(*g.face_shape(a)) for a in range(2)],
               fk=[z(*g.face_shape(a)) for a in range(2)])
    bad_phase = I.NasgPhase(Gamma=1.0, Pi=0.0, b=0.0, q=0.0, cp=1000.0, cv=700.0, k=0.1)
    cases = [
        dict(dt=0.0),
        dict(phases=(s.ph1, bad_phase)),
        dict(host_C=True),
    ]
    for c in cases:
        with pytest.raises((MgError, TypeError)) as e:
            if c.get("host_C"):
                # a host pointer where a device array is required (bypassing the binding's own check)
                import ctypes as C_
                st = B.MgState()
                host = np.ascontiguousarray(s.C)
                st.C = C_.c_void_p(host.ctypes.data)
                st.m1, st.m2, st.E = (C_.c_void_p(t.data_ptr()) for t in (d["m1"], d["m2"], d["E"]))
                for a in range(2):
                    st.mom[a] = C_.c_void_p(d["mom"][a].data_ptr())
                    st.uf[a] = C_.c_void_p(d["uf"][a].data_ptr())
                res = B.MgAssembly()
                res.lam, res.rhs = C_.c_void_p(out["lam"].data_ptr()), C_.c_void_p(out["b"].data_ptr())
                for a in range(2):
                    res.face_alpha[a] = C_.c_void_p(out["fa"][a].data_ptr())
                    res.face_k[a] = C_.c_void_p(out["fk"][a].data_ptr())
                ph = (B.MgPhase * 2)(B.make_phase(s.ph1), B.make_phase(s.ph2))
                B.check(B.load().mg_assemble_async(C_.byref(B.make_grid(g)), ph, s.dt, 0, C_.byref(st), C_.byref(res),
                                             None))
            else:
                B.assemble(g, c.get("phases", (s.ph1, s.ph2)), c.get("dt", s.dt), d["C"], d["m1"], d["m2"], d["E"],
                           d["mom"], d["uf"], out)
        if isinstance(e.value, MgError):
            assert e.value.status == MG_ERR_INVALID_ARG
    assert float(out["lam"].abs().sum()) == 0.0          # nothing written by a rejected call


@pytest.mark.parametrize("inner", [1, 2])
def test_full_size_mixed_solve_converges(torch_cuda, inner):
    """From (T^(adv), p^(adv)) the first residual is small against lambda_T
    (~1e16 at these units): mixed precision iterates on the correction from x0
    (the paper's defect-correction form) and reaches 1e-10 like FP64; the two
    agree to 1e-8 in the deviation from x0, per field."""
    from paper_2206_11294_gb300 import binding as B
    from paper_2206_11294_gb300.binding import Solver
    torch = torch_cuda
    s = I.bubbles_state_1024()
    g = s.grid
    _, d, out = _gpu_assemble(torch, s)
    xs = {}
    for prec in ("fp64", "mixed"):
        sv = Solver(g, precision=prec, rtol=1e-10, max_cycles=30, inner_cycles=inner)
        sv.set_coeffs(out["lam"], out["fa"], out["fk"])
        x = out["x0"].clone()
        st = sv.solve(out["b"], x)
        assert st["status"] == "MG_OK" and st["outer"] <= 6, (prec, st)
        xs[prec] = x.cpu().numpy()
        sv.close()
    x0 = out["x0"].cpu().numpy()
    dev = xs["fp64"] - x0
    for f in range(2):
        err = np.linalg.norm((xs["mixed"] - x0)[:, f] - dev[:, f]) / np.linalg.norm(dev[:, f])
        assert err <= 1e-8, (f, err)


# ---------------------------------------------------------------- Eq. 39
def _energy_case(torch, orc, g, seed):
    """The state, its assembled guess plus noise as the solution, and the corrected velocity and phase pressures
    (both from the oracle, so the energy step is compared on its own)."""
    s = _state(g, seed=seed)
    ref = orc.assemble(g, s.ph1, s.ph2, s.dt, s.C, s.m1, s.m2, s.E, s.mom, s.uf)
    rng = np.random.default_rng(seed)
    x = ref["x0"] + rng.normal(0, 1.0, ref["x0"].shape) * np.array([1.0, 300.0])
    rc = orc.correct(g, s.dt, s.sigma, x, s.C, s.kappa, ref["fa"], s.uf)
    rho1, rho2 = I.phase_density(s.T, s.p, s.ph1), I.phase_density(s.T, s.p, s.ph2)
    E1 = s.C * I.phase_energy(s.p, rho1, s.ph1)
    E2 = (1 - s.C) * I.phase_energy(s.p, rho2, s.ph2)
    return s, x, rc, E1, E2


def _flux_bound(g, ph, p, T, uf, dt):
    """64 ulps of the largest face term, through the divergence: the increment is a difference of face fluxes of
    size p u, mu u^2 / h and k T / h, evaluated in another order of operations than the oracle's."""
    U = max(float(np.abs(u).max()) for u in uf)
    P = max(float(np.abs(p).max()), max(abs(v) for s in g.bcp for v in s))
    Tm = max(float(np.abs(T).max()), max(abs(v) for s in g.bcT for v in s))
    F = P * U + ph.mu * 8 * U * U / g.h + ph.k * 4 * Tm / g.h
    return 64 * EPS * dt * 4 * g.dim * F / g.h


def _gpu_energy(torch, g, s, x, rc, E1, E2, in_place=False):
    from paper_2206_11294_gb300 import binding as B
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    e1, e2 = T(E1), T(E2)
    o1, o2 = (e1, e2) if in_place else (torch.empty_like(e1), torch.empty_like(e2))
    B.energy(g, (s.ph1, s.ph2), s.dt, T(x), T(s.C), T(rc["p1"]), T(rc["p2"]), [T(u) for u in rc["uf"]], e1, e2, o1, o2)
    torch.cuda.synchronize()
    return o1.cpu().numpy(), o2.cpu().numpy()


@pytest.mark.parametrize("name", list(GRIDS))
def test_energy_matches_oracle(torch_cuda, orc, name):
    g = GRIDS[name]
    s, x, rc, E1, E2 = _energy_case(torch_cuda, orc, g, 31)
    Z = np.zeros_like(E1)
    T = x[:, 0].reshape(E1.shape)
    ref = orc.energy(g, s.ph1, s.ph2, s.dt, s.C, rc["p1"], rc["p2"], T, rc["uf"], Z, Z)
    got1, got2 = _gpu_energy(torch_cuda, g, s, x, rc, Z, Z)
    for got, r, ph, p in ((got1, ref["E1"], s.ph1, rc["p1"]), (got2, ref["E2"], s.ph2, rc["p2"])):
        assert np.abs(r).max() > 0
        bound = _flux_bound(g, ph, p, T, rc["uf"], s.dt)
        _close(got, r, 1.0, scale=bound + 1e-12 * np.abs(r), what=f"dE {name}")
    # with the advected energies, in place
    ref = orc.energy(g, s.ph1, s.ph2, s.dt, s.C, rc["p1"], rc["p2"], T, rc["uf"], E1, E2)
    got1, got2 = _gpu_energy(torch_cuda, g, s, x, rc, E1, E2, in_place=True)
    for got, r, ph, p, E in ((got1, ref["E1"], s.ph1, rc["p1"], E1), (got2, ref["E2"], s.ph2, rc["p2"], E2)):
        bound = _flux_bound(g, ph, p, T, rc["uf"], s.dt) + 4 * EPS * np.abs(E)
        _close(got, r, 1.0, scale=bound + 1e-12 * np.abs(r - E), what=f"E {name}")


def test_energy_conservative_with_walls(torch_cuda, orc):
    """Walls all round: the volume sum of div F_i is zero up to rounding (each face flux is one value for its two
    cells, including the faces on the edge of a thread block's tile)."""
    g = GRIDS["2d_walls"]
    s, x, rc, _, _ = _energy_case(torch_cuda, orc, g, 32)
    s.C = np.full_like(s.C, 0.5)
    Z = np.zeros_like(s.C)
    got1, got2 = _gpu_energy(torch_cuda, g, s, x, rc, Z, Z)
    T = x[:, 0].reshape(Z.shape)
    for got, ph, p in ((got1, s.ph1, rc["p1"]), (got2, s.ph2, rc["p2"])):
        div = got / (0.5 * s.dt)
        per_cell = _flux_bound(g, ph, p, T, rc["uf"], s.dt) / (0.5 * s.dt)
        assert np.abs(div).max() > 1e3 * per_cell
        assert abs(div.sum()) <= per_cell * np.sqrt(g.N), (div.sum(), per_cell)


def test_energy_full_size_matches_oracle(torch_cuda, orc):
    """The 16-bubble 1024^2 state through the whole step on the device: assemble, solve, correct, energy; the
    energy against the oracle's on the device's own solution and corrected fields."""
    from paper_2206_11294_gb300 import binding as B
    from paper_2206_11294_gb300.binding import Solver
    torch = torch_cuda
    s = I.bubbles_state_1024()
    g = s.grid
    got, d, out = _gpu_assemble(torch, s)
    solver = Solver(g, rtol=1e-10)
    solver.set_coeffs(out["lam"], out["fa"], out["fk"])
    x = out["x0"].clone()
    st = solver.solve(out["b"], x)
    assert st["status"] == "MG_OK"
    uo = [torch.empty_like(u) for u in d["uf"]]
    p1, p2 = torch.empty_like(d["C"]), torch.empty_like(d["C"])
    B.correct(g, s.dt, s.sigma, x, d["C"], d["kappa"], out["fa"], d["uf"], uo, p1, p2)
    rho1, rho2 = I.phase_density(s.T, s.p, s.ph1), I.phase_density(s.T, s.p, s.ph2)
    E1 = s.C * I.phase_energy(s.p, rho1, s.ph1)
    E2 = (1 - s.C) * I.phase_energy(s.p, rho2, s.ph2)
    e1, e2 = (torch.from_numpy(E1).cuda(), torch.from_numpy(E2).cuda())
    o1, o2 = torch.empty_like(e1), torch.empty_like(e2)
    B.energy(g, (s.ph1, s.ph2), s.dt, x, d["C"], p1, p2, uo, e1, e2, o1, o2)
    torch.cuda.synchronize()
    xh = x.cpu().numpy()
    T = xh[:, 0].reshape(E1.shape)
    ufh = [u.cpu().numpy() for u in uo]
    p1h, p2h = p1.cpu().numpy(), p2.cpu().numpy()
    ref = orc.energy(g, s.ph1, s.ph2, s.dt, s.C, p1h, p2h, T, ufh, E1, E2)
    for got, r, ph, p, E in ((o1, ref["E1"], s.ph1, p1h, E1), (o2, ref["E2"], s.ph2, p2h, E2)):
        bound = _flux_bound(g, ph, p, T, ufh, s.dt) + 4 * EPS * np.abs(E)
        _close(got.cpu().numpy(), r, 1.0, scale=bound + 1e-12 * np.abs(r - E), what="E full size")
    solver.close()


def test_energy_invalid_arguments_rejected(torch_cuda, orc):
    from paper_2206_11294_gb300 import binding as B
    from paper_2206_11294_gb300.binding import MgError, MG_ERR_INVALID_ARG
    import dataclasses
    torch = torch_cuda
    g = GRIDS["2d_walls"]
    s, x, rc, E1, E2 = _energy_case(torch, orc, g, 33)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    xd, Cd, p1, p2, uf = T(x), T(s.C), T(rc["p1"]), T(rc["p2"]), [T(u) for u in rc["uf"]]
    e1, e2 = T(E1), T(E2)
    o1, o2 = torch.zeros_like(e1), torch.zeros_like(e2)
    bad = dataclasses.replace(s.ph1, mu=-1.0)
    cases = [
        dict(dt=-1.0),
        dict(phases=(bad, s.ph2)),
        dict(o1=p1),                 # an output over a neighbour-read input
        dict(o1=o2),
        dict(o1=e2),
    ]
    for c in cases:
        with pytest.raises(MgError) as e:
            B.energy(g, c.get("phases", (s.ph1, s.ph2)), c.get("dt", s.dt), xd, Cd, p1, p2, uf, e1, e2,
                     c.get("o1", o1), o2)
        assert e.value.status == MG_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert float(o1.abs().sum()) == 0.0 and float(o2.abs().sum()) == 0.0


def test_energy_of_an_absent_phase_is_unchanged(torch_cuda, orc):
    """Cells of one phase only (C exactly 0 or 1 in halves): the absent phase's energy comes back bit for bit."""
    g = GRIDS["2d_walls"]
    s, x, rc, E1, E2 = _energy_case(torch_cuda, orc, g, 34)
    C = np.zeros_like(s.C)
    C[:, :, : g.n[0] // 2] = 1.0
    s.C = C
    got1, got2 = _gpu_energy(torch_cuda, g, s, x, rc, E1, E2)
    np.testing.assert_array_equal(got1[C == 0.0], E1[C == 0.0])
    np.testing.assert_array_equal(got2[C == 1.0], E2[C == 1.0])
    assert np.any(got1[C == 1.0] != E1[C == 1.0]) and np.any(got2[C == 0.0] != E2[C == 0.0])
