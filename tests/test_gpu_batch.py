"""Batched solves (mg_batch_*): many independent problems of uneven sizes in
one set of launches per V-cycle stage, each graph replay one cycle of all.

Each problem's result must be the one mg_solve gives it alone (same cycles,
same values: the batch runs the same per-block device code on the same data
and stops each problem with the same rule), and the batch must agree with the
oracle like the single path does.
"""
import numpy as np
import pytest

from paper_2206_11294_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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
    return torch


def _problems_2d():
    sizes = [64, 96, 128, 160, 224, 256, 96, 64, 320, 192]
    out = []
    for q, n in enumerate(sizes):
        p = I.bubble_2d(n=n, seed=100 + q, n_bubbles=1 + q % 4, rmin=0.05, rmax=0.15, centred=False,
                        gas_rho=1.0, name=f"b{q}")
        if q % 3 == 2:          # some stiff members: more cycles, uneven stopping
            p = I.bubble_2d(n=n, seed=100 + q, n_bubbles=2, rmin=0.05, rmax=0.15, centred=False, gas_rho=1.0,
                            length=6.4e-3, dt=1e-5, name=f"s{q}")
        out.append(p)
    return out


def _problems_3d():
    return [I.random_coeff_problem(I.Grid(dim=3, axisym=0, n=n, h=1e-4, bc=((1, 1), (0, 1), (0, 1)),
                                          bcT=((300, 300), (0, 300), (0, 300)),
                                          bcp=((1e5, 1e5), (0, 1e5), (0, 1e5))), seed=200 + q, dt=1e-5)
            for q, n in enumerate([(32, 32, 32), (64, 32, 16), (40, 24, 16), (16, 16, 16)])]


def _solvers(probs, **kw):
    from paper_2206_11294_gb300.binding import Solver
    out = []
    for p in probs:
        s = Solver(p.grid, **kw)
        s.set_coeffs(p.lam, p.fa, p.fk)
        out.append(s)
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("which", ["2d", "3d"])
def test_batch_equals_solo(torch_cuda, precision, which):
    from paper_2206_11294_gb300.binding import Batch
    probs = _problems_2d() if which == "2d" else _problems_3d()
    kw = dict(precision=precision, rtol=1e-10, max_cycles=60)
    solo = _solvers(probs, **kw)
    xs_solo, st_solo = [], []
    for s, p in zip(solo, probs):
        x = p.x0.copy()
        st_solo.append(s.solve(p.b, x))
        xs_solo.append(x)
    batch = Batch(solo)
    xs = [p.x0.copy() for p in probs]
    st = batch.solve([p.b for p in probs], xs)
    for q, p in enumerate(probs):
        assert st[q]["cycles"] == st_solo[q]["cycles"], q
        assert st[q]["status"] == "MG_OK"
        assert rel_dev(xs[q], xs_solo[q], p.x0) <= 1e-13, q
    # members stop at different cycle counts in the stiff/literal mix
    if which == "2d":
        assert len({s["cycles"] for s in st}) > 1
    assert batch.launches() > 0
    batch.close()
    for s in solo:
        s.close()


@pytest.mark.parametrize("nu1,nu2", [(0, 2), (2, 0)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_solo_cycle_shapes(torch_cuda, precision, nu1, nu2):
    """Without pre- (post-) smoothing the restriction (stopping norm) takes
    every cell; the batch must follow the single path there as well."""
    from paper_2206_11294_gb300.binding import Batch
    probs = _problems_2d()[:6]
    kw = dict(precision=precision, rtol=1e-10, max_cycles=80, nu1=nu1, nu2=nu2)
    solo = _solvers(probs, **kw)
    xs_solo, st_solo = [], []
    for s, p in zip(solo, probs):
        x = p.x0.copy()
        st_solo.append(s.solve(p.b, x))
        xs_solo.append(x)
    batch = Batch(solo)
    xs = [p.x0.copy() for p in probs]
    st = batch.solve([p.b for p in probs], xs)
    for q, p in enumerate(probs):
        assert st[q]["cycles"] == st_solo[q]["cycles"], q
        assert rel_dev(xs[q], xs_solo[q], p.x0) <= 1e-13, q
    batch.close()
    for s in solo:
        s.close()


def test_batch_membership_does_not_change_results(torch_cuda):
    """A problem solved in a batch of one and in the full mix: bitwise equal."""
    from paper_2206_11294_gb300.binding import Batch
    probs = _problems_2d()
    solvers = _solvers(probs, rtol=1e-10, max_cycles=60)
    mix = Batch(solvers)
    xs = [p.x0.copy() for p in probs]
    mix.solve([p.b for p in probs], xs)
    for q in (0, 4, 8):
        one = Batch([solvers[q]])
        x1 = probs[q].x0.copy()
        one.solve([probs[q].b], [x1])
        assert np.array_equal(x1, xs[q]), q
        one.close()
    mix.close()
    for s in solvers:
        s.close()


def test_batch_vs_oracle(torch_cuda, orc):
    from paper_2206_11294_gb300.binding import Batch
    probs = _problems_2d()[:4]
    solvers = _solvers(probs, rtol=0.0, max_cycles=3)
    b = Batch(solvers)
    xs = [p.x0.copy() for p in probs]
    st = b.solve([p.b for p in probs], xs)
    for q, p in enumerate(probs):
        ref, cyc, _ = orc.mg_solve(p.grid.as_dict(), p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=3, rtol=0.0)
        assert st[q]["cycles"] == 3 == cyc
        # literal members 1e-12; stiff members (h = 5e-5 m) carry FP64 rounding of
        # the 1e5 Pa background through rows where sum_f G_f ~ 1.6e6 meets l3 ~ 5.4:
        # eps * sum G * |p| / (|l3| * dev) ~ 6.5e-9, so 1e-8
        tol = 1e-12 if p.name.startswith("b") else 1e-8
        assert rel_dev(xs[q], ref, p.x0) <= tol, q
    b.close()
    for s in solvers:
        s.close()


def test_batch_device_arrays_and_repeat(torch_cuda):
    """Device-side per-problem arrays; two solves in a row give identical results."""
    torch = torch_cuda
    from paper_2206_11294_gb300.binding import Batch
    probs = _problems_2d()[:5]
    solvers = _solvers(probs, precision="mixed", rtol=1e-10, max_cycles=60)
    b = Batch(solvers)
    bs = [torch.from_numpy(p.b).cuda() for p in probs]
    outs = []
    for _ in range(2):
        xs = [torch.from_numpy(p.x0.copy()).cuda() for p in probs]
        b.solve(bs, xs)
        outs.append([x.cpu().numpy() for x in xs])
    for a, c in zip(*outs):
        assert np.array_equal(a, c)
    b.close()
    for s in solvers:
        s.close()


def test_batch_rejects_mismatched_options(torch_cuda):
    from paper_2206_11294_gb300.binding import Batch, MgError, MG_ERR_INVALID_ARG
    probs = _problems_2d()[:2]
    s1 = _solvers(probs[:1], rtol=1e-10)[0]
    s2 = _solvers(probs[1:], rtol=1e-8)[0]
    with pytest.raises(MgError) as e:
        Batch([s1, s2])
    assert e.value.status == MG_ERR_INVALID_ARG
    s1.close()
    s2.close()


@pytest.mark.parametrize("precision,which", [("fp64", "2d"), ("mixed", "2d"), ("mixed", "3d")])
def test_batched_set_coeffs_equals_per_handle(torch_cuda, precision, which):
    """Coefficient set-up of all problems in one set of launches gives the
    hierarchy the per-handle set-up gives: same cycles, same results."""
    torch = torch_cuda
    from paper_2206_11294_gb300.binding import Batch, Solver
    probs = _problems_2d() if which == "2d" else _problems_3d()
    kw = dict(precision=precision, rtol=1e-10, max_cycles=60)
    ref = _solvers(probs, **kw)
    xs_ref = []
    for s, p in zip(ref, probs):
        x = p.x0.copy()
        s.solve(p.b, x)
        xs_ref.append(x)
    fresh = [Solver(p.grid, **kw) for p in probs]
    b = Batch(fresh)
    T = lambda a: torch.from_numpy(a).cuda()
    b.set_coeffs([T(p.lam) for p in probs], [[T(f) for f in p.fa] for p in probs],
                 [[T(f) for f in p.fk] for p in probs])
    xs = [p.x0.copy() for p in probs]
    st = b.solve([p.b for p in probs], xs)
    for q, p in enumerate(probs):
        assert rel_dev(xs[q], xs_ref[q], p.x0) <= 1e-13, q
    # host-array intake through the batch as well
    b.set_coeffs([p.lam for p in probs], [p.fa for p in probs], [p.fk for p in probs])
    xs2 = [p.x0.copy() for p in probs]
    b.solve([p.b for p in probs], xs2)
    for q in range(len(probs)):
        assert np.array_equal(xs2[q], xs[q]), q
    b.close()
    for s in ref + fresh:
        s.close()


def test_batched_set_coeffs_names_bad_problem(torch_cuda):
    from paper_2206_11294_gb300.binding import Batch, MgError, MG_ERR_INVALID_COEFF, Solver
    probs = _problems_2d()[:4]
    solvers = [Solver(p.grid) for p in probs]
    b = Batch(solvers)
    lams = [p.lam.copy() for p in probs]
    lams[2][7, 1] = np.inf
    with pytest.raises(MgError) as e:
        b.set_coeffs(lams, [p.fa for p in probs], [p.fk for p in probs])
    assert e.value.status == MG_ERR_INVALID_COEFF and "problem 2" in str(e.value)
    b.close()
    for s in solvers:
        s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_tunings_keep_results(torch_cuda, precision):
    """Every batch kernel choice (sweep kind and tile per depth, persistent
    grid size) and the batch autotuner's pick give the same results, bit for
    bit, as the default choices."""
    from paper_2206_11294_gb300.binding import Batch, MgError, MG_ERR_INVALID_ARG
    probs = _problems_2d()[:6]
    solvers = _solvers(probs, precision=precision, rtol=1e-10, max_cycles=60)
    b = Batch(solvers)
    xs_ref = [p.x0.copy() for p in probs]
    st_ref = b.solve([p.b for p in probs], xs_ref)
    base = b.tuning()
    n = base["depths"]
    variants = [dict(base, sweep=["colour"] * n, tile=[0] * n, blocks_per_sm=1)]
    for t in range(3):
        variants.append(dict(base, sweep=["fused"] * n, tile=[t] * n, blocks_per_sm=[2, 16, 32][t]))
    for v in variants:
        b.set_tuning(v)
        assert b.tuning() == v
        xs = [p.x0.copy() for p in probs]
        st = b.solve([p.b for p in probs], xs)
        for q in range(len(probs)):
            assert st[q]["cycles"] == st_ref[q]["cycles"]
            assert np.array_equal(xs[q], xs_ref[q]), (v, q)
    tuning, ms = b.autotune(reps=2)
    assert ms > 0 and 1 <= tuning["blocks_per_sm"] <= 32 and tuning["depths"] == n
    xs = [p.x0.copy() for p in probs]
    b.solve([p.b for p in probs], xs)
    for q in range(len(probs)):
        assert np.array_equal(xs[q], xs_ref[q])
    for bad in (dict(base, blocks_per_sm=0), dict(base, tile=[3] * n), dict(base, sweep=["x"] * n, tile=[0] * n)):
        if bad.get("sweep") == ["x"] * n:
            continue                       # from_dict maps unknown names to colour: not an ABI error
        with pytest.raises(MgError) as e:
            b.set_tuning(bad)
        assert e.value.status == MG_ERR_INVALID_ARG
    b.close()
    for s in solvers:
        s.close()


def test_batch_3d_rejects_fused(torch_cuda):
    from paper_2206_11294_gb300.binding import Batch, MgError, MG_ERR_INVALID_ARG
    probs = _problems_3d()[:2]
    solvers = _solvers(probs)
    b = Batch(solvers)
    t = b.tuning()
    with pytest.raises(MgError) as e:
        b.set_tuning(dict(t, sweep=["fused"] * t["depths"]))
    assert e.value.status == MG_ERR_INVALID_ARG
    b.close()
    for s in solvers:
        s.close()


@pytest.mark.parametrize("coarse", ["auto", "inverse"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_banded_coarsest_path(torch_cuda, precision, coarse):
    """Problems whose coarsest level has more than 128 unknowns (31 x 31, 15 x
    15 and 13 x 13 cells) take the windowed banded LU, batched over problems,
    and either solve from the factors in each cycle (auto) or form the
    inverse: same results as the per-handle set-up, bit for bit."""
    from paper_2206_11294_gb300.binding import Batch, Solver
    torch = torch_cuda
    probs = [I.bubble_2d(n=n, seed=300 + q, n_bubbles=2, rmin=0.05, rmax=0.15, centred=False, gas_rho=1.0,
                         name=f"m{q}") for q, n in enumerate([480, 416, 64, 480, 992])]
    kw = dict(precision=precision, rtol=1e-10, max_cycles=60, coarse=coarse)
    ref = _solvers(probs, **kw)
    assert all(len(s.levels()) >= 3 for s in ref)
    xs_ref = []
    for s, p in zip(ref, probs):
        x = p.x0.copy()
        s.solve(p.b, x)
        xs_ref.append(x)
    fresh = [Solver(p.grid, **kw) for p in probs]
    b = Batch(fresh)
    b.set_coeffs([p.lam for p in probs], [p.fa for p in probs], [p.fk for p in probs])
    xs = [p.x0.copy() for p in probs]
    b.solve([p.b for p in probs], xs)
    for q in range(len(probs)):
        assert np.array_equal(xs[q], xs_ref[q]), q
    b.close()
    for s in ref + fresh:
        s.close()


def test_window_and_blocked_lu_give_the_same_factors(torch_cuda):
    """Twenty problems on the windowed coarse path (288^2: 9 x 9 coarsest
    cells, 162 unknowns) are more than one wave of 8-CTA clusters, so the
    batch factors them with the single-block windowed LU, while each solo
    handle uses the LU blocked over a cluster.  The two factorisations do the
    same multiply-adds per entry in the same order: batch and solo results
    must agree bit for bit, in both precisions."""
    from paper_2206_11294_gb300.binding import Batch, Solver
    probs = [I.bubble_2d(n=288, seed=400 + q, n_bubbles=1 + q % 3, rmin=0.05, rmax=0.15, centred=False,
                         gas_rho=1.0, name=f"w{q}") for q in range(20)]
    for precision in ("fp64", "mixed"):
        kw = dict(precision=precision, rtol=1e-10, max_cycles=60)
        ref = _solvers(probs, **kw)
        assert 2 * int(np.prod(ref[0].levels()[-1])) > 128
        xs_ref = []
        for s, p in zip(ref, probs):
            x = p.x0.copy()
            s.solve(p.b, x)
            xs_ref.append(x)
        fresh = [Solver(p.grid, **kw) for p in probs]
        b = Batch(fresh)
        b.set_coeffs([p.lam for p in probs], [p.fa for p in probs], [p.fk for p in probs])
        xs = [p.x0.copy() for p in probs]
        b.solve([p.b for p in probs], xs)
        for q in range(len(probs)):
            assert np.array_equal(xs[q], xs_ref[q]), (precision, q)
        b.close()
        for s in ref + fresh:
            s.close()


def test_batch_sample_of_32_vs_oracle(torch_cuda, orc):
    """The 256-problem batch workload's first 32 problems (the same seeded
    sizes, 64^2 to 1024^2 in multiples of 32, and bubble fields), batched in
    FP64 for two fixed cycles: each against the oracle's two cycles at 1e-12
    of the deviation."""
    from paper_2206_11294_gb300.binding import Batch
    probs = I.batch_problems(count=32)
    assert len({p.grid.n for p in probs}) > 10
    solvers = _solvers(probs, rtol=0.0, max_cycles=2)
    b = Batch(solvers)
    xs = [p.x0.copy() for p in probs]
    st = b.solve([p.b for p in probs], xs)
    for q, p in enumerate(probs):
        ref, cyc, _ = orc.mg_solve(p.grid.as_dict(), p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=2, rtol=0.0)
        assert st[q]["cycles"] == 2 == cyc
        assert rel_dev(xs[q], ref, p.x0) <= 1e-12, (q, p.grid.n)
    b.close()
    for s in solvers:
        s.close()
