"""Kernel choices (mg_set_tuning) and the native autotuner (mg_autotune).

Every choice -- colour, fused, TMA-fed fused or fused-pair sweeps with any
tile shape per level, the cluster tail from any allowed level on 1, 8 or 16
CTAs, or none, dependent launches on or off -- runs the same
per-cell arithmetic in the same order, so solves must agree bit for bit and
stop after the same number of cycles."""
import numpy as np
import pytest

from paper_2206_11294_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _problems():
    W, D, A = I.BC_WALL, I.BC_DIRICHLET, I.BC_AXIS
    return {
        "2d": I.random_coeff_problem(I.Grid(dim=2, axisym=0, n=(192, 128, 1), h=1e-4, bc=((W, D), (D, W), (0, 0)),
                                            bcT=((0, 300), (300, 0), (0, 0)), bcp=((0, 1e5), (1e5, 0), (0, 0))),
                                     seed=71, dt=1e-5),
        "axi": I.bubble_axi(nr=64, nz=128),
        "3d": I.random_coeff_problem(I.Grid(dim=3, axisym=0, n=(64, 32, 32), h=1e-4, bc=((W, W), (W, W), (W, D)),
                                            bcT=((0, 0), (0, 0), (0, 300)), bcp=((0, 0), (0, 0), (0, 1e5))),
                                     seed=72, dt=1e-5),
    }


PROBS = _problems()


def _solve(p, tuning=None, **kw):
    """The coarsest solve by the inverse: the tail kernel, one of the choices
    under test, multiplies by it (the 3D problem's 8 x 4 x 4 coarsest level
    would otherwise solve from its factors and refuse every tail)."""
    from paper_2206_11294_gb300.binding import Solver
    s = Solver(p.grid, rtol=1e-10, max_cycles=60, coarse="inverse", **kw)
    s.set_coeffs(p.lam, p.fa, p.fk)
    if tuning is not None:
        s.set_tuning(tuning)
    x = p.x0.copy()
    st = s.solve(p.b, x)
    return s, x, st


def _variants(s):
    """Explicit tunings covering every kind of choice the hierarchy allows."""
    base = s.tuning()
    n = base["levels"]
    dim = s.grid.dim
    out = []
    colour = dict(base, sweep=["colour"] * n, tile=[0] * n, tail_level=n, tail_ctas=8, persistent=0)
    out.append(colour)
    out.append(dict(colour, persistent=1))
    out.append(dict(colour, overlap=0))                     # plain stream order instead of dependent launches
    out.append(dict(colour, overlap=0, persistent=1))
    out.append(dict(colour, sweep=["colour2"] * n))
    if dim == 2:
        for t in range(3):
            out.append(dict(colour, sweep=["fused"] * n, tile=[t] * n))
        for t in range(3):
            out.append(dict(colour, sweep=["async"] * n, tile=[t] * n))
        for t in range(3):
            out.append(dict(colour, sweep=["fused2"] * n, tile=[t] * n))
        out.append(dict(colour, sweep=["fused2" if l % 2 == 0 else "fused" for l in range(n)],
                        tile=[(l + 1) % 3 for l in range(n)]))
        out.append(dict(colour, sweep=["fused" if l % 2 else "colour" for l in range(n)],
                        tile=[l % 3 for l in range(n)]))
    sizes = s.levels()
    for l in range(1, n - 1):
        cells = int(np.prod(sizes[l]))
        if n - l <= 12 and cells <= 16384:
            for ctas in (1, 8, 16):
                out.append(dict(out[-1] if dim == 2 else colour, tail_level=l, tail_ctas=ctas))
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(PROBS))
def test_every_choice_gives_identical_results(torch_cuda, name, precision):
    from paper_2206_11294_gb300.binding import MgError
    p = PROBS[name]
    s0, x0, st0 = _solve(p, precision=precision)
    tried = 0
    for v in _variants(s0):
        try:
            s, x, st = _solve(p, tuning=v, precision=precision)
        except MgError as e:            # 16-CTA clusters where the device does not allow them, or a
            # one-block tail whose levels do not fit its shared memory
            assert (v["tail_ctas"] == 16 and "cluster size" in str(e)) or \
                (v["tail_ctas"] == 1 and "shared memory" in str(e)) or \
                ("async" in v["sweep"] and "does not fit" in str(e)), str(e)
            continue
        assert s.tuning()["sweep"] == v["sweep"]
        assert st["cycles"] == st0["cycles"], v
        assert np.array_equal(x, x0), v
        tried += 1
        s.close()
    assert tried >= 2
    s0.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["2d", "3d"])
def test_autotune_picks_valid_choice_and_keeps_results(torch_cuda, name, precision):
    p = PROBS[name]
    s0, x0, st0 = _solve(p, precision=precision)
    tuning, ms = s0.autotune(reps=3)
    assert ms > 0
    n = len(s0.levels())
    assert tuning["levels"] == n
    assert all(k in ("colour", "colour2", "fused", "async", "fused2") for k in tuning["sweep"])
    if p.grid.dim == 3:
        assert set(tuning["sweep"]) <= {"colour", "colour2"}
    assert tuning["tail_level"] >= n or 1 <= tuning["tail_level"] <= n - 2
    assert tuning["tail_ctas"] in (1, 8, 16)
    assert tuning["overlap"] in (0, 1)
    assert s0.tuning() == tuning
    x = p.x0.copy()
    st = s0.solve(p.b, x)                     # scratch overwritten by the tuner: same solve
    assert st["cycles"] == st0["cycles"]
    assert np.array_equal(x, x0)
    s0.close()


def test_set_tuning_rejects_bad_choices(torch_cuda):
    from paper_2206_11294_gb300.binding import MgError, MG_ERR_INVALID_ARG
    s3, _, _ = _solve(PROBS["3d"])
    s2, _, _ = _solve(PROBS["2d"])
    for s, mutate in [(s3, lambda t: t["sweep"].__setitem__(0, "fused")),
                      (s3, lambda t: t["sweep"].__setitem__(0, "async")),
                      (s2, lambda t: t["tile"].__setitem__(1, 3)),
                      (s2, lambda t: t.__setitem__("tail_level", 0)),
                      (s2, lambda t: t.__setitem__("tail_level", t["levels"] - 1)),
                      (s2, lambda t: t.update(tail_level=1, tail_ctas=12)),
                      (s2, lambda t: t.update(tail_level=1, tail_ctas=1)),   # 6144 FP64 cells: > 200 KB
                      # a valid sweep change with an invalid flag: nothing of it may be applied
                      (s2, lambda t: t.update(persistent=2, sweep=["fused"] + t["sweep"][1:])),
                      (s2, lambda t: t.update(overlap=2, sweep=["fused"] + t["sweep"][1:])),
                      (s2, lambda t: t.update(tail_level=1))]:      # level 1 of 192x128 has 6144 cells: allowed
        before = s.tuning()
        t = dict(before, sweep=list(before["sweep"]), tile=list(before["tile"]))
        mutate(t)
        if t.get("tail_level") == 1 and t.get("tail_ctas") == before["tail_ctas"]:
            s.set_tuning(t)                   # the valid one goes through
            assert s.tuning()["tail_level"] == 1
            s.set_tuning(before)
            continue
        with pytest.raises(MgError) as e:
            s.set_tuning(t)
        assert e.value.status == MG_ERR_INVALID_ARG
        assert s.tuning() == before
    s2.close()
    s3.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fused_pairs_in_w_cycles_and_smoothing(torch_cuda, precision):
    """Fused sweep pairs move a level's values to its second buffer and back
    within each cycle: W-cycles (two visits of each coarse level) and the
    public smoother (one pair: the values come back by a copy) give the colour
    sweeps' results bit for bit; a cycle shape whose pairs are odd in number
    (V(2,0)) is refused."""
    from paper_2206_11294_gb300.binding import MgError, MG_ERR_INVALID_ARG
    p = PROBS["2d"]
    s0, x0, st0 = _solve(p, precision=precision, cycle="W")
    n = s0.tuning()["levels"]
    pairs = dict(s0.tuning(), sweep=["fused2"] * n, tile=[0] * n, tail_level=n)
    s1, x1, st1 = _solve(p, tuning=pairs, precision=precision, cycle="W")
    assert st1["cycles"] == st0["cycles"] and np.array_equal(x1, x0)
    if precision == "fp64":
        a, b = p.x0.copy(), p.x0.copy()
        s0.set_tuning(dict(s0.tuning(), sweep=["colour"] * n))
        s0.smooth(p.b, a, sweeps=2)
        s1.smooth(p.b, b, sweeps=2)
        assert np.array_equal(a, b)
        s0.smooth(p.b, a, sweeps=3)
        s1.smooth(p.b, b, sweeps=3)
        assert np.array_equal(a, b)
    s2, _, _ = _solve(p, precision=precision, nu2=0)
    with pytest.raises(MgError) as e:
        s2.set_tuning(dict(s2.tuning(), sweep=["fused2"] * n, tile=[0] * n))
    assert e.value.status == MG_ERR_INVALID_ARG
    for s in (s0, s1, s2):
        s.close()


def test_table_reuses_measurement(torch_cuda):
    from paper_2206_11294_gb300.autotune import TuningTable
    p = PROBS["2d"]
    table = TuningTable(None)
    s1, _, _ = _solve(p)
    t1 = table.tune(s1, reps=2)
    s2, _, _ = _solve(p)
    t2 = table.tune(s2, reps=2)
    assert table.measured == 1 and table.reused == 1
    assert t2 == t1 and s2.tuning() == t1
    s1.close()
    s2.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tma_sweep_on_ragged_grid(torch_cuda, precision):
    """The TMA-fed sweep on a grid that no tile shape divides (200 x 72: tiles
    hang over the right and top edges, where the boxes are zero-filled): same
    result, bit for bit, as colour sweeps; a level it cannot run is refused.
    Mixed precision runs it with the FP64 blocks at jumps off: the TMA sweep
    stages the FP32 W in shared memory and has no FP64 branch, so with them on
    the finest level refuses it."""
    from paper_2206_11294_gb300.binding import MgError, MG_ERR_INVALID_ARG
    W, D = I.BC_WALL, I.BC_DIRICHLET
    p = I.random_coeff_problem(I.Grid(dim=2, axisym=0, n=(200, 72, 1), h=1e-4, bc=((D, W), (W, D), (0, 0)),
                                      bcT=((300, 0), (0, 300), (0, 0)), bcp=((1e5, 0), (0, 1e5), (0, 0))),
                               seed=73, dt=1e-5)
    if precision == "mixed":
        sj, _, stj = _solve(p, precision="mixed")
        assert stj["fp64_cells"] > 0
        bad = sj.tuning()
        bad["sweep"][0], bad["tile"][0] = "async", 1
        with pytest.raises(MgError) as e:
            sj.set_tuning(bad)
        assert e.value.status == MG_ERR_INVALID_ARG
        sj.close()
    kw = dict(precision=precision) if precision == "fp64" else dict(precision="mixed", fp64_jump_ratio=0.0)
    s0, x0, st0 = _solve(p, **kw)
    base = s0.tuning()
    n = base["levels"]
    sizes = s0.levels()
    # FP64 64 x 16 tiles need more than one block's shared memory; FP32 needs an even row length
    allowed = lambda l, t: (precision == "mixed" or t != 0) and (precision == "fp64" or sizes[l][0] % 2 == 0)
    for t in range(3):
        v = dict(base, sweep=["colour"] * n, tile=[0] * n, tail_level=n)
        for l in range(n - 1):
            if allowed(l, t):
                v["sweep"][l], v["tile"][l] = "async", t
        s, x, st = _solve(p, tuning=v, **kw)
        assert st["cycles"] == st0["cycles"]
        assert np.array_equal(x, x0), t
        s.close()
    if precision == "fp64":                           # 64 x 16 FP64 tiles: refused, handle unchanged
        bad = dict(base, sweep=list(base["sweep"]), tile=list(base["tile"]))
        bad["sweep"][0], bad["tile"][0] = "async", 0
        with pytest.raises(MgError) as e:
            s0.set_tuning(bad)
        assert e.value.status == MG_ERR_INVALID_ARG and "does not fit" in str(e.value)
        assert s0.tuning() == base
    s0.close()
