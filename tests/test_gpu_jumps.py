"""FP64 block updates at coefficient jumps inside the FP32 cycles of mixed
precision (mg_options.fp64_jump_ratio).

A finest-level cell whose interior faces' k or 1/rho differ by more than the
ratio (the cells along a bubble interface, where the density ratio is 1000)
applies its 2x2 block in FP64 in every FP32 sweep; every other cell stays
FP32.  Checked here: the marked cells are exactly the ones an independent
count from the face arrays finds (integer parity); marking changes nothing
in FP64 solves; mixed solves with and without it reach the FP64 oracle's
solution (literal regime: 1e-8 at the 1e-10 stop); batches equal solo solves
bit for bit with it on; the stiff cases' error at the 1e-10 stop stays within
twice the FP64 oracle's own error at the same stop (the stopping rule, not
the precision, sets that floor: see the test's docstring)."""
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


def rel_dev(x, ref, x0):
    return max(float(np.linalg.norm(x[:, f] - ref[:, f]) / max(np.linalg.norm(ref[:, f] - x0[:, f]), 1e-300))
               for f in range(2))


def expected_marks(p, ratio):
    """Cells whose interior faces' k or 1/rho differ by more than `ratio`, from
    the face arrays directly (numpy)."""
    g = p.grid
    n0, n1, n2 = g.n
    kmin = np.full((n2, n1, n0), np.inf)
    kmax = np.full((n2, n1, n0), -np.inf)
    amin, amax = kmin.copy(), kmax.copy()
    for a in range(g.dim):
        fk = p.fk[a].reshape(g.face_shape(a))
        fa = p.fa[a].reshape(g.face_shape(a))
        ax = 2 - a                              # numpy axis of axis a in (n2, n1, n0)
        m = g.n[a]
        for side in (0, 1):
            sl = [slice(None)] * 3
            sl[ax] = slice(side, side + m)
            kf, af = fk[tuple(sl)], fa[tuple(sl)]
            inner = np.ones((n2, n1, n0), bool)
            idx = [slice(None)] * 3
            idx[ax] = 0 if side == 0 else m - 1
            inner[tuple(idx)] = False           # the first / last cell's boundary face is not interior
            kmin = np.where(inner, np.minimum(kmin, kf), kmin)
            kmax = np.where(inner, np.maximum(kmax, kf), kmax)
            amin = np.where(inner, np.minimum(amin, af), amin)
            amax = np.where(inner, np.maximum(amax, af), amax)
    return (kmax > ratio * kmin) | (amax > ratio * amin)


def _cases():
    return {
        "bubble_2d": I.bubble_2d(192, seed=91, n_bubbles=4, rmin=0.05, rmax=0.15, centred=False),
        "axi": I.stiff(I.bubble_axi, 96, 192),
        "wall_3d": I.bubble_wall_3d(48, seed=92),
        "stiff_2d": I.stiff(I.bubble_2d, 128),
    }


CASES = _cases()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("ratio", [2.0, 1.5])
def test_marked_cells_are_the_jump_cells(torch_cuda, name, ratio):
    from paper_2206_11294_gb300.binding import Solver
    p = CASES[name]
    s = Solver(p.grid, precision="mixed", rtol=1e-10, max_cycles=80, fp64_jump_ratio=ratio)
    s.set_coeffs(p.lam, p.fa, p.fk)
    st = s.solve(p.b, p.x0.copy())
    want = int(expected_marks(p, ratio).sum())
    assert want > 0
    assert st["fp64_cells"] == want
    s.close()
    for kw in (dict(precision="fp64"), dict(precision="mixed", fp64_jump_ratio=0.0)):
        s = Solver(p.grid, rtol=1e-10, max_cycles=80, **kw)
        s.set_coeffs(p.lam, p.fa, p.fk)
        assert s.solve(p.b, p.x0.copy())["fp64_cells"] == 0
        s.close()


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_with_and_without_fp64_blocks_vs_oracle(torch_cuda, orc, name):
    """Both reach the oracle's solution: literal cases stop at 1e-10 and must be
    within 1e-8 of the converged oracle; stiff cases stop at 1e-10 and must be
    within twice the FP64 oracle's own distance at that stop (or 1e-8, the
    larger), since any solver stopped at 1e-10 carries cond x 1e-10 of
    algebraic error (measured up to 3.7e-8 for the oracle on the stiff parity
    cases)."""
    p = CASES[name]
    g = p.grid.as_dict()
    conv, _, _ = orc.mg_solve(g, p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=150, rtol=1e-13)
    o10, _, _ = orc.mg_solve(g, p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=150, rtol=1e-10)
    floor = max(1e-8, 2.0 * rel_dev(o10, conv, p.x0))
    from paper_2206_11294_gb300.binding import Solver
    for ratio in (2.0, 0.0):
        s = Solver(p.grid, precision="mixed", rtol=1e-10, max_cycles=150, fp64_jump_ratio=ratio)
        s.set_coeffs(p.lam, p.fa, p.fk)
        x = p.x0.copy()
        st = s.solve(p.b, x)
        assert st["status"] == "MG_OK"
        assert rel_dev(x, conv, p.x0) <= floor, (ratio, rel_dev(x, conv, p.x0), floor)
        s.close()


def test_batch_equals_solo_with_fp64_blocks(torch_cuda):
    from paper_2206_11294_gb300.binding import Batch, Solver
    probs = [CASES["bubble_2d"], CASES["stiff_2d"], I.bubble_2d(128, seed=93, n_bubbles=2, rmin=0.05, rmax=0.1,
                                                              centred=False)]
    solo = []
    for p in probs:
        s = Solver(p.grid, precision="mixed", rtol=1e-10, max_cycles=80)
        s.set_coeffs(p.lam, p.fa, p.fk)
        x = p.x0.copy()
        st = s.solve(p.b, x)
        solo.append((x, st))
        s.close()
    hs = [Solver(p.grid, precision="mixed", rtol=1e-10, max_cycles=80) for p in probs]
    b = Batch(hs)
    b.set_coeffs([p.lam for p in probs], [p.fa for p in probs], [p.fk for p in probs])
    xs = [p.x0.copy() for p in probs]
    sts = b.solve([p.b for p in probs], xs)
    for (x, st), xb, sb in zip(solo, xs, sts):
        assert sb["cycles"] == st["cycles"] and sb["fp64_cells"] == st["fp64_cells"] > 0
        assert np.array_equal(xb, x)
    b.close()
    for s in hs:
        s.close()
