"""The allocation-free norm entry point (mg_residual_norms_noalloc).

It serves callers that cannot allocate device memory (their device memory is
owned by another allocator, or their loop must not call cudaMalloc/cudaFree).
Checked through the C ABI against the handle-based mg_residual_norms on the
same device arrays, on two calls in a row (the second with a different state,
so a stale partial sum from the first call would show), at the tolerance the
other norm tests use (1e-12 relative), and against the CPU oracle's norms.
After a first call (which sets the scratch up), a call must leave the device's
free memory and torch's allocated bytes unchanged: it allocates nothing.
This file is collected last.
"""
import numpy as np
import pytest

from paper_2206_11294_gb300 import inputs as I

pytestmark = pytest.mark.gpu

W, D, A = I.BC_WALL, I.BC_DIRICHLET, I.BC_AXIS


def _problems():
    return [
        I.random_coeff_problem(I.Grid(dim=2, axisym=0, n=(200, 72, 1), h=1.0 / 200, bc=((D, W), (W, D), (0, 0)),
                                      bcT=((310, 0), (0, 290), (0, 0)), bcp=((1.1e5, 0), (0, 0.9e5), (0, 0))),
                               seed=61, dt=1e-7),
        I.random_coeff_problem(I.Grid(dim=2, axisym=1, n=(48, 104, 1), h=1e-4, bc=((A, D), (W, W), (0, 0)),
                                      bcT=((0, 300), (0, 0), (0, 0)), bcp=((0, 1e5), (0, 0), (0, 0))),
                               seed=62, dt=1e-5),
        I.random_coeff_problem(I.Grid(dim=3, axisym=0, n=(40, 24, 16), h=1e-4, bc=((D, D), (D, D), (W, D)),
                                      bcT=((300, 300), (300, 300), (0, 300)),
                                      bcp=((1e5, 1e5), (1e5, 1e5), (0, 1e5))), seed=63, dt=1e-5),
    ]


@pytest.mark.parametrize("q", [0, 1, 2])
def test_noalloc_norms_match_handle_norms_twice(q, orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_11294_gb300 import binding as B
    p = _problems()[q]
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    lam, fa, fk, b = T(p.lam), [T(f) for f in p.fa], [T(f) for f in p.fk], T(p.b)
    s = B.Solver(p.grid)
    s.set_coeffs(lam, fa, fk)
    rng = np.random.default_rng(q)
    states = [p.x0, p.x0 * (1.0 + 1e-3 * rng.standard_normal(p.x0.shape))]
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for x in states:                       # two calls in a row
        xd = T(x)
        ref = s.residual_norms(b, xd)
        B.residual_norms_noalloc(p.grid, lam, fa, fk, b, xd, out)
        got = out.cpu().numpy()
        assert np.allclose(got, ref, rtol=1e-12, atol=0), (got, ref)
        oref = orc.residual_norms(p.grid.as_dict(), p.lam, p.fa, p.fk, p.b, x)
        assert np.allclose(got, oref, rtol=1e-12, atol=0), (got, oref)
    # the entry point's reason to exist: a call allocates no device memory
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    B.residual_norms_noalloc(p.grid, lam, fa, fk, b, xd, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    s.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_11294_gb300 import binding as B
    import ctypes as C
    g = B.make_grid(I.Grid(dim=2, axisym=0, n=(4096, 4104, 1), h=1.0))
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = (C.c_void_p * 3)(C.c_void_p(dummy.data_ptr()), C.c_void_p(dummy.data_ptr()), None)
    st = B.load().mg_residual_norms_noalloc(C.byref(g), C.c_void_p(dummy.data_ptr()), p, p,
                                            C.c_void_p(dummy.data_ptr()), C.c_void_p(dummy.data_ptr()),
                                            C.c_void_p(dummy.data_ptr()), None)
    assert st == B.MG_ERR_INVALID_ARG
    assert "at most 65536" in B.last_error()
