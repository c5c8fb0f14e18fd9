"""mg_copy_h2d_async: host-to-device copies by a kernel from page-locked
memory.  Bytes must arrive exactly for every size (words of 16 bytes and a
ragged tail, empty included); anything other than page-locked host source,
device destination and 16-byte alignment is refused before any launch."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_11294_gb300 import binding
    binding.load()
    return torch


@pytest.mark.parametrize("nbytes", [0, 1, 15, 16, 17, 4104, 1 << 20, (37 << 20) + 3])
def test_copy_is_exact(torch_cuda, nbytes):
    torch = torch_cuda
    from paper_2206_11294_gb300.binding import copy_h2d
    rng = np.random.default_rng(nbytes)
    src = torch.from_numpy(rng.integers(0, 256, size=nbytes, dtype=np.uint8)).pin_memory()
    dst = torch.full((nbytes,), 7, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream(priority=-1)
    copy_h2d(dst, src, s)
    s.synchronize()
    assert torch.equal(dst.cpu(), src)


def test_copy_of_doubles_on_the_current_stream(torch_cuda):
    torch = torch_cuda
    from paper_2206_11294_gb300.binding import copy_h2d
    src = torch.randn(1001, 4, dtype=torch.float64).pin_memory()
    dst = copy_h2d(torch.empty(1001, 4, dtype=torch.float64, device="cuda"), src)
    torch.cuda.synchronize()
    assert torch.equal(dst.cpu(), src)


def test_copy_refuses_bad_arguments(torch_cuda):
    torch = torch_cuda
    from paper_2206_11294_gb300.binding import MG_ERR_INVALID_ARG, MgError, copy_h2d
    pinned = torch.zeros(4096, dtype=torch.uint8).pin_memory()
    dev = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    bad = [(dev, torch.zeros(4096, dtype=torch.uint8)),            # pageable source
           (dev[1:], pinned[1:]),                                   # misaligned
           (torch.zeros(4096, dtype=torch.uint8).pin_memory(), pinned),   # host destination
           (dev, dev.clone())]                                      # device source
    for d, s in bad:
        with pytest.raises(MgError) as e:
            copy_h2d(d, s)
        assert e.value.status == MG_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert int(dev.sum()) == 0
