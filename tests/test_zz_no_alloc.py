"""prop_fft2_noalloc: the batched 2-D DFT for callers that cannot allocate
device memory (a plugin whose host application owns every device
allocation, a program held to a fixed memory budget).  Its twiddle tables sit
in a fixed file-scope device array instead of a caller workspace.

Checked through the C ABI against prop_fft2 (which uses a caller workspace)
and against numpy.fft, within the tolerances of the FFT tests.  Calls of
different sizes and precisions alternate on one stream, each size coming back
after another one has rewritten the shared array, so that a stale or wrongly
offset twiddle table left by an earlier call would show.  This file is
collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# (nx, ny, precision): a sequence in which every size returns after others
SEQUENCE = [(1024, 1024, "fp32"), (384, 768, "fp64"), (64, 32, "fp32"), (1024, 1024, "fp32"),
            (16, 1024, "fp64"), (384, 768, "fp64"), (1024, 1024, "fp64"), (64, 32, "fp32")]
TOL = {"fp32": 2e-6, "fp64": 1e-13}


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2410_17446_gb300 import build, prop
    build.build()
    return prop


def _input(nx, ny):
    rng = np.random.default_rng(nx + 3 * ny)
    return rng.standard_normal((2, ny, nx)) + 1j * rng.standard_normal((2, ny, nx))


def test_noalloc_fft_alternating_sizes_and_precisions(P):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    for nx, ny, prec in SEQUENCE:
        p = P.PROP_FP32 if prec == "fp32" else P.PROP_FP64
        cdt = torch.complex64 if prec == "fp32" else torch.complex128
        x = _input(nx, ny)
        wb = P.prop_fft2_workspace_size(nx, ny, p)
        work = torch.empty(wb, dtype=torch.uint8, device="cuda")
        for inverse in (0, 1):
            ref = torch.tensor(x, dtype=cdt, device="cuda")
            P.prop_fft2(nx, ny, 2, p, inverse, ref, work, wb, stream)
            want = ref.cpu().numpy()
            npref = (np.fft.ifft2(x) if inverse else np.fft.fft2(x))
            d = torch.tensor(x, dtype=cdt, device="cuda")
            P.prop_fft2_noalloc(nx, ny, 2, p, inverse, d, stream)
            got = d.cpu().numpy()
            assert np.linalg.norm(got - want) / np.linalg.norm(want) < TOL[prec], (nx, ny, prec, inverse)
            assert np.linalg.norm(got - npref) / np.linalg.norm(npref) < TOL[prec], (nx, ny, prec, inverse)


def test_noalloc_rejects_bad_requests(P):
    import torch
    d = torch.zeros(4, dtype=torch.complex64, device="cuda")
    with pytest.raises(P.PropError) as e:
        P.prop_fft2_noalloc(100, 64, 1, P.PROP_FP32, 0, d, 0)
    assert e.value.status == P.PROP_E_UNSUPPORTED
    P.prop_fft2_noalloc(64, 64, 0, P.PROP_FP32, 0, d, 0)   # empty batch: nothing to do
