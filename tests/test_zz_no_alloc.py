"""prop_fft2_noalloc: the batched 2-D DFT for callers that cannot allocate
device memory (a plugin whose host application owns every device
allocation, a program held to a fixed memory budget).  Its twiddle tables sit
in a fixed file-scope device array instead of a caller workspace.

Checked through the C ABI against prop_fft2 (which uses a caller workspace),
within the tolerances of the FFT tests, on two calls in a row so that a stale
or shared scratch would show.  This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [(64, 32, "fp32"), (1024, 1024, "fp32"), (384, 768, "fp64"), (16, 1024, "fp64")]


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2410_17446_gb300 import build, prop
    build.build()
    return prop


@pytest.mark.parametrize("nx,ny,prec", CASES)
def test_noalloc_fft_matches_workspace_fft_twice(P, nx, ny, prec):
    import torch
    p = P.PROP_FP32 if prec == "fp32" else P.PROP_FP64
    cdt = torch.complex64 if prec == "fp32" else torch.complex128
    tol = 2e-6 if prec == "fp32" else 1e-13
    rng = np.random.default_rng(nx + 3 * ny)
    x = rng.standard_normal((2, ny, nx)) + 1j * rng.standard_normal((2, ny, nx))
    stream = torch.cuda.current_stream().cuda_stream
    wb = P.prop_fft2_workspace_size(nx, ny, p)
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    for inverse in (0, 1):
        ref = torch.tensor(x, dtype=cdt, device="cuda")
        P.prop_fft2(nx, ny, 2, p, inverse, ref, work, wb, stream)
        want = ref.cpu().numpy()
        for _ in range(2):
            d = torch.tensor(x, dtype=cdt, device="cuda")
            P.prop_fft2_noalloc(nx, ny, 2, p, inverse, d, stream)
            got = d.cpu().numpy()
            assert np.linalg.norm(got - want) / np.linalg.norm(want) < tol


def test_noalloc_rejects_bad_requests(P):
    import torch
    d = torch.zeros(4, dtype=torch.complex64, device="cuda")
    with pytest.raises(P.PropError) as e:
        P.prop_fft2_noalloc(100, 64, 1, P.PROP_FP32, 0, d, 0)
    assert e.value.status == P.PROP_E_UNSUPPORTED
    P.prop_fft2_noalloc(64, 64, 0, P.PROP_FP32, 0, d, 0)   # empty batch: nothing to do
