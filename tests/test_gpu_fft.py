"""The shared-memory radix FFT (every pass of the hot path) against numpy.fft."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(16, 16), (32, 64), (128, 64), (256, 256), (384, 768), (512, 128), (768, 384), (1024, 1024)]


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2410_17446_gb300 import build, prop
    build.build()
    return prop


@pytest.mark.parametrize("nx,ny", SHAPES)
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_fft2_forward_and_inverse(P, nx, ny, prec):
    import torch
    rng = np.random.default_rng(nx * 7 + ny)
    batch = 3
    x = rng.standard_normal((batch, ny, nx)) + 1j * rng.standard_normal((batch, ny, nx))
    cdt = torch.complex64 if prec == "fp32" else torch.complex128
    p = P.PROP_FP32 if prec == "fp32" else P.PROP_FP64
    tol = 2e-6 if prec == "fp32" else 1e-13
    wb = P.prop_fft2_workspace_size(nx, ny, p)
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    d = torch.tensor(x, dtype=cdt, device="cuda")
    P.prop_fft2(nx, ny, batch, p, 0, d, work, wb, torch.cuda.current_stream().cuda_stream)
    ref = np.fft.fft2(x)
    got = d.cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol
    P.prop_fft2(nx, ny, batch, p, 1, d, work, wb, torch.cuda.current_stream().cuda_stream)
    back = d.cpu().numpy()
    assert np.linalg.norm(back - x) / np.linalg.norm(x) < tol


def test_fft2_empty_batch_and_bad_size(P):
    import torch
    work = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    d = torch.zeros(4, dtype=torch.complex64, device="cuda")
    P.prop_fft2(64, 64, 0, P.PROP_FP32, 0, d, work, work.numel(), 0)
    with pytest.raises(P.PropError):
        P.prop_fft2(100, 64, 1, P.PROP_FP32, 0, d, work, work.numel(), 0)
