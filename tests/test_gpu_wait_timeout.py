"""Failure detection of the asynchronous tile copies, without a GPU fault: a
bounded mbarrier wait on a copy that never comes must end with PROP_E_TIMEOUT,
and the CUDA context must stay usable afterwards."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2410_17446_gb300 import build, prop
    build.build()
    return prop


def test_bounded_wait_reports_timeout_and_context_survives(P):
    import time
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    t0 = time.perf_counter()
    st = P.lib().prop_selftest_wait_timeout(stream)
    dt = time.perf_counter() - t0
    assert st == P.PROP_E_TIMEOUT, P.lib().prop_error_string(st)
    assert dt < 30.0
    # the same context still computes: a 2-D transform through the library
    rng = np.random.default_rng(3)
    x = rng.standard_normal((1, 64, 64)) + 1j * rng.standard_normal((1, 64, 64))
    wb = P.prop_fft2_workspace_size(64, 64, P.PROP_FP64)
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    d = torch.tensor(x, dtype=torch.complex128, device="cuda")
    P.prop_fft2(64, 64, 1, P.PROP_FP64, 0, d, work, wb, stream)
    ref = np.fft.fft2(x)
    assert np.linalg.norm(d.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-13
