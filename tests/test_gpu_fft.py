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


PLANS = [("block", "plain"), ("block", "warp"), ("warp", "plain"), ("warp", "warp"), ("warp", "tma")]


@pytest.fixture
def restore_plans(P):
    saved = {(n, p): P.prop_get_fft_plan(n, p) for n in (512, 1024) for p in (P.PROP_FP32, P.PROP_FP64)}
    yield
    for (n, p), pl in saved.items():
        P.prop_set_fft_plan(n, p, pl.rows, pl.cols, pl.rows_small, pl.cols_small)


@pytest.mark.parametrize("rows,cols", PLANS)
@pytest.mark.parametrize("nx,ny", [(1024, 1024), (512, 1024), (1024, 512), (512, 512)])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_fft2_every_plan(P, restore_plans, rows, cols, nx, ny, prec):
    """The warp row and column transforms (N = 512, 1024) against numpy.fft, in
    every combination with the block-wide ones (prop_fft2 has no tensor maps, so
    'tma' there means the plain-load column pass)."""
    import torch
    p = P.PROP_FP32 if prec == "fp32" else P.PROP_FP64
    R = {"block": P.PROP_ROWS_BLOCK, "warp": P.PROP_ROWS_WARP}[rows]
    Cc = {"tma": P.PROP_COLS_TMA, "plain": P.PROP_COLS_PLAIN, "warp": P.PROP_COLS_WARP}[cols]
    for n in {nx, ny}:
        P.prop_set_fft_plan(n, p, R, Cc)
    rng = np.random.default_rng(nx + 5 * ny)
    x = rng.standard_normal((2, ny, nx)) + 1j * rng.standard_normal((2, ny, nx))
    cdt = torch.complex64 if prec == "fp32" else torch.complex128
    tol = 2e-6 if prec == "fp32" else 1e-13
    wb = P.prop_fft2_workspace_size(nx, ny, p)
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    d = torch.tensor(x, dtype=cdt, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    P.prop_fft2(nx, ny, 2, p, 0, d, work, wb, s)
    ref = np.fft.fft2(x)
    assert np.linalg.norm(d.cpu().numpy() - ref) / np.linalg.norm(ref) < tol
    P.prop_fft2(nx, ny, 2, p, 1, d, work, wb, s)
    assert np.linalg.norm(d.cpu().numpy() - x) / np.linalg.norm(x) < tol


def test_plan_validation(P, restore_plans):
    with pytest.raises(P.PropError) as e:
        P.prop_set_fft_plan(256, P.PROP_FP32, P.PROP_ROWS_WARP, P.PROP_COLS_TMA)
    assert e.value.status == P.PROP_E_UNSUPPORTED
    with pytest.raises(P.PropError):
        P.prop_set_fft_plan(100, P.PROP_FP32, P.PROP_ROWS_BLOCK, P.PROP_COLS_TMA)
    P.prop_set_fft_plan(1024, P.PROP_FP32, P.PROP_ROWS_WARP, P.PROP_COLS_WARP, P.PROP_ROWS_BLOCK, P.PROP_COLS_PLAIN)
    pl = P.prop_get_fft_plan(1024, P.PROP_FP32)
    assert (pl.rows, pl.cols, pl.rows_small, pl.cols_small) == (P.PROP_ROWS_WARP, P.PROP_COLS_WARP,
                                                                P.PROP_ROWS_BLOCK, P.PROP_COLS_PLAIN)


@pytest.mark.parametrize("n", [256, 1024])
def test_autotuner_times_every_combination(P, restore_plans, n):
    """prop_fft_autotune times the round trip for each (rows, cols) combination
    that exists for n, returns the fastest under the 5 % rule and leaves the
    installed plan unchanged."""
    from paper_2410_17446_gb300 import autotune
    before = P.prop_get_fft_plan(n, P.PROP_FP32)
    rec = autotune.tune(n, P.PROP_FP32, reps=2, batch=4)
    after = P.prop_get_fft_plan(n, P.PROP_FP32)
    assert (before.rows, before.cols, before.rows_small, before.cols_small) == \
        (after.rows, after.cols, after.rows_small, after.cols_small)
    t = rec["round_trip_ms"]
    assert all(v > 0 for v in t.values())
    if n == 1024:
        assert set(t) == {"block+tma", "block+plain", "block+warp", "warp+tma", "warp+plain", "warp+warp"}
    else:
        assert set(t) == {"block+tma", "block+plain"} and rec["rows"] == "block"
    fastest = min(t, key=t.get)
    want = fastest if t[fastest] < 0.95 * t["block+tma"] else "block+tma"
    assert f"{rec['rows']}+{rec['cols']}" == want
    assert rec["rows_small"] in ("block", "warp") and rec["cols_small"] in ("tma", "plain", "warp")
