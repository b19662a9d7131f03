"""E3 from Gauss's law (Sec. 2) through the C ABI: prop_get_e3 against the
oracle's e3_from_transverse on the same field and medium.

The field is set directly (prop_set_field), so the check isolates the
recovery: FP64 to 1e-10 and FP32 to 1e-5 (relative L2), on the vector
workload's recipe (random n^2 with border, lambda/6) and on a homogeneous
n0 = 1.2 medium; then after propagation steps the recovered E3 of the GPU
field matches the oracle's E3 of the oracle's field."""
import math

import numpy as np
import pytest

from util import gpu_propagator, gpu_run, oracle_table, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2410_17446_gb300 import build, prop
    build.build()
    return prop


def _field(n, dx, seed):
    rng = np.random.default_rng(seed)
    x = (np.arange(n) - n // 2) * dx
    X, Y = np.meshgrid(x, x)
    env = np.exp(-(X ** 2 + Y ** 2) / (0.15 * n * dx) ** 2)
    return np.stack([env * (1 + 0.3 * rng.standard_normal((n, n))),
                     env * (0.4j + 0.3 * rng.standard_normal((n, n)))]).astype(np.complex128)


@pytest.mark.parametrize("prec,bar", [("fp64", 1e-10), ("fp32", 1e-5)])
@pytest.mark.parametrize("n", [64, 256])
def test_e3_matches_oracle_random_medium(P, prec, bar, n):
    from oracle import gauss
    from paper_2410_17446_gb300 import workloads as wl
    W = wl.vector_random_512(1, n=n)
    b = W.beams[0]
    pr = gpu_propagator(W, "vector_random_512", P.PROP_FP64 if prec == "fp64" else P.PROP_FP32)
    w = _field(n, b.grid.dx, n)
    pr.set_field(0, w)
    pr.set_medium(0, b.medium(0))
    got = pr.get_e3(0)
    ref = gauss.e3_from_transverse(w, b.medium(0), b.grid.dx, b.grid.dy, W.k0, W.n0)
    assert np.linalg.norm(ref) > 1e-3 * np.linalg.norm(w)
    assert rel_l2(got, ref) < bar


def test_e3_homogeneous_n0(P):
    """n0 = 1.2 and n^2 = n0^2: kz is taken with k0 n0."""
    from oracle import gauss
    from paper_2410_17446_gb300 import prop as Pm, tables, workloads as wl
    g = wl.Grid(128, 128, 0.2, 0.2)
    tab = tables.load("plain_scalar_64")
    pr = Pm.Propagator.from_table([(g.nx, g.ny, g.dx, g.dy)], 2 * math.pi, 1.2, 0.5, tab, ncomp=2,
                                  precision=P.PROP_FP64)
    w = _field(128, 0.2, 3)
    n2 = np.full((128, 128), 1.44, np.complex128)
    pr.set_field(0, w)
    pr.set_medium(0, n2)
    got = pr.get_e3(0)
    ref = gauss.e3_from_transverse(w, n2, g.dx, g.dy, 2 * math.pi, 1.2)
    assert rel_l2(got, ref) < 1e-10


def test_e3_after_steps(P):
    """Three FP64 steps of the vector workload's recipe at 64^2, then E3 of the
    GPU field against E3 of the oracle's field."""
    from oracle import gauss
    from oracle import propagator as orp
    from paper_2410_17446_gb300 import workloads as wl
    W = wl.vector_random_512(3, n=64)
    b = W.beams[0]
    pr = gpu_propagator(W, "vector_random_512", P.PROP_FP64, tol=1e-12)
    gpu_run(pr, W, 3)
    got = pr.get_e3(0)
    wref = orp.run(b, W.k0, W.n0, oracle_table("vector_random_512"), 2, 3, tol=1e-12)
    ref = gauss.e3_from_transverse(wref, b.medium(2), b.grid.dx, b.grid.dy, W.k0, W.n0)
    assert rel_l2(got, ref) < 1e-9


def test_e3_needs_a_vector_handle(P):
    from paper_2410_17446_gb300 import workloads as wl
    W = wl.plain_scalar_64(1)
    pr = gpu_propagator(W, "plain_scalar_64", P.PROP_FP64)
    with pytest.raises(P.PropError) as e:
        pr.get_e3(0)
    assert e.value.status == P.PROP_E_UNSUPPORTED
