"""Beams of uneven grid sizes advanced in lockstep, each Arnoldi pass one launch
over every grid (the multi-group step, Sec. 4's batched solves across beams).

The multi-group step runs the same per-system arithmetic as the grid-by-grid
step, so the fields agree with it and with the CPU oracle at the FP32 bar, and
the number of launches of each Arnoldi kernel is the number of lockstep Arnoldi
steps, whatever the number of grids."""
import numpy as np
import pytest

from util import gpu_propagator, gpu_run, oracle_table, rel_l2

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
ARNOLDI_KINDS = ("rows_fwd", "cols", "rows_inv", "gram", "gs_update")


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2410_17446_gb300 import build, prop
    build.build()
    return prop


def _workload(specs, nsteps, dz=0.5, name="uneven_mg"):
    """Scalar beams, one per (n, dx, eps, period, waist), each with its own sine product."""
    from paper_2410_17446_gb300 import workloads as wl
    beams = []
    for n, dx, eps, period, waist in specs:
        g = wl.Grid(n, n, dx, dx)
        width = max(8, n // 16)

        def med(s, g=g, eps=eps, period=period, width=width):
            return wl.sine_product_n2(g, eps, period, (s + 0.5) * dz, width, 0.2)

        beams.append(wl.Beam(g, wl.gaussian_beam(g, waist)[None], med, lambda s: True, width, 0.2))
    return wl.Workload(name, wl.K0, 1.0, dz, nsteps, 12, 1, "fp32", 20, 1e-7, beams)


def _oracle(W, beam, nsteps):
    from oracle import propagator as orp
    return orp.run(W.beams[beam], W.k0, W.n0, oracle_table("uneven_batch"), W.ncomp, nsteps, tol=1e-12)


def _launches(pr):
    prof = pr.profile()
    return {k: prof[k]["launches"] for k in ARNOLDI_KINDS}


UNEVEN = ((128, 0.25, 0.06, 1.3, 3.0), (256, 0.25, 0.05, 1.7, 4.0), (384, 0.25, 0.04, 1.2, 4.0),
          (256, 0.25, 0.03, 2.1, 5.0), (512, 0.25, 0.03, 2.0, 5.0))


def test_uneven_sizes_match_grid_by_grid_and_oracle(P):
    """Four grids (128, 256 twice, 384, 512) in one handle, two FP32 steps: the
    lockstep fields equal the grid-by-grid ones and, on the 128 and 256 grids,
    the FP64 oracle's, within the FP32 bar."""
    W = _workload(UNEVEN, 2)
    mg = gpu_run(gpu_propagator(W, "uneven_batch", P.PROP_FP32), W, 2)
    one = gpu_run(gpu_propagator(W, "uneven_batch", P.PROP_FP32, multigroup=False), W, 2)
    for i in range(len(W.beams)):
        assert rel_l2(mg[i], one[i]) < FP32_TOL, i
    for i in (0, 1, 3):
        assert rel_l2(mg[i], _oracle(W, i, 2)) < FP32_TOL, i


def test_launches_per_arnoldi_pass_do_not_grow_with_the_grids(P):
    """The same beam on 2 and on 4 grids (256^2, dx differing by 1e-12 relative,
    so each is its own grid and every solve takes the same Arnoldi steps): in
    lockstep each Arnoldi kernel launches as often for 4 grids as for 2, while
    grid by grid the launches double; every copy of the field agrees."""
    def specs(k):
        return [(256, 0.25 * (1 + 1e-12 * i), 0.05, 1.7, 4.0) for i in range(k)]

    counts, fields = {}, {}
    for k in (2, 4):
        for mgflag in (True, False):
            W = _workload(specs(k), 1)
            pr = gpu_propagator(W, "uneven_batch", P.PROP_FP32, multigroup=mgflag)
            fields[k, mgflag] = gpu_run(pr, W, 1)
            counts[k, mgflag] = _launches(pr)
    print("launches", counts)
    for kind in ("gram", "gs_update"):   # Arnoldi-only kernels
        assert counts[4, True][kind] == counts[2, True][kind], kind
        assert counts[4, False][kind] == 2 * counts[2, False][kind], kind
        assert counts[2, True][kind] * 2 <= counts[2, False][kind] + 2 * 4, kind
    for kind in ARNOLDI_KINDS:
        assert counts[4, True][kind] < counts[4, False][kind], kind
    ref = fields[2, False][0]
    for key, fl in fields.items():
        for f in fl:
            assert rel_l2(f, ref) < FP32_TOL, key


def test_radix3_and_1024_grids_in_lockstep(P):
    """768 and 1024 grids with a 128 one, one FP32 step: the lockstep fields equal
    the grid-by-grid ones within the FP32 bar."""
    W = _workload(((768, 0.25, 0.08, 2.3, 6.0), (1024, 0.25, 0.05, 1.7, 8.0), (128, 0.25, 0.06, 1.3, 3.0)), 1)
    mg = gpu_run(gpu_propagator(W, "uneven_batch", P.PROP_FP32), W, 1)
    one = gpu_run(gpu_propagator(W, "uneven_batch", P.PROP_FP32, multigroup=False), W, 1)
    for i in range(len(W.beams)):
        assert rel_l2(mg[i], one[i]) < FP32_TOL, i


def test_vector_grids_in_lockstep(P):
    """The vector operator (w1, w2) on 128 and 256 grids of the Gaussian random
    medium in one handle, two FP32 steps: lockstep equals grid by grid, and the
    128 beam equals the oracle's, within the FP32 bar."""
    from paper_2410_17446_gb300 import workloads as wl
    a, b = wl.vector_random_512(2, n=128), wl.vector_random_512(2, n=256)
    W = wl.Workload("vector_mg", a.k0, a.n0, a.dz, 2, a.npoles, 2, "fp32", 20, 1e-7, a.beams + b.beams)
    mg = gpu_run(gpu_propagator(W, "vector_random_512", P.PROP_FP32), W, 2)
    one = gpu_run(gpu_propagator(W, "vector_random_512", P.PROP_FP32, multigroup=False), W, 2)
    for i in range(2):
        assert rel_l2(mg[i], one[i]) < FP32_TOL, i
    from oracle import propagator as orp
    ref = orp.run(W.beams[0], W.k0, W.n0, oracle_table("vector_random_512"), 2, 2, tol=1e-12)
    assert rel_l2(mg[0], ref) < FP32_TOL
    assert np.linalg.norm(mg[1][1]) > 0
