"""Parity of the CUDA z-step (Eq. approx_prop) with the CPU oracle, through the C ABI.

Bars: relative L2 field error <= 1e-10 where FP64 runs, <= 1e-5 for the FP32
path (the accuracy bars of the method's configurations)."""
import math

import numpy as np
import pytest

from util import gpu_propagator, gpu_run, oracle_table, rel_l2, table_json

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2410_17446_gb300 import build, prop
    build.build()
    return prop


def oracle_run(W, table, nsteps, beam=0, tol=1e-12):
    from oracle import propagator as pr
    b = W.beams[beam]
    return pr.run(b, W.k0, W.n0, table, W.ncomp, nsteps, tol=tol)


def test_plain_scalar_64_fp64_full_run(P):
    """64^2, 12 poles, static sine-product medium with an absorbing border, 16 steps, FP64."""
    from paper_2410_17446_gb300 import workloads as wl
    W = wl.plain_scalar_64()
    pr = gpu_propagator(W, "plain_scalar_64", P.PROP_FP64, tol=1e-12)
    got = gpu_run(pr, W, W.nsteps)[0]
    ref = oracle_run(W, oracle_table("plain_scalar_64"), W.nsteps)
    assert rel_l2(got, ref) < FP64_TOL
    it = pr.iterations()
    assert it.min() >= 1


@pytest.mark.parametrize("n,steps", [(128, 3), (256, 1)])
def test_batched_scalar_fp32_reduced(P, n, steps):
    """z-varying sine-product medium with border, 16 poles, complex FP32 path."""
    from paper_2410_17446_gb300 import workloads as wl
    W = wl.batched_scalar_1024(steps, n=n)
    pr = gpu_propagator(W, "batched_scalar_1024", P.PROP_FP32)
    got = gpu_run(pr, W, steps)[0]
    ref = oracle_run(W, oracle_table("batched_scalar_1024"), steps, tol=1e-12)
    assert rel_l2(got, ref) < FP32_TOL


@pytest.mark.parametrize("prec,tol", [("fp32", FP32_TOL), ("fp64", FP64_TOL)])
def test_homogeneous_aperture_against_closed_form(P, prec, tol):
    """Homogeneous medium: the step is IFFT[r(zeta_fs) FFT w] (Eq. approx_fs_prop)
    and no GMRES iteration is needed."""
    from oracle import propagator as orp
    from paper_2410_17446_gb300 import workloads as wl
    W = wl.homogeneous_aperture_1024(20, n=256)
    pr = gpu_propagator(W, "homogeneous_aperture_1024", P.PROP_FP64 if prec == "fp64" else P.PROP_FP32)
    got = gpu_run(pr, W, 20)[0]
    g = W.beams[0].grid
    ref = orp.homogeneous_rational_step(W.beams[0].w0, g.dx, g.dy, W.k0, oracle_table("homogeneous_aperture_1024"), 20)
    assert rel_l2(got, ref) < tol
    assert pr.iterations().max() == 0


def test_uneven_beams_in_one_handle(P):
    """Beams of different grid sizes (and one repeated size) share one handle."""
    from paper_2410_17446_gb300 import workloads as wl
    W = wl.uneven_batch(nbeams=3, nsteps=2, sizes=(64, 128))
    pr = gpu_propagator(W, "uneven_batch", P.PROP_FP32)
    got = gpu_run(pr, W, 2)
    T = oracle_table("uneven_batch")
    for i in range(3):
        assert rel_l2(got[i], oracle_run(W, T, 2, beam=i)) < FP32_TOL


def test_zero_field_stays_zero(P):
    from paper_2410_17446_gb300 import workloads as wl
    W = wl.plain_scalar_64(2)
    pr = gpu_propagator(W, "plain_scalar_64", P.PROP_FP32)
    pr.set_field(0, np.zeros((1, 64, 64), np.complex128))
    out = gpu_run(pr, W, 2)[0]
    assert np.all(out == 0)


def test_noconv_leaves_field_unchanged(P):
    from paper_2410_17446_gb300 import workloads as wl
    W = wl.plain_scalar_64(1)
    pr = gpu_propagator(W, "plain_scalar_64", P.PROP_FP64, tol=1e-15, max_restarts=1, restart=2)
    pr.set_medium(0, W.beams[0].medium(0))
    with pytest.raises(P.PropError) as e:
        pr.step()
    assert e.value.status == P.PROP_E_NOCONV
    np.testing.assert_array_equal(pr.get_field(0), W.beams[0].w0)


def test_homogeneous_aperture_full_size_100_steps(P):
    """1024^2, 100 steps, FP32: the configuration as benchmarked, against the
    closed-form rational step IFFT[r(zeta_fs)^100 FFT w0] (Eq. approx_fs_prop)."""
    from oracle import propagator as orp
    from paper_2410_17446_gb300 import workloads as wl
    W = wl.homogeneous_aperture_1024()
    pr = gpu_propagator(W, "homogeneous_aperture_1024", P.PROP_FP32)
    got = gpu_run(pr, W, W.nsteps)[0]
    g = W.beams[0].grid
    ref = orp.homogeneous_rational_step(W.beams[0].w0, g.dx, g.dy, W.k0, oracle_table("homogeneous_aperture_1024"),
                                        W.nsteps)
    assert rel_l2(got, ref) < FP32_TOL


@pytest.mark.parametrize("n,plan", [(256, None), (1024, None), (1024, ("warp", "warp")), (1024, ("block", "plain"))])
def test_batched_scalar_solutions_satisfy_the_shifted_systems(P, n, plan):
    """Full size (and a reduced one): after a GPU step the oracle rebuilds every
    pole's solution x_k = (Z_fs - p_k)^-1 w + e_k from the GPU's correction e_k,
    checks its residual ||w - (Z - p_k) x_k|| with the oracle's own operator,
    and recombines r(Z) w = r0 w + sum r_k x_k (Eq. approx_prop) against the
    GPU's new field."""
    from oracle import operators as ops
    from paper_2410_17446_gb300 import workloads as wl
    saved = P.prop_get_fft_plan(n, P.PROP_FP32)
    if plan is not None:   # FFT pass variants (same arithmetic): warp rows and columns, or plain-load columns
        P.prop_set_fft_plan(n, P.PROP_FP32, {"block": P.PROP_ROWS_BLOCK, "warp": P.PROP_ROWS_WARP}[plan[0]],
                            {"plain": P.PROP_COLS_PLAIN, "warp": P.PROP_COLS_WARP}[plan[1]])
    W = wl.batched_scalar_1024(1, n=n)
    T = oracle_table("batched_scalar_1024")
    try:
        pr = gpu_propagator(W, "batched_scalar_1024", P.PROP_FP32)
        got = gpu_run(pr, W, 1)[0]
    finally:
        P.prop_set_fft_plan(n, P.PROP_FP32, saved.rows, saved.cols, saved.rows_small, saved.cols_small)
    b = W.beams[0]
    w0 = b.w0
    med = ops.Medium(b.medium(0), b.grid.dx, b.grid.dy, W.k0, W.n0, 1)
    out = T.r0 * w0
    worst = 0.0
    for k, (p, r) in enumerate(zip(T.poles, T.residues)):
        x = med.freespace_solve(w0, p) + pr.get_correction(0, k)
        res = np.linalg.norm(w0 - med.apply_shifted(x, p)) / np.linalg.norm(w0)
        worst = max(worst, res)
        out = out + r * x
    assert worst < 1e-4, worst          # FP32 solves: residual well below the field
    assert rel_l2(got, out) < 1e-6      # the GPU's residue sum and free-space part
    assert pr.iterations().min() >= 1


def test_small_vector_fp64(P):
    """Two-component (w1, w2) propagation with psi and cross-polarisation terms, FP64, 16^2."""
    from paper_2410_17446_gb300 import workloads as wl
    W = wl.small_vector(16)
    pr = gpu_propagator(W, "plain_scalar_64", P.PROP_FP64, tol=1e-12)
    got = gpu_run(pr, W, 2)[0]
    ref = oracle_run(W, oracle_table("plain_scalar_64"), 2)
    assert rel_l2(got, ref) < FP64_TOL


@pytest.mark.parametrize("n,steps,prec", [(64, 3, "fp32"), (128, 1, "fp64")])
def test_vector_random_reduced(P, n, steps, prec):
    """Gaussian random medium (l = lambda, seed 7) with border, x-polarised beam, 14 poles."""
    from paper_2410_17446_gb300 import workloads as wl
    W = wl.vector_random_512(steps, n=n)
    pr = gpu_propagator(W, "vector_random_512", P.PROP_FP32 if prec == "fp32" else P.PROP_FP64,
                        **({} if prec == "fp32" else {"tol": 1e-12}))
    got = gpu_run(pr, W, steps)[0]
    ref = oracle_run(W, oracle_table("vector_random_512"), steps)
    assert rel_l2(got, ref) < (FP32_TOL if prec == "fp32" else FP64_TOL)
    assert np.linalg.norm(got[1]) > 0        # cross-polarisation has coupled energy into w2


def test_vector_random_full_size_solutions(P):
    """512^2 vector step: every pole's x_k = (Z_fs - p_k)^-1 w + e_k satisfies
    (Z - p_k) x_k = w under the oracle's operator, and the GPU field is
    r0 w + sum r_k x_k."""
    from oracle import operators as ops
    from paper_2410_17446_gb300 import workloads as wl
    W = wl.vector_random_512(1)
    T = oracle_table("vector_random_512")
    pr = gpu_propagator(W, "vector_random_512", P.PROP_FP32)
    b = W.beams[0]
    got = gpu_run(pr, W, 1)[0]
    med = ops.Medium(b.medium(0), b.grid.dx, b.grid.dy, W.k0, W.n0, 2)
    out = T.r0 * b.w0
    worst = 0.0
    for k, (p, r) in enumerate(zip(T.poles, T.residues)):
        x = med.freespace_solve(b.w0, p) + pr.get_correction(0, k)
        worst = max(worst, np.linalg.norm(b.w0 - med.apply_shifted(x, p)) / np.linalg.norm(b.w0))
        out = out + r * x
    assert worst < 1e-4, worst
    assert rel_l2(got, out) < 1e-6


def test_hard_scattering_beam_fp32_six_steps(P):
    """The hardest beam of the uneven batch (eps = 0.083, period 1.498 lambda:
    first-order scattering lands next to the evanescent boundary, where the poles
    crowd) at 128^2, six FP32 steps against the FP64 oracle."""
    from paper_2410_17446_gb300 import workloads as wl
    g = wl.Grid(128, 128, 0.25, 0.25)
    dz = 0.5

    def med(s):
        return wl.sine_product_n2(g, 0.0831792411594809, 1.4983412918408128, (s + 0.5) * dz, 8, 0.2)

    beam = wl.Beam(g, wl.gaussian_beam(g, 2.827372867618358)[None], med, lambda s: True, 8, 0.2)
    W = wl.Workload("hard_beam_128", wl.K0, 1.0, dz, 6, 12, 1, "fp32", 20, 1e-7, [beam])
    pr = gpu_propagator(W, "uneven_batch", P.PROP_FP32)
    got = gpu_run(pr, W, 6)[0]
    ref = oracle_run(W, oracle_table("uneven_batch"), 6)
    assert rel_l2(got, ref) < FP32_TOL


def test_uneven_384_and_768_beams_solutions(P):
    """The radix-3 grids of the uneven batch (384 = 3 8 16, 768 = 3 16 16) in one
    handle with a repeated 384 beam: after one FP32 step every beam's pole
    solutions x_k = (Z_fs - p_k)^-1 w + e_k satisfy (Z - p_k) x_k = w under the
    oracle's operator, and the GPU field is r0 w + sum r_k x_k (Eq. approx_prop)."""
    from oracle import operators as ops
    from paper_2410_17446_gb300 import workloads as wl
    dz = 0.5
    beams = []
    for n, eps, period, waist in ((384, 0.05, 1.7, 4.0), (768, 0.08, 2.3, 6.0), (384, 0.03, 1.2, 3.0)):
        g = wl.Grid(n, n, 0.25, 0.25)
        width = max(8, n // 16)

        def med(s, g=g, eps=eps, period=period, width=width):
            return wl.sine_product_n2(g, eps, period, (s + 0.5) * dz, width, 0.2)

        beams.append(wl.Beam(g, wl.gaussian_beam(g, waist)[None], med, lambda s: True, width, 0.2))
    W = wl.Workload("uneven_384_768", wl.K0, 1.0, dz, 1, 12, 1, "fp32", 20, 1e-7, beams)
    T = oracle_table("uneven_batch")
    pr = gpu_propagator(W, "uneven_batch", P.PROP_FP32)
    got = gpu_run(pr, W, 1)
    for i, b in enumerate(W.beams):
        med = ops.Medium(b.medium(0), b.grid.dx, b.grid.dy, W.k0, W.n0, 1)
        out = T.r0 * b.w0
        worst = 0.0
        for k, (p, r) in enumerate(zip(T.poles, T.residues)):
            x = med.freespace_solve(b.w0, p) + pr.get_correction(i, k)
            worst = max(worst, np.linalg.norm(b.w0 - med.apply_shifted(x, p)) / np.linalg.norm(b.w0))
            out = out + r * x
        assert worst < 1e-4, (i, worst)
        assert rel_l2(got[i], out) < 1e-6, i


def test_mean_and_freespace_preconditioners_agree(P):
    """The preconditioner changes only how GMRES gets there (Sec. 4.2): the
    default constant-index preconditioner and the n = n0 free-space one give the
    same FP64 field, and the oracle's, on the 64^2 workload with its border."""
    from paper_2410_17446_gb300 import workloads as wl
    W = wl.plain_scalar_64(4)
    fields, its = {}, {}
    for pc in (P.PROP_PRECOND_MEAN, P.PROP_PRECOND_FREESPACE):
        pr = gpu_propagator(W, "plain_scalar_64", P.PROP_FP64, tol=1e-12, precond=pc)
        fields[pc] = gpu_run(pr, W, 4)[0]
        its[pc] = int(pr.stats().total_iters)
    ref = oracle_run(W, oracle_table("plain_scalar_64"), 4)
    assert rel_l2(fields[P.PROP_PRECOND_MEAN], ref) < FP64_TOL
    assert rel_l2(fields[P.PROP_PRECOND_FREESPACE], ref) < FP64_TOL
    print("Arnoldi steps: mean", its[P.PROP_PRECOND_MEAN], "free space", its[P.PROP_PRECOND_FREESPACE])
    assert its[P.PROP_PRECOND_MEAN] < its[P.PROP_PRECOND_FREESPACE]


def test_repeat_runs_agree_to_rounding(P):
    """The FP64 Gram sums and norms are accumulated with atomics into 16 stripes,
    so the summation order, and with it the last bits, may change from run to
    run: two runs of the same 3 FP32 steps agree far inside the FP32 bar."""
    from paper_2410_17446_gb300 import workloads as wl
    W = wl.batched_scalar_1024(3, n=256)
    a = gpu_run(gpu_propagator(W, "batched_scalar_1024", P.PROP_FP32), W, 3)[0]
    b = gpu_run(gpu_propagator(W, "batched_scalar_1024", P.PROP_FP32), W, 3)[0]
    assert rel_l2(a, b) < 1e-6
