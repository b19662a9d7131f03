"""Pins of the AAA-Lawson oracle (Sec. 3.1) to values fixed outside it."""
import json
import math
import os

import numpy as np
import pytest

from oracle import aaa_lawson as al

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "paper_numbers.json")))
TABLES = os.path.join(os.path.dirname(HERE), "paper_2410_17446_gb300", "tables")


def test_target_closed_forms():
    """g(zeta) = exp(iK(-1+sqrt(1+zeta))) at points where sqrt is known exactly
    (Eq. expop_prop; decaying branch of Eq. exp_prop_planewave)."""
    K = 2.7
    z = np.array([0.0, -1.0, 3.0, -5.0, 8.0])
    want = np.array([1.0, np.exp(-1j * K), np.exp(1j * K), np.exp(-1j * K) * np.exp(-2 * K),
                     np.exp(2j * K)])
    np.testing.assert_allclose(al.target(z, K), want, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("key", ["aaa_lawson_dz_half", "aaa_lawson_dz_five"])
def test_paper_fit_error_level(key):
    """The mean fit error the paper prints for AAA-Lawson on Re zeta in [-4, 2],
    evaluated (as its plots are) on a uniform sampling of the interval; within 10x."""
    c = GOLD[key]
    K = 2 * math.pi * c["n0"] * c["dz"]
    Z = np.linspace(c["lo"], c["hi"], 2000).astype(np.complex128)
    T = al.fit(K, c["npoles"], c["lo"], c["hi"], Z=Z)
    # the paper approximates exp(iK sqrt(1+zeta)); g differs by the unit factor e^{-iK}
    err = np.abs(T(Z.real) * np.exp(1j * K) - np.exp(1j * K * np.sqrt(1 + Z)))
    assert T.npoles == c["npoles"]
    assert c["mean_error"] / 10 <= err.mean() <= c["mean_error"] * 10, err.mean()


def test_aaa_recovers_a_rational_function():
    """A type (3,3) rational function is reproduced exactly by 4 support points:
    poles, residues and constant come back (textbook special case of AAA)."""
    q = np.array([-1.3 - 0.4j, 0.2 - 1.1j, 1.7 - 0.25j])
    a = np.array([0.7 + 0.2j, -1.1 + 0.5j, 0.3 - 0.9j])
    c0 = 0.4 - 0.3j
    f = lambda z: c0 + (a[None, :] / (z[:, None] - q[None, :])).sum(1)
    Z = np.linspace(-3, 3, 400).astype(np.complex128)
    idx, w = al.aaa(Z, f(Z), 4)
    p, r, r0 = al.partial_fractions(Z[idx], w * f(Z)[idx], w)
    order = np.argsort(q.real)
    np.testing.assert_allclose(p, q[order], atol=1e-10)
    np.testing.assert_allclose(r, a[order], atol=1e-10)
    assert abs(r0 - c0) < 1e-10


def test_partial_fractions_equal_barycentric():
    """Eq. (pf_expan_eq): the partial-fraction form equals the barycentric
    quotient it was derived from, away from the poles."""
    T = al.fit(math.pi, 12, -8.5, 2.0, im_shifts=(0.2,))
    rng = np.random.default_rng(3)
    z = rng.uniform(-8.5, 2, 500) + 1j * rng.uniform(0, 0.3, 500)
    # rebuild alpha, beta from the same fit
    Zs = al.sample_set(-8.5, 2.0, im_shifts=(0.2,))
    F = al.target(Zs, math.pi)
    idx, w = al.aaa(Zs, F, 13)
    alpha, beta, _ = al.lawson(Zs, F, idx, w)
    p, res, r0 = al.partial_fractions(Zs[idx], alpha, beta)
    bary = al.bary_eval(z, Zs[idx], alpha, beta)
    pf = al.pf_eval(z, p, res, r0)
    assert np.max(np.abs(bary - pf)) / np.max(np.abs(bary)) < 1e-10
    np.testing.assert_allclose(p, T.poles, atol=1e-12)


@pytest.mark.parametrize("name", ["plain_scalar_64", "homogeneous_aperture_1024", "batched_scalar_1024",
                                  "vector_random_512", "uneven_batch"])
def test_committed_tables(name):
    """Each committed pole table: no pole inside the region that holds the
    operator's spectrum (Re zeta in the fit range, 0 <= Im zeta <= the
    absorbing strip), so every shifted system of Eq. (W_k_def) is nonsingular;
    and the fit is accurate on its real domain away from the branch point."""
    d = json.load(open(os.path.join(TABLES, name + ".json")))
    T = al.PoleTable.from_json(d)
    top = max(T.im_shifts) if T.im_shifts else 0.0
    dx = np.maximum(0.0, np.maximum(T.lo - T.poles.real, T.poles.real - T.hi))
    dy = np.maximum(0.0, np.maximum(-T.poles.imag, T.poles.imag - top))
    assert np.all(np.hypot(dx, dy) > 5e-4), np.hypot(dx, dy).min()
    z = np.linspace(T.lo, T.hi, 20001)
    z = z[np.abs(z + 1) > 0.05]
    err = np.abs(T(z) - al.target(z, T.K))
    assert err.max() < 1e-3, err.max()
    assert T.npoles == d["npoles"]


def test_committed_table_is_reproducible():
    """The table generator is deterministic: refitting gives the stored poles."""
    from oracle import make_tables
    from paper_2410_17446_gb300 import workloads as wl
    d = json.load(open(os.path.join(TABLES, "plain_scalar_64.json")))
    T = make_tables.table_for(wl.plain_scalar_64(1))
    np.testing.assert_allclose(T.poles, al.PoleTable.from_json(d).poles, rtol=1e-9, atol=1e-12)
