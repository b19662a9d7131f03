"""Pins of the shifted and rotated Padé oracle (Sec. 3.1) to facts fixed outside it."""
import json
import math
import os

import numpy as np
import pytest

pytest.importorskip("mpmath")

from oracle import aaa_lawson as al   # noqa: E402
from oracle import pade               # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "paper_numbers.json")))
ALPHA = math.pi / 8


def test_pade_of_exp_is_the_textbook_approximant():
    """[2/2] Padé of e^Y (series 1/n!) is (1 + Y/2 + Y^2/12)/(1 - Y/2 + Y^2/12)."""
    c = [1.0 / math.factorial(n) for n in range(5)]
    p, q = pade.pade(c, 2, 2)
    np.testing.assert_allclose([complex(x) for x in p], [1, 0.5, 1 / 12], atol=1e-40 + 1e-15)
    np.testing.assert_allclose([complex(x) for x in q], [1, -0.5, 1 / 12], atol=1e-15)


def test_taylor_series_sums_to_the_rotated_target():
    """The series of h(Y) = exp(iK(-1 + e^{i a/2} sqrt(1+Y))) summed at |Y| = 0.3
    equals h computed directly, and h equals g(zeta) = exp(iK(-1+sqrt(1+zeta)))
    on the real zeta axis (the rotation keeps the decaying branch there)."""
    K = 2.7
    c = np.array([complex(x) for x in pade.taylor(K, ALPHA, 80)])
    for Y in (0.3, -0.3j, 0.2 + 0.2j):
        direct = np.exp(1j * K * (-1 + np.exp(0.5j * ALPHA) * np.sqrt(1 + Y)))
        assert abs(np.polyval(c[::-1], Y) - direct) < 1e-13
    z = np.array([-3.0, -1.5, -0.5, 0.0, 1.5])
    Y = (1 + z) * np.exp(-1j * ALPHA) - 1
    h = np.exp(1j * K * (-1 + np.exp(0.5j * ALPHA) * np.sqrt(1 + Y)))
    np.testing.assert_allclose(h, al.target(z, K), rtol=1e-13, atol=1e-14)


def test_partial_fractions_equal_the_quotient():
    """Eq. pf_expan_eq for the Padé quotient: r0 + sum r_k/(zeta - p_k) = P(Y)/Q(Y)."""
    K = math.pi
    T = pade.rotated_pade_table(K, 10, ALPHA)
    z = np.concatenate([np.linspace(-4, 2, 101), np.linspace(-4, 2, 23) + 0.3j])
    q = pade.rotated_pade_eval(z, K, 10, ALPHA)
    assert np.max(np.abs(T(z) - q) / np.abs(q)) < 1e-9
    assert T.npoles == 10
    # the rotation puts the poles below the real axis, along the turned branch cut
    assert np.all(T.poles.imag < 0)


def test_plain_pade_matches_the_taylor_series_to_order_2N():
    """alpha = 0: the [N/N] approximant agrees with g to O(zeta^{2N+1}) at zeta = 0,
    so halving zeta cuts the error by about 2^{2N+1}."""
    K = math.pi
    T = pade.rotated_pade_table(K, 4, 0.0)
    e1 = abs(T(np.array([0.2]))[0] - al.target(np.array([0.2]), K)[0])
    e2 = abs(T(np.array([0.1]))[0] - al.target(np.array([0.1]), K)[0])
    assert 2 ** 7 < e1 / e2 < 2 ** 11


def test_paper_statements_at_half_wavelength():
    """Sec. 3.1, dz = 0.5 lambda, n0 = 1.0003: the (10,10) Padé approximant is
    more accurate than the (25,25) AAA-Lawson fit (mean error ~2.3e-11) around
    zeta = 0, substantially worse elsewhere, and degrades near zeta = -1."""
    c = GOLD["aaa_lawson_dz_half"]
    K = 2 * math.pi * c["n0"] * c["dz"]
    T = pade.rotated_pade_table(K, 10, ALPHA)
    z = np.linspace(-4, 2, 2001)
    err = np.abs(T(z) - al.target(z, K))
    at = lambda x: err[np.argmin(np.abs(z - x))]
    assert at(0.0) < c["mean_error"]
    assert at(-0.95) > 1e4 * c["mean_error"]
    assert at(2.0) > c["mean_error"]
    assert err.mean() > 100 * c["mean_error"]


def test_paper_statements_at_five_wavelengths():
    """Sec. 3.1, dz = 5 lambda: across the propagating range the Padé errors are
    5 to 8 orders of magnitude above the (28,28) AAA-Lawson mean error (~1.19e-8);
    checked on the median over (-1, 0] with one decade of slack each side."""
    c = GOLD["aaa_lawson_dz_five"]
    K = 2 * math.pi * c["n0"] * c["dz"]
    T = pade.rotated_pade_table(K, 10, ALPHA)
    z = np.linspace(-1, 0, 1001)[1:]
    ratio = np.median(np.abs(T(z) - al.target(z, K))) / c["mean_error"]
    assert 1e4 <= ratio <= 1e9, ratio
