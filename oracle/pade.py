"""Padé approximants of the exponential propagator, shifted and rotated (Sec. 3.1).

Oracle (test infrastructure).  Sec. 3.1 compares AAA-Lawson with the older
construction: a (10,10) Padé approximant of exp(iK sqrt(1 + zeta)), built from
the Taylor coefficients of the exponential operator as functions of K, shifted
to the branch point zeta = -1 and rotated about it by pi/8.

Reading (the paper gives no formula): write 1 + zeta = e^{i alpha} (1 + Y), i.e.

    Y = (1 + zeta) e^{-i alpha} - 1,     alpha = pi/8,

so that sqrt(1 + zeta) = e^{i alpha/2} sqrt(1 + Y) with the principal root in Y.
On the real zeta axis this is the decaying branch of Eq. exp_prop_planewave
(arg(1 + zeta) in {0, pi} maps to arg(1 + Y) in {-alpha, pi - alpha}), and the
branch cut, the ray arg(1 + zeta) = alpha - pi, is turned by alpha about
zeta = -1 into the lower half-plane.  The target is

    h(Y) = exp(iK (-1 + e^{i alpha/2} sqrt(1 + Y)))  =  g(zeta),

whose Taylor series about Y = 0 (zeta_0 = -1 + e^{i alpha}: the point zeta = 0
turned by alpha about -1) is formed term by term: the binomial series of
sqrt(1 + Y), then the exponential of a power series by the recurrence
n f_n = sum_{k=1..n} k a_k f_{n-k} (from f' = a' f).  The [N/N] Padé
approximant P/Q (Q(0) = 1) matches that series through Y^{2N}; its partial
fractions in Y become partial fractions in zeta because Y is linear in zeta:
Y - y_k = e^{-i alpha} (zeta - p_k) with p_k = -1 + (1 + y_k) e^{i alpha}, so
r_k = e^{i alpha} a_k for the Y-residue a_k, and r0 = P_N / Q_N.  With
alpha = 0 this is the plain Padé approximant about zeta = 0.

The series and the Padé linear system are ill-conditioned in double precision
for large K (the paper says (10,10) sits at the practical limit of its
computation), so they are evaluated in multiple precision (mpmath, 60 digits)
and rounded once to complex128 at the end.
"""
from __future__ import annotations

import math

import numpy as np

from .aaa_lawson import PoleTable

DPS = 60


def _mp():
    import mpmath
    mpmath.mp.dps = DPS
    return mpmath


def sqrt1p_series(n: int):
    """Coefficients of (1 + Y)^{1/2} = sum binom(1/2, m) Y^m, m < n (mpmath)."""
    mp = _mp()
    c = [mp.mpf(1)]
    for m in range(1, n):
        c.append(c[-1] * (mp.mpf(1) / 2 - (m - 1)) / m)
    return c


def exp_series(a, n: int):
    """Coefficients of exp(A(Y)) for A = sum a_m Y^m, m < n: f_0 = e^{a_0},
    m f_m = sum_{k=1..m} k a_k f_{m-k}."""
    mp = _mp()
    f = [mp.exp(a[0])]
    for m in range(1, n):
        s = mp.mpc(0)
        for k in range(1, m + 1):
            s += k * a[k] * f[m - k]
        f.append(s / m)
    return f


def taylor(K: float, alpha: float, n: int):
    """First n Taylor coefficients of h(Y) = exp(iK(-1 + e^{i alpha/2} sqrt(1+Y))) about Y = 0."""
    mp = _mp()
    s = sqrt1p_series(n)
    rot = mp.expjpi(mp.mpf(alpha) / (2 * mp.pi)) if alpha else mp.mpc(1)
    iK = mp.mpc(0, K)
    a = [iK * rot * s[m] for m in range(n)]
    a[0] -= iK
    return exp_series(a, n)


def pade(c, L: int, M: int):
    """[L/M] Padé coefficients (p[0..L], q[0..M], q[0] = 1) of the series c:
    sum_j q_j c_{L+i-j} = 0 for i = 1..M, then p_i = sum_{j<=min(i,M)} q_j c_{i-j}."""
    mp = _mp()
    A = mp.matrix(M, M)
    b = mp.matrix(M, 1)
    for i in range(1, M + 1):
        for j in range(1, M + 1):
            idx = L + i - j
            A[i - 1, j - 1] = c[idx] if idx >= 0 else 0
        b[i - 1] = -c[L + i]
    qv = mp.lu_solve(A, b)
    q = [mp.mpc(1)] + [qv[j] for j in range(M)]
    p = []
    for i in range(L + 1):
        s = mp.mpc(0)
        for j in range(0, min(i, M) + 1):
            s += q[j] * c[i - j]
        p.append(s)
    return p, q


def rotated_pade_table(K: float, N: int = 10, alpha: float = math.pi / 8) -> PoleTable:
    """Partial fractions in zeta of the [N/N] Padé approximant of h about Y = 0."""
    mp = _mp()
    c = taylor(K, alpha, 2 * N + 1)
    p, q = pade(c, N, N)
    # roots of Q (highest degree first for polyroots)
    ys = mp.polyroots(list(reversed(q)), maxsteps=400, extraprec=4 * DPS)
    dq = [j * q[j] for j in range(1, N + 1)]            # Q'
    rot = mp.expjpi(mp.mpf(alpha) / mp.pi) if alpha else mp.mpc(1)   # e^{i alpha}
    poles, res = [], []
    for y in ys:
        Py = sum(p[i] * y ** i for i in range(N + 1))
        dQy = sum(dq[j] * y ** j for j in range(N))
        a = Py / dQy
        poles.append(complex(-1 + (1 + y) * rot))
        res.append(complex(a * rot))
    r0 = complex(p[N] / q[N])
    order = np.argsort(np.array(poles).real)
    return PoleTable(K, np.array(poles)[order], np.array(res)[order], r0, -4.0, 2.0, (), float("nan"))


def rotated_pade_eval(z: np.ndarray, K: float, N: int = 10, alpha: float = math.pi / 8) -> np.ndarray:
    """P(Y)/Q(Y) at Y = (1+z) e^{-i alpha} - 1 from the Padé coefficients directly
    (the quotient form, to check the partial fractions against)."""
    c = taylor(K, alpha, 2 * N + 1)
    p, q = pade(c, N, N)
    pc = np.array([complex(x) for x in p])
    qc = np.array([complex(x) for x in q])
    Y = (1 + np.asarray(z, np.complex128)) * np.exp(-1j * alpha) - 1
    return np.polyval(pc[::-1], Y) / np.polyval(qc[::-1], Y)
