"""AAA-Lawson rational approximation of the exponential propagator (Sec. 3.1).

Oracle (test infrastructure).  The function approximated is the one whose
partial fractions the propagator sums, with the e^{-iK} factor of Eq.
(Wk_define) folded in:

    g(zeta) = exp(i K (-1 + sqrt(1 + zeta))),   K = k0 n0 dz   (Eq. expop_prop),

on the branch with Im sqrt >= 0, so evanescent waves (zeta < -1) decay (Eq.
exp_prop_planewave).  For real or upper-half-plane zeta the principal square
root is that branch.

The algorithm is the one the paper adopts from Nakatsukasa & Trefethen (2020):
  1. AAA: greedy choice of support points for a barycentric form
     r = sum_j w_j f_j/(z - z_j) / sum_j w_j/(z - z_j); each step adds the
     sample of largest error and takes w as the smallest right singular vector
     of the Loewner matrix.  P+1 support points give type (P, P).
  2. Lawson: with the support points fixed, separate numerator and
     denominator coefficients alpha, beta are refitted by iteratively
     reweighted least squares on the linearised error f*D - N, each weight
     multiplied by the current error modulus and renormalised, moving the
     approximant toward minimax.  The iterate of smallest maximum error is kept.
  3. Partial fractions (Eq. pf_expan_eq): the poles are the finite
     generalised eigenvalues of the arrowhead pencil of the denominator, each
     residue is N(p)/D'(p), and the constant is r(inf) = sum alpha/sum beta.
In the partial-fraction form r(zeta) = r0 + sum_k r_k/(zeta - p_k):
p_k = b_kN, r_k = e^{-iK} a_kN and r0 = e^{-iK} alpha_NN/beta_NN.
"""
from __future__ import annotations

import dataclasses
import json
import math
from typing import Optional, Sequence

import numpy as np
import scipy.linalg


def target(z: np.ndarray, K: float) -> np.ndarray:
    """g(zeta) = exp(iK(-1 + sqrt(1+zeta))) on the decaying branch."""
    z = np.asarray(z, dtype=np.complex128)
    return np.exp(1j * K * (np.sqrt(1.0 + z) - 1.0))


def sample_set(lo: float, hi: float, m_uniform: int = 2000, cluster_min: Optional[float] = None,
               m_cluster: int = 200, im_shifts: Sequence[float] = ()) -> np.ndarray:
    """Fit samples: a uniform grid on [lo, hi]; optionally geometric clustering
    toward the branch point zeta = -1 down to ``cluster_min``; and copies shifted
    by +i*s for each s in ``im_shifts`` (the strip an absorbing Im n^2 moves the
    spectrum into).  Clustering buys accuracy next to the branch point at the
    price of poles closer to the real axis (slower shifted solves)."""
    u = np.linspace(lo, hi, m_uniform)
    z = u
    if cluster_min is not None:
        d = np.geomspace(cluster_min, 0.5, m_cluster)
        z = np.concatenate([u, -1.0 - d, -1.0 + d])
    z = np.unique(z)
    z = z[(z >= lo) & (z <= hi)].astype(np.complex128)
    parts = [z] + [z + 1j * s for s in im_shifts if s > 0]
    return np.concatenate(parts)


def aaa(Z: np.ndarray, F: np.ndarray, n_support: int):
    """AAA greedy barycentric fit with ``n_support`` support points.

    Returns (support indices into Z, barycentric weights w).
    """
    Z = np.asarray(Z, np.complex128)
    F = np.asarray(F, np.complex128)
    free = np.ones(Z.size, dtype=bool)
    R = np.full(Z.size, F.mean())
    idx = []
    w = None
    for _ in range(n_support):
        j = int(np.argmax(np.where(free, np.abs(F - R), -1.0)))
        idx.append(j)
        free[j] = False
        zs, fs = Z[idx], F[idx]
        C = 1.0 / (Z[free, None] - zs[None, :])          # Cauchy matrix
        L = (F[free, None] - fs[None, :]) * C            # Loewner matrix
        _, _, Vh = np.linalg.svd(L, full_matrices=False)
        w = Vh[-1].conj()                                 # smallest right singular vector
        R = F.copy()
        R[free] = (C @ (w * fs)) / (C @ w)
    return np.array(idx), w


def bary_eval(z: np.ndarray, zs: np.ndarray, alpha: np.ndarray, beta: np.ndarray) -> np.ndarray:
    """N(z)/D(z) with N = sum alpha_j/(z-z_j), D = sum beta_j/(z-z_j); at z = z_j the limit alpha_j/beta_j."""
    z = np.asarray(z, np.complex128)
    out = np.empty(z.shape, np.complex128)
    flat = z.ravel()
    diff = flat[:, None] - zs[None, :]
    hit = diff == 0
    with np.errstate(divide="ignore", invalid="ignore"):
        C = 1.0 / diff
        val = (C @ alpha) / (C @ beta)
    rows, cols = np.nonzero(hit)
    val[rows] = alpha[cols] / beta[cols]
    out.ravel()[:] = val
    return out


def lawson(Z: np.ndarray, F: np.ndarray, idx: np.ndarray, w: np.ndarray, iters: int = 60):
    """Lawson IRLS refinement of the barycentric coefficients (support fixed).

    At the support points the linearised residual is written in its
    multiplied-through limit f_j beta_j - alpha_j, scaled by the distance to the
    nearest other sample so that it weighs like its neighbours.
    Returns (alpha, beta, max error over all samples) of the best iterate.
    """
    Z = np.asarray(Z, np.complex128)
    F = np.asarray(F, np.complex128)
    zs, fs = Z[idx], F[idx]
    m = zs.size
    free = np.ones(Z.size, dtype=bool)
    free[idx] = False
    Zf, Ff = Z[free], F[free]
    C = 1.0 / (Zf[:, None] - zs[None, :])
    h = np.array([np.partition(np.abs(Z - z), 1)[1] for z in zs])

    def errors(a, b):
        return np.abs(Ff - (C @ a) / (C @ b)), np.abs(fs - a / b)

    alpha, beta = w * fs, w.copy()           # the AAA iterate, written non-interpolatorily
    ef, es = errors(alpha, beta)
    best = (max(ef.max(), es.max()), alpha.copy(), beta.copy())
    wf = np.ones(Zf.size)
    ws = np.ones(m)
    for _ in range(iters):
        wf = wf * ef
        ws = ws * es
        tot = wf.sum() + ws.sum()
        if not np.isfinite(tot) or tot == 0.0:
            break
        wf, ws = wf / tot, ws / tot
        sf = np.sqrt(wf)[:, None]
        A_free = np.hstack([sf * (Ff[:, None] * C), -sf * C])
        A_sup = np.hstack([np.diag(np.sqrt(ws) * fs / h), -np.diag(np.sqrt(ws) / h)])
        _, _, Vh = np.linalg.svd(np.vstack([A_free, A_sup]), full_matrices=False)
        v = Vh[-1].conj()
        beta, alpha = v[:m], v[m:]
        ef, es = errors(alpha, beta)
        e = max(ef.max(), es.max())
        if np.isfinite(e) and e < best[0]:
            best = (e, alpha.copy(), beta.copy())
    return best[1], best[2], best[0]


def partial_fractions(zs: np.ndarray, alpha: np.ndarray, beta: np.ndarray):
    """Poles, residues and constant of N/D (Eq. pf_expan_eq).

    Poles: finite eigenvalues of the pencil (E, B) with
    E = [[0, beta^T], [1, diag(zs)]], B = diag(0, 1, ..., 1).
    Residues: N(p)/D'(p) with D'(z) = -sum beta_j/(z - z_j)^2.
    """
    m = zs.size
    E = np.zeros((m + 1, m + 1), np.complex128)
    E[0, 1:] = beta
    E[1:, 0] = 1.0
    E[1:, 1:] = np.diag(zs)
    B = np.eye(m + 1, dtype=np.complex128)
    B[0, 0] = 0.0
    ev = scipy.linalg.eigvals(E, B)
    p = ev[np.isfinite(ev)]
    p = p[np.abs(p) < 1e12]
    Cp = 1.0 / (p[:, None] - zs[None, :])
    res = (Cp @ alpha) / (-(Cp ** 2) @ beta)
    r0 = alpha.sum() / beta.sum()
    order = np.argsort(p.real)
    return p[order], res[order], r0


def pf_eval(z, poles, residues, r0) -> np.ndarray:
    z = np.asarray(z, np.complex128)
    return r0 + (residues[None, :] / (z.ravel()[:, None] - poles[None, :])).sum(axis=1).reshape(z.shape)


@dataclasses.dataclass
class PoleTable:
    """r(zeta) = r0 + sum_k residues[k]/(zeta - poles[k]) ~ g(zeta)."""
    K: float
    poles: np.ndarray
    residues: np.ndarray
    r0: complex
    lo: float
    hi: float
    im_shifts: tuple
    fit_max_err: float
    support: Optional[np.ndarray] = None

    @property
    def npoles(self) -> int:
        return int(self.poles.size)

    def __call__(self, z):
        return pf_eval(z, self.poles, self.residues, self.r0)

    def to_json(self) -> dict:
        return {
            "K": self.K, "npoles": self.npoles,
            "poles": [[float(p.real), float(p.imag)] for p in self.poles],
            "residues": [[float(r.real), float(r.imag)] for r in self.residues],
            "r0": [float(np.real(self.r0)), float(np.imag(self.r0))],
            "domain": [self.lo, self.hi], "im_shifts": list(self.im_shifts),
            "fit_max_err": self.fit_max_err,
        }

    @staticmethod
    def from_json(d: dict) -> "PoleTable":
        return PoleTable(
            K=d["K"], poles=np.array([complex(a, b) for a, b in d["poles"]]),
            residues=np.array([complex(a, b) for a, b in d["residues"]]),
            r0=complex(*d["r0"]), lo=d["domain"][0], hi=d["domain"][1],
            im_shifts=tuple(d.get("im_shifts", ())), fit_max_err=d.get("fit_max_err", float("nan")))


def fit(K: float, npoles: int, lo: float, hi: float = 2.0, im_shifts: Sequence[float] = (),
        m_uniform: int = 2000, cluster_min: Optional[float] = None, lawson_iters: int = 60,
        Z: Optional[np.ndarray] = None) -> PoleTable:
    """AAA-Lawson fit of g on [lo, hi] (plus the Im strip), as partial fractions."""
    if Z is None:
        Z = sample_set(lo, hi, m_uniform, cluster_min, 200, im_shifts)
    F = target(Z, K)
    idx, w = aaa(Z, F, npoles + 1)
    alpha, beta, err = lawson(Z, F, idx, w, lawson_iters)
    p, res, r0 = partial_fractions(Z[idx], alpha, beta)
    return PoleTable(K, p, res, r0, lo, hi, tuple(im_shifts), float(err), Z[idx])


def fit_domain(nx: int, ny: int, dx: float, dy: float, k0n0: float, delta_min_re: float) -> float:
    """Lower end of the fit range: min(-4, zeta_min + min Re delta - 0.5), where
    zeta_min = -(kx_max^2 + ky_max^2)/(k0 n0)^2 is the grid's most evanescent
    free-space eigenvalue (Sec. 3: Re zeta = -(kx^2+ky^2)/(k0 n0)^2)."""
    kx_max = math.pi / dx
    ky_max = math.pi / dy
    zmin = -(kx_max ** 2 + ky_max ** 2) / k0n0 ** 2
    return min(-4.0, zmin + min(0.0, delta_min_re) - 0.5)
