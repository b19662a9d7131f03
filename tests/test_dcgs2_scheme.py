"""The delayed re-orthogonalisation (DCGS2) recurrences of the GPU Arnoldi step,
restated in FP64 NumPy and checked against what Arnoldi must produce: an
orthonormal basis and the Arnoldi relation B Q_J = Q_{J+1} Hbar_J.

Step j holds final v_0..v_{j-1} and the once-projected candidate u = v_j.  With
w = B u, a = V^H u, b = V^H w, c = <u, u>, d = <u, w>, rho^2 = c - |a|^2:
column j-1 becomes h[:j, j-1] += a, h[j, j-1] = rho; q_j = (u - V a)/rho;
column j's first projection is h[i, j] = (b_i - t_i)/rho (i < j),
h[j, j] = (d - a^H b)/rho^2 - t_j/rho with t = Hbar a over the final columns;
and u_{j+1} = w/rho - sum_{i<j} (b_i/rho) v_i - ((d - a^H b)/rho^2) q_j.
"""
import numpy as np


def dcgs2_arnoldi(B, r0, m, leak=0.0):
    """leak: subtract only (1 - leak) of each first projection (and record the
    column accordingly), a deliberate loss of orthogonality that the delayed
    re-orthogonalisation of the next step must remove exactly."""
    n = r0.size
    V = np.zeros((n, m + 2), complex)
    H = np.zeros((m + 1, m), complex)
    V[:, 0] = r0 / np.linalg.norm(r0)
    for j in range(m + 1):
        u = V[:, j].copy()
        w = B @ u if j < m else np.zeros(n, complex)
        Vj = V[:, :j]
        a, b = Vj.conj().T @ u, Vj.conj().T @ w
        c, d = np.vdot(u, u).real, np.vdot(u, w)
        rho = np.sqrt(c - np.vdot(a, a).real)
        if j >= 1:                                   # column j-1 is final now
            H[:j, j - 1] += a
            H[j, j - 1] = rho
        q = (u - Vj @ a) / rho
        V[:, j] = q
        if j == m:
            break
        t = H[: j + 1, :j] @ a                       # Hbar a over the final columns
        ahb = np.vdot(a, b)
        gam = np.concatenate([b / rho, [(d - ahb) / rho ** 2]]) * (1.0 - leak)
        # column j, first projection: (b_i - t_i)/rho and (d - a^H b)/rho^2 - t_j/rho when leak = 0
        H[: j + 1, j] = gam - t / rho
        V[:, j + 1] = w / rho - V[:, : j + 1] @ gam  # the next candidate, once projected
    return V[:, : m + 1], H


def test_dcgs2_gives_orthonormal_basis_and_arnoldi_relation():
    rng = np.random.default_rng(4)
    n, m = 200, 20
    A = np.eye(n) + 0.3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    A[0, 1] += 5.0                                   # non-normal
    r0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    Q, H = dcgs2_arnoldi(A, r0, m)
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(m + 1)) < 1e-12
    assert np.linalg.norm(A @ Q[:, :m] - Q @ H) < 1e-11 * np.linalg.norm(A)
    assert np.allclose(np.tril(H, -2), 0.0)          # upper Hessenberg


def test_dcgs2_gmres_solution_matches_direct_solve():
    rng = np.random.default_rng(9)
    n, m = 60, 30                                    # m < n: no exact breakdown (rho > 0 throughout)
    A = np.eye(n) + 0.2 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 0j
    Q, H = dcgs2_arnoldi(A, b, m)
    beta = np.linalg.norm(b)
    g = np.zeros(m + 1, complex)
    g[0] = beta
    y = np.linalg.lstsq(H, g, rcond=None)[0]
    x = Q[:, :m] @ y
    assert np.linalg.norm(A @ x - b) < 1e-10 * beta
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-9 * np.linalg.norm(x)


def test_dcgs2_removes_a_large_loss_of_orthogonality():
    """With 1% of every projection left in the candidates the products a are
    large, so the corrections h[:, j-1] += a, rho^2 = c - |a|^2 and t = Hbar a
    must all be right for the basis and the Arnoldi relation to come out exact."""
    rng = np.random.default_rng(6)
    n, m = 150, 16
    A = np.eye(n) + 0.4 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    r0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    Q, H = dcgs2_arnoldi(A, r0, m, leak=1e-2)
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(m + 1)) < 1e-12
    assert np.linalg.norm(A @ Q[:, :m] - Q @ H) < 1e-11 * np.linalg.norm(A)
