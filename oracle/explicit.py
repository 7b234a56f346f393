"""Explicit least-squares LRE (n <= 5) -- test infrastructure only.

Follows Sec. II of arXiv:1602.08604 literally:
  Eq. (5)  Omega_i = 2^{-n/2} (x)_k sigma_{i_k},  i = sum_k i_k 4^{n-k}
  Eq. (2)  gamma_i^(j) = Tr(|Psi><Psi|^(j) Omega_i)   (rows of X)
  Eq. (3)  theta_LS = (X^T X)^{-1} sum_j p_j Gamma^(j)   (Cholesky solve)
  Eq. (4)  mu = sum_i theta_i Omega_i
The measurement set is the 6^n Pauli eigenprojectors (Sec. III), ordered by
basis b = sum_q a_q 3^{n-q} (a in X,Y,Z) and outcome o = sum_q o_q 2^{n-q}
(o_q = 0 for the +1 eigenvector).  p_j is the frequency of outcome o within
its basis (counts / shots of that basis).
"""
import numpy as np

SIGMA = np.array([
    [[1, 0], [0, 1]],
    [[0, 1], [1, 0]],
    [[0, -1j], [1j, 0]],
    [[1, 0], [0, -1]],
], dtype=np.complex128)

_S = 1.0 / np.sqrt(2.0)
# single-qubit eigenvectors: EIG[a][o], o = 0 is the +1 eigenvalue of sigma_{a+1}
EIG = np.array([
    [[_S, _S], [_S, -_S]],
    [[_S, 1j * _S], [_S, -1j * _S]],
    [[1, 0], [0, 1]],
], dtype=np.complex128)


def omega_basis(n):
    """All 4^n matrices Omega_i of Eq. (5), shape (4^n, d, d)."""
    mats = [np.array([[1.0 + 0j]])]
    for _ in range(n):
        mats = [np.kron(m, s) for m in mats for s in SIGMA]
    return np.array(mats) * 2.0 ** (-n / 2.0)


def measurement_vectors(n):
    """|Psi_j> for j = (b, o), shape (3^n, 2^n, d)."""
    vecs = [[np.array([1.0 + 0j])]]  # vecs[b][o]
    for _ in range(n):
        vecs = [[np.kron(v, EIG[a][o]) for v in row for o in range(2)]
                for row in vecs for a in range(3)]
        # reorder outcomes so the new qubit is the least significant bit
    B = 3 ** n
    d = 2 ** n
    out = np.array(vecs).reshape(B, d, d)
    return out


def design_matrix(n):
    """X with rows Gamma^(j)^T, j = b*2^n + o; shape (6^n, 4^n), real."""
    om = omega_basis(n)
    psi = measurement_vectors(n).reshape(-1, 2 ** n)
    X = np.einsum("jk,ikl,jl->ji", psi.conj(), om, psi, optimize=True)
    if np.max(np.abs(X.imag)) > 1e-12:
        raise AssertionError("design matrix is not real")
    return X.real.copy()


def ls_theta(counts, shots, n, X=None):
    """theta_LS of Eq. (3) in the orthonormal Omega scale (4^n,).

    counts: (3^n, 2^n) integers; shots: scalar or (3^n,) per-basis totals.
    """
    if X is None:
        X = design_matrix(n)
    c = np.asarray(counts, dtype=np.float64)
    N = np.broadcast_to(np.asarray(shots, dtype=np.float64), (c.shape[0],))
    p = (c / N[:, None]).reshape(-1)
    XtX = X.T @ X
    rhs = X.T @ p
    L = np.linalg.cholesky(XtX)
    y = np.linalg.solve(L, rhs)
    return np.linalg.solve(L.T, y)


def expectations_from_theta(theta, n):
    """Pauli expectation estimates t_i = 2^{n/2} theta_i (t_0 = 1)."""
    return np.asarray(theta) * 2.0 ** (n / 2.0)


def mu_from_theta(theta, n):
    """mu = sum_i theta_i Omega_i, Eq. (4)."""
    om = omega_basis(n)
    return np.einsum("i,ikl->kl", np.asarray(theta, dtype=np.complex128), om)
