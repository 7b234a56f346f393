"""The 4^n-operator variant of the LRE (Sec. VI) -- test infrastructure only.

Sec. VI remarks that reducing the measurement operators from the 6^n Pauli
eigenprojectors to 4^n lowers the cost of step (i) from O(12^n) to O(8^n).
The paper names no operator set.  Reading: the minimal informationally
complete subset of the Pauli eigenprojectors, per qubit
    E_0 = |0><0|,  E_1 = |1><1|,  E_2 = |+><+|,  E_3 = |+i><+i|
(the +1 eigenvector of X and of Y, both eigenvectors of Z); each n-qubit
operator E_j = (x)_q E_{j_q} (j = sum j_q 4^{n-q}, qubit 1 first) still has
2^n nonzeros in the basis of Eq. (5), so 4^n operators x 2^n nonzeros per
operator gives the paper's O(8^n).  The frequency of E_j is read from the
Pauli counts: qubit q in E_0/E_1 is the Z basis with outcome 0/1, E_2 the
X basis with outcome 0, E_3 the Y basis with outcome 0, so
    p_j = c_b(o) / N   with   b, o  fixed by j  (uniform shots N).

`ls_theta` is Eq. (3) literally with these 4^n rows: build X explicitly from
the projectors and Omega_i (Eq. 5) and solve the normal equations (n <= 5).
X^T X = G^{(x)n} is no longer diagonal (G below, a pinned fact); X is square
and invertible, so the LS estimate is the exact solution of X theta = p.
`kron_theta` applies the same inverse qubit by qubit (X = X_1^{(x)n}), for
the sizes the explicit solve cannot reach; it is pinned against ls_theta.
"""
import numpy as np

from . import explicit

_S = 1.0 / np.sqrt(2.0)
# per-qubit projector vectors: |0>, |1>, |+>, |+i>
VEC = np.array([[1, 0], [0, 1], [_S, _S], [_S, 1j * _S]], dtype=np.complex128)
# the (axis, outcome) of the Pauli count that estimates each projector's
# probability: axis 0 = X, 1 = Y, 2 = Z; outcome 0 = the +1 eigenvector
SOURCE = [(2, 0), (2, 1), (0, 0), (1, 0)]


def operator_vectors(n):
    """|psi_j> for j = sum j_q 4^{n-q}, shape (4^n, 2^n)."""
    vecs = [np.array([1.0 + 0j])]
    for _ in range(n):
        vecs = [np.kron(v, w) for v in vecs for w in VEC]
    return np.array(vecs)


def design_matrix(n):
    """X_{j,i} = Tr(|psi_j><psi_j| Omega_i) (Eq. 2 with the 4^n operators)."""
    om = explicit.omega_basis(n)
    psi = operator_vectors(n)
    X = np.einsum("jk,ikl,jl->ji", psi.conj(), om, psi, optimize=True)
    if np.max(np.abs(X.imag)) > 1e-12:
        raise AssertionError("design matrix is not real")
    return X.real.copy()


def source_index(j, n):
    """(basis b, outcome o) of the Pauli count that estimates operator j."""
    b = o = 0
    for q in range(n):
        jq = (j >> (2 * (n - 1 - q))) & 3
        a, oq = SOURCE[jq]
        b = 3 * b + a
        o = 2 * o + oq
    return b, o


def frequencies(counts, shots, n):
    """p_j for the 4^n operators from Pauli counts [3^n][2^n], uniform shots."""
    c = np.asarray(counts)
    p = np.empty(4 ** n, np.float64)
    for j in range(4 ** n):
        b, o = source_index(j, n)
        p[j] = c[b, o] / float(shots)
    return p


def ls_theta(counts, shots, n):
    """theta of Eq. (3) by the normal equations (Cholesky), n <= 5."""
    X = design_matrix(n)
    p = frequencies(counts, shots, n)
    A = X.T @ X
    L = np.linalg.cholesky(A)
    y = np.linalg.solve(L, X.T @ p)
    return np.linalg.solve(L.T, y)


def kron_theta(counts, shots, n):
    """The same estimate as t_P = 2^{n/2} theta_P, with X^{-1} = (X_1^{-1})^{(x)n}
    applied one qubit at a time to the frequency tensor."""
    X1 = design_matrix(1)
    inv = np.linalg.inv(X1) * np.sqrt(2.0)          # t = 2^{1/2} theta per qubit
    p = frequencies(counts, shots, n).reshape((4,) * n) if n > 0 else np.ones(1)
    for q in range(n):
        p = np.moveaxis(np.tensordot(inv, p, axes=([1], [q])), 0, q)
    return p.reshape(-1)


# The per-qubit inverse in count units: with uniform shots N the frequency
# of E_0, E_1 (Z basis) and E_2 (X basis), E_3 (Y basis) give, for one qubit,
#   <I> = p_0 + p_1,  <X> = 2 p_2 - p_0 - p_1,  <Y> = 2 p_3 - p_0 - p_1,  <Z> = p_0 - p_1
# (rows: I, X, Y, Z; columns: E_0..E_3), all integer coefficients.
R_INT = np.array([[1, 1, 0, 0],
                  [-1, -1, 2, 0],
                  [-1, -1, 0, 2],
                  [1, -1, 0, 0]], dtype=np.int64)


def selected_counts(counts, n):
    """u_j = c_b(o) for the (basis, outcome) that estimates operator j."""
    c = np.asarray(counts)
    return np.array([c[source_index(j, n)] for j in range(4 ** n)], dtype=np.int64)


def exact_sums(counts, n):
    """S = R^{(x)n} u in exact int64 (|S| <= N 3^n)."""
    s = selected_counts(counts, n).reshape((4,) * n) if n > 0 else np.ones(1, np.int64)
    for q in range(n):
        s = np.moveaxis(np.tensordot(R_INT, s, axes=([1], [q])), 0, q)
    return s.reshape(-1)


def exact_theta(counts, shots, n):
    """t_P = S_P / N: one correctly rounded division of exact integers."""
    return exact_sums(counts, n).astype(np.float64) / float(shots)
