"""Step (iii) physical projection -- test infrastructure only.

Sec. II step (iii) of arXiv:1602.08604 pulls mu back to the closest density
matrix with the fast algorithm of Smolin, Gambetta and Smith (PRL 108,
070502, 2012), which the paper cites but does not restate.  That algorithm
(their Sec. "Algorithm"): diagonalise mu = V diag(lambda) V^dag with the
eigenvalues in decreasing order; set a = 0 and i = d; while
lambda_i + a/i < 0, add lambda_i to a, set lambda_i = 0 and decrease i; then
add a/i to lambda_1..lambda_i; return V diag(lambda') V^dag.  The paper's
"closest under the matrix 2-norm" is read as the Frobenius norm, the one
that algorithm minimises.

`simplex_projection` is an independent route to the same spectrum (the
Euclidean projection onto the probability simplex by sorting and a
threshold), used only to cross-check `smolin`.
"""
import numpy as np


def smolin_eigenvalues(lam_desc):
    """Corrected spectrum (decreasing order) by the Smolin et al. loop."""
    lam = np.array(lam_desc, dtype=np.float64, copy=True)
    d = lam.shape[0]
    a = 0.0
    i = d
    while i > 0 and lam[i - 1] + a / i < 0:
        a += lam[i - 1]
        lam[i - 1] = 0.0
        i -= 1
    lam[:i] += a / i
    return lam


def smolin(mu):
    """(rho_hat, eigenvalues of mu decreasing, eigenvalues of rho_hat decreasing)."""
    mu = np.asarray(mu, dtype=np.complex128)
    H = 0.5 * (mu + mu.conj().T)
    w, V = np.linalg.eigh(H)
    order = np.argsort(w)[::-1]
    w = w[order]
    V = V[:, order]
    lam = smolin_eigenvalues(w)
    rho = (V * lam[None, :]) @ V.conj().T
    return rho, w, lam


def simplex_projection(lam):
    """Euclidean projection of a real vector onto {x >= 0, sum x = 1}."""
    v = np.asarray(lam, dtype=np.float64)
    u = np.sort(v)[::-1]
    css = np.cumsum(u)
    k = np.arange(1, len(u) + 1)
    cond = u - (css - 1.0) / k > 0
    r = k[cond][-1]
    tau = (css[r - 1] - 1.0) / r
    return np.maximum(v - tau, 0.0)
