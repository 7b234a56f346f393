"""Seeded quantum states and their Born probabilities under Pauli bases.

Only the forward model lives here (state -> Pauli expectations -> outcome
probabilities of each of the 3^n product bases).  Index conventions are the
ones stated in synth/__init__.py.
"""
import numpy as np

PAULI_1Q = np.array([
    [[1, 0], [0, 1]],
    [[0, 1], [1, 0]],
    [[0, -1j], [1j, 0]],
    [[1, 0], [0, -1]],
], dtype=np.complex128)


def ternary_digits(b, n):
    """Digits a_1..a_n (qubit 1 first) of basis index b, shape (..., n)."""
    b = np.asarray(b, dtype=np.int64)
    out = np.empty(b.shape + (n,), dtype=np.int64)
    x = b.copy()
    for q in range(n - 1, -1, -1):
        out[..., q] = x % 3
        x //= 3
    return out


def binary_digits(o, n):
    o = np.asarray(o, dtype=np.int64)
    return np.stack([(o >> (n - 1 - q)) & 1 for q in range(n)], axis=-1)


def pauli_index_of(p_digits):
    """Canonical index sum_q p_q 4^(n-q) from digits (..., n)."""
    p = np.asarray(p_digits, dtype=np.int64)
    n = p.shape[-1]
    w = 4 ** np.arange(n - 1, -1, -1, dtype=np.int64)
    return (p * w).sum(axis=-1)


def compatible_pauli_table(n):
    """idx[b, m]: canonical index of the Pauli string with support mask m
    (bit n-q of m is qubit q) whose non-identity letters follow basis b."""
    B = 3 ** n
    a = ternary_digits(np.arange(B), n)            # (B, n)
    m = binary_digits(np.arange(2 ** n), n)        # (d, n)
    p = np.where(m[None, :, :] == 1, a[:, None, :] + 1, 0)
    return pauli_index_of(p)


def _fwht_last(x):
    """Unnormalised Walsh-Hadamard transform along the last axis."""
    x = np.array(x, dtype=np.float64, copy=True)
    d = x.shape[-1]
    h = 1
    while h < d:
        y = x.reshape(x.shape[:-1] + (d // (2 * h), 2, h))
        a = y[..., 0, :].copy()
        bb = y[..., 1, :]
        y[..., 0, :] = a + bb
        y[..., 1, :] = a - bb
        x = y.reshape(x.shape)
        h *= 2
    return x


def pauli_expectations(rho):
    """<P> = Tr(rho P) for every n-qubit Pauli string, canonical order.

    Uses P[r, r^x] = (-1)^{|r&z|} (-i)^{|x&z|} for the string with X/Y
    support x and Z/Y support z.
    """
    rho = np.asarray(rho, dtype=np.complex128)
    d = rho.shape[0]
    n = d.bit_length() - 1
    r = np.arange(d)
    out = np.zeros(4 ** n, dtype=np.float64)
    xs = binary_digits(np.arange(d), n)            # (d, n) bits of x (and of z)
    popc = xs.sum(axis=1)                          # popcount of 0..d-1
    z = np.arange(d)
    for x in range(d):
        v = rho[r ^ x, r]                          # Tr picks rho[c, r] P[r, c]
        w = _fwht_last(v.real) + 1j * _fwht_last(v.imag)   # sum_r v[r](-1)^{r.z}
        xz = popc[x & z]
        ph = (-1j) ** xz
        val = (ph * w).real
        xd = xs[x]
        zd = xs                                     # (d, n)
        p = np.where(xd[None, :] == 1, np.where(zd == 1, 2, 1), np.where(zd == 1, 3, 0))
        out[pauli_index_of(p)] = val
    return out


def born_probabilities(expect, n):
    """p[b, o] = 2^-n sum_m <P(b, m)> (-1)^{|o&m|}  (float64, (3^n, 2^n))."""
    idx = compatible_pauli_table(n)
    e = np.asarray(expect, dtype=np.float64)[idx]
    p = _fwht_last(e) / float(2 ** n)
    return p


def born_probabilities_direct(rho):
    """Brute-force p[b, o] = <psi_bo| rho |psi_bo> (small n only)."""
    rho = np.asarray(rho, dtype=np.complex128)
    d = rho.shape[0]
    n = d.bit_length() - 1
    s = 1 / np.sqrt(2)
    vec = {0: [np.array([s, s]), np.array([s, -s])],
           1: [np.array([s, 1j * s]), np.array([s, -1j * s])],
           2: [np.array([1, 0], dtype=complex), np.array([0, 1], dtype=complex)]}
    P = np.zeros((3 ** n, d))
    for b in range(3 ** n):
        a = ternary_digits(b, n)
        for o in range(d):
            ob = binary_digits(o, n)
            psi = np.array([1.0 + 0j])
            for q in range(n):
                psi = np.kron(psi, vec[int(a[q])][int(ob[q])])
            P[b, o] = np.real(np.vdot(psi, rho @ psi))
    return P


# ---------------------------------------------------------------- states

def ginibre_state(n, rank, seed):
    """Seeded rank-`rank` Ginibre density matrix G G^dag / Tr (complex128)."""
    rng = np.random.default_rng(seed)
    d = 2 ** n
    G = rng.standard_normal((d, rank)) + 1j * rng.standard_normal((d, rank))
    rho = G @ G.conj().T
    return rho / np.trace(rho).real


def ginibre_mixture(n, rank, seed):
    """Random-rank mixture used by the batched workload (same as Ginibre)."""
    return ginibre_state(n, rank, seed)


def ghz_noise_expectation(p_digits, p_noise):
    """Closed-form <P> of (1-p)|GHZ><GHZ| + p I/d for digit arrays (..., n)."""
    p = np.asarray(p_digits)
    is_id = np.all(p == 0, axis=-1)
    iz = np.all((p == 0) | (p == 3), axis=-1)
    nz = np.sum(p == 3, axis=-1)
    xy = np.all((p == 1) | (p == 2), axis=-1)
    ny = np.sum(p == 2, axis=-1)
    val = np.zeros(p.shape[:-1])
    val = np.where(iz & (nz % 2 == 0), 1.0 - p_noise, val)
    re = np.where(ny % 4 == 0, 1.0, np.where(ny % 4 == 2, -1.0, 0.0))
    val = np.where(xy, (1.0 - p_noise) * re, val)
    val = np.where(is_id, 1.0, val)
    return val


def ghz_noise_expectations(n, p_noise):
    i = np.arange(4 ** n)
    digits = np.stack([(i >> (2 * (n - 1 - q))) & 3 for q in range(n)], axis=-1)
    return ghz_noise_expectation(digits, p_noise)


def ghz_noise_state(n, p_noise):
    d = 2 ** n
    g = np.zeros(d, dtype=np.complex128)
    g[0] = g[-1] = 1 / np.sqrt(2)
    return (1 - p_noise) * np.outer(g, g.conj()) + p_noise * np.eye(d) / d


def haar_bloch_vectors(n, seed, shrink=1.0):
    """Bloch vectors (n, 3) of seeded Haar-random single-qubit pure states,
    shrunk by `shrink` (per-qubit depolarising)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return shrink * v


def product_state(bloch):
    rho = np.array([[1.0 + 0j]])
    for r in bloch:
        q = 0.5 * (PAULI_1Q[0] + r[0] * PAULI_1Q[1] + r[1] * PAULI_1Q[2] + r[2] * PAULI_1Q[3])
        rho = np.kron(rho, q)
    return rho


def maximally_mixed(n):
    d = 2 ** n
    return np.eye(d, dtype=np.complex128) / d
