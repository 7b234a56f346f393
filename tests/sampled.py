"""Sampled parity checks at sizes the oracle cannot finish whole (helpers for
the GPU tests, not a test module).

theta: Pauli strings are drawn in blocks.  A block fixes non-identity
letters on n - K sites and leaves K sites free; every string that keeps the
fixed letters and puts any letter (I, X, Y, Z) on the free sites has its 3^k
compatible bases among the block's 3^K bases (the fixed sites' axes are
fixed, the free sites range over X, Y, Z).  So one gather of 3^K count rows
serves strings of every identity count k = 0..K, and the oracle's per-entry
direct sum (Sec. III: the sum over the compatible groups, divided by N 3^k)
runs on them in chunks of bounded memory.

rho: sampled elements by the direct element sum of Sec. IV (the 2^n strings
of the element's x-mask group) from the GPU's theta, each within a relative
1e-6 of the FP64 value (absolute 1e-12 for elements that are zero).
"""
import numpy as np

from oracle import direct


def _index(letters, n):
    return int(sum(int(letters[q]) << (2 * (n - 1 - q)) for q in range(n)))


def _block_bases(n, fixed_sites, fixed_letters, free_sites):
    """Basis indices of the block: axes of the fixed sites from their letters,
    every axis on the free sites (qubit 1 = most significant ternary digit)."""
    axes = np.zeros(n, np.int64)
    for q, p in zip(fixed_sites, fixed_letters):
        axes[q] = p - 1
    K = len(free_sites)
    out = np.empty(3 ** K, np.int64)
    for j in range(3 ** K):
        a = axes.copy()
        x = j
        for q in reversed(free_sites):
            a[q] = x % 3
            x //= 3
        out[j] = int(sum(int(a[q]) * 3 ** (n - 1 - q) for q in range(n)))
    return out


def block_entries(n, rng, K, quota):
    """One block: (indices, block bases).  quota[k] strings with k identity
    letters (all there are, when fewer)."""
    free = sorted(rng.choice(n, size=K, replace=False).tolist())
    fixed = [q for q in range(n) if q not in free]
    letters_fixed = rng.integers(1, 4, size=len(fixed))
    idx = []
    from math import comb
    for k in range(K + 1):
        avail = comb(K, k) * 3 ** (K - k)
        want = min(quota.get(k, 0), avail)
        seen = set()
        while len(seen) < want:
            lt = np.zeros(n, np.int64)
            lt[fixed] = letters_fixed
            ids = rng.choice(K, size=k, replace=False)
            fl = rng.integers(1, 4, size=K)
            fl[ids] = 0
            lt[free] = fl
            seen.add(_index(lt, n))
        idx.extend(sorted(seen))
    return np.array(idx, np.int64), _block_bases(n, fixed, letters_fixed, free)


def check_theta_blocks(n, theta_host, shots, rows_for, rng, blocks, K, quota, max_rows=30000):
    """Bit-exact comparison of theta_host[i] with the oracle's S_i / (N 3^k) on
    the sampled strings.  rows_for(bases) returns the count rows of those
    bases (the same input the GPU read).  Returns (entries checked, counts per
    k, first mismatch or None)."""
    checked, per_k = 0, {}
    for _ in range(blocks):
        idx, bases = block_entries(n, rng, K, quota)
        pos = {int(b): j for j, b in enumerate(bases)}
        rows = rows_for(bases)                                  # (3^K, 2^n)
        ks = np.array([direct.identity_letters(i, n) for i in idx])
        order = np.argsort(ks)
        start = 0
        while start < len(order):                               # chunks of at most max_rows rows
            tot, stop = 0, start
            while stop < len(order) and (tot == 0 or tot + 3 ** int(ks[order[stop]]) <= max_rows):
                tot += 3 ** int(ks[order[stop]])
                stop += 1
            sel = idx[order[start:stop]]
            want = direct.estimate_entries(n, sel, lambda b: rows[[pos[int(x)] for x in b]], shots)
            got = theta_host[sel]
            bad = np.nonzero(got != want)[0]
            if len(bad):
                i = int(sel[bad[0]])
                return checked, per_k, (i, float(got[bad[0]]), float(want[bad[0]]))
            checked += len(sel)
            for k in ks[order[start:stop]]:
                per_k[int(k)] = per_k.get(int(k), 0) + 1
            start = stop
    return checked, per_k, None


def check_rho_elements(n, theta_host, rho_at, rng, count, n_diag):
    """count sampled rho elements (n_diag of them on the diagonal) against the
    oracle's direct element sum of theta_host; rho_at(r, c) returns the GPU's
    complex values.  Returns (max relative error, relative Frobenius error
    over the sample)."""
    d = 2 ** n
    r = rng.integers(0, d, count)
    c = rng.integers(0, d, count)
    c[:n_diag] = r[:n_diag]
    ref = direct.mu_elements(theta_host, n, r, c)
    got = np.asarray(rho_at(r, c), dtype=np.complex128)
    err = np.abs(got - ref)
    tol = 1e-6 * np.abs(ref) + 1e-12
    rel = float(np.max(err / np.maximum(np.abs(ref), 1e-300)))
    assert np.all(err <= tol), (rel, int(np.argmax(err - tol)))
    return rel, float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
