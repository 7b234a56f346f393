"""Seeded multinomial count samplers (CPU twins of synth/csrc/gen.cu).

Every random word comes from Philox4x32-10 keyed by the 64-bit seed, with a
counter that names (shot, basis, stream, call).  Every decision is an
integer comparison against a uint32 threshold computed once on the host, so
the CPU and GPU samplers give identical counts.

Samplers
  * cdf      generic: inverse-CDF over per-basis uint32 thresholds
             (shot s uses word s&3 of the call with counter (s>>2, b, 0x11, 0)).
  * ghz      (1-p)|GHZ><GHZ| + p I/d sampled directly: with probability p a
             uniform outcome, else the GHZ outcome law of basis b.
  * product  product of single-qubit states: one word per qubit and shot.
  * mixed    the maximally mixed state I/d at any shot number, by binary
             splitting: every qubit's outcome is a fair coin, so the shots c
             at a node of the outcome tree (qubit 1 first) send
             Binomial(c, 1/2) of them to bit 0, drawn exactly as the number of
             set bits among c fair random bits (node (q, v) reads words
             4g..4g+3 of the calls with counter (g, b, 0x44, (1 << q) | v),
             the first c bits, word by word from the least significant bit).
             Cost n S / 128 calls per basis instead of n S / 4.
"""
import numpy as np

from .philox import philox4x32, seed_key
from .states import ternary_digits

STREAM_CDF = 0x11
STREAM_GHZ = 0x22
STREAM_PROD = 0x33
STREAM_SPLIT = 0x44


def prob_threshold(p):
    """uint32 threshold t with P(word < t) ~= p (t = round(p 2^32), clamped)."""
    t = np.floor(np.asarray(p, dtype=np.float64) * 4294967296.0 + 0.5)
    return np.clip(t, 0, 4294967295).astype(np.uint32)


def cdf_thresholds(probs):
    """Per-basis uint32 thresholds (B, d-1) from float64 probabilities (B, d)."""
    p = np.clip(np.asarray(probs, dtype=np.float64), 0.0, None)
    p = p / p.sum(axis=1, keepdims=True)
    cum = np.cumsum(p, axis=1)[:, :-1]
    t = np.floor(cum * 4294967296.0)
    return np.clip(t, 0, 4294967295).astype(np.uint32)


def _hist(outcomes, d, dtype):
    B = outcomes.shape[0]
    flat = outcomes + (np.arange(B, dtype=np.int64)[:, None] * d)
    c = np.bincount(flat.ravel(), minlength=B * d).reshape(B, d)
    return c.astype(dtype)


def sample_cdf(thresholds, shots, seed, bases=None, dtype=np.int32):
    """Counts (len(bases), d) by inverse-CDF sampling (d = thresholds.shape[1]+1)."""
    thr = np.asarray(thresholds, dtype=np.uint32)
    B, dm1 = thr.shape
    d = dm1 + 1
    bases = np.arange(B, dtype=np.int64) if bases is None else np.asarray(bases, dtype=np.int64)
    k0, k1 = seed_key(seed)
    s = np.arange(shots, dtype=np.int64)
    out = np.zeros((len(bases), d), dtype=dtype)
    step = max(1, (1 << 22) // max(shots, 1))
    for lo in range(0, len(bases), step):
        bb = bases[lo:lo + step]
        w = philox4x32((s >> 2)[None, :], bb[:, None], STREAM_CDF, 0, k0, k1)
        u = np.choose((s & 3)[None, :].repeat(len(bb), 0), w)
        o = np.empty_like(u, dtype=np.int64)
        for j, b in enumerate(bb):
            o[j] = np.searchsorted(thr[b], u[j], side="right")
        out[lo:lo + step] = _hist(o, d, dtype)
    return out


def ghz_sample_outcomes(n, p_noise_thr, shots, seed, bases):
    """Outcome indices (len(bases), shots) of the direct GHZ+white-noise sampler."""
    bases = np.asarray(bases, dtype=np.int64)
    d = 1 << n
    k0, k1 = seed_key(seed)
    a = ternary_digits(bases, n)                                # (B, n)
    bit = (1 << (n - 1 - np.arange(n))).astype(np.int64)        # qubit q -> bit n-1-q (0-based q)
    zmask = ((a == 2) * bit).sum(axis=1)                        # (B,)
    ny = (a == 1).sum(axis=1)
    s = np.arange(shots, dtype=np.int64)
    w0, w1, w2, _ = philox4x32(s[None, :], bases[:, None], STREAM_GHZ, 0, k0, k1)
    w0 = w0.astype(np.int64); w1 = w1.astype(np.int64); w2 = w2.astype(np.int64)
    noise = w0 < int(p_noise_thr)
    u = w1 & (d - 1)
    zm = zmask[:, None]
    with_z = (u & ~zm) | np.where((w2 & 1) == 1, zm, 0)
    pc = np.zeros_like(u)
    t = u.copy()
    while np.any(t):
        pc ^= t & 1
        t >>= 1
    par = ((ny >> 1) & 1)[:, None]
    no_z = np.where(((ny % 2) == 0)[:, None] & (pc != par), u ^ 1, u)
    ghz = np.where(zm != 0, with_z, no_z)
    return np.where(noise, u, ghz)


def sample_ghz(n, p_noise, shots, seed, bases=None, dtype=np.int32):
    B = 3 ** n
    bases = np.arange(B, dtype=np.int64) if bases is None else np.asarray(bases, dtype=np.int64)
    thr = int(prob_threshold(p_noise))
    d = 1 << n
    out = np.zeros((len(bases), d), dtype=dtype)
    step = max(1, (1 << 22) // max(shots, 1))
    for lo in range(0, len(bases), step):
        bb = bases[lo:lo + step]
        o = ghz_sample_outcomes(n, thr, shots, seed, bb)
        out[lo:lo + step] = _hist(o, d, dtype)
    return out


def product_thresholds(bloch):
    """uint32 thresholds (n, 3): P(o_q = 0 | axis a) = (1 + r_a)/2."""
    r = np.asarray(bloch, dtype=np.float64)
    return prob_threshold((1.0 + r) / 2.0)


def sample_product(bloch, shots, seed, bases=None, dtype=np.int32):
    thr = product_thresholds(bloch)                             # (n, 3)
    n = thr.shape[0]
    d = 1 << n
    B = 3 ** n
    bases = np.arange(B, dtype=np.int64) if bases is None else np.asarray(bases, dtype=np.int64)
    k0, k1 = seed_key(seed)
    out = np.zeros((len(bases), d), dtype=dtype)
    s = np.arange(shots, dtype=np.int64)
    step = max(1, (1 << 21) // max(shots, 1))
    for lo in range(0, len(bases), step):
        bb = bases[lo:lo + step]
        a = ternary_digits(bb, n)                               # (B, n)
        o = np.zeros((len(bb), shots), dtype=np.int64)
        for call in range((n + 3) // 4):
            w = philox4x32(s[None, :], bb[:, None], STREAM_PROD, call, k0, k1)
            for j in range(4):
                q = 4 * call + j
                if q >= n:
                    break
                t = thr[q][a[:, q]].astype(np.int64)[:, None]
                bitv = (w[j].astype(np.int64) >= t).astype(np.int64)
                o |= bitv << (n - 1 - q)
        out[lo:lo + step] = _hist(o, d, dtype)
    return out


def exact_counts(probs, shots, dtype=np.int32):
    """Infinite-shot counts N p when every N p is an integer (asserted)."""
    x = np.asarray(probs, dtype=np.float64) * shots
    c = np.rint(x)
    if np.max(np.abs(x - c)) > 1e-6:
        raise ValueError("N*p is not integral for this state and shot count")
    c = c.astype(np.int64)
    if np.any(c.sum(axis=1) != shots):
        raise ValueError("rounded rows do not sum to the shot count")
    return c.astype(dtype)


def _popcount32(x):
    x = x.astype(np.uint64)
    c = np.zeros(x.shape, dtype=np.int64)
    for k in range(32):
        c += ((x >> np.uint64(k)) & np.uint64(1)).astype(np.int64)
    return c


def fair_binomial(c, b, node, k0, k1):
    """Binomial(c, 1/2) for each basis b (arrays of equal length): the number
    of set bits among the first c bits of node `node`'s word stream."""
    c = np.asarray(c, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    out = np.zeros(len(c), dtype=np.int64)
    calls = (c + 127) // 128
    for g in range(int(calls.max()) if len(c) else 0):
        live = calls > g
        if not np.any(live):
            break
        words = philox4x32(np.uint32(g), b[live], STREAM_SPLIT, np.uint32(node), k0, k1)
        cl = c[live]
        acc = np.zeros(int(live.sum()), dtype=np.int64)
        for k in range(4):
            first = 128 * g + 32 * k                  # index of this word's first bit
            nb = np.clip(cl - first, 0, 32)           # bits of this word inside the first c
            mask = np.where(nb >= 32, np.uint64(0xFFFFFFFF),
                            (np.uint64(1) << nb.astype(np.uint64)) - np.uint64(1))
            acc += _popcount32(words[k].astype(np.uint64) & mask)
        out[live] += acc
    return out


def sample_mixed(n, shots, seed, bases=None, dtype=np.int32):
    """Counts of the maximally mixed n-qubit state (every basis uniform over
    its 2^n outcomes), drawn by binary splitting of the shots."""
    B = 3 ** n
    d = 1 << n
    bases = np.arange(B, dtype=np.int64) if bases is None else np.asarray(bases, dtype=np.int64)
    k0, k1 = seed_key(seed)
    # slot v << (n - q) holds node (q, v): the node and its left child share a slot
    c = np.zeros((len(bases), d), dtype=np.int64)
    c[:, 0] = shots
    for q in range(n):
        half = 1 << (n - q - 1)
        for v in range(1 << q):
            slot = v << (n - q)
            c0 = fair_binomial(c[:, slot], bases, (1 << q) | v, k0, k1)
            c[:, slot + half] = c[:, slot] - c0
            c[:, slot] = c0
    return c.astype(dtype)
