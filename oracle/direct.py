"""ctypes binding and build step for oracle/direct.c -- test infrastructure only."""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "direct.c")
_LIB = os.path.join(_HERE, "_direct.so")
_lib = None


def build(force=False):
    """Compile direct.c with gcc + OpenMP into oracle/_direct.so."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", _LIB + ".tmp"]
    subprocess.check_call(cmd)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        p = ctypes.c_void_p
        i64 = ctypes.c_int64
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_set_threads.restype = ctypes.c_int
        L.oracle_direct_sums.argtypes = [ctypes.c_int, p, ctypes.c_int, i64, i64, p, p]
        L.oracle_direct_sums.restype = ctypes.c_int
        L.oracle_direct_weighted.argtypes = [ctypes.c_int, p, ctypes.c_int, p, i64, i64, p, p]
        L.oracle_direct_weighted.restype = ctypes.c_int
        L.oracle_theta_uniform.argtypes = [ctypes.c_int, p, p, i64, p]
        L.oracle_theta_weighted.argtypes = [ctypes.c_int, p, p, p]
        L.oracle_direct_mu_elements.argtypes = [ctypes.c_int, p, p, p, i64, p, p]
        L.oracle_direct_mu.argtypes = [ctypes.c_int, p, p, p]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(t=0):
    return lib().oracle_set_threads(int(t))


def _kind(counts):
    if counts.dtype == np.int32:
        return 0
    if counts.dtype == np.int16:
        return 1
    raise TypeError("counts must be int32 or int16")


def parity_sums(counts, n, b0=0, b1=None, S=None, diag=None):
    """Integer sums S (4^n int64) and X^T X diagonal (group counts) for
    groups [b0, b1); `counts` holds rows b0..b1-1."""
    counts = np.ascontiguousarray(counts)
    b1 = b0 + counts.shape[0] if b1 is None else b1
    P = 4 ** n
    S = np.zeros(P, np.int64) if S is None else S
    diag = np.zeros(P, np.int64) if diag is None else diag
    rc = lib().oracle_direct_sums(n, _ptr(counts), _kind(counts), b0, b1, _ptr(S), _ptr(diag))
    if rc != 0:
        raise MemoryError("oracle_direct_sums failed")
    return S, diag


def estimate(counts, shots, n):
    """Pauli expectation estimates t (4^n FP64, t[0] = 1) by the direct sum.

    shots: int (uniform, exact-integer path) or (3^n,) array (FP64 path)."""
    counts = np.ascontiguousarray(counts)
    P = 4 ** n
    t = np.empty(P, np.float64)
    if np.ndim(shots) == 0:
        S, diag = parity_sums(counts, n)
        lib().oracle_theta_uniform(n, _ptr(S), _ptr(diag), int(shots), _ptr(t))
        return t
    sh = np.ascontiguousarray(np.asarray(shots, dtype=np.int64))
    acc = np.zeros(P, np.float64)
    diag = np.zeros(P, np.int64)
    rc = lib().oracle_direct_weighted(n, _ptr(counts), _kind(counts), _ptr(sh), 0,
                                      counts.shape[0], _ptr(acc), _ptr(diag))
    if rc != 0:
        raise MemoryError("oracle_direct_weighted failed")
    lib().oracle_theta_weighted(n, _ptr(acc), _ptr(diag), _ptr(t))
    return t


def mu(t, n):
    """mu (complex128 d x d) by the per-group direct sum."""
    t = np.ascontiguousarray(np.asarray(t, dtype=np.float64))
    d = 2 ** n
    re = np.empty((d, d), np.float64)
    im = np.empty((d, d), np.float64)
    lib().oracle_direct_mu(n, _ptr(t), _ptr(re), _ptr(im))
    return re + 1j * im


def mu_elements(t, n, rows, cols):
    t = np.ascontiguousarray(np.asarray(t, dtype=np.float64))
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    cols = np.ascontiguousarray(np.asarray(cols, dtype=np.int64))
    re = np.empty(len(rows), np.float64)
    im = np.empty(len(rows), np.float64)
    lib().oracle_direct_mu_elements(n, _ptr(t), _ptr(rows), _ptr(cols), len(rows), _ptr(re), _ptr(im))
    return re + 1j * im


def compatible_bases(i, n):
    """Basis indices (increasing) of the groups whose locations include Pauli
    index i: the non-identity letters fix those digits, identity sites range
    over X, Y, Z."""
    digits = [(i >> (2 * (n - 1 - q))) & 3 for q in range(n)]  # qubit 1 first
    bases = [0]
    for p in digits:
        if p == 0:
            bases = [3 * b + a for b in bases for a in range(3)]
        else:
            bases = [3 * b + (p - 1) for b in bases]
    return bases


def parity_sum_entries(n, indices, rows_for):
    """S_i for selected Pauli indices.  rows_for(bases) must return the counts
    rows (len(bases), 2^n) of those bases (int32 or int16)."""
    L = lib()
    if not hasattr(L, "_entries_set"):
        L.oracle_direct_entries.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        L._entries_set = True
    idx = np.asarray(indices, dtype=np.int64)
    all_bases, offs = [], []
    for i in idx:
        offs.append(len(all_bases))
        all_bases.extend(compatible_bases(int(i), n))
    rows = np.ascontiguousarray(rows_for(np.array(all_bases, dtype=np.int64)))
    offs = np.ascontiguousarray(np.array(offs, dtype=np.int64))
    S = np.empty(len(idx), np.int64)
    L.oracle_direct_entries(n, _ptr(rows), _kind(rows), _ptr(np.ascontiguousarray(idx)), _ptr(offs),
                            len(idx), _ptr(S))
    return S


def identity_letters(i, n):
    return sum(((int(i) >> (2 * q)) & 3) == 0 for q in range(n))


def estimate_entries(n, indices, rows_for, shots):
    """t_i = S_i / (N 3^k) for selected indices (uniform shots)."""
    S = parity_sum_entries(n, indices, rows_for)
    k = np.array([identity_letters(i, n) for i in indices])
    return S.astype(np.float64) / (float(shots) * (3.0 ** k))
