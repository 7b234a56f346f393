"""Build and ctypes binding of the device count generators (synth/csrc/gen.cu).

Input synthesis for GPU tests and benchmarks: the counts land directly in
device memory and are bit-identical to synth.counts on the CPU.
"""
import ctypes
import os
import subprocess

import numpy as np

from .counts import prob_threshold, product_thresholds
from .philox import seed_key

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "gen.cu")
LIB = os.path.join(HERE, "_gen.so")
_lib = None


def build(force=False):
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
    subprocess.check_call([nvcc, "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
                           "-gencode", "arch=compute_103a,code=sm_103a", SRC, "-o", LIB + ".tmp"])
    os.replace(LIB + ".tmp", LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise ImportError(f"{LIB} missing: run synth.gen.build()")
        L = ctypes.CDLL(LIB)
        p, i, i64, u32, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
        L.synth_gen_cdf.argtypes = [p, i, i64, i64, i64, u64, p, i, p]
        L.synth_gen_ghz.argtypes = [i, u32, i64, i64, i64, u64, p, i, p]
        L.synth_gen_product.argtypes = [p, i, i64, i64, i64, u64, p, i, p]
        L.synth_gen_ghz_records.argtypes = [i, u32, i64, i64, i64, u64, p, p]
        L.synth_gen_mixed.argtypes = [i, i64, i64, i64, u64, p, i, p]
        for f in (L.synth_gen_cdf, L.synth_gen_ghz, L.synth_gen_product, L.synth_gen_ghz_records,
                  L.synth_gen_mixed):
            f.restype = i
        _lib = L
    return _lib


def _kind(t):
    import torch
    return 1 if t.dtype == torch.int16 else 0


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _seed(seed):
    return int(seed) & 0xFFFFFFFFFFFFFFFF


def gen_cdf(thr_dev, n, shots, seed, counts, b0=0):
    rc = lib().synth_gen_cdf(thr_dev.data_ptr(), n, b0, counts.shape[0], shots, _seed(seed),
                             counts.data_ptr(), _kind(counts), _stream())
    if rc != 0:
        raise RuntimeError(f"synth_gen_cdf: cuda error {rc}")


def gen_ghz(n, p_noise, shots, seed, counts, b0=0):
    thr = int(prob_threshold(p_noise))
    rc = lib().synth_gen_ghz(n, thr, b0, counts.shape[0], shots, _seed(seed), counts.data_ptr(),
                             _kind(counts), _stream())
    if rc != 0:
        raise RuntimeError(f"synth_gen_ghz: cuda error {rc}")


def gen_product(bloch, shots, seed, counts, b0=0):
    import torch
    thr = torch.from_numpy(product_thresholds(bloch).astype(np.uint32).view(np.int32).ravel().copy())
    thr = thr.to(counts.device)
    n = len(bloch)
    rc = lib().synth_gen_product(thr.data_ptr(), n, b0, counts.shape[0], shots, _seed(seed),
                                 counts.data_ptr(), _kind(counts), _stream())
    torch.cuda.current_stream().synchronize()
    if rc != 0:
        raise RuntimeError(f"synth_gen_product: cuda error {rc}")


def gen_ghz_records(n, p_noise, seed, records, b0=0):
    """records: uint16-valued device tensor [bases][shots] (int16 storage)."""
    thr = int(prob_threshold(p_noise))
    nb, shots = records.shape
    rc = lib().synth_gen_ghz_records(n, thr, b0, nb, shots, _seed(seed), records.data_ptr(), _stream())
    if rc != 0:
        raise RuntimeError(f"synth_gen_ghz_records: cuda error {rc}")


def gen_mixed(n, shots, seed, counts, b0=0):
    """Maximally mixed state counts by binary splitting (synth.counts.sample_mixed)."""
    rc = lib().synth_gen_mixed(n, b0, counts.shape[0], shots, _seed(seed), counts.data_ptr(), _kind(counts),
                               _stream())
    if rc != 0:
        raise RuntimeError(f"synth_gen_mixed: cuda error {rc}")
