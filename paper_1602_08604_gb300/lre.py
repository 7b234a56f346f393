"""ctypes binding of include/lre.h (argument marshalling only).

Every function mirrors the C entry point of the same name.  Device buffers
are passed as torch CUDA tensors (only their data pointers cross the ABI);
streams as torch.cuda.Stream or raw handles.  A non-OK status raises
LreError.  If liblre.so has not been built, loading fails loudly.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblre.so")

LRE_OK = 0
LRE_ERR_INVALID_ARG = 1
LRE_ERR_UNSUPPORTED = 2
LRE_ERR_SHOTS_MISMATCH = 3
LRE_ERR_OOM = 4
LRE_ERR_CUDA = 5
LRE_ERR_TIMEOUT = 6
LRE_ERR_EIG_FAILED = 7

LRE_COUNTS_I32 = 0
LRE_COUNTS_I16 = 1
LRE_SHOTS_U16 = 2

LRE_FOLD_FWHT = 0
LRE_FOLD_TENSOR = 1
LRE_FOLD_TENSOR_SPLIT = 2

LRE_HOST_COUNTS_I32 = 0
LRE_HOST_COUNTS_I16 = 1
LRE_HOST_RECORDS_U16 = 2

class lre_instance(ctypes.Structure):
    """Mirror of the C struct lre_instance (one batched instance)."""
    _fields_ = [("counts", ctypes.c_void_p), ("kind", ctypes.c_int32), ("n", ctypes.c_int32),
                ("shots", ctypes.c_int64), ("theta", ctypes.c_void_p), ("rho", ctypes.c_void_p)]


# (name, restype, argtypes) for every symbol declared in include/lre.h
_p = ctypes.c_void_p
_i = ctypes.c_int
_i64 = ctypes.c_int64
_sz = ctypes.c_size_t
SIGNATURES = [
    ("lre_create", _i, [ctypes.POINTER(_p), _i]),
    ("lre_destroy", None, [_p]),
    ("lre_set_workspace_limit", _i, [_p, _sz]),
    ("lre_workspace_size", _i, [_p, _i, _i, _i, ctypes.POINTER(_sz)]),
    ("lre_parity_sums", _i, [_p, _p, _i, _i, _i64, _p, _p]),
    ("lre_estimate", _i, [_p, _p, _i, _p, _i64, _i, _p, _p, _p]),
    ("lre_slab_sums", _i, [_p, _p, _i, _i, _i64, _p, _p, _p]),
    ("lre_weight", _i, [_p, _p, _i, _i64, _i64, _i64, _p, _p]),
    ("lre_estimate_ic4", _i, [_p, _p, _i, _i64, _i, _p, _p, _p]),
    ("lre_stream_begin", _i, [_p, _i, _i, _i64]),
    ("lre_stream_chunk", _i, [_p, _p, _i64, _i64, _p]),
    ("lre_stream_end", _i, [_p, _p, _p, _p]),
    ("lre_stream_checkpoint", _i, [_p, _p, _sz, ctypes.POINTER(_sz), _p]),
    ("lre_stream_resume", _i, [_p, _p, _sz, _p]),
    ("lre_assemble", _i, [_p, _p, _i, _p, _p]),
    ("lre_assemble_noalloc", _i, [_p, _i, _p, _p]),
    ("lre_project", _i, [_p, _p, _i, _p, _p, _p, _p]),
    ("lre_histogram", _i, [_p, _p, _i64, _i64, _i, _p, _i, _p]),
    ("lre_estimate_host", _i, [_p, _p, _i, _i64, _i, _p, _p, _p]),
    ("lre_batch_run", _i, [_p, _p, _i, _p]),
    ("lre_batch_tune", _i, [_p, _p, _i, _p, ctypes.POINTER(ctypes.c_float)]),
    ("lre_batch_schedule", _i, [_p] + [ctypes.POINTER(_i)] * 4),
    ("lre_set_fold_path", _i, [_p, _i]),
    ("lre_sync", _i, [_p, _p]),
    ("lre_status_string", ctypes.c_char_p, [_i]),
    ("lre_last_error", ctypes.c_char_p, [_p]),
    ("lre_profile", _i, [_p, _i]),
    ("lre_profile_count", _i, [_p]),
    ("lre_profile_get", _i, [_p, _i, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_float)]),
    ("lre_launch_count", ctypes.c_uint64, [_p]),
]

_lib = None


class LreError(RuntimeError):
    def __init__(self, status, detail=""):
        self.status = status
        msg = load().lre_status_string(status).decode()
        super().__init__(f"lre status {status} ({msg}){': ' + detail if detail else ''}")


def load():
    """Load liblre.so (built by paper_1602_08604_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_1602_08604_gb300/build.py "
                              "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _kind(t):
    import torch
    if t.dtype == torch.int32:
        return LRE_COUNTS_I32
    if t.dtype == torch.int16:
        return LRE_COUNTS_I16
    raise TypeError("counts must be an int32 or int16 tensor")


def _check(st, ctx=None):
    if st != LRE_OK:
        # with no context, lre_last_error(NULL) holds the calling thread's
        # lre_assemble_noalloc failure (empty for the other calls)
        detail = load().lre_last_error(ctx).decode()
        raise LreError(st, detail)


def lre_create(device=0):
    ctx = ctypes.c_void_p()
    _check(load().lre_create(ctypes.byref(ctx), int(device)))
    return ctx.value


def lre_destroy(ctx):
    load().lre_destroy(ctx)


def lre_set_workspace_limit(ctx, nbytes):
    _check(load().lre_set_workspace_limit(ctx, int(nbytes)), ctx)


def lre_workspace_size(ctx, n, kind=LRE_COUNTS_I32, per_basis_shots=False):
    out = ctypes.c_size_t()
    _check(load().lre_workspace_size(ctx, int(n), int(kind), int(bool(per_basis_shots)),
                                     ctypes.byref(out)), ctx)
    return out.value


def lre_parity_sums(ctx, counts, n, S, row_total_bound=0, stream=None):
    _check(load().lre_parity_sums(ctx, _ptr(counts), _kind(counts), int(n), int(row_total_bound),
                                  _ptr(S), _stream(stream)), ctx)


def lre_estimate(ctx, counts, shots, n, theta, rho=None, stream=None, kind=None):
    """shots: int (uniform) or an int64 device tensor of per-basis totals.
    kind: LRE_COUNTS_* from the tensor's dtype by default; LRE_SHOTS_U16 for
    a [3^n][shots] tensor of 16-bit shot records (any 16-bit dtype)."""
    if isinstance(shots, int):
        sp, su = None, shots
    else:
        sp, su = _ptr(shots), 0
    k = _kind(counts) if kind is None else int(kind)
    _check(load().lre_estimate(ctx, _ptr(counts), k, sp, int(su), int(n), _ptr(theta),
                               _ptr(rho), _stream(stream)), ctx)


def lre_slab_sums(ctx, slab, n, ident, own, row_total_bound=0, stream=None):
    """slab: [3^(n-1)][2^n] counts of one qubit-1 axis; ident, own: int64 [4^(n-1)]."""
    _check(load().lre_slab_sums(ctx, _ptr(slab), _kind(slab), int(n), int(row_total_bound), _ptr(ident),
                                _ptr(own), _stream(stream)), ctx)


def lre_weight(ctx, S, n, first, shots, theta, stream=None):
    """theta[j] = S[j] / (N 3^k(first + j)) for the block of len(S) sums."""
    _check(load().lre_weight(ctx, _ptr(S), int(n), int(first), int(S.numel()), int(shots), _ptr(theta),
                             _stream(stream)), ctx)


def lre_estimate_ic4(ctx, counts, shots, n, theta, rho=None, stream=None):
    """The 4^n-operator estimate (|0>, |1>, |+>, |+i> per qubit) from Pauli counts."""
    _check(load().lre_estimate_ic4(ctx, _ptr(counts), _kind(counts), int(shots), int(n), _ptr(theta), _ptr(rho),
                                   _stream(stream)), ctx)


def lre_stream_begin(ctx, n, kind, shots):
    _check(load().lre_stream_begin(ctx, int(n), int(kind), int(shots)), ctx)


def lre_stream_chunk(ctx, counts, first_basis, stream=None):
    """counts: device [num_bases][2^n] tensor of bases first_basis..."""
    _check(load().lre_stream_chunk(ctx, _ptr(counts), int(first_basis), int(counts.shape[0]), _stream(stream)), ctx)


def lre_stream_end(ctx, theta, rho=None, stream=None):
    _check(load().lre_stream_end(ctx, _ptr(theta), _ptr(rho), _stream(stream)), ctx)


def lre_stream_checkpoint(ctx, stream=None):
    """The streamed state as bytes (host memory)."""
    need = ctypes.c_size_t()
    _check(load().lre_stream_checkpoint(ctx, None, 0, ctypes.byref(need), _stream(stream)), ctx)
    buf = ctypes.create_string_buffer(need.value)
    _check(load().lre_stream_checkpoint(ctx, buf, need.value, ctypes.byref(need), _stream(stream)), ctx)
    return buf.raw


def lre_stream_resume(ctx, state, stream=None):
    _check(load().lre_stream_resume(ctx, state, len(state), _stream(stream)), ctx)


def lre_assemble(ctx, theta, n, rho, stream=None):
    _check(load().lre_assemble(ctx, _ptr(theta), int(n), _ptr(rho), _stream(stream)), ctx)


def lre_assemble_noalloc(theta, n, rho, stream=None):
    """Step (ii) without any device allocation (fixed 32 MiB scratch, n <= 10)."""
    _check(load().lre_assemble_noalloc(_ptr(theta), int(n), _ptr(rho), _stream(stream)))


def lre_project(ctx, rho_in, n, rho_out, eig_mu=None, eig_rho=None, stream=None):
    _check(load().lre_project(ctx, _ptr(rho_in), int(n), _ptr(rho_out), _ptr(eig_mu), _ptr(eig_rho),
                              _stream(stream)), ctx)


def lre_histogram(ctx, records, n, counts, stream=None):
    """records: uint16-valued tensor [bases][shots] (torch.uint16 or int16 view)."""
    B, S = records.shape
    _check(load().lre_histogram(ctx, _ptr(records), int(B), int(S), int(n), _ptr(counts),
                                _kind(counts), _stream(stream)), ctx)


def lre_estimate_host(ctx, host_in, host_kind, shots, n, theta_host, rho_host=None, stream=None):
    """host_in / theta_host / rho_host: pinned CPU tensors (data pointers only)."""
    _check(load().lre_estimate_host(ctx, _ptr(host_in), int(host_kind), int(shots), int(n),
                                    _ptr(theta_host), _ptr(rho_host), _stream(stream)), ctx)


def _instances(items):
    """items: iterable of (counts, shots, n, theta, rho_or_None) device tensors."""
    arr = (lre_instance * len(items))()
    for k, (counts, shots, n, theta, rho) in enumerate(items):
        arr[k] = lre_instance(_ptr(counts), _kind(counts), int(n), int(shots), _ptr(theta), _ptr(rho))
    return arr


def lre_batch_run(ctx, items, stream=None):
    arr = items if isinstance(items, ctypes.Array) else _instances(items)
    _check(load().lre_batch_run(ctx, ctypes.cast(arr, ctypes.c_void_p), len(arr), _stream(stream)), ctx)


def lre_batch_tune(ctx, items, stream=None):
    """Pick the fastest batched schedule for this batch; returns ms per launch."""
    arr = items if isinstance(items, ctypes.Array) else _instances(items)
    ms = ctypes.c_float()
    _check(load().lre_batch_tune(ctx, ctypes.cast(arr, ctypes.c_void_p), len(arr), _stream(stream),
                                 ctypes.byref(ms)), ctx)
    return ms.value


def lre_batch_schedule(ctx):
    """The context's batched schedule as a dict (jmax, ctas_per_sm, first_unit, unit)."""
    v = [ctypes.c_int() for _ in range(4)]
    _check(load().lre_batch_schedule(ctx, *[ctypes.byref(x) for x in v]), ctx)
    return dict(zip(("jmax", "ctas_per_sm", "first_unit", "unit"), (x.value for x in v)))


def lre_set_fold_path(ctx, path):
    """LRE_FOLD_TENSOR (default; tcgen05 first pass for int16 counts), LRE_FOLD_TENSOR_SPLIT (also int32
    counts, as two fp16 planes) or LRE_FOLD_FWHT."""
    _check(load().lre_set_fold_path(ctx, int(path)), ctx)


def lre_sync(ctx, stream=None):
    _check(load().lre_sync(ctx, _stream(stream)), ctx)


def lre_status_string(status):
    return load().lre_status_string(int(status)).decode()


def lre_last_error(ctx):
    return load().lre_last_error(ctx).decode()


def lre_profile(ctx, enable=True):
    _check(load().lre_profile(ctx, int(bool(enable))), ctx)


def lre_profile_count(ctx):
    return load().lre_profile_count(ctx)


def lre_profile_get(ctx, i):
    name = ctypes.c_char_p()
    ms = ctypes.c_float()
    _check(load().lre_profile_get(ctx, int(i), ctypes.byref(name), ctypes.byref(ms)), ctx)
    return name.value.decode(), ms.value


def lre_profile_records(ctx):
    return [lre_profile_get(ctx, i) for i in range(lre_profile_count(ctx))]


def lre_launch_count(ctx):
    return int(load().lre_launch_count(ctx))
