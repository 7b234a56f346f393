"""Workspace canaries (a substitute for a device memory checker, none of
which runs on this pool): with a 64 KiB guard of a fixed pattern after the
context's workspace, every entry point, on every path and at sizes that span
the kernels' tile shapes and ragged tails, must leave the guard whole."""
import ctypes

import numpy as np
import pytest

from tests.gpu_util import ctx_and_lre, need_gpu

pytestmark = pytest.mark.gpu


def _hooks(lre):
    L = lre.load()
    L.lre_debug_set_canaries.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.lre_debug_set_canaries.restype = ctypes.c_int
    L.lre_debug_check_canaries.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]
    L.lre_debug_check_canaries.restype = ctypes.c_int
    L.lre_debug_set_first_pass.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.lre_debug_set_first_pass.restype = ctypes.c_int
    return L


def _intact(L, ctx):
    ok = ctypes.c_int(-1)
    assert L.lre_debug_check_canaries(ctx, ctypes.byref(ok)) == 0
    return ok.value == 1


@pytest.mark.parametrize("n,dt,shots,path,variant", [
    (1, np.int32, 100, 1, 1), (5, np.int16, 1000, 1, 1), (7, np.int16, 1000, 1, 1),
    (8, np.int32, 4096, 2, 1), (10, np.int16, 2047, 1, 1), (10, np.int32, 1000, 0, 1),
    (11, np.int16, 1000, 1, 2), (12, np.int16, 1000, 0, 0)])
def test_estimate_paths_stay_inside_the_workspace(n, dt, shots, path, variant):
    torch = need_gpu()
    from synth import gen
    lre, ctx = ctx_and_lre()
    L = _hooks(lre)
    try:
        assert L.lre_debug_set_canaries(ctx, 1) == 0
        assert L.lre_debug_set_first_pass(ctx, variant) == 0
        lre.lre_set_fold_path(ctx, path)
        c = torch.empty((3 ** n, 2 ** n), dtype=torch.int16 if dt == np.int16 else torch.int32, device="cuda")
        gen.gen_ghz(n, 0.05, shots, 5 + n, c)
        theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
        rho = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device="cuda")
        S = torch.empty(4 ** n, dtype=torch.int64, device="cuda")
        lre.lre_estimate(ctx, c, shots, n, theta, rho)
        lre.lre_parity_sums(ctx, c, n, S, row_total_bound=shots)
        lre.lre_assemble(ctx, theta, n, rho)
        lre.lre_sync(ctx)
        assert _intact(L, ctx)
        lre.lre_estimate_ic4(ctx, c, shots, n, theta, rho)
        lre.lre_sync(ctx)
        assert _intact(L, ctx)
        if n >= 2:
            m = 3 ** (n - 1)
            ident = torch.empty(4 ** (n - 1), dtype=torch.int64, device="cuda")
            own = torch.empty_like(ident)
            lre.lre_slab_sums(ctx, c[m:2 * m], n, ident, own, row_total_bound=shots)
            lre.lre_sync(ctx)
            assert _intact(L, ctx)
        if n >= 7 and variant == 1:               # the streamed first pass takes tile ranges
            lre.lre_stream_begin(ctx, n, lre.LRE_COUNTS_I16 if dt == np.int16 else lre.LRE_COUNTS_I32, shots)
            for b0 in range(0, 3 ** n, 729):
                lre.lre_stream_chunk(ctx, c[b0:b0 + 729], b0)
            lre.lre_stream_end(ctx, theta, rho)
            lre.lre_sync(ctx)
            assert _intact(L, ctx)
    finally:
        lre.lre_destroy(ctx)


@pytest.mark.parametrize("n", [6, 11])
def test_projection_stays_inside_the_workspace(n):
    torch = need_gpu()
    from synth import gen
    lre, ctx = ctx_and_lre()
    L = _hooks(lre)
    try:
        assert L.lre_debug_set_canaries(ctx, 1) == 0
        c = torch.empty((3 ** n, 2 ** n), dtype=torch.int16, device="cuda")
        gen.gen_ghz(n, 0.05, 1000, 9 + n, c)
        theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
        mu = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device="cuda")
        lre.lre_estimate(ctx, c, 1000, n, theta, mu)
        out = torch.empty_like(mu)
        em = torch.empty(2 ** n, dtype=torch.float64, device="cuda")
        lre.lre_project(ctx, mu, n, out)                  # Krylov path from d = 2048
        lre.lre_project(ctx, mu, n, out, eig_mu=em)        # reduction path
        lre.lre_sync(ctx)
        assert _intact(L, ctx)
    finally:
        lre.lre_destroy(ctx)


def test_batch_stays_inside_the_workspace():
    torch = need_gpu()
    from tests.test_gpu_batch import _instance
    lre, ctx = ctx_and_lre()
    L = _hooks(lre)
    try:
        assert L.lre_debug_set_canaries(ctx, 1) == 0
        items = []
        for k, n in enumerate((3, 5, 7, 9)):
            cc = _instance(n, 70 + k, 1500, np.int32)
            th = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
            rh = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device="cuda")
            items.append((torch.from_numpy(cc).cuda(), 1500, n, th, rh))
        lre.lre_batch_run(ctx, items)
        lre.lre_sync(ctx)
        assert _intact(L, ctx)
    finally:
        lre.lre_destroy(ctx)
