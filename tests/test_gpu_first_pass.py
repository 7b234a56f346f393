"""The two first-pass kernels (register-only and TMA pipeline) produce the
same int32 partial sums (test hook lre_debug_first_pass)."""
import ctypes

import numpy as np
import pytest

from tests.gpu_util import ctx_and_lre, need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,dt", [(7, np.int32), (7, np.int16), (8, np.int16), (9, np.int32)])
def test_pipeline_equals_register_kernel(n, dt):
    torch = need_gpu()
    lre, ctx = ctx_and_lre()
    L = lre.load()
    f = L.lre_debug_first_pass
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    try:
        rng = np.random.default_rng(n)
        counts = rng.multinomial(1000, np.ones(2 ** n) / 2 ** n, size=3 ** n).astype(dt)
        c = torch.from_numpy(counts).cuda()
        size = 3 ** (n - 6) * 2 ** (n - 6) * 4096
        outs = []
        for variant in (0, 1):
            o = torch.full((size,), -7, dtype=torch.int32, device="cuda")
            kind = lre.LRE_COUNTS_I16 if dt == np.int16 else lre.LRE_COUNTS_I32
            assert f(ctx, c.data_ptr(), kind, n, o.data_ptr(), variant,
                     torch.cuda.current_stream().cuda_stream) == 0
            lre.lre_sync(ctx)
            outs.append(o.cpu().numpy())
        bad = np.nonzero(outs[0] != outs[1])[0]
        if len(bad):
            tile, rem = bad // 4096, bad % 4096
            pytest.fail(f"{len(bad)} of {size} differ; tiles {np.unique(tile)[:8]}, "
                        f"plB {np.unique(rem // 64)[:8]}, plA {np.unique(rem % 64)[:8]}, "
                        f"sample ref {outs[0][bad[:4]]} got {outs[1][bad[:4]]}")
    finally:
        lre.lre_destroy(ctx)


@pytest.mark.parametrize("n,dt", [(10, np.int16), (11, np.int32), (12, np.int16)])
def test_fused_second_pass_equals_unfused(n, dt):
    """The first pass fused with the second through L2 gives the same exact
    integer parity sums as the two passes run separately."""
    torch = need_gpu()
    from synth import gen
    c = torch.empty((3 ** n, 2 ** n), dtype=torch.int16 if dt == np.int16 else torch.int32, device="cuda")
    gen.gen_ghz(n, 0.05, 1000, 77 + n, c)
    res = []
    for variant, kernel in ((2, "fold_first9_fused"), (1, "fold_first6")):
        lre, ctx = ctx_and_lre()  # one context per variant: no shared workspace
        try:
            f = lre.load().lre_debug_set_first_pass
            f.argtypes = [ctypes.c_void_p, ctypes.c_int]
            f.restype = ctypes.c_int
            lre.lre_set_fold_path(ctx, lre.LRE_FOLD_FWHT)  # both sides on the ALU kernels
            assert f(ctx, variant) == 0
            S = torch.full((4 ** n,), -1, dtype=torch.int64, device="cuda")
            lre.lre_profile(ctx, True)
            lre.lre_parity_sums(ctx, c, n, S, row_total_bound=1000)
            lre.lre_sync(ctx)
            assert kernel in {k for k, _ in lre.lre_profile_records(ctx)}
            res.append(S)
        finally:
            lre.lre_destroy(ctx)
    assert torch.equal(res[0], res[1])
    assert int(res[1][0]) == 1000 * 3 ** n
