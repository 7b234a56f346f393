"""TMA-staged fold passes (the passes after the six-qubit first pass) against
the per-thread-load passes: identical parity sums and theta for every pass
shape (J = 1, 2, 3; store, parity and final modes)."""
import ctypes

import numpy as np
import pytest

from tests.gpu_util import ctx_and_lre, need_gpu

pytestmark = pytest.mark.gpu


def _hook(lre):
    f = lre.load().lre_debug_set_generic_tma
    f.argtypes = [ctypes.c_void_p, ctypes.c_int]
    f.restype = ctypes.c_int
    return f


# plans: 7 = 6+1, 8 = 6+2, 9 = 6+3, 10 = 6+3+1, 11 = 6+3+2, 12 = 6+3+3, 13 = 6+3+3+1
@pytest.mark.parametrize("n", [7, 8, 9, 10, 11, 12, 13])
def test_tma_passes_equal_register_passes(n):
    torch = need_gpu()
    from synth import gen
    c = torch.empty((3 ** n, 2 ** n), dtype=torch.int16, device="cuda")
    gen.gen_ghz(n, 0.05, 1000, 500 + n, c)
    out = {}
    for on in (1, 0):  # each setting in a context of its own: no shared workspace
        lre, ctx = ctx_and_lre()
        try:
            assert _hook(lre)(ctx, on) == 0
            S = torch.full((4 ** n,), -1, dtype=torch.int64, device="cuda")
            theta = torch.full((4 ** n,), -1.0, dtype=torch.float64, device="cuda")
            lre.lre_profile(ctx, True)
            lre.lre_parity_sums(ctx, c, n, S, row_total_bound=1000)
            lre.lre_estimate(ctx, c, 1000, n, theta)
            lre.lre_sync(ctx)
            names = {k for k, _ in lre.lre_profile_records(ctx)}
            # the TMA kernels take the store and parity passes (finals stay
            # in the register kernel), so any plan with more than one pass
            # after the first, or a parity last pass, launches one
            assert ("fold_tma" in names) == bool(on), names
            out[on] = (S, theta)
        finally:
            lre.lre_destroy(ctx)
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1])
    assert int(out[1][0][0]) == 1000 * 3 ** n
