"""The final fold pass's division (one FP64 multiply, then an exact 128-bit
integer remainder and round-to-nearest-even) against IEEE division of the
same exact integers (numpy float64): bit for bit, for signs, |S| = D, the
largest |S| and divisors up to 2^53 - 1.  (An exact tie would need a
quotient with 54 significant bits, i.e. |S| >= 2^53, so none occurs.)"""
import ctypes

import numpy as np
import pytest

from tests.gpu_util import ctx_and_lre, need_gpu

pytestmark = pytest.mark.gpu

DIVISORS = [1, 2, 3, 4, 7, 1000, 1023 * 3 ** 7, 1000 * 3 ** 14, 2047 * 3 ** 14, 3 ** 33, 2 ** 52 - 1, 2 ** 52,
            2 ** 52 + 1, 2 ** 53 - 1, 6 * 3 ** 20]


@pytest.mark.parametrize("D", DIVISORS)
def test_division_matches_ieee(D):
    torch = need_gpu()
    lre, ctx = ctx_and_lre()
    f = lre.load().lre_debug_div
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    try:
        rng = np.random.default_rng(D % 100003)
        lim = min(D, 2 ** 53 - 1)
        S = np.concatenate([
            rng.integers(-lim, lim + 1, 200000, dtype=np.int64),
            rng.integers(-(2 ** 53 - 1), 2 ** 53, 50000, dtype=np.int64),
            np.array([1, -1, D, -D, D // 2, D // 2 + 1, -(D // 2), max(D - 1, 1), 2 ** 52, 2 ** 53 - 1,
                      -(2 ** 53 - 1), 0], dtype=np.int64),
        ])
        S = S[np.abs(S) < 2 ** 53]
        dS = torch.from_numpy(S).cuda()
        out = torch.empty(len(S), dtype=torch.float64, device="cuda")
        assert f(ctx, dS.data_ptr(), len(S), D, out.data_ptr(), torch.cuda.current_stream().cuda_stream) == 0
        torch.cuda.synchronize()
        want = S.astype(np.float64) / np.float64(D)
        got = out.cpu().numpy()
        bad = np.nonzero(got.view(np.int64) != want.view(np.int64))[0]
        assert len(bad) == 0, (S[bad[:5]], got[bad[:5]], want[bad[:5]])
    finally:
        lre.lre_destroy(ctx)
