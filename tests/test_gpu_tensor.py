"""Tensor-core form of the first fold pass (tcgen05.mma kind::f16, exact
small integers, FP32 accumulation in TMEM): bit-identical to the FWHT path
and to the oracle."""
import numpy as np
import pytest

from oracle import direct
from tests.gpu_util import ctx_and_lre, need_gpu

pytestmark = pytest.mark.gpu


def _counts(torch, n, shots, seed, dt=np.int16):
    from synth import gen
    c = torch.empty((3 ** n, 2 ** n), dtype=torch.int16 if dt == np.int16 else torch.int32, device="cuda")
    gen.gen_ghz(n, 0.05, shots, seed, c)
    return c


@pytest.mark.parametrize("n", [7, 8, 10, 11])
def test_tensor_parity_sums_equal_fwht(n):
    torch = need_gpu()
    lre, ctx = ctx_and_lre()
    try:
        c = _counts(torch, n, 1000, 90 + n)
        res = []
        for path in (lre.LRE_FOLD_FWHT, lre.LRE_FOLD_TENSOR):
            lre.lre_set_fold_path(ctx, path)
            S = torch.empty(4 ** n, dtype=torch.int64, device="cuda")
            lre.lre_parity_sums(ctx, c, n, S, row_total_bound=1000)
            lre.lre_sync(ctx)
            res.append(S)
        assert torch.equal(res[0], res[1])
    finally:
        lre.lre_destroy(ctx)


def test_tensor_theta_matches_oracle_and_worst_case_counts():
    torch = need_gpu()
    lre, ctx = ctx_and_lre()
    try:
        lre.lre_set_fold_path(ctx, lre.LRE_FOLD_TENSOR)
        n = 7
        rng = np.random.default_rng(3)
        # worst case for the fp16 bias trick: counts up to 1023 (1023 shots)
        raw = rng.multinomial(1023, np.r_[0.9, np.full(2 ** n - 1, 0.1 / (2 ** n - 1))], size=3 ** n)
        raw = raw.astype(np.int16)
        theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
        lre.lre_estimate(ctx, torch.from_numpy(raw).cuda(), 1023, n, theta)
        lre.lre_sync(ctx)
        np.testing.assert_array_equal(theta.cpu().numpy(), direct.estimate(raw, 1023, n))
        # 1024 shots and int32 counts take the FWHT path and stay exact
        raw2 = rng.multinomial(1024, np.ones(2 ** n) / 2 ** n, size=3 ** n).astype(np.int16)
        lre.lre_estimate(ctx, torch.from_numpy(raw2).cuda(), 1024, n, theta)
        lre.lre_sync(ctx)
        np.testing.assert_array_equal(theta.cpu().numpy(), direct.estimate(raw2, 1024, n))
    finally:
        lre.lre_destroy(ctx)
