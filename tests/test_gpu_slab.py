"""One instance split by the axis of qubit 1 (lre_slab_sums, lre_weight and
the orchestration in paper_1602_08604_gb300/shard.py), all three slabs on
one GPU: each slab's shares equal the oracle's direct sums over that slab's
basis groups only (Sec. III), bit for bit, and the combined theta equals
lre_estimate's and the oracle's estimate bit for bit."""
import numpy as np
import pytest

from oracle import direct
from tests.gpu_util import ctx_and_lre, need_gpu

pytestmark = pytest.mark.gpu


def _counts(n, N, seed, dtype):
    rng = np.random.default_rng(seed)
    p = rng.dirichlet(np.full(2 ** n, 0.5), size=3 ** n)
    return np.stack([rng.multinomial(N, row) for row in p]).astype(dtype)


@pytest.mark.parametrize("n,dtype,shots", [(2, np.int32, 100), (5, np.int32, 1000), (7, np.int16, 1000),
                                           (8, np.int16, 2047), (8, np.int32, 40000)])
def test_slab_sums_and_sharded_theta(n, dtype, shots):
    torch = need_gpu()
    from paper_1602_08604_gb300 import shard
    c = _counts(n, shots, 50 + n, dtype)
    cd = torch.from_numpy(c).cuda()
    plan = shard.SlabPlan(n, 1)
    lre, ctx = ctx_and_lre()
    try:
        slabs = {}
        for a in range(3):
            lo, hi = plan.rows(a)
            slabs[a] = cd[lo:hi]
            ident = torch.full((plan.block,), -7, dtype=torch.int64, device="cuda")
            own = torch.full((plan.block,), -7, dtype=torch.int64, device="cuda")
            lre.lre_slab_sums(ctx, slabs[a], n, ident, own, row_total_bound=shots)
            lre.lre_sync(ctx)
            S, _ = direct.parity_sums(c[lo:hi], n, b0=lo, b1=hi)
            olo, ohi = plan.own_range(a)
            np.testing.assert_array_equal(ident.cpu().numpy(), S[: plan.block])
            np.testing.assert_array_equal(own.cpu().numpy(), S[olo:ohi])
            assert not np.any(S[plan.block:olo]) and not np.any(S[ohi:])   # the slab feeds nothing else
        theta = shard.estimate_sharded(lre, ctx, slabs, shots, n)
        t1 = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
        lre.lre_estimate(ctx, cd, shots, n, t1)
        lre.lre_sync(ctx)
        assert torch.equal(theta, t1)
        np.testing.assert_array_equal(theta.cpu().numpy(), direct.estimate(c, shots, n))
    finally:
        lre.lre_destroy(ctx)


def test_weight_checks_and_block_offsets():
    torch = need_gpu()
    lre, ctx = ctx_and_lre()
    try:
        n, N = 3, 10
        S = torch.tensor([30, -30, 270, 7], dtype=torch.int64, device="cuda")
        t = torch.empty(4, dtype=torch.float64, device="cuda")
        lre.lre_weight(ctx, S, n, 0, N, t)          # indices 0..3: k = 3, 2, 2, 2
        lre.lre_sync(ctx)
        assert t.cpu().tolist() == [30 / 270, -30 / 90, 270 / 90, 7 / 90]
        with pytest.raises(lre.LreError):
            lre.lre_weight(ctx, S, n, 4 ** n - 2, N, t)  # beyond 4^n
    finally:
        lre.lre_destroy(ctx)
