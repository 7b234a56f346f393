"""lre_estimate on device shot records (LRE_SHOTS_U16): the per-basis
results of Sec. III given as one outcome index per shot.  The call
histograms them into counts on the device and runs the same fold; theta must
equal the oracle's estimate from the records' counts bit for bit, rho within
relative Frobenius 1e-6."""
import numpy as np
import pytest

from oracle import direct
from tests.gpu_util import ctx_and_lre, need_gpu, rel_fro

pytestmark = pytest.mark.gpu


def _records(n, shots, seed):
    """Shot records [3^n][shots] (uint16 outcome indices, shuffled per basis)
    and their counts."""
    rng = np.random.default_rng(seed)
    d = 2 ** n
    p = rng.dirichlet(np.full(d, 0.3), size=3 ** n)
    counts = np.stack([rng.multinomial(shots, row) for row in p])
    rec = np.empty((3 ** n, shots), np.uint16)
    for b in range(3 ** n):
        r = np.repeat(np.arange(d, dtype=np.uint16), counts[b])
        rng.shuffle(r)
        rec[b] = r
    return rec, counts


@pytest.mark.parametrize("n,shots", [(3, 1000), (7, 1000), (9, 1000), (9, 2047), (5, 40000)])
def test_estimate_from_device_records(n, shots):
    torch = need_gpu()
    rec, counts = _records(n, shots, 10 + n)
    lre, ctx = ctx_and_lre()
    try:
        r = torch.from_numpy(rec.view(np.int16)).cuda()
        theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
        rho = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device="cuda")
        lre.lre_estimate(ctx, r, shots, n, theta, rho, kind=lre.LRE_SHOTS_U16)
        lre.lre_sync(ctx)
        t_ref = direct.estimate(counts.astype(np.int32), shots, n)
        np.testing.assert_array_equal(theta.cpu().numpy(), t_ref)
        assert rel_fro(rho.cpu().numpy(), direct.mu(t_ref, n)) <= 1e-6
    finally:
        lre.lre_destroy(ctx)


def test_records_argument_checks():
    torch = need_gpu()
    n, shots = 7, 64
    rec, _ = _records(n, shots, 3)
    lre, ctx = ctx_and_lre()
    try:
        r = torch.from_numpy(rec.view(np.int16)).cuda()
        theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
        per_basis = torch.full((3 ** n,), shots, dtype=torch.int64, device="cuda")
        with pytest.raises(lre.LreError) as e:        # records carry uniform shots only
            lre.lre_estimate(ctx, r, per_basis, n, theta, kind=lre.LRE_SHOTS_U16)
        assert e.value.status == lre.LRE_ERR_INVALID_ARG
        rec[17, 5] = 2 ** n                           # an outcome index out of range
        r = torch.from_numpy(rec.view(np.int16)).cuda()
        lre.lre_estimate(ctx, r, shots, n, theta, kind=lre.LRE_SHOTS_U16)
        with pytest.raises(lre.LreError) as e:
            lre.lre_sync(ctx)
        assert e.value.status == lre.LRE_ERR_INVALID_ARG
    finally:
        lre.lre_destroy(ctx)
