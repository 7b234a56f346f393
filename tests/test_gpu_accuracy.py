"""Sec. V statistics at scale: the maximally mixed state through the whole
GPU path.  The mean-squared error of mu follows the closed form
((10/3)^n - 3^-n)/(d S) (pinned on the CPU oracle at n = 3, 4 over many
seeds); at n = 10 one draw already sums about a million squared
coefficients, so it lands within a few per cent.  The projection can only
move the estimate closer to the (physical) truth."""
import pytest

from tests.gpu_util import ctx_and_lre, need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shots", [256, 2047])
def test_mse_law_at_n10(shots):
    torch = need_gpu()
    import bench
    lre, ctx = ctx_and_lre()
    try:
        pt = bench.accuracy_point(lre, ctx, torch, 10, shots, 77)
    finally:
        lre.lre_destroy(ctx)
    assert pt["theta_I"] == 1.0
    assert abs(pt["hs_mu_ratio"] - 1.0) < 0.05, pt
    assert pt["hs_rho_hat"] <= pt["hs_mu"], pt
    assert 0.0 <= pt["infidelity_rho_hat"] < 1.0, pt
