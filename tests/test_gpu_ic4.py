"""The 4^n-operator variant (Sec. VI; |0>, |1>, |+>, |+i> per qubit) on the
GPU against the oracle (oracle/ic4.py, pinned against Eq. 3's normal
equations): theta bit for bit (exact integer sums, one correctly rounded
division by N), rho within 1e-6 relative Frobenius."""
import numpy as np
import pytest

from oracle import direct, ic4
from tests.gpu_util import ctx_and_lre, need_gpu, rel_fro

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 9])
@pytest.mark.parametrize("dtype", [np.int16, np.int32])
def test_ic4_theta_and_rho_match_oracle(n, dtype):
    torch = need_gpu()
    rng = np.random.default_rng(70 + n)
    N = 999
    p = rng.dirichlet(np.full(2 ** n, 0.7), size=3 ** n)
    c = np.stack([rng.multinomial(N, row) for row in p]).astype(dtype)
    lre, ctx = ctx_and_lre()
    try:
        theta = torch.full((4 ** n,), float("nan"), dtype=torch.float64, device="cuda")
        rho = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device="cuda")
        lre.lre_estimate_ic4(ctx, torch.from_numpy(c).cuda(), N, n, theta, rho)
        lre.lre_sync(ctx)
        want = ic4.exact_theta(c, N, n)
        np.testing.assert_array_equal(theta.cpu().numpy(), want)
        assert rel_fro(rho.cpu().numpy(), direct.mu(want, n)) <= 1e-6
    finally:
        lre.lre_destroy(ctx)
