"""Oracle anchors for the fold pass plans between the exhaustive sizes and
the headline: n = 11 (passes of 6 + 3 + 2 qubits), 12 (6 + 3 + 3) and 13
(6 + 3 + 3 + 1), GHZ + 5 % white noise, 1000 shots per basis, int16 counts
drawn on the device.  theta through the default (tensor-core) path must
equal the FWHT path's bit for bit over the whole vector, and the oracle's
per-entry direct sum bit for bit on about 10^4 sampled coefficients
stratified over k = 0..8 identity letters (tests/sampled.py); sampled rho
elements match the direct element sum within a relative 1e-6."""
import numpy as np
import pytest

from tests import sampled
from tests.gpu_util import ctx_and_lre, need_gpu

pytestmark = pytest.mark.gpu

QUOTA = {0: 250, 1: 250, 2: 250, 3: 250, 4: 250, 5: 150, 6: 100, 7: 24, 8: 1}


@pytest.mark.parametrize("n", [11, 12, 13])
def test_large_n_theta_anchored_to_oracle(n):
    torch = need_gpu()
    from synth import gen
    shots = 1000
    counts = torch.empty((3 ** n, 2 ** n), dtype=torch.int16, device="cuda")
    gen.gen_ghz(n, 0.05, shots, 1300 + n, counts)
    thetas, rho = [], None
    for path in ("tensor", "fwht"):
        lre, ctx = ctx_and_lre()
        try:
            lre.lre_set_fold_path(ctx, lre.LRE_FOLD_TENSOR if path == "tensor" else lre.LRE_FOLD_FWHT)
            theta = torch.full((4 ** n,), float("nan"), dtype=torch.float64, device="cuda")
            r = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device="cuda") if path == "tensor" else None
            lre.lre_estimate(ctx, counts, shots, n, theta, r)
            lre.lre_sync(ctx)
            thetas.append(theta)
            rho = r if r is not None else rho
        finally:
            lre.lre_destroy(ctx)
    assert torch.equal(thetas[0], thetas[1])
    t_host = thetas[0].cpu().numpy()
    del thetas
    rng = np.random.default_rng(100 + n)
    rows_for = lambda b: counts[torch.from_numpy(np.asarray(b)).cuda()].cpu().numpy()
    checked, per_k, bad = sampled.check_theta_blocks(n, t_host, shots, rows_for, rng,
                                                     blocks=7, K=8, quota=QUOTA)
    assert bad is None, bad
    assert checked >= 10_000 and sorted(per_k) == list(range(9)), (checked, per_k)
    rho_at = lambda r, c: rho[torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda()].cpu().numpy()
    sampled.check_rho_elements(n, t_host, rho_at, rng, count=4096, n_diag=512)
