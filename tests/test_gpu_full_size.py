"""The headline workload at its full size, in the launch configuration
bench.py times: n = 14 GHZ + 5 % white noise, 3^14 bases x 2^14 outcomes of
int16 counts (156.7 GB) drawn on the device, lre_estimate with the default
(tensor-core) path.  The oracle cannot run the whole estimate, so it checks
sampled outputs it can compute one by one: Pauli coefficients from their 3^k
compatible bases (counts regenerated on the CPU by the same counter-based
generator) bit for bit, rho elements from the GPU theta by the direct
element sum (Sec. IV) within 1e-6, plus exact invariants: theta_I = 1 and a
Hermitian rho."""
import numpy as np
import pytest

from tests.gpu_util import ctx_and_lre, need_gpu

pytestmark = pytest.mark.gpu


def test_n14_headline_sampled_parity():
    torch = need_gpu()
    free, total = torch.cuda.mem_get_info()
    if free < 215e9:
        pytest.skip("the n = 14 workload needs about 210 GB of device memory")
    import bench
    wl = bench.WORKLOADS["n14"]
    n = wl["n"]
    lre, ctx = ctx_and_lre()
    try:
        counts = bench.make_counts(torch, wl, torch.device("cuda", 0))
        theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
        rho = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device="cuda")
        lre.lre_estimate(ctx, counts, wl["shots"], n, theta, rho)
        lre.lre_sync(ctx)
        del counts
        assert float(theta[0]) == 1.0
        chk = bench.spot_check(torch, wl, theta, rho, n_entries=128, n_rho=64)
        assert chk["theta_bit_exact"], chk
        assert chk["rho_max_rel_err"] <= 1e-6, chk
        rng = np.random.default_rng(7)
        r = torch.from_numpy(rng.integers(0, 2 ** n, 256)).cuda()
        c = torch.from_numpy(rng.integers(0, 2 ** n, 256)).cuda()
        assert torch.equal(rho[r, c], torch.conj(rho[c, r]))
        tr = torch.diagonal(rho).real.double().sum().item()
        assert abs(tr - 1.0) < 1e-4
    finally:
        lre.lre_destroy(ctx)
