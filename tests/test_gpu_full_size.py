"""The headline workload at its full size, in the launch configuration
bench.py times: n = 14 GHZ + 5 % white noise, 3^14 bases x 2^14 outcomes of
int16 counts (156.7 GB) drawn on the device, lre_estimate with the default
(tensor-core) path.  The oracle cannot run the whole estimate, so it checks
sampled outputs it can compute one by one (tests/sampled.py): about 10^4
Pauli coefficients stratified over k = 0..8 identity letters, from the count
rows of their compatible bases (the rows the GPU read), bit for bit; 10^4
rho elements (10^3 of them diagonal) by the direct element sum of Sec. IV
from the GPU theta, each within a relative 1e-6; and exact invariants:
theta_I = 1, a Hermitian rho of unit trace."""
import numpy as np
import pytest

from tests import sampled
from tests.gpu_util import ctx_and_lre, need_gpu

pytestmark = pytest.mark.gpu

# strings per identity count k in each block of 8 free sites (all there are
# for k = 7, 8); seven blocks give about 10^4 strings
QUOTA = {0: 250, 1: 250, 2: 250, 3: 250, 4: 250, 5: 150, 6: 100, 7: 24, 8: 1}


def test_n14_headline_sampled_parity():
    torch = need_gpu()
    torch.cuda.empty_cache()          # what earlier tests left in the caching allocator
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
    finally:
        lre.lre_destroy(ctx)                      # frees the fold workspace
    t_host = theta.cpu().numpy()
    del theta
    assert t_host[0] == 1.0
    rng = np.random.default_rng(7)
    rows_for = lambda b: counts[torch.from_numpy(np.asarray(b)).cuda()].cpu().numpy()
    checked, per_k, bad = sampled.check_theta_blocks(n, t_host, wl["shots"], rows_for, rng,
                                                     blocks=7, K=8, quota=QUOTA)
    assert bad is None, bad
    assert checked >= 10_000 and sorted(per_k) == list(range(9)), (checked, per_k)
    del counts
    rho_at = lambda r, c: rho[torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda()].cpu().numpy()
    sampled.check_rho_elements(n, t_host, rho_at, rng, count=10_000, n_diag=1_000)
    r = torch.from_numpy(rng.integers(0, 2 ** n, 4096)).cuda()
    c = torch.from_numpy(rng.integers(0, 2 ** n, 4096)).cuda()
    assert torch.equal(rho[r, c], torch.conj(rho[c, r]))
    tr = torch.diagonal(rho).real.double().sum().item()
    assert abs(tr - 1.0) < 1e-4


def test_n14_projection_paths_agree_and_give_a_density_matrix():
    """Step (iii) at d = 16384 (beyond the FP64 oracle's reach): the Lanczos
    path and the tridiagonal-reduction path agree within 1e-6 relative
    Frobenius and 1e-9 on the spectrum, and the result is a density matrix
    (Hermitian, unit trace, non-negative spectrum summing to one)."""
    torch = need_gpu()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < 215e9:
        pytest.skip("the n = 14 workload needs about 210 GB of device memory")
    import ctypes

    import bench
    wl = bench.WORKLOADS["n14"]
    n = wl["n"]
    d = 2 ** n
    lre, ctx = ctx_and_lre()
    try:
        counts = bench.make_counts(torch, wl, torch.device("cuda", 0))
        theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
        mu = torch.empty((d, d), dtype=torch.complex64, device="cuda")
        lre.lre_estimate(ctx, counts, wl["shots"], n, theta, mu)
        lre.lre_sync(ctx)
        del counts, theta
        torch.cuda.empty_cache()
        f = lre.load().lre_debug_set_project_mode
        f.argtypes = [ctypes.c_void_p, ctypes.c_int]
        f.restype = ctypes.c_int
        outs, eigs = [], []
        for mode in (1, 2):                     # Lanczos, then the reduction
            assert f(ctx, mode) == 0
            out = torch.empty_like(mu)
            er = torch.empty(d, dtype=torch.float64, device="cuda")
            lre.lre_project(ctx, mu, n, out, eig_rho=er)
            lre.lre_sync(ctx)
            outs.append(out)
            eigs.append(er)
        diff = torch.linalg.vector_norm((outs[0] - outs[1]).to(torch.complex128))
        ref = torch.linalg.vector_norm(outs[1].to(torch.complex128))
        assert float(diff / ref) <= 1e-6
        assert float((eigs[0] - eigs[1]).abs().max()) <= 1e-9
        lam = eigs[0]
        # the kept eigenvalues sum to Tr mu, 1 up to the complex64 rounding of its diagonal
        assert float(lam.min()) >= 0.0 and abs(float(lam.sum()) - 1.0) < 1e-6
        rho = outs[0]
        assert abs(float(torch.diagonal(rho).real.double().sum()) - 1.0) < 1e-4
        rng = np.random.default_rng(3)
        r = torch.from_numpy(rng.integers(0, d, 4096)).cuda()
        c = torch.from_numpy(rng.integers(0, d, 4096)).cuda()
        assert torch.equal(rho[r, c], torch.conj(rho[c, r]))
    finally:
        lre.lre_destroy(ctx)
