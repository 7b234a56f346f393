"""Step (iii): the eigenvalue-first projection (tridiagonal reduction,
bisection, inverse iteration for the smaller of the kept / dropped sets)
against the oracle's Smolin projection, and against the full
eigendecomposition path on larger sizes."""
import ctypes

import numpy as np
import pytest

from oracle import project
from synth import counts as sc
from synth import states as st
from tests.gpu_util import ctx_and_lre, need_gpu, rel_fro

pytestmark = pytest.mark.gpu


def _mode(lre, ctx, m):
    f = lre.load().lre_debug_set_project_mode
    f.argtypes = [ctypes.c_void_p, ctypes.c_int]
    f.restype = ctypes.c_int
    assert f(ctx, m) == 0


def _hermitian_with_spectrum(lam, seed):
    """U diag(lam) U^dag for a Haar-random U, rounded to an exactly Hermitian
    complex64 matrix with a real diagonal."""
    d = len(lam)
    rng = np.random.default_rng(seed)
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    q = q * (np.diag(r) / np.abs(np.diag(r)))
    m = (q * lam) @ q.conj().T
    m = m.astype(np.complex64)
    m = np.triu(m) + np.triu(m, 1).conj().T
    m[np.diag_indices(d)] = m.diagonal().real
    return m


def _check(lre, ctx, torch, m, n):
    mu = torch.from_numpy(m).cuda()
    out = torch.empty_like(mu)
    em = torch.empty(2 ** n, dtype=torch.float64, device="cuda")
    er = torch.empty(2 ** n, dtype=torch.float64, device="cuda")
    lre.lre_project(ctx, mu, n, out, em, er)
    lre.lre_sync(ctx)
    ref, lam_mu, lam = project.smolin(m.astype(np.complex128))
    got = out.cpu().numpy()
    assert rel_fro(got, ref) <= 1e-6
    np.testing.assert_allclose(em.cpu().numpy(), lam_mu, atol=1e-9)
    np.testing.assert_allclose(er.cpu().numpy(), lam, atol=1e-9)
    return got, lam


@pytest.mark.parametrize("n,N", [(6, 100), (7, 1000), (8, 50), (9, 1000), (10, 200)])
def test_partial_projection_kept_form_matches_oracle(n, N):
    """LRE estimates of rank-2 states from finite shots: few eigenvalues kept."""
    torch = need_gpu()
    lre, ctx = ctx_and_lre()
    try:
        rho = st.ginibre_state(n, 2, seed=40 + n)
        thr = sc.cdf_thresholds(st.born_probabilities(st.pauli_expectations(rho), n))
        counts = sc.sample_cdf(thr, N, seed=41 + n)
        mu = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device="cuda")
        theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
        lre.lre_estimate(ctx, torch.from_numpy(counts).cuda(), N, n, theta, mu)
        lre.lre_sync(ctx)
        _, lam = _check(lre, ctx, torch, mu.cpu().numpy(), n)
        assert 0 < (lam > 0).sum() <= 2 ** (n - 1)
    finally:
        lre.lre_destroy(ctx)


@pytest.mark.parametrize("n", [6, 8, 9])
def test_partial_projection_dropped_form_matches_oracle(n):
    """Mostly positive spectrum with a few negative eigenvalues: the dropped
    set is the smaller one."""
    torch = need_gpu()
    lre, ctx = ctx_and_lre()
    try:
        d = 2 ** n
        rng = np.random.default_rng(n)
        lam = rng.uniform(0.2, 1.0, d)
        lam[:5] = -rng.uniform(0.001, 0.02, 5)
        lam /= lam.sum()
        _, out_lam = _check(lre, ctx, torch, _hermitian_with_spectrum(lam, 7 + n), n)
        assert (out_lam > 0).sum() > d // 2
    finally:
        lre.lre_destroy(ctx)


def test_partial_projection_clustered_and_degenerate():
    """Kept eigenvalues in tight clusters (equal before complex64 rounding)."""
    torch = need_gpu()
    lre, ctx = ctx_and_lre()
    try:
        n = 7
        d = 2 ** n
        lam = np.full(d, -1e-4)
        lam[-3:] = 0.25              # a three-fold cluster
        lam[-6:-3] = 0.08            # and another
        lam[-7] = 0.01
        lam[:-7] += np.linspace(0, 1e-5, d - 7)
        lam /= lam.sum()
        got, out_lam = _check(lre, ctx, torch, _hermitian_with_spectrum(lam, 99), n)
        assert (out_lam > 0).sum() == 7
    finally:
        lre.lre_destroy(ctx)


def test_partial_projection_of_physical_state_is_identity():
    torch = need_gpu()
    lre, ctx = ctx_and_lre()
    try:
        n = 6
        m = st.ginibre_state(n, 2 ** n, seed=5).astype(np.complex64)
        m = np.triu(m) + np.triu(m, 1).conj().T
        m[np.diag_indices(2 ** n)] = m.diagonal().real
        w = np.linalg.eigvalsh(m.astype(np.complex128))
        assert w.min() > 0
        mu = torch.from_numpy(m).cuda()
        out = torch.empty_like(mu)
        lre.lre_project(ctx, mu, n, out)
        lre.lre_sync(ctx)
        np.testing.assert_array_equal(out.cpu().numpy(), m)
    finally:
        lre.lre_destroy(ctx)


@pytest.mark.parametrize("n", [11, 12])
def test_partial_equals_full_path(n):
    """GHZ + noise estimates at larger sizes: eigenvalue-first against the
    full eigendecomposition (both FP64 on the GPU)."""
    torch = need_gpu()
    lre, ctx = ctx_and_lre()
    try:
        from synth import gen
        c = torch.empty((3 ** n, 2 ** n), dtype=torch.int16, device="cuda")
        gen.gen_ghz(n, 0.05, 1000, 900 + n, c)
        theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
        mu = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device="cuda")
        lre.lre_estimate(ctx, c, 1000, n, theta, mu)
        del c
        outs, eigs = [], []
        for mode in (0, 1):
            _mode(lre, ctx, mode)
            out = torch.full_like(mu, float("nan"))  # nothing left from the other mode
            er = torch.full((2 ** n,), float("nan"), dtype=torch.float64, device="cuda")
            lre.lre_project(ctx, mu, n, out, eig_rho=er)
            lre.lre_sync(ctx)
            outs.append(out.cpu().numpy())
            eigs.append(er.cpu().numpy())
        assert rel_fro(outs[1], outs[0]) <= 1e-6
        np.testing.assert_allclose(eigs[1], eigs[0], atol=1e-12)
        assert (eigs[1] > 0).sum() < 2 ** (n - 1)
    finally:
        lre.lre_destroy(ctx)
