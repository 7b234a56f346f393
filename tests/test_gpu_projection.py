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
        for mode in (0, 2):
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


@pytest.mark.parametrize("n", [11, 12])
def test_partial_projection_large_n_matches_oracle(n):
    """GHZ + noise estimates at d = 2048 and 4096 (the largest size the FP64
    oracle's dense eigendecomposition finishes in seconds): the default
    projection against the oracle's Smolin projection of the same complex64
    mu, within 1e-6 relative Frobenius, both spectra within 1e-9."""
    torch = need_gpu()
    lre, ctx = ctx_and_lre()
    try:
        from synth import gen
        c = torch.empty((3 ** n, 2 ** n), dtype=torch.int16, device="cuda")
        gen.gen_ghz(n, 0.05, 1000, 700 + n, c)
        theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
        mu = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device="cuda")
        lre.lre_estimate(ctx, c, 1000, n, theta, mu)
        lre.lre_sync(ctx)
        del c
        _, lam = _check(lre, ctx, torch, mu.cpu().numpy(), n)
        assert 0 < (lam > 0).sum() < 2 ** (n - 1)
    finally:
        lre.lre_destroy(ctx)


def _project_krylov(lre, ctx, torch, m, n):
    """lre_project without eig_mu (the Krylov path's case); returns the
    projection, its spectrum and the names of the launches it made."""
    mu = torch.from_numpy(m).cuda()
    out = torch.full_like(mu, float("nan"))
    er = torch.full((2 ** n,), float("nan"), dtype=torch.float64, device="cuda")
    lre.lre_profile(ctx, True)
    lre.lre_project(ctx, mu, n, out, eig_rho=er)
    lre.lre_sync(ctx)
    names = [k for k, _ in lre.lre_profile_records(ctx)]
    lre.lre_profile(ctx, False)
    return out.cpu().numpy(), er.cpu().numpy(), names


@pytest.mark.parametrize("n", [11, 12])
def test_krylov_projection_of_estimates_matches_oracle(n):
    """GHZ + noise estimates (a few dozen kept eigenvalues): the Lanczos path
    decides the threshold from the top of the spectrum, certifies it and
    rebuilds the kept form; against the oracle's Smolin projection of the same
    complex64 mu (1e-6 relative Frobenius, spectrum within 1e-9)."""
    torch = need_gpu()
    lre, ctx = ctx_and_lre()
    try:
        from synth import gen
        c = torch.empty((3 ** n, 2 ** n), dtype=torch.int16, device="cuda")
        gen.gen_ghz(n, 0.05, 1000, 500 + n, c)
        theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
        mu = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device="cuda")
        lre.lre_estimate(ctx, c, 1000, n, theta, mu)
        lre.lre_sync(ctx)
        del c
        m = mu.cpu().numpy()
        got, er, names = _project_krylov(lre, ctx, torch, m, n)
        assert "kry_matvec" in names and "hetrd(cusolver)" not in names, sorted(set(names))
        ref, _, lam = project.smolin(m.astype(np.complex128))
        assert rel_fro(got, ref) <= 1e-6
        np.testing.assert_allclose(er, lam, atol=1e-9)
        assert 0 < (lam > 0).sum() < 2 ** (n - 1)
    finally:
        lre.lre_destroy(ctx)


def test_krylov_projection_dropped_form_matches_oracle():
    """A mostly positive spectrum with five negative eigenvalues (d = 2048):
    the threshold comes from Smolin's walk over the smallest eigenvalues and
    the rebuild is mu + sI minus the dropped directions."""
    torch = need_gpu()
    lre, ctx = ctx_and_lre()
    try:
        n = 11
        d = 2 ** n
        rng = np.random.default_rng(31)
        lam = rng.uniform(0.2, 1.0, d)
        lam[:5] = -rng.uniform(0.05, 0.2, 5) * lam.mean()
        lam /= lam.sum()
        m = _hermitian_with_spectrum(lam, 8)
        mu = torch.from_numpy(m).cuda()
        out = torch.full_like(mu, float("nan"))
        lre.lre_profile(ctx, True)
        lre.lre_project(ctx, mu, n, out)
        lre.lre_sync(ctx)
        names = [k for k, _ in lre.lre_profile_records(ctx)]
        lre.lre_profile(ctx, False)
        assert "kry_matvec" in names and "hetrd(cusolver)" not in names, sorted(set(names))
        ref, _, lam_ref = project.smolin(m.astype(np.complex128))
        assert rel_fro(out.cpu().numpy(), ref) <= 1e-6
        assert (lam_ref > 0).sum() == d - 5
    finally:
        lre.lre_destroy(ctx)


def test_krylov_projection_with_degenerate_kept_cluster_is_right():
    """Kept eigenvalues equal before complex64 rounding (a three-fold and a
    two-fold cluster): Lanczos sees such clusters late, so either the
    certification run catches a missed copy and the call takes the reduction
    path, or the copies were found; the projection must match the oracle
    either way."""
    torch = need_gpu()
    lre, ctx = ctx_and_lre()
    try:
        n = 11
        d = 2 ** n
        rng = np.random.default_rng(12)
        lam = -rng.uniform(0, 2e-5, d)
        lam[-3:] = 0.3
        lam[-5:-3] = 0.15
        lam[-6] = 0.05
        lam /= lam.sum()
        m = _hermitian_with_spectrum(lam, 13)
        got, er, names = _project_krylov(lre, ctx, torch, m, n)
        ref, _, lam_ref = project.smolin(m.astype(np.complex128))
        assert rel_fro(got, ref) <= 1e-6
        np.testing.assert_allclose(er, lam_ref, atol=1e-9)
        assert (lam_ref > 0).sum() == 6
    finally:
        lre.lre_destroy(ctx)


def test_krylov_equals_reduction_path_n13():
    """n = 13 estimate (beyond the FP64 oracle's reach): the Lanczos path and
    the tridiagonal-reduction path agree within 1e-6 relative Frobenius and
    1e-9 on the spectrum."""
    torch = need_gpu()
    lre, ctx = ctx_and_lre()
    try:
        n = 13
        from synth import gen
        c = torch.empty((3 ** n, 2 ** n), dtype=torch.int16, device="cuda")
        gen.gen_ghz(n, 0.05, 1000, 613, c)
        theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
        mu = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device="cuda")
        lre.lre_estimate(ctx, c, 1000, n, theta, mu)
        lre.lre_sync(ctx)
        del c, theta
        outs, eigs = [], []
        for mode in (1, 2):
            _mode(lre, ctx, mode)
            out = torch.full_like(mu, float("nan"))
            er = torch.full((2 ** n,), float("nan"), dtype=torch.float64, device="cuda")
            lre.lre_profile(ctx, True)
            lre.lre_project(ctx, mu, n, out, eig_rho=er)
            lre.lre_sync(ctx)
            names = [k for k, _ in lre.lre_profile_records(ctx)]
            lre.lre_profile(ctx, False)
            assert ("kry_matvec" in names) == (mode == 1), sorted(set(names))
            outs.append(out.cpu().numpy())
            eigs.append(er.cpu().numpy())
        assert rel_fro(outs[0], outs[1]) <= 1e-6
        np.testing.assert_allclose(eigs[0], eigs[1], atol=1e-9)
    finally:
        lre.lre_destroy(ctx)
