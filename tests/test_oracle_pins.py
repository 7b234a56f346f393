"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test targets a plausible mistake: a dropped X^T X term, a wrong sign of
a Gamma entry, a transposed index order, a wrong Y phase, a wrong 1/(N 3^k)
weight, or a wrong projection loop.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import direct, explicit, project
from synth import counts as sc
from synth import states as st

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# --------------------------------------------------- Sec. III statements

def test_gamma_vectors_n1_match_paper():
    # Sec. III: (1/sqrt2)(1,+-1,0,0), (1/sqrt2)(1,0,+-1,0), (1/sqrt2)(1,0,0,+-1)
    X = explicit.design_matrix(1) * np.sqrt(2)
    want = np.array([[1, 1, 0, 0], [1, -1, 0, 0], [1, 0, 1, 0], [1, 0, -1, 0],
                     [1, 0, 0, 1], [1, 0, 0, -1]], dtype=float)
    np.testing.assert_allclose(X, want, atol=1e-12)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_xtx_is_kron_power_of_diag3111(n):
    # Sec. III: X^T X = diag{3,1,1,1} for one qubit and its tensor power for n
    X = explicit.design_matrix(n)
    want = np.array([[1.0]])
    for _ in range(n):
        want = np.kron(want, np.diag([3.0, 1.0, 1.0, 1.0]))
    np.testing.assert_allclose(X.T @ X, want, atol=1e-12)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_direct_diag_equals_3_pow_identity_count(n):
    rng = np.random.default_rng(n)
    c = rng.integers(0, 50, size=(3 ** n, 2 ** n)).astype(np.int32)
    _, diag = direct.parity_sums(c, n)
    i = np.arange(4 ** n)
    k = sum(((i >> (2 * q)) & 3) == 0 for q in range(n))
    np.testing.assert_array_equal(diag, 3 ** k)


def test_omega_orthonormal_and_index_order():
    # Sec. II: Tr(Omega_i Omega_j) = delta_ij; Eq. (5) index i = sum i_k 4^{n-k}
    om = explicit.omega_basis(2)
    G = np.einsum("ikl,jlk->ij", om, om)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)
    # index 4*1 + 3 = 7 is sigma_x (x) sigma_z / 2 (qubit 1 most significant)
    want = np.kron(explicit.SIGMA[1], explicit.SIGMA[3]) / 2
    np.testing.assert_allclose(om[7], want, atol=1e-15)


# --------------------------------------------------- hand-checked fixtures

def test_n1_handchecked_explicit_and_direct():
    g = _load("n1_handchecked.json")
    for case in g["cases"]:
        c = np.array(case["counts"], dtype=np.int32)
        N = case["shots"]
        t_exp = explicit.expectations_from_theta(explicit.ls_theta(c, N, 1), 1)
        t_dir = direct.estimate(c, N, 1)
        np.testing.assert_allclose(t_exp, case["t"], atol=1e-14)
        np.testing.assert_array_equal(t_dir, np.array(case["t"]))
        if "mu_re" in case:
            mu = direct.mu(t_dir, 1)
            np.testing.assert_allclose(mu.real, case["mu_re"], atol=1e-15)
            np.testing.assert_allclose(mu.imag, case["mu_im"], atol=1e-15)
            mu_e = explicit.mu_from_theta(explicit.ls_theta(c, N, 1), 1)
            np.testing.assert_allclose(mu_e, mu, atol=1e-14)


def test_n1_projection_handchecked():
    g = _load("n1_handchecked.json")
    phys, outside = g["cases"]
    mu = direct.mu(np.array(phys["t"]), 1)
    rho, lam_mu, lam = project.smolin(mu)
    np.testing.assert_allclose(rho, mu, atol=1e-14)
    mu = direct.mu(np.array(outside["t"]), 1)
    rho, lam_mu, lam = project.smolin(mu)
    s3 = np.sqrt(3.0)
    np.testing.assert_allclose(lam_mu, [(1 + s3) / 2, (1 - s3) / 2], atol=1e-14)
    want = 0.5 * (explicit.SIGMA[0] + (explicit.SIGMA[1] + explicit.SIGMA[2] + explicit.SIGMA[3]) / s3)
    np.testing.assert_allclose(rho, want, atol=1e-14)
    np.testing.assert_allclose(lam, [1.0, 0.0], atol=1e-14)


def test_n2_bell_exact_counts():
    g = _load("n2_bell_exact.json")
    c = np.array(g["counts"], dtype=np.int32)
    want = np.zeros(16)
    for k, v in g["t_nonzero"].items():
        want[int(k)] = v
    t = direct.estimate(c, g["shots"], 2)
    np.testing.assert_array_equal(t, want)
    t_e = explicit.expectations_from_theta(explicit.ls_theta(c, g["shots"], 2), 2)
    np.testing.assert_allclose(t_e, want, atol=1e-13)
    np.testing.assert_allclose(direct.mu(t, 2).real, g["mu_re"], atol=1e-15)
    np.testing.assert_allclose(direct.mu(t, 2).imag, 0, atol=1e-15)


def test_n1_closed_form_random_counts():
    # one qubit: t_I = 1, t_a = (c_a0 - c_a1)/N exactly
    rng = np.random.default_rng(3)
    for _ in range(20):
        N = int(rng.integers(1, 5000))
        c0 = rng.integers(0, N + 1, size=3)
        c = np.stack([c0, N - c0], axis=1).astype(np.int32)
        t = direct.estimate(c, N, 1)
        want = np.array([1.0] + [(int(c[a, 0]) - int(c[a, 1])) / N for a in range(3)])
        np.testing.assert_array_equal(t, want)


# --------------------------------------------------- infinite-shot counts

@pytest.mark.parametrize("n", [2, 3, 4])
def test_ghz_white_noise_infinite_shots_exact(n):
    p = Fraction(1, 10)
    d = 2 ** n
    probs = st.born_probabilities(st.ghz_noise_expectations(n, float(p)), n)
    N = 10 * d
    c = sc.exact_counts(probs, N)
    t = direct.estimate(c, N, n)
    # exact rational <P> of (1-p)GHZ + p I/d, rounded once
    want = np.zeros(4 ** n)
    for i in range(4 ** n):
        dig = [(i >> (2 * (n - 1 - q))) & 3 for q in range(n)]
        if all(x == 0 for x in dig):
            want[i] = 1.0
        elif all(x in (0, 3) for x in dig) and sum(x == 3 for x in dig) % 2 == 0:
            want[i] = float(1 - p)
        elif all(x in (1, 2) for x in dig):
            ny = sum(x == 2 for x in dig)
            want[i] = float((1 - p) * (1 if ny % 4 == 0 else (-1 if ny % 4 == 2 else 0)))
    np.testing.assert_array_equal(t, want)


def test_product_of_eigenstates_infinite_shots():
    # |0> (x) |+> (x) |+i>: <P> = prod_q <sigma_{p_q}>_q, probabilities in {0,1/2,1}/...
    bloch = np.array([[0, 0, 1.0], [1.0, 0, 0], [0, 1.0, 0]])
    rho = st.product_state(bloch)
    n = 3
    probs = st.born_probabilities_direct(rho)
    c = sc.exact_counts(probs, 8)
    t = direct.estimate(c, 8, n)
    single = [{0: 1, 1: 0, 2: 0, 3: 1}, {0: 1, 1: 1, 2: 0, 3: 0}, {0: 1, 1: 0, 2: 1, 3: 0}]
    want = np.array([np.prod([single[q][(i >> (2 * (n - 1 - q))) & 3] for q in range(n)])
                     for i in range(4 ** n)], dtype=float)
    np.testing.assert_array_equal(t, want)


def test_maximally_mixed_infinite_shots():
    n = 4
    d = 2 ** n
    c = np.ones((3 ** n, d), dtype=np.int32)
    t = direct.estimate(c, d, n)
    want = np.zeros(4 ** n)
    want[0] = 1
    np.testing.assert_array_equal(t, want)
    mu = direct.mu(t, n)
    np.testing.assert_allclose(mu, np.eye(d) / d, atol=1e-15)


# --------------------------------------------------- cross-method agreement

@pytest.mark.parametrize("n,seed", [(2, 0), (3, 1), (4, 2)])
def test_explicit_ls_matches_direct_sum(n, seed):
    rng = np.random.default_rng(seed)
    N = 1000
    raw = rng.multinomial(N, np.ones(2 ** n) / 2 ** n, size=3 ** n).astype(np.int32)
    t_dir = direct.estimate(raw, N, n)
    t_exp = explicit.expectations_from_theta(explicit.ls_theta(raw, N, n), n)
    np.testing.assert_allclose(t_dir, t_exp, atol=1e-12, rtol=0)
    assert t_dir[0] == 1.0
    mu_d = direct.mu(t_dir, n)
    mu_e = explicit.mu_from_theta(explicit.ls_theta(raw, N, n), n)
    np.testing.assert_allclose(mu_d, mu_e, atol=1e-13)
    np.testing.assert_allclose(np.trace(mu_d), 1.0, atol=1e-14)
    np.testing.assert_allclose(mu_d, mu_d.conj().T, atol=0)


def test_weighted_shots_match_explicit():
    n = 3
    rng = np.random.default_rng(7)
    N = rng.integers(100, 2000, size=3 ** n)
    c = np.stack([rng.multinomial(int(x), np.ones(8) / 8) for x in N]).astype(np.int32)
    t_dir = direct.estimate(c, N, n)
    t_exp = explicit.expectations_from_theta(explicit.ls_theta(c, N, n), n)
    np.testing.assert_allclose(t_dir, t_exp, atol=1e-12)


def test_int16_counts_equal_int32():
    n = 3
    rng = np.random.default_rng(9)
    c = rng.multinomial(1000, np.ones(8) / 8, size=27).astype(np.int32)
    np.testing.assert_array_equal(direct.parity_sums(c, n)[0],
                                  direct.parity_sums(c.astype(np.int16), n)[0])


def test_mu_elements_match_full():
    n = 4
    rng = np.random.default_rng(5)
    t = rng.standard_normal(4 ** n)
    t[0] = 1.0
    full = direct.mu(t, n)
    r = rng.integers(0, 16, 40)
    cc = rng.integers(0, 16, 40)
    np.testing.assert_allclose(direct.mu_elements(t, n, r, cc), full[r, cc], atol=1e-15)


def test_mu_of_true_expectations_is_the_state():
    # Eq. (4) inverts Eq. (1): sum_i Tr(rho Omega_i) Omega_i = rho
    rho = st.ginibre_state(3, 2, seed=11)
    t = st.pauli_expectations(rho)
    np.testing.assert_allclose(direct.mu(t, 3), rho, atol=1e-14)


# --------------------------------------------------- projection (step iii)

def test_smolin_matches_simplex_projection():
    rng = np.random.default_rng(4)
    for _ in range(50):
        lam = np.sort(rng.standard_normal(16) * 0.2 + 1 / 16)[::-1]
        lam = lam - (lam.sum() - 1) / 16
        np.testing.assert_allclose(project.smolin_eigenvalues(lam),
                                   np.sort(project.simplex_projection(lam))[::-1], atol=1e-14)


def test_projection_optimality_and_psd_fixed_point():
    rng = np.random.default_rng(6)
    n = 3
    raw = rng.multinomial(20, np.ones(8) / 8, size=27).astype(np.int32)
    mu = direct.mu(direct.estimate(raw, 20, n), n)
    rho, lam_mu, lam = project.smolin(mu)
    assert lam_mu.min() < 0            # low shots: mu is unphysical
    w = np.linalg.eigvalsh(rho)
    assert w.min() > -1e-12
    np.testing.assert_allclose(np.trace(rho), 1.0, atol=1e-12)
    for s in range(30):
        sigma = st.ginibre_state(n, 1 + s % 4, seed=100 + s)
        ip = np.vdot(mu - rho, sigma - rho).real     # <mu-rho, sigma-rho>_F <= 0
        assert ip <= 1e-12
    # physical mu is a fixed point (Sec. V: large N_0)
    rho2, _, _ = project.smolin(rho)
    np.testing.assert_allclose(rho2, rho, atol=1e-13)


# --------------------------------------------------- Sec. V statistics

@pytest.mark.parametrize("n", [3, 4])
def test_maximally_mixed_mse_law(n):
    """E Tr(mu - rho)^2 = ((10/3)^n - 3^-n)/(d S) for the maximally-mixed
    state with S shots per basis; Sec. V's asymptote (1/N_0)(5/6)^n with
    N = 6^n N_0 is this without the 3^-n term."""
    d = 2 ** n
    S = 64
    thr = sc.cdf_thresholds(np.full((3 ** n, d), 1.0 / d))
    vals = []
    for seed in range(200):
        c = sc.sample_cdf(thr, S, seed)
        t = direct.estimate(c, S, n)
        err = t.copy()
        err[0] -= 1.0
        vals.append((err[1:] ** 2).sum() / d)
    vals = np.array(vals)
    want = ((10 / 3) ** n - 3.0 ** (-n)) / (d * S)
    se = vals.std(ddof=1) / np.sqrt(len(vals))
    assert abs(vals.mean() - want) < 4 * se, (vals.mean(), want, se)
    # a 1/(N 2^k) weight instead of 1/(N 3^k) would be far outside
    assert abs(vals.mean() - want) < 0.1 * want


def test_entry_spot_values_match_full_direct_sum():
    n = 5
    rng = np.random.default_rng(12)
    c = rng.multinomial(1000, np.ones(32) / 32, size=243).astype(np.int16)
    S, _ = direct.parity_sums(c, n)
    idx = rng.integers(0, 4 ** n, 64)
    np.testing.assert_array_equal(direct.parity_sum_entries(n, idx, lambda b: c[b]), S[idx])
    assert direct.compatible_bases(0, 1) == [0, 1, 2]
    assert direct.compatible_bases(4 * 3 + 0, 2) == [6, 7, 8]   # Z(x)I: a_1 = Z


@pytest.mark.parametrize("n", [4, 5])
def test_estimate_entries_match_full_estimate_every_k(n):
    # the per-entry checker used at full size (S_i / (N 3^k) over the 3^k
    # compatible groups) against the full direct sum, bit for bit, on every
    # index (so every identity count k = 0..n), and against the explicit
    # least-squares solve of Eq. (3) at n = 4 (independent of both)
    N = 997
    rng = np.random.default_rng(40 + n)
    p = rng.dirichlet(np.ones(2 ** n), size=3 ** n)
    c = np.stack([rng.multinomial(N, row) for row in p]).astype(np.int32)
    idx = np.arange(4 ** n)
    t_entries = direct.estimate_entries(n, idx, lambda b: c[b], N)
    t_full = direct.estimate(c, N, n)
    np.testing.assert_array_equal(t_entries, t_full)
    ks = np.array([direct.identity_letters(i, n) for i in idx])
    assert set(ks.tolist()) == set(range(n + 1))
    if n == 4:
        t_ls = explicit.expectations_from_theta(explicit.ls_theta(c, N, n), n)
        assert np.max(np.abs(t_entries - t_ls)) < 1e-12
    # identity letters are counted per base-4 digit, whatever its position
    assert direct.identity_letters(0, n) == n
    assert direct.identity_letters(3 * 4 ** (n - 1), n) == n - 1     # Z on qubit 1
    assert direct.identity_letters(1, n) == n - 1                    # X on qubit n
