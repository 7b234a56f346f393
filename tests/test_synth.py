"""Seeded input generators: known-answer vectors and law checks."""
import numpy as np
import pytest

from synth import counts as sc
from synth import states as st
from synth.philox import philox4x32


def test_philox_known_answers():
    # Known-answer vectors of Philox4x32-10 (Salmon et al., SC'11 reference suite)
    cases = [
        ((0, 0, 0, 0), (0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
        ((0xffffffff,) * 4, (0xffffffff,) * 2, (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
        ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
         (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
    ]
    for ctr, key, want in cases:
        got = philox4x32(*ctr, *key)
        assert tuple(int(x) for x in got) == want


@pytest.mark.parametrize("n", [1, 2, 3])
def test_born_fast_matches_direct(n):
    rho = st.ginibre_state(n, 2, seed=n)
    fast = st.born_probabilities(st.pauli_expectations(rho), n)
    np.testing.assert_allclose(fast, st.born_probabilities_direct(rho), atol=1e-14)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_ghz_closed_form_matches_state(n):
    np.testing.assert_allclose(st.pauli_expectations(st.ghz_noise_state(n, 0.1)),
                               st.ghz_noise_expectations(n, 0.1), atol=1e-14)


def _tv(counts, probs):
    f = counts / counts.sum(axis=1, keepdims=True)
    return np.abs(f - probs).sum(axis=1).max()


def test_ghz_direct_sampler_follows_born_law():
    n = 3
    probs = st.born_probabilities(st.ghz_noise_expectations(n, 0.05), n)
    c = sc.sample_ghz(n, 0.05, 200000, seed=1)
    assert np.all(c.sum(axis=1) == 200000)
    assert _tv(c, probs) < 0.01


def test_product_sampler_follows_born_law():
    n = 3
    bloch = st.haar_bloch_vectors(n, seed=2, shrink=0.95)
    probs = st.born_probabilities_direct(st.product_state(bloch))
    c = sc.sample_product(bloch, 200000, seed=3)
    assert _tv(c, probs) < 0.01


def test_cdf_sampler_follows_born_law_and_subsets():
    n = 2
    probs = st.born_probabilities(st.pauli_expectations(st.ginibre_state(n, 2, seed=5)), n)
    thr = sc.cdf_thresholds(probs)
    c = sc.sample_cdf(thr, 100000, seed=4)
    assert _tv(c, probs) < 0.01
    sub = sc.sample_cdf(thr, 100000, seed=4, bases=[3, 7])
    np.testing.assert_array_equal(sub, c[[3, 7]])
    sub = sc.sample_ghz(4, 0.1, 1000, seed=9, bases=[5, 80])
    np.testing.assert_array_equal(sub, sc.sample_ghz(4, 0.1, 1000, seed=9)[[5, 80]])


def test_mixed_splitting_sampler_is_the_multinomial_of_I_over_d():
    # rows sum to the shots exactly; every count has the Binomial(S, 1/d)
    # mean and variance; the root split (qubit 1) is Binomial(S, 1/2);
    # subsets of bases reproduce the full draw
    n, S = 4, 100000
    d = 2 ** n
    c = sc.sample_mixed(n, S, seed=21)
    assert np.all(c.sum(axis=1) == S)
    x = c.astype(np.float64).ravel()
    mean, var = S / d, S / d * (1 - 1 / d)
    assert abs(x.mean() - mean) < 1e-9                      # the totals fix the mean exactly
    assert abs(x.var() / var - 1) < 0.15
    half = c[:, : d // 2].sum(axis=1).astype(np.float64)   # outcomes with o_1 = 0
    assert abs(half.mean() - S / 2) < 4 * np.sqrt(S / 4 / len(half))
    assert abs(half.var() / (S / 4) - 1) < 0.4
    np.testing.assert_array_equal(sc.sample_mixed(n, S, seed=21, bases=[5, 44]), c[[5, 44]])


def test_fair_binomial_counts_the_set_bits_of_its_stream():
    # brute force on one node: the first c bits of the stream, one at a time
    from synth.philox import philox4x32, seed_key
    k0, k1 = seed_key(77)
    for c in (1, 31, 32, 33, 127, 128, 129, 300):
        bits = []
        for g in range((c + 127) // 128):
            w = philox4x32(np.uint32(g), np.uint32(9), sc.STREAM_SPLIT, np.uint32(5), k0, k1)
            for k in range(4):
                v = int(w[k])
                bits.extend((v >> i) & 1 for i in range(32))
        want = sum(bits[:c])
        got = sc.fair_binomial(np.array([c]), np.array([9]), 5, k0, k1)[0]
        assert got == want, (c, got, want)
