"""CPU checks of the sampled parity helpers (tests/sampled.py) used at sizes
the oracle cannot finish whole: every sampled string's compatible bases lie
in its block, the check passes on the oracle's own theta over every identity
count, and it catches one planted wrong coefficient and one wrong rho
element."""
import numpy as np

from oracle import direct
from tests import sampled


def test_block_strings_draw_on_their_block_only():
    rng = np.random.default_rng(1)
    n, K = 9, 5
    idx, bases = sampled.block_entries(n, rng, K, {k: 10 for k in range(K + 1)})
    block = set(bases.tolist())
    assert len(block) == 3 ** K
    ks = set()
    for i in idx:
        assert set(direct.compatible_bases(int(i), n)) <= block
        ks.add(direct.identity_letters(int(i), n))
    assert ks == set(range(K + 1))


def test_sampled_theta_and_rho_checks_pass_and_catch_a_planted_error():
    n, N = 7, 500
    rng = np.random.default_rng(2)
    c = rng.multinomial(N, np.ones(2 ** n) / 2 ** n, size=3 ** n).astype(np.int16)
    t = direct.estimate(c, N, n)
    rows_for = lambda b: c[np.asarray(b)]
    q = {k: 6 for k in range(6)}
    checked, per_k, bad = sampled.check_theta_blocks(n, t, N, rows_for, np.random.default_rng(3), 3, 5, q)
    assert bad is None and checked > 0 and sorted(per_k) == list(range(6))
    idx, _ = sampled.block_entries(n, np.random.default_rng(3), 5, q)
    t_bad = t.copy()
    t_bad[idx[len(idx) // 2]] = np.nextafter(t_bad[idx[len(idx) // 2]], 2.0)   # one ulp off
    _, _, bad = sampled.check_theta_blocks(n, t_bad, N, rows_for, np.random.default_rng(3), 3, 5, q)
    assert bad is not None and bad[0] == idx[len(idx) // 2]
    mu = direct.mu(t, n).astype(np.complex64)
    sampled.check_rho_elements(n, t, lambda r, cc: mu[r, cc], np.random.default_rng(4), 300, 40)
    r0 = int(np.random.default_rng(4).integers(0, 2 ** n, 300)[0])   # the first sampled (diagonal) element
    mu[r0, r0] *= 1 + 1e-5
    try:
        sampled.check_rho_elements(n, t, lambda r, cc: mu[r, cc], np.random.default_rng(4), 300, 40)
        caught = False
    except AssertionError:
        caught = True
    assert caught
