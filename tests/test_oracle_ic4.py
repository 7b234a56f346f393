"""Pins of the 4^n-operator oracle (oracle/ic4.py; Sec. VI's variant, read
as the minimal informationally complete subset |0>, |1>, |+>, |+i> of the
Pauli eigenprojectors per qubit) against what the mathematics fixes."""
import numpy as np
import pytest

from oracle import direct, ic4
from synth import counts as sc
from synth import states as st


def test_single_qubit_rows_and_normal_matrix():
    s = 1 / np.sqrt(2)
    X1 = ic4.design_matrix(1)
    # |0><0| = (I+Z)/2, |1><1| = (I-Z)/2, |+><+| = (I+X)/2, |+i><+i| = (I+Y)/2
    np.testing.assert_allclose(X1, s * np.array([[1, 0, 0, 1], [1, 0, 0, -1], [1, 1, 0, 0], [1, 0, 1, 0]]),
                               atol=1e-15)
    G = np.array([[2, .5, .5, 0], [.5, .5, 0, 0], [.5, 0, .5, 0], [0, 0, 0, 1]])
    for n in (1, 2, 3):
        X = ic4.design_matrix(n)
        Gn = np.ones((1, 1))
        for _ in range(n):
            Gn = np.kron(Gn, G)
        np.testing.assert_allclose(X.T @ X, Gn, atol=1e-12)   # not diagonal, unlike Sec. III's
        assert X.shape == (4 ** n, 4 ** n) and np.linalg.matrix_rank(X) == 4 ** n   # square, invertible
        # every operator keeps 2^n nonzeros in the basis of Eq. (5): 4^n x 2^n = 8^n
        assert all(np.count_nonzero(np.abs(row) > 1e-12) == 2 ** n for row in X)


def test_sources_are_the_right_pauli_counts():
    assert ic4.source_index(0, 1) == (2, 0)       # |0>: Z basis, outcome 0
    assert ic4.source_index(1, 1) == (2, 1)       # |1>: Z basis, outcome 1
    assert ic4.source_index(2, 1) == (0, 0)       # |+>: X basis, +1
    assert ic4.source_index(3, 1) == (1, 0)       # |+i>: Y basis, +1
    assert ic4.source_index(2 * 4 + 1, 2) == (0 * 3 + 2, 0 * 2 + 1)   # |+> (x) |1>


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_exact_integer_form_equals_the_normal_equations(n):
    rng = np.random.default_rng(n)
    N = 500
    c = rng.multinomial(N, np.ones(2 ** n) / 2 ** n, size=3 ** n)
    t_ls = ic4.ls_theta(c, N, n) * 2.0 ** (n / 2)
    np.testing.assert_allclose(ic4.exact_theta(c, N, n), t_ls, atol=1e-12)
    np.testing.assert_allclose(ic4.kron_theta(c, N, n), t_ls, atol=1e-12)
    assert abs(np.abs(ic4.exact_sums(c, n)).max()) <= N * 3 ** n


def test_infinite_shot_counts_give_the_exact_expectations():
    # GHZ + white noise with rational Born probabilities: every operator
    # frequency is exact, so the estimate is the state's <P> (the whole
    # coefficient vector, including the ones the 4^n operators reach only
    # through the inverse of the non-diagonal X^T X)
    for n in (2, 3):
        d = 2 ** n
        N = 10 * d
        probs = st.born_probabilities(st.ghz_noise_expectations(n, 0.1), n)
        c = sc.exact_counts(probs, N)
        want = st.ghz_noise_expectations(n, 0.1)
        np.testing.assert_allclose(ic4.exact_theta(c, N, n), want, atol=1e-14)


def test_one_qubit_equals_the_pauli_estimate_and_differs_beyond():
    # with one qubit both estimators use every count of their bases alike
    c1 = np.array([[70, 30], [50, 50], [80, 20]])
    np.testing.assert_array_equal(ic4.exact_theta(c1, 100, 1), [1.0, 0.4, 0.0, 0.6])
    np.testing.assert_array_equal(direct.estimate(c1.astype(np.int32), 100, 1), [1.0, 0.4, 0.0, 0.6])
    # from two qubits on the 4^n form ignores the -1 outcomes of X and Y
    rng = np.random.default_rng(3)
    c = rng.multinomial(400, np.ones(4) / 4, size=9)
    assert not np.allclose(ic4.exact_theta(c, 400, 2), direct.estimate(c.astype(np.int32), 400, 2))
