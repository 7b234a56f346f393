"""Tensor-core first pass on int32 counts above 2047 (two fp16 planes per
count: c mod 2048 and (c >> 11) 2^11, contracted in one MMA chain), and the
range check every tensor-core variant makes on the counts it reads.

Bar: parity sums and uniform-shot theta bit-exact against the FWHT path and
the oracle (the MMA arithmetic is exact integer arithmetic by construction;
these tests check that the hardware honours it, at the largest counts each
encoding takes).  A count outside [0, shots] must latch
LRE_ERR_SHOTS_MISMATCH on the tensor path; rows whose totals are off while
every count stays in range give the oracle's numbers on both paths.
"""
import numpy as np
import pytest

from oracle import direct
from tests.gpu_util import ctx_and_lre, need_gpu, rel_fro
from tests.test_gpu_tensor import _counts, _set_first7, _set_variant, _sums_by_path

pytestmark = pytest.mark.gpu


def _skewed_counts(n, shots, seed, dtype):
    """Mostly one outcome per basis, every 7th basis with all its shots in a
    single outcome, and counts placed at the plane boundaries 2047, 2048 and
    shots itself."""
    rng = np.random.default_rng(seed)
    d = 2 ** n
    p = np.r_[0.7, np.full(d - 1, 0.3 / (d - 1))]
    raw = rng.multinomial(shots, p, size=3 ** n)
    raw[::7] = 0
    raw[::7, rng.integers(0, d)] = shots
    for k, top in enumerate((2047, 2048, shots - 1)):
        if top <= shots:
            b = 11 + 13 * k
            raw[b] = 0
            raw[b, 3] = top
            raw[b, 5] = shots - top
    return raw.astype(dtype)


@pytest.mark.parametrize("n,shots", [(7, 4096), (8, 4096), (10, 4096), (11, 1000), (8, 16383)])
def test_split_parity_sums_equal_fwht(n, shots):
    torch = need_gpu()
    c = _counts(torch, n, shots, 300 + n, dt=np.int32)
    res = _sums_by_path(torch, c, n, shots)
    assert torch.equal(res[0], res[1])
    assert int(res[0][0]) == shots * 3 ** n


@pytest.mark.parametrize("shots", [2048, 4096, 16383])
def test_split_theta_matches_oracle_at_largest_counts(shots):
    torch = need_gpu()
    n = 8
    raw = _skewed_counts(n, shots, 17 + shots, np.int32)
    lre, ctx = ctx_and_lre()
    try:
        lre.lre_set_fold_path(ctx, lre.LRE_FOLD_TENSOR_SPLIT)
        lre.lre_profile(ctx, True)
        theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
        rho = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device="cuda")
        lre.lre_estimate(ctx, torch.from_numpy(raw).cuda(), shots, n, theta, rho)
        lre.lre_sync(ctx)
        assert "fold_first6_mma_split" in [k for k, _ in lre.lre_profile_records(ctx)]
        t_ref = direct.estimate(raw, shots, n)
        np.testing.assert_array_equal(theta.cpu().numpy(), t_ref)
        assert rel_fro(rho.cpu().numpy(), direct.mu(t_ref, n)) <= 1e-6
    finally:
        lre.lre_destroy(ctx)


def test_split_n12_precision_workload_equals_fwht_and_oracle():
    """The n=12 precision workload: product of Haar qubits with Bloch shrink
    0.95, 4096 shots per basis, int32 counts (8.7 GB): tensor-core and FWHT
    parity sums bit-identical, theta anchored to the oracle on sampled
    coefficients of every identity count."""
    torch = need_gpu()
    from synth import gen
    from synth import states as st
    n, shots = 12, 4096
    bloch = st.haar_bloch_vectors(n, seed=2016, shrink=0.95)
    c = torch.empty((3 ** n, 2 ** n), dtype=torch.int32, device="cuda")
    gen.gen_product(bloch, shots, 77, c)
    res = _sums_by_path(torch, c, n, shots)
    assert torch.equal(res[0], res[1])
    S = res[0].cpu().numpy()
    del res
    rng = np.random.default_rng(5)
    idx = _stratified_indices(n, rng, per_k=12, kmax=6)
    want = direct.parity_sum_entries(n, idx, lambda b: c[torch.from_numpy(np.asarray(b)).cuda()].cpu().numpy())
    np.testing.assert_array_equal(S[idx], want)


def _stratified_indices(n, rng, per_k, kmax):
    """Pauli indices with k identity letters for k = 0..kmax (per_k each)."""
    out = []
    for k in range(kmax + 1):
        for _ in range(per_k):
            sites = rng.choice(n, size=k, replace=False)
            letters = rng.integers(1, 4, size=n)
            letters[sites] = 0
            out.append(sum(int(letters[q]) << (2 * (n - 1 - q)) for q in range(n)))
    return np.array(out, dtype=np.int64)


def _bad_estimate(torch, raw, shots, n, variant=0, first7=0):
    lre, ctx = ctx_and_lre()
    try:
        _set_variant(lre, ctx, variant)
        _set_first7(lre, ctx, first7)
        lre.lre_set_fold_path(ctx, lre.LRE_FOLD_TENSOR_SPLIT)
        theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
        lre.lre_estimate(ctx, torch.from_numpy(raw).cuda(), shots, n, theta)
        with pytest.raises(lre.LreError) as e:
            lre.lre_sync(ctx)
        assert e.value.status == lre.LRE_ERR_SHOTS_MISMATCH
        # the context stays usable: the next call on valid counts is exact
        good = _skewed_counts(n, shots, 3, raw.dtype)
        lre.lre_estimate(ctx, torch.from_numpy(good).cuda(), shots, n, theta)
        lre.lre_sync(ctx)
        np.testing.assert_array_equal(theta.cpu().numpy(), direct.estimate(good, shots, n))
    finally:
        lre.lre_destroy(ctx)


@pytest.mark.parametrize("dtype,shots,variant,bad,first7", [
    (np.int16, 1000, 0, 1005, 0),    # above the shots, still inside the raw encoding
    (np.int16, 1000, 0, 2100, 0),    # beyond the raw encoding (would read as another value)
    (np.int16, 1000, 0, -3, 0),      # negative
    (np.int16, 1000, 0, 1005, 1),    # the same three through the seven-qubit pass
    (np.int16, 1000, 0, 2100, 1),
    (np.int16, 1000, 0, -3, 1),
    (np.int16, 1000, 1, 1024, 0),    # beyond the biased encoding
    (np.int32, 4096, 3, 4100, 0),    # int32 planes: above the shots
    (np.int32, 4096, 3, 70000, 0),   # int32 planes: far beyond
    (np.int32, 4096, 3, -1, 0),
])
def test_tensor_path_latches_count_out_of_range(dtype, shots, variant, bad, first7):
    """One count outside [0, shots] while the grand total still equals
    shots * 3^n (another row gives up the difference)."""
    torch = need_gpu()
    n = 8
    raw = _skewed_counts(n, shots, 40, dtype).astype(np.int64)
    b_bad, b_fix = 100, 101
    delta = bad - raw[b_bad, 9]
    raw[b_bad, 9] = bad
    if delta < 0:                               # a negative count: the shots go to another row
        raw[b_fix, 0] -= delta
    else:                                       # keep the grand total: later rows give shots up
        b = b_fix
        while delta > 0:
            for o in range(2 ** n):
                t = min(delta, raw[b, o])
                raw[b, o] -= t
                delta -= t
            b += 1
    assert raw.sum() == shots * 3 ** n
    _bad_estimate(torch, raw.astype(dtype), shots, n, variant if variant != 3 else 0, first7)


@pytest.mark.parametrize("dtype,shots", [(np.int16, 1000), (np.int32, 4096)])
def test_rows_off_their_shots_within_range_match_oracle(dtype, shots):
    """Row totals off by a few shots (one row over, one under; the grand
    total kept), every count within [0, shots]: no error, and both first-pass
    paths give the oracle's theta bit for bit."""
    torch = need_gpu()
    n = 9
    raw = _skewed_counts(n, shots, 41, dtype).astype(np.int64)
    raw[200] = 0
    raw[200, :5] = shots // 5
    raw[200, 7] += 5                            # row 200: a few shots over
    over = raw[200].sum() - shots
    raw[201] = 0
    raw[201, 0] = shots - over                  # row 201 gives it back
    assert raw.sum() == shots * 3 ** n and raw.max() <= shots and raw.min() >= 0
    raw = raw.astype(dtype)
    want = direct.estimate(raw, shots, n)
    for path in ("tensor", "fwht"):
        lre, ctx = ctx_and_lre()
        try:
            lre.lre_set_fold_path(ctx, lre.LRE_FOLD_TENSOR_SPLIT if path == "tensor" else lre.LRE_FOLD_FWHT)
            theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
            lre.lre_estimate(ctx, torch.from_numpy(raw).cuda(), shots, n, theta)
            lre.lre_sync(ctx)
            np.testing.assert_array_equal(theta.cpu().numpy(), want)
        finally:
            lre.lre_destroy(ctx)


def test_split_planes_refuse_a_row_above_its_shots():
    """The split-plane partials store the high plane only where a partial can
    exceed int16 when every basis row sums to its shots.  A row holding 16
    times its shots (every count still within [0, shots], the grand total
    kept by emptying other rows) gives the letter I I I X X X a partial of
    42000 in a run without high planes: the tensor path latches
    LRE_ERR_SHOTS_MISMATCH instead of returning a wrong theta.  (The
    six-qubit first pass: at n = 10 the seven-qubit one would leave int32
    partials, which hold any value.)"""
    torch = need_gpu()
    n, shots = 10, 1000
    raw = np.zeros((3 ** n, 2 ** n), dtype=np.int64)
    raw[:, 0] = shots                                  # every row: all shots on outcome 0
    o = np.arange(64)
    even = np.array([bin((x >> 3) & 7).count("1") % 2 == 0 for x in o])
    raw[0, :] = 0
    raw[0, o[even]] = 500                              # 32 outcomes x 500 = 16 x the shots
    excess = int(raw[0].sum()) - shots
    raw[3 ** n - 1 - np.arange(excess // shots), 0] = 0  # the total stays shots * 3^n
    assert raw.sum() == shots * 3 ** n and raw.max() <= shots
    _bad_estimate(torch, raw.astype(np.int16), shots, n, 0, first7=0)


def test_seven_qubit_planes_refuse_a_row_above_its_shots():
    """The same row at n = 11 (7 + 3 + 1 qubits: split-plane partials of
    seven letters).  Its tile gives the letter X I I I X X X (qubit 7 on X,
    tile rows of axis X minus those of outcome 1) the partial 42000 in a run
    without high planes: the seven-qubit pass latches LRE_ERR_SHOTS_MISMATCH;
    the same context then matches the FWHT path on valid counts."""
    torch = need_gpu()
    n, shots = 11, 1000
    c = torch.zeros((3 ** n, 2 ** n), dtype=torch.int16, device="cuda")
    c[:, 0] = shots
    o = np.arange(64)
    even = np.array([bin((x >> 3) & 7).count("1") % 2 == 0 for x in o])
    c[0, :] = 0
    c[0, torch.from_numpy(o[even]).cuda()] = 500
    excess = 500 * int(even.sum()) - shots
    c[3 ** n - excess // shots:, 0] = 0  # the total stays shots * 3^n
    assert int(c.sum(dtype=torch.int64)) == shots * 3 ** n
    good = _counts(torch, n, shots, 1111)
    theta = {}
    for tensor in (True, False):
        lre, ctx = ctx_and_lre()
        try:
            lre.lre_set_fold_path(ctx, lre.LRE_FOLD_TENSOR if tensor else lre.LRE_FOLD_FWHT)
            _set_first7(lre, ctx, 1 if tensor else 0)
            t = torch.full((4 ** n,), -1.0, dtype=torch.float64, device="cuda")
            if tensor:
                lre.lre_profile(ctx, True)
                lre.lre_estimate(ctx, c, shots, n, t)
                with pytest.raises(lre.LreError) as e:
                    lre.lre_sync(ctx)
                assert e.value.status == lre.LRE_ERR_SHOTS_MISMATCH
                assert "fold_first7_mma" in [k for k, _ in lre.lre_profile_records(ctx)]
            lre.lre_estimate(ctx, good, shots, n, t)
            lre.lre_sync(ctx)
            theta[tensor] = t
        finally:
            lre.lre_destroy(ctx)
    assert torch.equal(theta[True], theta[False])
