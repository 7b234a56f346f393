"""Tensor-core form of the first fold pass (tcgen05.mma kind::f16, exact
small integers, FP32 accumulation in TMEM): bit-identical to the FWHT path
and to the oracle, for both operand encodings (raw counts read as fp16 bit
patterns, and fp16(1024 + c)), and the raw pass folding seven qubits
bit-identical to the six-qubit one."""
import ctypes

import numpy as np
import pytest

from oracle import direct
from tests.gpu_util import ctx_and_lre, need_gpu

pytestmark = pytest.mark.gpu


def _counts(torch, n, shots, seed, dt=np.int16):
    from synth import gen
    c = torch.empty((3 ** n, 2 ** n), dtype=torch.int16 if dt == np.int16 else torch.int32, device="cuda")
    gen.gen_ghz(n, 0.05, shots, seed, c)
    return c


def _set_variant(lre, ctx, biased):
    f = lre.load().lre_debug_set_mma_variant
    f.argtypes = [ctypes.c_void_p, ctypes.c_int]
    f.restype = ctypes.c_int
    assert f(ctx, biased) == 0


def _sums_by_path(torch, c, n, bound, biased=0):
    """Parity sums through the tensor-core path, then the FWHT path, each in
    a context of its own (no workspace shared between the two)."""
    res = []
    for tensor in (True, False):
        lre, ctx = ctx_and_lre()
        try:
            _set_variant(lre, ctx, biased)
            lre.lre_set_fold_path(ctx, lre.LRE_FOLD_TENSOR_SPLIT if tensor else lre.LRE_FOLD_FWHT)
            S = torch.full((4 ** n,), -1, dtype=torch.int64, device="cuda")
            lre.lre_profile(ctx, True)
            lre.lre_parity_sums(ctx, c, n, S, row_total_bound=bound)
            lre.lre_sync(ctx)
            names = [k for k, _ in lre.lre_profile_records(ctx)]
            assert any(k.startswith(("fold_first6_mma", "fold_first7_mma")) for k in names) == tensor, names
            res.append(S)
        finally:
            lre.lre_destroy(ctx)
    return res


@pytest.mark.parametrize("biased", [0, 1])
@pytest.mark.parametrize("n", [7, 8, 10, 11])
def test_tensor_parity_sums_equal_fwht(n, biased):
    torch = need_gpu()
    c = _counts(torch, n, 1000, 90 + n)
    res = _sums_by_path(torch, c, n, 1000, biased)
    assert torch.equal(res[0], res[1])


@pytest.mark.parametrize("biased,top", [(0, 2047), (1, 1023)])
def test_tensor_theta_matches_oracle_at_largest_counts(biased, top):
    """Counts up to the largest value each encoding keeps exact; one count
    above it sends the call down the FWHT path, still exact."""
    torch = need_gpu()
    lre, ctx = ctx_and_lre()
    try:
        _set_variant(lre, ctx, biased)
        lre.lre_set_fold_path(ctx, lre.LRE_FOLD_TENSOR)
        n = 8
        rng = np.random.default_rng(3 + biased)
        p = np.r_[0.9, np.full(2 ** n - 1, 0.1 / (2 ** n - 1))]
        raw = rng.multinomial(top, p, size=3 ** n)
        raw[::7, 0] = top  # full-weight rows: every count in one outcome
        raw[::7, 1:] = 0
        raw = raw.astype(np.int16)
        theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
        lre.lre_estimate(ctx, torch.from_numpy(raw).cuda(), top, n, theta)
        lre.lre_sync(ctx)
        np.testing.assert_array_equal(theta.cpu().numpy(), direct.estimate(raw, top, n))
        raw2 = rng.multinomial(top + 1, np.ones(2 ** n) / 2 ** n, size=3 ** n).astype(np.int16)
        lre.lre_estimate(ctx, torch.from_numpy(raw2).cuda(), top + 1, n, theta)
        lre.lre_sync(ctx)
        np.testing.assert_array_equal(theta.cpu().numpy(), direct.estimate(raw2, top + 1, n))
    finally:
        lre.lre_destroy(ctx)


def test_tensor_first_pass_n12_equals_fwht():
    """Headline-shaped case: many tiles per CTA, both level-B warp pairs and
    every ring slot in use."""
    torch = need_gpu()
    n = 12
    c = _counts(torch, n, 1000, 1234)
    res = _sums_by_path(torch, c, n, 1000)
    assert torch.equal(res[0], res[1])
    assert int(res[0][0]) == 1000 * 3 ** n


def _bound_rows(torch, n, shots, seed):
    """GHZ + noise counts with two whole tile rows (729 consecutive bases)
    driven to the partial-sum bound: every shot in outcome 0 (all partials
    +3^k N) and every shot in the all-ones outcome (sign by parity)."""
    c = _counts(torch, n, shots, seed)
    c[0:729] = 0
    c[0:729, 0] = shots
    c[729:1458] = 0
    c[729:1458, 2 ** n - 1] = shots
    return c


# shots per basis around the partial-sum sizes the split planes meet: 729 x 44
# fits int16 and 729 x 45 does not (the all-identity partial), 2047 is the
# largest raw count (729 x 2047 < 2^21 in the 24-bit planes).
@pytest.mark.parametrize("shots", [44, 45, 1000, 2047])
def test_split_planes_at_bound_partials_equal_fwht(shots):
    torch = need_gpu()
    n = 10
    c = _bound_rows(torch, n, shots, 500 + shots)
    res = _sums_by_path(torch, c, n, shots)
    assert torch.equal(res[0], res[1])
    assert int(res[0][0]) == shots * 3 ** n


def test_split_plane_theta_matches_oracle():
    """theta through the tensor first pass and the split planes, with whole
    tile rows at the partial-sum bound, against the oracle."""
    torch = need_gpu()
    lre, ctx = ctx_and_lre()
    try:
        n, shots = 10, 45
        lre.lre_set_fold_path(ctx, lre.LRE_FOLD_TENSOR)
        c = _bound_rows(torch, n, shots, 77)
        theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
        lre.lre_estimate(ctx, c, shots, n, theta)
        lre.lre_sync(ctx)
        np.testing.assert_array_equal(theta.cpu().numpy(), direct.estimate(c.cpu().numpy(), shots, n))
    finally:
        lre.lre_destroy(ctx)


@pytest.mark.parametrize("n,consumers,discard", [(10, 0, 0), (11, 0, 0), (12, 0, 0), (12, 1, 0), (12, 100, 1),
                                                 (12, 0, 1)])
def test_fused_first_and_second_pass_equals_unfused(n, consumers, discard):
    """The tensor-core first pass fused with the second through an L2 ring
    (test hook: first-pass variant 2; consumers: CTAs on the second pass, 0
    the default; discard: consumed ring lines dropped from L2) gives the
    unfused path's parity sums and theta bit for bit."""
    torch = need_gpu()
    c = _counts(torch, n, 1000, 60 + n)
    out = []
    for variant in (1, 2):
        lre, ctx = ctx_and_lre()
        try:
            f = lre.load().lre_debug_set_first_pass
            f.argtypes = [ctypes.c_void_p, ctypes.c_int]
            f.restype = ctypes.c_int
            assert f(ctx, variant) == 0
            g = lre.load().lre_debug_set_fused_consumers
            g.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
            g.restype = ctypes.c_int
            assert g(ctx, consumers, discard) == 0
            lre.lre_profile(ctx, True)
            S = torch.full((4 ** n,), -1, dtype=torch.int64, device="cuda")
            lre.lre_parity_sums(ctx, c, n, S, row_total_bound=1000)
            theta = torch.full((4 ** n,), float("nan"), dtype=torch.float64, device="cuda")
            lre.lre_estimate(ctx, c, 1000, n, theta)
            lre.lre_sync(ctx)
            names = [k for k, _ in lre.lre_profile_records(ctx)]
            assert ("fold_first9_mma" in names) == (variant == 2), names
            out.append((S, theta))
        finally:
            lre.lre_destroy(ctx)
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


def _set_first7(lre, ctx, on):
    f = lre.load().lre_debug_set_first7
    f.argtypes = [ctypes.c_void_p, ctypes.c_int]
    f.restype = ctypes.c_int
    assert f(ctx, on) == 0


def _set_generic_tma(lre, ctx, on):
    f = lre.load().lre_debug_set_generic_tma
    f.argtypes = [ctypes.c_void_p, ctypes.c_int]
    f.restype = ctypes.c_int
    assert f(ctx, on) == 0


def _sums_six_seven(torch, c, n, bound, generic_tma=1):
    """Parity sums with the seven-qubit raw first pass, then the six-qubit
    one, each in a context of its own, outputs pre-filled."""
    res = []
    for on in (1, 0):
        lre, ctx = ctx_and_lre()
        try:
            _set_first7(lre, ctx, on)
            _set_generic_tma(lre, ctx, generic_tma)
            lre.lre_set_fold_path(ctx, lre.LRE_FOLD_TENSOR)
            S = torch.full((4 ** n,), -1, dtype=torch.int64, device="cuda")
            lre.lre_profile(ctx, True)
            lre.lre_parity_sums(ctx, c, n, S, row_total_bound=bound)
            lre.lre_sync(ctx)
            names = [k for k, _ in lre.lre_profile_records(ctx)]
            assert ("fold_first7_mma" in names) == bool(on), names
            assert ("fold_first6_mma" in names) == (not on), names
            res.append(S)
        finally:
            lre.lre_destroy(ctx)
    return res


# 8 = 7+1 and 9 = 7+2 (int32 partials: the next pass is the last), 10 = 7+3,
# 11 = 7+3+1, 12 = 7+3+2 and 13 = 7+3+3 (split-plane partials)
@pytest.mark.parametrize("n", [8, 9, 10, 11, 12, 13])
def test_seven_qubit_first_pass_equals_six(n):
    torch = need_gpu()
    c = _counts(torch, n, 1000, 700 + n)
    a, b = _sums_six_seven(torch, c, n, 1000)
    assert torch.equal(a, b)
    assert int(a[0]) == 1000 * 3 ** n


def test_seven_qubit_int32_partials_equal_six():
    """Without the TMA-staged second pass the seven-qubit pass writes int32
    partials instead of split planes."""
    torch = need_gpu()
    n = 11
    c = _counts(torch, n, 1000, 811)
    a, b = _sums_six_seven(torch, c, n, 1000, generic_tma=0)
    assert torch.equal(a, b)


# shots around the seven-qubit partial sizes: 2187 x 14 fits int16 and 2187 x
# 15 does not (the all-identity partial), 729 x 44 / 45 the same for six
# identities, 2047 the largest raw count (2187 x 2047 < 2^23).
@pytest.mark.parametrize("shots", [14, 15, 44, 45, 2047])
def test_seven_qubit_split_planes_at_bound_partials(shots):
    """Three whole tile rows (one supertile row, 3 x 729 bases) with every
    shot in outcome 0, three more with every shot in the all-ones outcome:
    the partials of seven qubits reach +-3^k N."""
    torch = need_gpu()
    n = 11
    c = _counts(torch, n, shots, 900 + shots)
    c[0:2187] = 0
    c[0:2187, 0] = shots
    c[2187:4374] = 0
    c[2187:4374, 2 ** n - 1] = shots
    a, b = _sums_six_seven(torch, c, n, shots)
    assert torch.equal(a, b)
    fwht = _sums_by_path(torch, c, n, shots)[1]
    assert torch.equal(a, fwht)


@pytest.mark.parametrize("n", [8, 9])
def test_seven_qubit_theta_matches_oracle(n):
    """theta through the seven-qubit pass against the oracle's direct sums,
    counts up to the largest raw count with full-weight rows."""
    torch = need_gpu()
    lre, ctx = ctx_and_lre()
    try:
        lre.lre_set_fold_path(ctx, lre.LRE_FOLD_TENSOR)
        _set_first7(lre, ctx, 1)
        top = 2047
        rng = np.random.default_rng(40 + n)
        p = np.r_[0.5, np.full(2 ** n - 1, 0.5 / (2 ** n - 1))]
        raw = rng.multinomial(top, p, size=3 ** n)
        raw[::5, 0] = top
        raw[::5, 1:] = 0
        raw[1::11, :] = 0
        raw[1::11, -1] = top
        raw = raw.astype(np.int16)
        theta = torch.full((4 ** n,), -1.0, dtype=torch.float64, device="cuda")
        lre.lre_profile(ctx, True)
        lre.lre_estimate(ctx, torch.from_numpy(raw).cuda(), top, n, theta)
        lre.lre_sync(ctx)
        assert "fold_first7_mma" in [k for k, _ in lre.lre_profile_records(ctx)]
        np.testing.assert_array_equal(theta.cpu().numpy(), direct.estimate(raw, top, n))
    finally:
        lre.lre_destroy(ctx)
