"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bar (from the method's arithmetic):
  * integer parity sums S and uniform-shot theta: bit-exact (theta is one
    correctly rounded FP64 division of two exact integers on both sides);
  * per-basis-shot theta: |dtheta| <= 1e-12 (FP64 sums in a different order);
  * rho (complex64 output of an FP64 butterfly): relative Frobenius <= 1e-6;
  * projection: relative Frobenius <= 1e-6 against the oracle's projection of
    the same complex64 mu, spectra within 1e-9.
"""
import numpy as np
import pytest

from oracle import direct, project
from synth import counts as sc
from synth import states as st
from tests.gpu_util import ctx_and_lre, need_gpu, rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    lre, ctx = ctx_and_lre()
    yield torch, lre, ctx
    lre.lre_destroy(ctx)


def _ginibre_counts(n, N, seed, dtype=np.int32):
    rho = st.ginibre_state(n, 2, seed=seed)
    thr = sc.cdf_thresholds(st.born_probabilities(st.pauli_expectations(rho), n))
    return sc.sample_cdf(thr, N, seed=seed + 1, dtype=dtype)


@pytest.mark.parametrize("path", ["tensor", "fwht"])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("dtype", [np.int32, np.int16])
def test_theta_bit_exact_and_rho(env, n, dtype, path):
    """Both first-pass paths (the tensor-core one applies to int16 counts with
    n >= 6; every other case runs the FWHT kernels under either setting)."""
    torch, lre, ctx = env
    N = 1000
    counts = _ginibre_counts(n, N, seed=10 * n, dtype=dtype)
    c = torch.from_numpy(counts).cuda()
    theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
    rho = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device="cuda")
    lre.lre_set_fold_path(ctx, lre.LRE_FOLD_TENSOR if path == "tensor" else lre.LRE_FOLD_FWHT)
    try:
        lre.lre_estimate(ctx, c, N, n, theta, rho)
        lre.lre_sync(ctx)
    finally:
        lre.lre_set_fold_path(ctx, lre.LRE_FOLD_TENSOR)
    t_ref = direct.estimate(counts, N, n)
    np.testing.assert_array_equal(theta.cpu().numpy(), t_ref)
    assert rel_fro(rho.cpu().numpy(), direct.mu(t_ref, n)) <= 1e-6


@pytest.mark.parametrize("n,bound", [(3, 0), (6, 0), (7, 0), (7, 1000), (8, 1000)])
def test_parity_sums_bit_exact(env, n, bound):
    torch, lre, ctx = env
    counts = _ginibre_counts(n, 1000, seed=77 + n)
    S = torch.empty(4 ** n, dtype=torch.int64, device="cuda")
    lre.lre_parity_sums(ctx, torch.from_numpy(counts).cuda(), n, S, row_total_bound=bound)
    lre.lre_sync(ctx)
    np.testing.assert_array_equal(S.cpu().numpy(), direct.parity_sums(counts, n)[0])


@pytest.mark.parametrize("n", [2, 5, 7])
def test_per_basis_shots(env, n):
    torch, lre, ctx = env
    rng = np.random.default_rng(n)
    N = rng.integers(500, 10001, size=3 ** n)
    probs = st.born_probabilities(st.pauli_expectations(st.ginibre_state(n, 3, seed=n)), n)
    probs = np.clip(probs, 0, None)
    probs /= probs.sum(axis=1, keepdims=True)
    counts = np.stack([rng.multinomial(int(N[b]), probs[b]) for b in range(3 ** n)]).astype(np.int32)
    theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
    lre.lre_estimate(ctx, torch.from_numpy(counts).cuda(), torch.from_numpy(N.astype(np.int64)).cuda(),
                     n, theta)
    lre.lre_sync(ctx)
    np.testing.assert_allclose(theta.cpu().numpy(), direct.estimate(counts, N, n), atol=1e-12, rtol=0)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_assemble_matches_direct_mu(env, n):
    torch, lre, ctx = env
    rng = np.random.default_rng(100 + n)
    t = rng.uniform(-1, 1, 4 ** n)
    t[0] = 1.0
    rho = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device="cuda")
    lre.lre_assemble(ctx, torch.from_numpy(t).cuda(), n, rho)
    lre.lre_sync(ctx)
    assert rel_fro(rho.cpu().numpy(), direct.mu(t, n)) <= 1e-6


@pytest.mark.parametrize("n,N", [(1, 100), (2, 20), (3, 30), (5, 50), (7, 100)])
def test_projection_matches_oracle(env, n, N):
    torch, lre, ctx = env
    counts = _ginibre_counts(n, N, seed=300 + n)
    theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
    mu = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device="cuda")
    lre.lre_estimate(ctx, torch.from_numpy(counts).cuda(), N, n, theta, mu)
    out = torch.empty_like(mu)
    em = torch.empty(2 ** n, dtype=torch.float64, device="cuda")
    er = torch.empty(2 ** n, dtype=torch.float64, device="cuda")
    lre.lre_project(ctx, mu, n, out, em, er)
    lre.lre_sync(ctx)
    mu_h = mu.cpu().numpy().astype(np.complex128)
    ref, lam_mu, lam = project.smolin(mu_h)
    assert rel_fro(out.cpu().numpy(), ref) <= 1e-6
    np.testing.assert_allclose(em.cpu().numpy(), lam_mu, atol=1e-9)
    np.testing.assert_allclose(er.cpu().numpy(), lam, atol=1e-9)
    w = np.linalg.eigvalsh(out.cpu().numpy().astype(np.complex128))
    assert w.min() > -1e-6 and abs(np.trace(out.cpu().numpy()) - 1) < 1e-5


def test_projection_of_physical_state_is_identity(env):
    torch, lre, ctx = env
    n = 4
    m = st.ginibre_state(n, 16, seed=5).astype(np.complex64)
    m = np.triu(m) + np.triu(m, 1).conj().T          # exactly Hermitian in complex64
    m[np.diag_indices(2 ** n)] = m.diagonal().real
    mu = torch.from_numpy(m).cuda()
    out = torch.empty_like(mu)
    lre.lre_project(ctx, mu, n, out)
    lre.lre_sync(ctx)
    np.testing.assert_array_equal(out.cpu().numpy(), mu.cpu().numpy())


@pytest.mark.parametrize("n,B,S", [(5, 243, 777), (5, 243, 800), (2, 9, 40), (10, 300, 4096),
                                   (14, 40, 32760)])
def test_histogram_ingest(env, n, B, S):
    """Scalar and eight-records-per-load paths (S a multiple of 8 or not),
    the generic kernel below n = 3, packed 16-bit bins up to 32760 shots in
    one bin."""
    torch, lre, ctx = env
    rng = np.random.default_rng(8 + n)
    rec = rng.integers(0, 2 ** n, size=(B, S)).astype(np.uint16)
    rec[0, :] = 2 ** n - 1      # every shot in one bin (odd index: the high half of a word)
    rec[1, :] = 0               # and in bin 0
    want = np.stack([np.bincount(r, minlength=2 ** n) for r in rec.astype(np.int64)])
    dev = torch.from_numpy(rec.view(np.int16)).cuda()
    for dt in (torch.int32, torch.int16):
        out = torch.full((B, 2 ** n), -3, dtype=dt, device="cuda")
        lre.lre_histogram(ctx, dev, n, out)
        lre.lre_sync(ctx)
        np.testing.assert_array_equal(out.cpu().numpy(), want)


def test_histogram_rejects_out_of_range_record(env):
    torch, lre, ctx = env
    n = 6
    rec = np.zeros((27, 64), dtype=np.uint16)
    rec[5, 7] = 2 ** n
    out = torch.empty((27, 2 ** n), dtype=torch.int16, device="cuda")
    lre.lre_histogram(ctx, torch.from_numpy(rec.view(np.int16)).cuda(), n, out)
    with pytest.raises(lre.LreError) as e:
        lre.lre_sync(ctx)
    assert e.value.status == lre.LRE_ERR_INVALID_ARG


def test_device_generators_match_cpu(env):
    torch, lre, ctx = env
    from synth import gen
    n = 6
    c = torch.empty((3 ** n, 2 ** n), dtype=torch.int16, device="cuda")
    gen.gen_ghz(n, 0.05, 1000, 42, c)
    np.testing.assert_array_equal(c.cpu().numpy(), sc.sample_ghz(n, 0.05, 1000, 42, dtype=np.int16))
    bloch = st.haar_bloch_vectors(n, seed=3, shrink=0.95)
    c32 = torch.empty((3 ** n, 2 ** n), dtype=torch.int32, device="cuda")
    gen.gen_product(bloch, 500, 7, c32)
    np.testing.assert_array_equal(c32.cpu().numpy(), sc.sample_product(bloch, 500, 7))
    probs = st.born_probabilities(st.pauli_expectations(st.ginibre_state(4, 2, seed=1)), 4)
    thr = sc.cdf_thresholds(probs)
    c4 = torch.empty((81, 16), dtype=torch.int32, device="cuda")
    gen.gen_cdf(torch.from_numpy(thr.view(np.int32)).cuda(), 4, 1000, 5, c4)
    np.testing.assert_array_equal(c4.cpu().numpy(), sc.sample_cdf(thr, 1000, 5))


def test_errors_and_latched_status(env):
    torch, lre, ctx = env
    n = 3
    counts = torch.from_numpy(_ginibre_counts(n, 100, seed=1)).cuda()
    theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
    with pytest.raises(lre.LreError) as e:
        lre.lre_estimate(ctx, counts, 0, n, theta)
    assert e.value.status == lre.LRE_ERR_INVALID_ARG
    with pytest.raises(lre.LreError) as e:
        lre.lre_estimate(ctx, counts, 100, 15, theta)
    assert e.value.status == lre.LRE_ERR_UNSUPPORTED
    lre.lre_estimate(ctx, counts, 101, n, theta)      # wrong shots: latched, not raised
    with pytest.raises(lre.LreError) as e:
        lre.lre_sync(ctx)
    assert e.value.status == lre.LRE_ERR_SHOTS_MISMATCH
    lre.lre_sync(ctx)                                # cleared
    ctx2 = lre.lre_create(0)
    try:
        lre.lre_set_workspace_limit(ctx2, 1024)
        big = torch.from_numpy(_ginibre_counts(8, 100, seed=2)).cuda()
        th = torch.empty(4 ** 8, dtype=torch.float64, device="cuda")
        with pytest.raises(lre.LreError) as e:
            lre.lre_estimate(ctx2, big, 100, 8, th)
        assert e.value.status == lre.LRE_ERR_OOM
    finally:
        lre.lre_destroy(ctx2)


@pytest.mark.parametrize("n,kind,chunk", [(6, "records", 0), (7, "i16", 0), (8, "i32", 0), (3, "records", 0),
                                         (9, "records", 1), (9, "i16", 1500000), (10, "records", 3000000),
                                         (8, "i32", 1)])
def test_estimate_host_matches_device_path(env, n, kind, chunk):
    """End to end from pinned host memory (records histogrammed on device)
    gives the same bits as the device path and the oracle; chunk > 0 forces
    small streamed chunks (rounded up to one tile row of 729 bases), so the
    first fold pass runs on many chunks."""
    torch, lre, ctx = env
    import ctypes
    L = lre.load()
    f = L.lre_debug_set_host_chunk
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    f.restype = ctypes.c_int
    assert f(ctx, chunk if chunk else 256 << 20) == 0
    from synth import gen
    N = 1000
    if kind == "records":
        rec_dev = torch.empty((3 ** n, N), dtype=torch.int16, device="cuda")
        gen.gen_ghz_records(n, 0.05, 31, rec_dev)
        rec = rec_dev.cpu().numpy().view(np.uint16)
        np.testing.assert_array_equal(rec, sc.ghz_sample_outcomes(n, int(sc.prob_threshold(0.05)), N, 31,
                                                                  np.arange(3 ** n)))
        host_in = torch.from_numpy(rec.view(np.int16)).pin_memory()
        counts = np.stack([np.bincount(r, minlength=2 ** n) for r in rec.astype(np.int64)]).astype(np.int32)
        hk = lre.LRE_HOST_RECORDS_U16
    else:
        dt = np.int16 if kind == "i16" else np.int32
        counts = _ginibre_counts(n, N, seed=n, dtype=dt)
        host_in = torch.from_numpy(counts).pin_memory()
        hk = lre.LRE_HOST_COUNTS_I16 if kind == "i16" else lre.LRE_HOST_COUNTS_I32
    th = torch.empty(4 ** n, dtype=torch.float64).pin_memory()
    rh = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64).pin_memory()
    try:
        lre.lre_estimate_host(ctx, host_in, hk, N, n, th, rh)
    finally:
        assert f(ctx, 256 << 20) == 0
    t_ref = direct.estimate(counts, N, n)
    np.testing.assert_array_equal(th.numpy(), t_ref)
    assert rel_fro(rh.numpy(), direct.mu(t_ref, n)) <= 1e-6


@pytest.mark.parametrize("n,shift", [(10, 0), (11, 0), (12, 0), (13, 0), (10, 1), (12, 1)])
def test_assemble_tiled_passes_sampled(env, n, shift):
    """n >= 10 uses the shared-memory tiled passes (6 + 4 + ... qubits) on the
    Hermitian half, and a mirror pass for the rest of rho; shift = 1 hands
    theta over at an address that is 8 but not 16 bytes aligned: the same
    bits."""
    torch, lre, ctx = env
    rng = np.random.default_rng(500 + n)
    t = rng.uniform(-1, 1, 4 ** n)
    t[0] = 1.0
    d = 2 ** n
    rho = torch.empty((d, d), dtype=torch.complex64, device="cuda")
    if shift:
        buf = torch.empty(4 ** n + 2, dtype=torch.float64, device="cuda")
        th = buf[1:1 + 4 ** n]
        assert th.data_ptr() % 16 == 8
        th.copy_(torch.from_numpy(t))
        lre.lre_assemble(ctx, th, n, rho)
        aligned = torch.empty_like(rho)
        lre.lre_assemble(ctx, torch.from_numpy(t).cuda(), n, aligned)
        lre.lre_sync(ctx)
        assert torch.equal(rho, aligned)
    else:
        lre.lre_assemble(ctx, torch.from_numpy(t).cuda(), n, rho)
    lre.lre_sync(ctx)
    r = rng.integers(0, d, 300)
    c = rng.integers(0, d, 300)
    r[:20] = c[:20]                                   # include diagonal elements
    ref = direct.mu_elements(t, n, r, c)
    got = rho[torch.from_numpy(r).cuda(), torch.from_numpy(c).cuda()].cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-6 * np.max(np.abs(ref))
    tr = torch.diagonal(rho).sum().item()
    assert abs(tr - 1) < 1e-4
    assert torch.equal(rho, rho.conj().T)             # exactly Hermitian


@pytest.mark.parametrize("n,chunk,mode", [(9, 1, "forced"), (10, 3000000, "forced"), (8, 0, "forced"),
                                          (10, 3000000, "limit")])
def test_estimate_host_records_without_dense_counts(env, n, chunk, mode):
    """Shot records folded by the tensor-core first pass from tile-grouped
    records (no dense device counts), forced by the test hook or chosen
    because the workspace limit leaves no room for the dense counts: the same
    bits as the device path and the oracle."""
    torch, lre, ctx0 = env
    import ctypes
    from synth import gen
    ctx = lre.lre_create(0)
    L = lre.load()
    hooks = {}
    for name in ("lre_debug_set_host_chunk", "lre_debug_set_records_direct"):
        f = getattr(L, name)
        f.argtypes = [ctypes.c_void_p, ctypes.c_int64 if name.endswith("chunk") else ctypes.c_int]
        f.restype = ctypes.c_int
        hooks[name] = f
    try:
        N = 1000
        assert hooks["lre_debug_set_host_chunk"](ctx, chunk if chunk else 256 << 20) == 0
        if mode == "forced":
            assert hooks["lre_debug_set_records_direct"](ctx, 1) == 0
        else:
            lre.lre_set_workspace_limit(ctx, 100 << 20)  # room for the records path, not for dense counts
        rec_dev = torch.empty((3 ** n, N), dtype=torch.int16, device="cuda")
        gen.gen_ghz_records(n, 0.05, 77 + n, rec_dev)
        rec = rec_dev.cpu().numpy().view(np.uint16)
        host_in = torch.from_numpy(rec.view(np.int16)).pin_memory()
        counts = np.stack([np.bincount(r, minlength=2 ** n) for r in rec.astype(np.int64)]).astype(np.int32)
        th = torch.empty(4 ** n, dtype=torch.float64).pin_memory()
        rh = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64).pin_memory()
        lre.lre_profile(ctx, True)
        lre.lre_estimate_host(ctx, host_in, lre.LRE_HOST_RECORDS_U16, N, n, th, rh)
        names = {k for k, _ in lre.lre_profile_records(ctx)}
        lre.lre_profile(ctx, False)
        assert "fold_first6_mma_records" in names and "histogram" not in names, names
        t_ref = direct.estimate(counts, N, n)
        np.testing.assert_array_equal(th.numpy(), t_ref)
        assert rel_fro(rh.numpy(), direct.mu(t_ref, n)) <= 1e-6
    finally:
        lre.lre_destroy(ctx)
