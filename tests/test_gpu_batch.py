"""Batched form: many instances of uneven n and shots in one persistent
launch give exactly the per-instance lre_estimate results (and the oracle's
theta bit for bit where the oracle is fast)."""
import numpy as np
import pytest

from oracle import direct
from synth import counts as sc
from synth import states as st
from tests.gpu_util import ctx_and_lre, need_gpu

pytestmark = pytest.mark.gpu


def _instance(n, seed, shots, dtype):
    rho = st.ginibre_mixture(n, 1 + seed % 4, seed=seed)
    thr = sc.cdf_thresholds(st.born_probabilities(st.pauli_expectations(rho), n))
    return sc.sample_cdf(thr, shots, seed=seed + 7, dtype=dtype)


@pytest.fixture(scope="module")
def batch():
    torch = need_gpu()
    rng = np.random.default_rng(11)
    specs = [(n, int(np.exp(rng.uniform(np.log(500), np.log(10000)))), dt)
             for n, dt in [(1, np.int32), (2, np.int16), (3, np.int32), (4, np.int32), (5, np.int16),
                           (6, np.int32), (7, np.int32), (7, np.int16), (8, np.int32), (9, np.int32),
                           (3, np.int16), (5, np.int32)]]
    items, host = [], []
    for k, (n, shots, dt) in enumerate(specs):
        c = _instance(n, 40 + k, shots, dt)
        host.append((c, shots, n))
        theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
        rho = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device="cuda") if k % 5 != 3 else None
        items.append((torch.from_numpy(c).cuda(), shots, n, theta, rho))
    return torch, items, host


def _check_against_single(torch, lre, ctx, items, host):
    for (c, shots, n, theta, rho), (ch, _, _) in zip(items, host):
        t1 = torch.empty_like(theta)
        r1 = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device="cuda") if rho is not None else None
        lre.lre_estimate(ctx, c, shots, n, t1, r1)
        lre.lre_sync(ctx)
        assert torch.equal(theta, t1), n
        if rho is not None:
            assert torch.equal(rho, r1), n
        if n <= 6:
            np.testing.assert_array_equal(theta.cpu().numpy(), direct.estimate(ch, shots, n))


def test_batch_equals_per_instance_and_oracle(batch):
    torch, items, host = batch
    lre, ctx = ctx_and_lre()
    try:
        lre.lre_batch_run(ctx, items)
        lre.lre_sync(ctx)
        _check_against_single(torch, lre, ctx, items, host)
    finally:
        lre.lre_destroy(ctx)


def test_batch_tune_then_run(batch):
    torch, items, host = batch
    lre, ctx = ctx_and_lre()
    try:
        ms = lre.lre_batch_tune(ctx, items)
        sch = lre.lre_batch_schedule(ctx)
        assert sch["jmax"] in (2, 3) and sch["ctas_per_sm"] in (1, 2)
        assert sch["first_unit"] in (256, 1024) and sch["unit"] in (256, 1024, 4096)
        assert ms > 0
        for _, _, _, theta, rho in items:
            theta.fill_(float("nan"))
        lre.lre_batch_run(ctx, items)
        lre.lre_sync(ctx)
        _check_against_single(torch, lre, ctx, items, host)
    finally:
        lre.lre_destroy(ctx)


# the autotuner may keep any of its candidates: each must give the same
# results (J = 2 and 3 first passes staged, int16 and int32 counts, small and
# large units, one and two CTAs per SM)
@pytest.mark.parametrize("sched", [(2, 1, 256, 256), (2, 2, 1024, 4096), (3, 1, 1024, 256),
                                   (3, 2, 256, 1024), (3, 2, 1024, 4096)])
def test_every_schedule_matches_per_instance(batch, sched):
    import ctypes
    torch, items, host = batch
    lre, ctx = ctx_and_lre()
    try:
        f = lre.load().lre_debug_set_batch_schedule
        f.argtypes = [ctypes.c_void_p] + [ctypes.c_int] * 4
        f.restype = ctypes.c_int
        assert f(ctx, *sched) == 0
        assert tuple(lre.lre_batch_schedule(ctx).values()) == sched
        for _, _, _, theta, rho in items:
            theta.fill_(float("nan"))
            if rho is not None:
                rho.fill_(float("nan"))
        lre.lre_batch_run(ctx, items)
        lre.lre_sync(ctx)
        _check_against_single(torch, lre, ctx, items, host)
    finally:
        lre.lre_destroy(ctx)


def test_batch_rejects_large_n(batch):
    torch, items, host = batch
    lre, ctx = ctx_and_lre()
    try:
        c = torch.zeros((3 ** 10, 2 ** 10), dtype=torch.int32, device="cuda")
        th = torch.empty(4 ** 10, dtype=torch.float64, device="cuda")
        with pytest.raises(lre.LreError) as e:
            lre.lre_batch_run(ctx, [(c, 100, 10, th, None)])
        assert e.value.status == lre.LRE_ERR_UNSUPPORTED
    finally:
        lre.lre_destroy(ctx)


def test_batch_captured_in_a_cuda_graph_replays_on_new_counts(batch):
    """The batched launch recorded in a CUDA graph: replaying it after the
    counts change in place gives exactly the per-instance results on the new
    counts."""
    torch, items, host = batch
    lre, ctx = ctx_and_lre()
    try:
        small = [it for it in items if it[2] <= 7]
        lre.lre_batch_run(ctx, small)          # uncaptured run: workspace and pass table
        lre.lre_sync(ctx)
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            lre.lre_batch_run(ctx, small, stream=torch.cuda.current_stream())
        rng = np.random.default_rng(5)
        new_host = []
        for (c, shots, n, theta, rho) in small:
            fresh = _instance(n, int(rng.integers(1000, 2000)), shots,
                              np.int16 if c.dtype == torch.int16 else np.int32)
            c.copy_(torch.from_numpy(fresh))
            theta.zero_()
            new_host.append((fresh, shots, n))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        lre.lre_sync(ctx)
        _check_against_single(torch, lre, ctx, small, new_host)
    finally:
        lre.lre_destroy(ctx)


def test_batch_capture_without_uncaptured_run_is_refused(batch):
    torch, items, host = batch
    lre, ctx = ctx_and_lre()
    try:
        small = [it for it in items if it[2] <= 5]
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        err = None
        with torch.cuda.graph(g, stream=s):
            try:
                lre.lre_batch_run(ctx, small, stream=torch.cuda.current_stream())
            except lre.LreError as ex:
                err = ex
        assert err is not None and err.status == lre.LRE_ERR_UNSUPPORTED
    finally:
        lre.lre_destroy(ctx)


def test_batch_bounded_wait_runs_out_then_context_recovers(batch):
    """Failure detection without a fault: a test hook makes one pass of the
    table wait for a unit that never exists, with the wait bounded at 20 ms.
    The persistent kernel must return (every CTA leaves once the wait gives
    up), lre_sync must report LRE_ERR_TIMEOUT, and the same context must then
    run the batch correctly."""
    import ctypes
    import time
    torch, items, host = batch
    lre, ctx = ctx_and_lre()
    f = lre.load().lre_debug_batch_fault
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    f.restype = ctypes.c_int
    try:
        assert f(ctx, 20, 1) == 0
        t0 = time.perf_counter()
        lre.lre_batch_run(ctx, items)
        with pytest.raises(lre.LreError) as e:
            lre.lre_sync(ctx)
        assert e.value.status == lre.LRE_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 1.5        # gave up at its 20 ms bound, not the default 2 s
        assert f(ctx, 0, -1) == 0
        for _, _, _, theta, rho in items:
            theta.fill_(float("nan"))
        lre.lre_batch_run(ctx, items)
        lre.lre_sync(ctx)
        # the oracle reads the counts as they are now on the device (another
        # test of this module replaces some instances' counts in place)
        now = [(c.cpu().numpy(), shots, n) for c, shots, n, _, _ in items]
        _check_against_single(torch, lre, ctx, items, now)
    finally:
        lre.lre_destroy(ctx)
