"""Streamed steps (i)+(ii) (lre_stream_*): counts arriving in chunks of whole
tile rows give theta and rho bit-identical to lre_estimate on the whole
matrix (and theta to the oracle); a checkpoint taken half-way and resumed in
a new context gives the same; counts generated on the device chunk by chunk
just before they are folded (the whole matrix never exists) give the same
as the materialised path."""
import numpy as np
import pytest

from oracle import direct
from tests.gpu_util import ctx_and_lre, need_gpu

pytestmark = pytest.mark.gpu


def _whole(torch, lre, counts, shots, n):
    lre_, ctx = ctx_and_lre()
    try:
        theta = torch.empty(4 ** n, dtype=torch.float64, device="cuda")
        rho = torch.empty((2 ** n, 2 ** n), dtype=torch.complex64, device="cuda")
        lre.lre_estimate(ctx, counts, shots, n, theta, rho)
        lre.lre_sync(ctx)
        return theta, rho
    finally:
        lre.lre_destroy(ctx)


def _chunks(n, rows):
    B = 3 ** n
    return [(b, min(B, b + rows)) for b in range(0, B, rows)]


@pytest.mark.parametrize("n,dt,shots,rows", [(7, "i16", 1000, 729), (10, "i16", 1000, 2 * 729),
                                             (10, "i32", 4096, 3 * 729), (11, "i16", 1000, 27 * 729)])
def test_stream_equals_whole_matrix(n, dt, shots, rows):
    torch = need_gpu()
    from synth import gen
    c = torch.empty((3 ** n, 2 ** n), dtype=torch.int16 if dt == "i16" else torch.int32, device="cuda")
    gen.gen_ghz(n, 0.05, shots, 800 + n, c)
    lre, ctx = ctx_and_lre()
    try:
        t0, r0 = _whole(torch, lre, c, shots, n)
        kind = lre.LRE_COUNTS_I16 if dt == "i16" else lre.LRE_COUNTS_I32
        lre.lre_stream_begin(ctx, n, kind, shots)
        for b0, b1 in _chunks(n, rows):
            lre.lre_stream_chunk(ctx, c[b0:b1], b0)
        theta = torch.full_like(t0, float("nan"))
        rho = torch.full_like(r0, float("nan"))
        lre.lre_stream_end(ctx, theta, rho)
        lre.lre_sync(ctx)
        assert torch.equal(theta, t0) and torch.equal(rho, r0)
        if n <= 7:
            np.testing.assert_array_equal(theta.cpu().numpy(), direct.estimate(c.cpu().numpy(), shots, n))
    finally:
        lre.lre_destroy(ctx)


@pytest.mark.parametrize("n,dt,shots", [(10, "i16", 1000), (9, "i32", 4096)])
def test_checkpoint_and_resume_in_a_new_context(n, dt, shots):
    torch = need_gpu()
    from synth import gen
    c = torch.empty((3 ** n, 2 ** n), dtype=torch.int16 if dt == "i16" else torch.int32, device="cuda")
    gen.gen_ghz(n, 0.05, shots, 900 + n, c)
    from paper_1602_08604_gb300 import lre
    t0, _ = _whole(torch, lre, c, shots, n)
    kind = lre.LRE_COUNTS_I16 if dt == "i16" else lre.LRE_COUNTS_I32
    parts = _chunks(n, 729)
    half = len(parts) // 2
    ctx = lre.lre_create(0)
    try:
        lre.lre_stream_begin(ctx, n, kind, shots)
        for b0, b1 in parts[:half]:
            lre.lre_stream_chunk(ctx, c[b0:b1], b0)
        state = lre.lre_stream_checkpoint(ctx)
        with pytest.raises(lre.LreError) as e:        # chunks come in order
            lre.lre_stream_chunk(ctx, c[parts[-1][0]:parts[-1][1]], parts[-1][0])
        assert e.value.status == lre.LRE_ERR_INVALID_ARG
    finally:
        lre.lre_destroy(ctx)
    # a 64-byte header and the partials of the tile rows done: 3 bytes each
    # where the tensor pass writes split planes (n = 10), else int32
    per = 3 if n == 10 else 4
    assert len(state) == 64 + half * 2 ** (n - 6) * 4096 * per
    ctx = lre.lre_create(0)
    try:
        lre.lre_stream_resume(ctx, state)
        with pytest.raises(lre.LreError):                # not all bases in yet
            lre.lre_stream_end(ctx, torch.empty_like(t0))
        lre.lre_stream_resume(ctx, state)
        for b0, b1 in parts[half:]:
            lre.lre_stream_chunk(ctx, c[b0:b1], b0)
        theta = torch.full_like(t0, float("nan"))
        lre.lre_stream_end(ctx, theta)
        lre.lre_sync(ctx)
        assert torch.equal(theta, t0)
    finally:
        lre.lre_destroy(ctx)


def test_counts_generated_chunk_by_chunk_equal_the_materialised_path():
    """Fused generation: the device generator fills a two-slot ring of
    chunks, each folded before its slot is refilled; no count matrix."""
    torch = need_gpu()
    from synth import gen
    n, shots, rows = 11, 1000, 9 * 729
    full = torch.empty((3 ** n, 2 ** n), dtype=torch.int16, device="cuda")
    gen.gen_ghz(n, 0.05, shots, 77, full)
    from paper_1602_08604_gb300 import lre
    t0, r0 = _whole(torch, lre, full, shots, n)
    del full
    ring = [torch.empty((rows, 2 ** n), dtype=torch.int16, device="cuda") for _ in range(2)]
    ctx = lre.lre_create(0)
    try:
        lre.lre_stream_begin(ctx, n, lre.LRE_COUNTS_I16, shots)
        for k, (b0, b1) in enumerate(_chunks(n, rows)):
            buf = ring[k % 2][: b1 - b0]
            gen.gen_ghz(n, 0.05, shots, 77, buf, b0=b0)
            lre.lre_stream_chunk(ctx, buf, b0)
        theta = torch.empty_like(t0)
        rho = torch.empty_like(r0)
        lre.lre_stream_end(ctx, theta, rho)
        lre.lre_sync(ctx)
        assert torch.equal(theta, t0) and torch.equal(rho, r0)
    finally:
        lre.lre_destroy(ctx)
