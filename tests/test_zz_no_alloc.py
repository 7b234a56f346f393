"""lre_assemble_noalloc: step (ii) for callers that cannot allocate device
memory (for example an application whose own allocator already holds the
GPU's memory, or a service that keeps cudaMalloc off its request path).

Its output must match lre_assemble's on the same theta, within the rho
tolerance the other tests use (relative Frobenius 1e-6), on two calls in a
row of different sizes, since every call reuses the same fixed scratch
array.  This file is collected last so that a stop-at-first-failure run has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from tests.gpu_util import need_gpu, rel_fro

pytestmark = pytest.mark.gpu


def _theta(n, seed):
    rng = np.random.default_rng(seed)
    t = rng.uniform(-1, 1, 4 ** n)
    t[0] = 1.0
    return t


def test_noalloc_matches_lre_assemble_on_consecutive_calls():
    torch = need_gpu()
    from paper_1602_08604_gb300 import lre
    ctx = lre.lre_create(0)
    try:
        for n, seed in ((10, 1), (7, 2)):            # largest supported n, then a smaller one
            d = 2 ** n
            theta = torch.from_numpy(_theta(n, seed)).cuda()
            ref = torch.empty((d, d), dtype=torch.complex64, device="cuda")
            lre.lre_assemble(ctx, theta, n, ref)
            got = torch.full((d, d), float("nan"), dtype=torch.complex64, device="cuda")
            lre.lre_assemble_noalloc(theta, n, got)
            torch.cuda.synchronize()
            assert rel_fro(got.cpu().numpy(), ref.cpu().numpy()) <= 1e-6
    finally:
        lre.lre_destroy(ctx)


def test_noalloc_second_call_takes_no_device_memory():
    """After the first call on the device has loaded the scratch array and the
    kernels, a call leaves the device's free memory exactly as it was."""
    torch = need_gpu()
    from paper_1602_08604_gb300 import lre
    n = 10
    d = 2 ** n
    theta = torch.from_numpy(_theta(n, 3)).cuda()
    rho = torch.empty((d, d), dtype=torch.complex64, device="cuda")
    lre.lre_assemble_noalloc(theta, n, rho)          # set-up call
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        lre.lre_assemble_noalloc(theta, n, rho)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = need_gpu()
    from paper_1602_08604_gb300 import lre
    theta = torch.zeros(4 ** 11, dtype=torch.float64, device="cuda")
    rho = torch.empty((2 ** 11, 2 ** 11), dtype=torch.complex64, device="cuda")
    with pytest.raises(lre.LreError) as e:
        lre.lre_assemble_noalloc(theta, 11, rho)
    assert e.value.status == lre.LRE_ERR_UNSUPPORTED
    assert "n <= 10" in str(e.value)                  # the reason is readable without a context
