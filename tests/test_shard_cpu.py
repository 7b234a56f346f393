"""One instance split over ranks by the axis of qubit 1 (paper_1602_08604_gb300
/shard.py): the slab plan, the reduce-scatter of the identity block and the
assembly of theta, run as gloo ranks on the CPU.  Each rank's device work is
stood in for by the oracle: the slab's shares are the oracle's direct sums
over the slab's basis groups only (Sec. III), and the weight is the oracle's
S / (N 3^k).  The combined theta must equal the oracle's estimate of the
whole count matrix bit for bit, for 1, 2, 3 and 4 ranks (with 4, one rank
holds no slab and only weights its slice of the identity block)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _counts(n, N, seed):
    rng = np.random.default_rng(seed)
    p = rng.dirichlet(np.ones(2 ** n), size=3 ** n)
    return np.stack([rng.multinomial(N, row) for row in p]).astype(np.int32)


def _oracle_parts(n, N, c):
    from oracle import direct
    from paper_1602_08604_gb300.shard import SlabPlan
    plan = SlabPlan(n, 1)

    def slab_sums(a):
        lo, hi = plan.rows(a)
        S, _ = direct.parity_sums(c[lo:hi], n, b0=lo, b1=hi)     # the slab's groups only
        olo, ohi = plan.own_range(a)
        return torch.from_numpy(S[: plan.block].copy()), torch.from_numpy(S[olo:ohi].copy())

    def weight(S, first):
        idx = np.arange(first, first + S.numel())
        k = np.array([direct.identity_letters(int(i), n) for i in idx])
        return torch.from_numpy(S.numpy().astype(np.float64) / (float(N) * 3.0 ** k))

    return slab_sums, weight


def _worker(rank, world, port, q, n, N, seed):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import direct
    from paper_1602_08604_gb300 import shard
    c = _counts(n, N, seed)
    plan = shard.SlabPlan(n, world)
    slab_sums, weight = _oracle_parts(n, N, c)
    pieces = shard.step_i(plan, rank, slab_sums, weight, torch.device("cpu"))
    theta = shard.gather_theta(plan, pieces, torch.device("cpu")).numpy()
    want = direct.estimate(c, N, n)
    covered = sum(t.numel() for _, t in pieces)
    q.put((rank, bool(np.array_equal(theta, want)), covered, plan.axes(rank)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [1, 2, 3, 4])
def test_sharded_step_i_equals_oracle(world):
    import multiprocessing as mp
    n, N = 5, 777
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, n, N, 31)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert all(ok for _, ok, _, _ in res), res
    # every coefficient is weighted by exactly one rank
    assert sum(cov for _, _, cov, _ in res) == 4 ** n
    assert sorted(a for _, _, _, axes in res for a in axes) == [0, 1, 2]


def test_slab_plan_ranges():
    from paper_1602_08604_gb300.shard import SlabPlan
    p = SlabPlan(4, 3)
    assert p.block == 64 and p.chunk == 22
    assert [p.ident_range(r) for r in range(3)] == [(0, 22), (22, 44), (44, 64)]
    assert [p.own_range(a) for a in range(3)] == [(64, 128), (128, 192), (192, 256)]
    assert [p.rows(a) for a in range(3)] == [(0, 27), (27, 54), (54, 81)]
    p4 = SlabPlan(4, 4)
    assert p4.axes(3) == [] and p4.ident_range(3) == (48, 64)
