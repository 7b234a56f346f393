"""One LRE instance across several GPUs, one process per GPU (host-side
orchestration; every step of the arithmetic runs in liblre's kernels).

The 3^n bases are split by the axis a of qubit 1 into three slabs of 3^(n-1)
rows (Sec. III's basis groups partitioned by their first letter); slab a
lives on rank a mod world.  lre_slab_sums folds a slab over qubits 2..n and
returns
  * its share of the strings whose qubit-1 letter is I (every slab adds to
    them), and
  * the strings whose qubit-1 letter is a + 1, which only slab a feeds.
One reduce-scatter (sum) of the identity block gives every rank a slice of
it; lre_weight turns each rank's slice and its own blocks into theta
(Eq. 3's 1/(N 3^k)).  The pieces are disjoint ranges of theta in Eq. (5)
order; gather_theta assembles the whole vector where it is needed (step ii).
"""
import torch
import torch.distributed as dist


class SlabPlan:
    """Which rank holds which qubit-1 axis, and which slice of the identity
    block (4^(n-1) strings) each rank weights after the reduce-scatter."""

    def __init__(self, n, world):
        if n < 2:
            raise ValueError("the split needs n >= 2")
        self.n, self.world = n, world
        self.block = 4 ** (n - 1)
        self.owner = [a % world for a in range(3)]
        self.chunk = -(-self.block // world)            # ceil: the last slice is shorter or empty

    def axes(self, rank):
        return [a for a in range(3) if self.owner[a] == rank]

    def rows(self, a):
        """Row range of slab a in the full [3^n][2^n] count matrix."""
        m = 3 ** (self.n - 1)
        return a * m, (a + 1) * m

    def ident_range(self, rank):
        lo = min(rank * self.chunk, self.block)
        return lo, min(lo + self.chunk, self.block)

    def own_range(self, a):
        return (a + 1) * self.block, (a + 2) * self.block


def _world(group):
    return dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1


def step_i(plan, rank, slab_sums, weight, device, group=None):
    """Step (i) of this rank: slab_sums(a) -> (ident, own) int64 [4^(n-1)]
    for each axis the rank holds; weight(S, first) -> FP64 theta of the block
    S starting at Pauli index `first`.  Returns [(first, theta piece)]."""
    pieces = []
    ident = torch.zeros(plan.chunk * plan.world, dtype=torch.int64, device=device)
    for a in plan.axes(rank):
        i_a, o_a = slab_sums(a)
        ident[: plan.block] += i_a
        lo, _ = plan.own_range(a)
        pieces.append((lo, weight(o_a, lo)))
    mine = torch.empty(plan.chunk, dtype=torch.int64, device=device)
    if plan.world > 1:
        dist.reduce_scatter_tensor(mine, ident, op=dist.ReduceOp.SUM, group=group)
    else:
        mine.copy_(ident)
    lo, hi = plan.ident_range(rank)
    if hi > lo:
        pieces.append((lo, weight(mine[: hi - lo].contiguous(), lo)))
    return pieces


def gather_theta(plan, pieces, device, group=None):
    """The whole theta on every rank (the pieces are disjoint)."""
    theta = torch.zeros(4 ** plan.n, dtype=torch.float64, device=device)
    for first, t in pieces:
        theta[first: first + t.numel()] = t
    if plan.world > 1:
        dist.all_reduce(theta, op=dist.ReduceOp.SUM, group=group)
    return theta


def estimate_sharded(lre, ctx, slabs, shots, n, group=None, stream=None):
    """theta of one instance whose slabs (axis -> device [3^(n-1)][2^n]
    counts) are spread over the ranks of `group`; returns the full theta on
    every rank."""
    rank = dist.get_rank(group) if _world(group) > 1 else 0
    plan = SlabPlan(n, _world(group))
    device = next(iter(slabs.values())).device if slabs else torch.device("cuda", torch.cuda.current_device())
    block = plan.block

    def slab_sums(a):
        ident = torch.empty(block, dtype=torch.int64, device=device)
        own = torch.empty(block, dtype=torch.int64, device=device)
        lre.lre_slab_sums(ctx, slabs[a], n, ident, own, row_total_bound=shots, stream=stream)
        return ident, own

    def weight(S, first):
        t = torch.empty(S.numel(), dtype=torch.float64, device=device)
        lre.lre_weight(ctx, S, n, first, shots, t, stream=stream)
        return t

    pieces = step_i(plan, rank, slab_sums, weight, device, group)
    lre.lre_sync(ctx, stream)
    return gather_theta(plan, pieces, device, group)
