"""Slab sharding of one tensor over the ranks of a process group (one GPU each).

Y is split along one observed letter m into contiguous slabs, one per rank.  The
numerator and denominator of Eq. 3.6-3.8 are sums over the entries of Y, so for
a factor that does not hold m each rank's num and den over its slab are partial
sums: an all-reduce (sum) of them gives the whole tensor's, and every rank
applies the same update of Eq. 3.4 to its replica of that factor (replicas stay
bit-identical, since every rank reduces the same values in the same order).  A
factor that holds m only meets entries of its own slab rows, so each rank
updates its rows locally.  The factors keep Algorithm 1's Gauss-Seidel order.
The loss is the all-reduced sum of the slabs' losses.

Communication per sweep: two all-reduces of the size of each factor that does
not hold m (a few hundred KB for the benchmark shapes); none for the others.
"""
from __future__ import annotations

from ._nef import Plan, split_model


def slab_bounds(n: int, world: int, rank: int):
    """Rows [lo, hi) of rank `rank` when n rows are split into `world` contiguous
    slabs whose sizes differ by at most one."""
    base, extra = divmod(int(n), int(world))
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def slab_sweeps(ops, local, iters, allreduce):
    """`iters` sweeps of Algorithm 1 on one slab: factor l is updated in place by
    ops.update(l) when local[l] (it holds the split letter), else from the
    num/den of ops.numden(l) summed over the slabs by allreduce (in place) and
    applied by ops.apply_update(l, num, den)."""
    for _ in range(int(iters)):
        for l, is_local in enumerate(local):
            if is_local:
                ops.update(l)
            else:
                num, den = ops.numden(l)
                allreduce(num)
                allreduce(den)
                ops.apply_update(l, num, den)


class SlabFit:
    """A fit of `model_str` whose tensor is split along observed letter `m` over
    the ranks of a torch.distributed process group.

    ``dims`` are the full sizes; this rank's plan covers rows slab_bounds(dims[m],
    world, rank) of letter m.  ``fit`` takes this rank's slab of Y (and of the
    mask), the slab rows of the factors that hold m and full replicas of the
    others (CUDA tensors as for Plan.fit), and updates them in place."""

    def __init__(self, model_str: str, dims: dict, m: str, precision: str = "bf16", group=None, **plan_kw):
        import torch.distributed as dist
        obs, _, terms = split_model(model_str)
        if m not in obs:
            raise ValueError(f"{m!r} is not an observed letter of {model_str!r}")
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.lo, self.hi = slab_bounds(dims[m], self.world, self.rank)
        sdims = dict(dims)
        sdims[m] = self.hi - self.lo
        if sdims[m] < 1:
            raise ValueError("more ranks than rows of the split letter")
        self.local = [m in t for t in terms]
        self.plan = Plan(model_str, sdims, precision=precision, **plan_kw)

    def _allreduce(self, t):
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)

    def fit(self, Y, mask, factors, alpha, beta, iters):
        plan = self.plan

        class Ops:
            def update(self, l):
                plan.update(l, Y, mask, factors, alpha, beta)

            def numden(self, l):
                return plan.numden(l, Y, mask, factors, alpha, beta)

            def apply_update(self, l, num, den):
                plan.apply_update(l, factors, num, den, alpha, beta)

        slab_sweeps(Ops(), self.local, iters, self._allreduce)

    def loss(self, Y, mask, factors, alpha, beta):
        """(sum, count) over the whole tensor: the slabs' losses, all-reduced."""
        import torch
        s, c = plan_loss = self.plan.loss(Y, mask, factors, alpha, beta)
        t = torch.tensor([s, float(c)], dtype=torch.float64, device=Y.device)
        self._allreduce(t)
        del plan_loss
        return float(t[0]), int(t[1])
