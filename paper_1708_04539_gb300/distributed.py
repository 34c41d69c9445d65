"""Partitioned selected inversion of ONE matrix over several ranks (one GPU
each, torch.distributed), with a single exchange step.

The subtrees below the top of the supernodal tree are independent once the
selected inverse of the top is known: a supernode K inside the subtree of a
root r reads Ainv only inside that subtree and at R_r x R_r (the rows of
R_K outside the subtree lie in R_r).  So rank 0 sweeps the top once, sends
each subtree root's block G_r = Ainv(R_r, R_r) to the rank that owns the
subtree (the one exchange step), and every rank then sweeps its own
subtrees.  The partition itself (pselinv_partition), the restricted sweeps
(pselinv_set_subset) and the block transfers (pselinv_export_block /
pselinv_import_block) are library calls; this module only orders them and
moves the blocks between ranks.  Every rank holds the whole factorisation
(each factors the same matrix).
"""
from __future__ import annotations

import numpy as np


def subtree_roots(owner, parent):
    """Supernodes that head a rank's subtree: owned, with a parent in the top
    (or none)."""
    owner = np.asarray(owner)
    parent = np.asarray(parent)
    out = []
    for k in range(owner.size):
        if owner[k] >= 0 and (parent[k] < 0 or owner[parent[k]] < 0):
            out.append(k)
    return out


def exchange_plan(owner, parent, c):
    """(root, destination rank, block scalars) of every block rank 0 sends:
    the roots owned by another rank whose R_r is not empty."""
    return [(r, int(owner[r]), int(c[r]) * int(c[r])) for r in subtree_roots(owner, parent)
            if owner[r] != 0 and c[r] > 0]


def run_partitioned(ops, owner, parent, c, rank, world, dist):
    """One rank's share of the partitioned sweep.

    ops: sweep(subset_rank) runs the restricted sweep (-1 = the top);
         export(K) -> block (a tensor of c_K^2 scalars on the wire's device);
         new_block(K) -> an empty such block; import_(K, block).
    Blocks travel with dist.send / dist.recv, in the order of
    exchange_plan, so both sides agree on every message.  Returns the number
    of blocks this rank sent or received."""
    plan = exchange_plan(owner, parent, c)
    moved = 0
    if rank == 0:
        ops.sweep(-1)
        for root, dst, _ in plan:
            if world > 1:
                dist.send(ops.export(root), dst=dst)
                moved += 1
    else:
        for root, dst, _ in plan:
            if dst == rank:
                buf = ops.new_block(root)
                dist.recv(buf, src=0)
                ops.import_(root, buf)
                moved += 1
    ops.sweep(rank)
    return moved


class LibraryOps:
    """The device side of run_partitioned through the library handle `h`
    (blocks are device tensors for NCCL, host tensors for gloo)."""

    def __init__(self, h, owner, precision, stream=None, wire_device="cuda"):
        import torch
        self.h, self.owner, self.precision, self.stream = h, owner, precision, stream
        self.torch = torch
        st = h.structure()
        self.c = np.diff(st["rows_ptr"])
        self.dtype = torch.complex128 if h.dtype == 2 else torch.float64
        self.wire = wire_device

    def sweep(self, subset_rank):
        if not np.any(np.asarray(self.owner) == subset_rank):
            return  # nothing of this rank's (or no top)
        self.h.set_subset(self.owner, subset_rank)
        self.h.selinv(precision=self.precision, stream=self.stream)
        self.h.sync(stream=self.stream)

    def new_block(self, K):
        return self.torch.empty(int(self.c[K]) ** 2, dtype=self.dtype, device=self.wire)

    def export(self, K):
        buf = self.torch.empty(int(self.c[K]) ** 2, dtype=self.dtype, device="cuda")
        self.h.export_block(K, buf, stream=self.stream)
        return buf.to(self.wire)

    def import_(self, K, buf):
        self.h.import_block(K, buf.to("cuda"), stream=self.stream)
