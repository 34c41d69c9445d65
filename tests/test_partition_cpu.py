"""Partitioned sweep of one matrix over several ranks: the host side on the
CPU (pselinv_partition on host-only handles, the exchange plan, and the
exchange itself over two gloo ranks with stand-in blocks).  The device side
(restricted sweeps, block export and import) is checked on the GPU in
test_gpu_partition.py."""
from __future__ import annotations

import os
import socket
import sys

import numpy as np
import pytest

import gen
import paper_1708_04539_gb300 as ps
from paper_1708_04539_gb300.binding import supernodal_coordinates
from paper_1708_04539_gb300.distributed import exchange_plan, run_partitioned, subtree_roots

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROBLEMS = [
    lambda: gen.upwind_3d(14, 701, max_sn=64),
    lambda: gen.conv_diff_2d(40, 702, max_sn=32),
    lambda: gen.dg_blocks(5, 16, 703, max_sn=48),
]


def _host(p):
    from paper_1708_04539_gb300 import build
    build.build()
    return ps.SelInv.from_problem(p, host_only=True)


@pytest.mark.parametrize("nranks", [1, 2, 3, 8])
@pytest.mark.parametrize("make", PROBLEMS)
def test_partition_is_a_top_and_whole_subtrees(make, nranks):
    p = make()
    h = _host(p)
    st = h.structure()
    owner = h.partition(nranks)
    parent = st["sn_parent"]
    ns = int(st["nsuper"])
    assert owner.shape == (ns,) and owner.min() >= -1 and owner.max() < nranks
    if nranks == 1:
        assert np.all(owner == 0)
    for k in range(ns):
        if owner[k] < 0 and parent[k] >= 0:
            assert owner[parent[k]] < 0  # the top is closed towards the roots
        if owner[k] >= 0 and parent[k] >= 0 and owner[parent[k]] >= 0:
            assert owner[parent[k]] == owner[k]  # whole subtrees
    # load balance: no rank above twice the mean of the owned flops
    w = st["sn_width"].astype(float)
    c = np.diff(st["rows_ptr"]).astype(float)
    f = 4 * c * c * w + 4 * c * w * w + 4 / 3 * w ** 3
    load = np.array([f[owner == q].sum() for q in range(nranks)])
    assert load.max() <= 2.0 * load.mean() + 1e-9
    h.close()


@pytest.mark.parametrize("make", PROBLEMS)
def test_root_blocks_cover_every_outside_read(make):
    """Every entry of Ainv that a supernode of a subtree reads outside its
    subtree (R_K x R_K minus the subtree's columns) lies in G_r of the
    subtree's root: the single exchange step is enough."""
    p = make()
    h = _host(p)
    st = h.structure()
    owner = h.partition(3)
    parent = st["sn_parent"]
    first = np.asarray(st["sn_first"])
    width = np.asarray(st["sn_width"])
    roots = subtree_roots(owner, parent)
    root_of = {}
    for k in range(int(st["nsuper"]) - 1, -1, -1):
        if k in roots:
            root_of[k] = k
        elif owner[k] >= 0:
            root_of[k] = root_of[parent[k]]
    members = {}
    for k, r in root_of.items():
        members.setdefault(r, set()).update(range(first[k], first[k] + width[k]))
    for k, r in root_of.items():
        Rk = st["rows"][st["rows_ptr"][k]:st["rows_ptr"][k + 1]]
        Rr = set(st["rows"][st["rows_ptr"][r]:st["rows_ptr"][r + 1]].tolist())
        outside = [x for x in Rk.tolist() if x not in members[r]]
        assert set(outside) <= Rr, (k, r)
    plan = exchange_plan(owner, parent, np.diff(st["rows_ptr"]))
    for root, dst, size in plan:
        assert owner[root] == dst != 0 and size == np.diff(st["rows_ptr"])[root] ** 2
    h.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class FakeOps:
    """Stand-in for the device: storage slots hold values; the top sweep on
    rank 0 writes a known value into every slot of the top supernodes;
    export / import gather and write G_K through the structure's coordinates."""

    def __init__(self, st, owner, rank):
        import torch
        self.torch = torch
        self.st, self.owner, self.rank = st, owner, rank
        rows, cols = supernodal_coordinates(st)
        self.slot = {(int(r), int(c)): i for i, (r, c) in enumerate(zip(rows, cols))}
        self.store = np.zeros(int(st["storage_size"]))
        self.sweeps = []
        self.sn_of_slot = np.zeros(self.store.size, dtype=np.int64)
        for K in range(int(st["nsuper"])):
            o = int(st["sn_offset"][K])
            e = int(st["sn_offset"][K + 1]) if K + 1 < int(st["nsuper"]) else self.store.size
            self.sn_of_slot[o:e] = K

    def truth(self):
        return np.sin(np.arange(self.store.size) * 0.37) + 2.0

    def sweep(self, subset):
        self.sweeps.append(subset)
        if subset == -1:
            mask = self.owner[self.sn_of_slot] == -1
            self.store[mask] = self.truth()[mask]

    def _idx(self, K):
        R = self.st["rows"][self.st["rows_ptr"][K]:self.st["rows_ptr"][K + 1]]
        return np.array([self.slot[(int(a), int(b))] for b in R for a in R], dtype=np.int64)

    def new_block(self, K):
        c = int(self.st["rows_ptr"][K + 1] - self.st["rows_ptr"][K])
        return self.torch.zeros(c * c, dtype=self.torch.float64)

    def export(self, K):
        return self.torch.from_numpy(self.store[self._idx(K)].copy())

    def import_(self, K, buf):
        self.store[self._idx(K)] = buf.numpy()


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = gen.upwind_3d(12, 704, max_sn=64)
    h = _host(p)
    st = h.structure()
    owner = h.partition(world)
    ops = FakeOps(st, owner, rank)
    moved = run_partitioned(ops, owner, st["sn_parent"], np.diff(st["rows_ptr"]), rank, world, dist)
    # every block this rank received holds rank 0's top values exactly
    ok = True
    for root, dst, _ in exchange_plan(owner, st["sn_parent"], np.diff(st["rows_ptr"])):
        if dst == rank:
            idx = ops._idx(root)
            ok = ok and np.array_equal(ops.store[idx], ops.truth()[idx])
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, moved, ops.sweeps, ok))
    h.close()


def test_exchange_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    (r0, m0, s0, ok0), (r1, m1, s1, ok1) = out
    assert s0 == [-1, 0] and s1 == [1]
    assert m0 == m1 > 0  # rank 0 sent as many blocks as rank 1 received
    assert ok0 and ok1
