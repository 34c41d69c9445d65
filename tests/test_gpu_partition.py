"""Partitioned sweep of one matrix, emulated rank by rank on one GPU: each
"rank" is its own handle (every rank factors the whole matrix); rank 0
sweeps the top, exports every subtree root's block G_r = Ainv(R_r, R_r),
the owning rank imports it and sweeps its subtrees.  The supernodes each
rank computed must equal a single full sweep.  No two ranks' kernels run at
the same time and none waits on another: the ranks run one after another.
"""
from __future__ import annotations

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_04539_gb300 import build
    build.build()
    return _t


class DirectDist:
    """A stand-in for torch.distributed between emulated ranks in one
    process: send() stores the block, recv() returns it."""

    def __init__(self):
        self.q = {}

    def send(self, t, dst):
        self.q.setdefault(dst, []).append(t.clone())

    def recv(self, t, src):
        t.copy_(self.q[self._rank].pop(0))


@pytest.mark.parametrize("prec_name", ["fp64", "split"])
@pytest.mark.parametrize("world,make", [
    (2, lambda: gen.upwind_3d(16, 711, max_sn=64)),
    (3, lambda: gen.dg_blocks(5, 16, 712, max_sn=48)),
    (4, lambda: gen.stencil27_complex(10, 713, max_sn=64)),
])
def test_partitioned_sweep_equals_full_sweep(torch, world, make, prec_name):
    import paper_1708_04539_gb300 as ps
    from paper_1708_04539_gb300.distributed import LibraryOps, run_partitioned
    prec = ps.PREC_FP64 if prec_name == "fp64" else ps.PREC_OZAKI_FP16
    p = make()
    vals = torch.from_numpy(np.ascontiguousarray(p.values)).cuda()
    ref = ps.SelInv.from_problem(p)
    ref.factor(vals)
    if prec == ps.PREC_OZAKI_FP16:  # every level split, in all handles alike
        nlev = ref.structure()["nlevels"]
        triples = [(lev, 3, 0) for lev in range(nlev)]
        ref.plan_set(triples, prec)
    ref.selinv(precision=prec)
    full = ref.get_selected(layout=ps.LAYOUT_SUPERNODAL)
    st = ref.structure()
    owner = ref.partition(world)
    assert (owner == -1).any() and len(set(owner[owner >= 0].tolist())) == world
    dist = DirectDist()
    handles = []
    for rank in range(world):
        h = ps.SelInv.from_problem(p)
        h.factor(vals)
        if prec == ps.PREC_OZAKI_FP16:
            h.plan_set(triples, prec)
        handles.append(h)
    c = np.diff(st["rows_ptr"])
    moved = 0
    for rank in range(world):  # rank 0 first: it sends before the others receive
        dist._rank = rank
        ops = LibraryOps(handles[rank], owner, prec)
        moved += run_partitioned(ops, owner, st["sn_parent"], c, rank, world, dist)
    assert moved > 0 and all(len(v) == 0 for v in dist.q.values())
    # every supernode from the rank that owns it (the top from rank 0)
    ends = list(st["sn_offset"][1:]) + [int(st["storage_size"])]
    scale = np.abs(full).max()
    for rank in range(world):
        got = handles[rank].get_selected(layout=ps.LAYOUT_SUPERNODAL)
        for K in range(int(st["nsuper"])):
            if owner[K] == rank or (rank == 0 and owner[K] == -1):
                a, b = int(st["sn_offset"][K]), int(ends[K])
                assert np.abs(got[a:b] - full[a:b]).max() <= 1e-13 * scale, (rank, K)
    for h in handles + [ref]:
        h.sync()
        h.close()
