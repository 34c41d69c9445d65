"""The allocation-free entry point against the handle-based path.

pselinv_block_inverse_noalloc serves callers that cannot allocate device
memory (a framework's caching allocator owns the device, or cudaMalloc's
device-wide synchronisation is not allowed where they run).  For a matrix
that forms a single supernode, the handle-based path (pselinv_factor +
pselinv_selinv) returns A^{-1} as the supernode's diagonal block; the
allocation-free call, given the factored block, must return the same
matrix.  Two calls in a row check that the shared scratch array left by one
call does not leak into the next.  This file is collected last on purpose.
"""
from __future__ import annotations

import numpy as np
import pytest

import gen
from helpers import normwise_error

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_04539_gb300 import build
    build.build()
    return _t


def _reference(torch, p):
    """Factored block and A^{-1} from the handle-based entry points."""
    import paper_1708_04539_gb300 as ps
    h = ps.SelInv.from_problem(p, relax_pct=0)
    st = h.structure()
    assert st["nsuper"] == 1 and st["storage_size"] == p.n * p.n
    h.factor(torch.from_numpy(p.values).cuda())
    lu = h.get_selected(layout=ps.LAYOUT_FACTORS)
    h.selinv()
    ainv = h.get_selected(layout=ps.LAYOUT_SUPERNODAL)
    h.close()
    return lu, ainv


def _noalloc(torch, lu, n):
    from paper_1708_04539_gb300.binding import block_inverse_noalloc
    dev_lu = torch.from_numpy(lu.copy()).cuda()
    out = torch.full_like(dev_lu, float("nan"))
    block_inverse_noalloc(dev_lu, out, s=n)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_handle_path_twice(torch):
    cases = [gen.dense(200, 51, max_sn=256),
             gen.dense(77, 52, complex_values=True, max_sn=256),
             gen.dense(256, 53, max_sn=256)]
    for p in cases:
        lu, ainv = _reference(torch, p)
        first = _noalloc(torch, lu, p.n)
        second = _noalloc(torch, lu, p.n)
        assert normwise_error(first, ainv) < TOL
        assert normwise_error(second, ainv) < TOL
        assert np.array_equal(first, second)
        # and against the definition of the inverse, A A^{-1} = I
        a = p.dense()
        inv = first.reshape(p.n, p.n, order="F")
        assert np.abs(a @ inv - np.eye(p.n)).max() < 1e-12


def test_noalloc_rejects_oversized_block(torch):
    import ctypes
    import paper_1708_04539_gb300 as ps
    from paper_1708_04539_gb300.binding import NOALLOC_MAX_S, block_inverse_noalloc
    s = NOALLOC_MAX_S + 1
    blk = torch.zeros((s, s), dtype=torch.float64, device="cuda")
    out = torch.zeros_like(blk)
    with pytest.raises(ValueError):
        block_inverse_noalloc(blk, out, s=s)
    # the library itself refuses it too (no launch is made)
    lib = ps.load_library()
    rc = lib.pselinv_block_inverse_noalloc(ps.F64, s, ctypes.c_void_p(blk.data_ptr()), s,
                                           ctypes.c_void_p(out.data_ptr()), s, None)
    assert rc == -1


def test_noalloc_library_rejects_host_pointers(torch):
    """A host buffer never reaches a kernel: the library checks where its
    pointers live before launching."""
    import ctypes
    import paper_1708_04539_gb300 as ps
    lib = ps.load_library()
    host = np.eye(8)
    dev = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    hp, dp = ctypes.c_void_p(host.ctypes.data), ctypes.c_void_p(dev.data_ptr())
    assert lib.pselinv_block_inverse_noalloc(ps.F64, 8, hp, 8, dp, 8, None) == -1
    assert lib.pselinv_block_inverse_noalloc(ps.F64, 8, dp, 8, hp, 8, None) == -1
