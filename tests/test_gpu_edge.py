"""Degenerate shapes of Algorithm 1 on the GPU, FP64 and split, against the
oracle: a 1 x 1 matrix (one supernode, no row structure), a diagonal
matrix (every column its own root: C = {} everywhere, so Ainv_KK = D_K
alone), a forest of independent blocks (several roots, the sweep's first
level holds them all), a single supernode wider than the others' cut
(dense), and supernode widths that leave ragged 64-row tiles and partial
32-wide K blocks in the sliced products."""
from __future__ import annotations

import numpy as np
import pytest

import gen
import oracle
from gen.problems import _finish_small
from test_gpu_parity import compare_full, TOL_FP64

pytestmark = pytest.mark.gpu

TOL_SPLIT = 1e-9


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_04539_gb300 import build
    build.build()
    return _t


def run(torch, p, prec, relax=20):
    import paper_1708_04539_gb300 as ps
    h = ps.SelInv.from_problem(p, relax_pct=relax)
    h.factor(torch.from_numpy(np.ascontiguousarray(p.values)).cuda())
    if prec == ps.PREC_OZAKI_FP16:  # every level through the sliced products
        nlev = h.structure()["nlevels"]
        h.plan_set([(lev, 3, 0) for lev in range(nlev)], ps.PREC_OZAKI_FP16)
    h.selinv(precision=prec)
    st = h.structure()
    sn = h.get_selected(layout=ps.LAYOUT_SUPERNODAL)
    pa = h.get_selected()
    h.sync()
    h.close()
    return st, sn, pa


def diagonal(n, seed, complex_values=False):
    idx = np.arange(n)
    return _finish_small(n, idx, idx, seed, complex_values, f"diag_{n}", 16)


def forest(seed):
    """Three independent tridiagonal blocks of 40, 17 and 70 unknowns."""
    rows, cols, off = [np.arange(0)], [np.arange(0)], 0
    for m in (40, 17, 70):
        i = np.arange(m - 1) + off
        rows += [np.arange(off, off + m), i, i + 1]
        cols += [np.arange(off, off + m), i + 1, i]
        off += m
    return _finish_small(off, np.concatenate(rows), np.concatenate(cols), seed, False,
                         "forest", 16)


CASES = [
    ("one", lambda: diagonal(1, 951)),
    ("one_c", lambda: diagonal(1, 952, complex_values=True)),
    ("diagonal", lambda: diagonal(40, 953)),
    ("forest", lambda: forest(954)),
    ("dense_one_supernode", lambda: gen.dense(100, 955, max_sn=256)),
    ("ragged_tiles", lambda: gen.random_struct_sym(211, 0.05, 956, max_sn=37)),
]


@pytest.mark.parametrize("split", [False, True], ids=["fp64", "split"])
@pytest.mark.parametrize("name,maker", CASES, ids=[c[0] for c in CASES])
def test_degenerate_shapes_match_oracle(torch, name, maker, split):
    import paper_1708_04539_gb300 as ps
    p = maker()
    prec = ps.PREC_OZAKI_FP16 if split else ps.PREC_FP64
    st, sn, pa = run(torch, p, prec)
    sel, _ = compare_full(p, st, sn, 0, 20, tol=TOL_SPLIT if split else TOL_FP64)
    ref = oracle.extract(sel, p.colptr, p.rowind)
    assert np.max(np.abs(pa - ref)) <= (TOL_SPLIT if split else TOL_FP64) * np.max(np.abs(ref))
    if name.startswith("one") or name == "diagonal":
        # no row structure anywhere: Ainv_KK = U_KK^{-1} L_KK^{-1} = 1 / a_kk
        assert np.allclose(pa, 1.0 / p.values, rtol=1e-14, atol=0)
