"""Nested-dissection ordering of the library (``pselinv_order_nd``, host
only): a valid, deterministic permutation; separators after the parts they
separate (a connected component keeps a contiguous range); less fill than
the natural order on grid and random graphs; and the whole host pipeline
(symbolic analysis, oracle selected inversion) consumes it unchanged."""
from __future__ import annotations

import dataclasses

import numpy as np
import pytest

import gen
import oracle
import paper_1708_04539_gb300 as ps


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1708_04539_gb300 import build
    build.build()


def fill(p, perm):
    """Stored entries of L (diagonal blocks' lower halves plus panels) for
    the strict (relax 0) supernodes of the ordering perm."""
    h = ps.SelInv(p.n, p.colptr, p.rowind, perm, relax_pct=0, host_only=True)
    st = h.structure()
    w, rp = st["sn_width"], st["rows_ptr"]
    return int(sum(int(w[k]) * (int(w[k]) + 1) // 2 + int(w[k]) * int(rp[k + 1] - rp[k])
                   for k in range(st["nsuper"])))


MAKERS = [
    ("grid2d", lambda: gen.conv_diff_2d(31, 1)),
    ("grid3d", lambda: gen.upwind_3d(12, 2)),
    ("random", lambda: gen.random_struct_sym(300, 0.02, 5)),
    ("tridiag", lambda: gen.tridiagonal(300, 3)),
    ("arrow", lambda: gen.arrow(200, 4)),
    ("dense", lambda: gen.dense(60, 6)),
    ("dg", lambda: gen.dg_blocks(3, 8, 7)),
]


@pytest.mark.parametrize("name,make", MAKERS, ids=[m[0] for m in MAKERS])
@pytest.mark.parametrize("leaf", [1, 16, 64])
def test_valid_and_deterministic(name, make, leaf):
    p = make()
    a = ps.order_nd(p.n, p.colptr, p.rowind, leaf=leaf)
    b = ps.order_nd(p.n, p.colptr, p.rowind, leaf=leaf)
    assert a.dtype == np.int64 and np.array_equal(np.sort(a), np.arange(p.n))
    assert np.array_equal(a, b)


@pytest.mark.parametrize("name,make", MAKERS[:3], ids=[m[0] for m in MAKERS[:3]])
def test_less_fill_than_natural_order(name, make):
    p = make()
    nd = fill(p, ps.order_nd(p.n, p.colptr, p.rowind, leaf=16))
    natural = fill(p, np.arange(p.n))
    assert nd < 0.75 * natural, (nd, natural)
    # within reach of the generators' geometric dissection on grids
    if name.startswith("grid"):
        assert nd <= 1.25 * fill(p, p.perm)


def test_separator_last_on_a_path():
    """On a path the first separator is one middle vertex, ordered last, and
    each half keeps a contiguous range before it."""
    p = gen.tridiagonal(63, 9)
    perm = ps.order_nd(p.n, p.colptr, p.rowind, leaf=1)
    last = int(perm[-1])
    assert 20 <= last <= 42
    left = set(range(last)), set(range(last + 1, p.n))
    first_block = set(int(v) for v in perm[:len(left[0])])
    assert first_block in left


def test_components_keep_contiguous_ranges():
    """A block-diagonal pattern (two grids): each connected component is
    ordered within one contiguous range of positions."""
    a, b = gen.conv_diff_2d(9, 1), gen.conv_diff_2d(7, 2)
    n = a.n + b.n
    colptr = np.concatenate([a.colptr, a.colptr[-1] + b.colptr[1:]])
    rowind = np.concatenate([a.rowind, b.rowind + a.n])
    perm = ps.order_nd(n, colptr, rowind, leaf=4)
    assert np.array_equal(np.sort(perm), np.arange(n))
    comp = (perm >= a.n).astype(int)
    assert np.count_nonzero(np.diff(comp)) == 1


def test_errors_and_empty():
    p = gen.conv_diff_2d(5, 1)
    with pytest.raises(ps.PselinvError) as e:
        ps.order_nd(p.n, p.colptr, p.rowind, leaf=0)
    assert e.value.code == -1
    # drop one off-diagonal entry: the pattern is no longer symmetric
    j = 0
    k = int(p.colptr[j + 1]) - 1
    colptr = p.colptr.copy()
    colptr[j + 1:] -= 1
    rowind = np.delete(p.rowind, k)
    with pytest.raises(ps.PselinvError) as e:
        ps.order_nd(p.n, colptr, rowind)
    assert e.value.code == -2
    assert ps.order_nd(0, np.zeros(1, np.int64), np.zeros(0, np.int64)).size == 0


@pytest.mark.parametrize("name,make", [MAKERS[0], MAKERS[2]], ids=["grid2d", "random"])
def test_host_pipeline_consumes_the_ordering(name, make):
    """The library's symbolic analysis under the ND ordering equals the
    oracle's (independent) analysis bit for bit, and the oracle's selected
    inverse under it equals the one under the generator's ordering (A^{-1}
    does not depend on the ordering)."""
    p = make()
    q = dataclasses.replace(p, perm=ps.order_nd(p.n, p.colptr, p.rowind, leaf=16))
    h = ps.SelInv.from_problem(q, relax_pct=20, host_only=True)
    st = h.structure()
    s = oracle.analyze(q, relax_pct=20)
    assert st["nsuper"] == s.nsup
    assert np.array_equal(st["etree"], s.parent)
    x = oracle.extract(oracle.selected_inverse(q), q.colptr, q.rowind)
    y = oracle.extract(oracle.selected_inverse(p), p.colptr, p.rowind)
    assert np.abs(x - y).max() <= 1e-12 * np.abs(y).max()


def test_analyze_orders_by_nested_dissection_on_request():
    """perm None with nd_leaf > 0: the analysis uses pselinv_order_nd's
    ordering (the structure reports it); nd_leaf 0 keeps the natural order;
    a negative nd_leaf is refused."""
    p = gen.upwind_3d(8, 4)
    h = ps.SelInv(p.n, p.colptr, p.rowind, None, nd_leaf=16, host_only=True)
    assert np.array_equal(h.structure()["perm"], ps.order_nd(p.n, p.colptr, p.rowind, leaf=16))
    h0 = ps.SelInv(p.n, p.colptr, p.rowind, None, host_only=True)
    assert np.array_equal(h0.structure()["perm"], np.arange(p.n))
    with pytest.raises(ps.PselinvError):
        ps.SelInv(p.n, p.colptr, p.rowind, None, nd_leaf=-1, host_only=True)
