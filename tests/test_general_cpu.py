"""Host analysis of general patterns (pselinv_analyze_general, CPU only):
the structures and orderings against the independent general oracle.

With strict supernodes (relax 0) every supernode's R_L and R_U are the
oracle's C_L and C_U of its last column, and columns join a supernode
exactly when the oracle's structures chain (j + 1 in C_L(j) and C_U(j),
sizes one apart).  With relaxation the supernodal structures contain the
scalar ones and are closed under the supernodal updates.  Nothing here
launches a kernel."""
from __future__ import annotations

import numpy as np
import pytest

import gen
import oracle
import paper_1708_04539_gb300 as ps
from paper_1708_04539_gb300.binding import inverse_coordinates
from helpers import csc_cols


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1708_04539_gb300 import build
    build.build()


CASES = [
    ("random", lambda: gen.general_random(60, 0.05, 501, max_sn=8)),
    ("random_c", lambda: gen.general_random(50, 0.06, 502, complex_values=True, max_sn=8)),
    ("oneway", lambda: gen.upwind_oneway_2d(9, 503, max_sn=16)),
    ("upper", lambda: gen.general_random(30, 0.2, 504, triangle="upper", row_scramble=False)),
    ("lower", lambda: gen.general_random(30, 0.2, 505, triangle="lower", row_scramble=False)),
    ("sym_pattern", lambda: gen.conv_diff_2d(8, 506, max_sn=16)),
]


def _handle(p, relax, **kw):
    return ps.SelInv.from_general_problem(p, relax_pct=relax, host_only=True, **kw)


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_strict_structures_match_oracle(name, make):
    p = make()
    h = _handle(p, 0)
    st = h.structure()
    g = oracle.ganalyze(p)
    assert st["general"]
    assert np.array_equal(st["perm"], p.meta.get("cperm", p.perm))
    assert np.array_equal(st["rperm"], p.meta.get("rperm", p.perm))
    first = list(st["sn_first"]) + [p.n]
    for K in range(st["nsuper"]):
        f, l = first[K], first[K + 1] - 1
        assert np.array_equal(st["rows"][st["rows_ptr"][K]:st["rows_ptr"][K + 1]], g.col_l(l))
        assert np.array_equal(st["urows"][st["urows_ptr"][K]:st["urows_ptr"][K + 1]], g.row_u(l))
        for j in range(f, l):  # the strict rule inside the supernode
            assert j + 1 in g.col_l(j) and j + 1 in g.row_u(j)
            assert g.col_l(j).size == g.col_l(j + 1).size + 1
            assert g.row_u(j).size == g.row_u(j + 1).size + 1
        if l + 1 < p.n and st["sn_width"][K] < p.max_supernode:  # and no longer
            j = l
            assert not (j + 1 in g.col_l(j) and j + 1 in g.row_u(j) and
                        g.col_l(j).size == g.col_l(j + 1).size + 1 and
                        g.row_u(j).size == g.row_u(j + 1).size + 1)
    h.close()


@pytest.mark.parametrize("relax", [0, 20, 100])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_storage_covers_the_oracle_pattern(name, make, relax):
    """The storage holds every entry of the oracle's pattern of (L+U)^T; the
    value map sends each entry of A to Atilde's position, and the output map
    to the transposed one (Eq. sel_entries)."""
    p = make()
    h = _handle(p, relax)
    st = h.structure()
    rows, cols = inverse_coordinates(st)
    key = rows * p.n + cols
    g = oracle.ganalyze(p)
    orows, ocols = g.inverse_pattern()
    assert np.all(np.isin(orows * p.n + ocols, key))
    assert np.unique(key).size == key.size
    irp = np.empty(p.n, dtype=np.int64)
    irp[st["rperm"]] = np.arange(p.n)
    icp = np.empty(p.n, dtype=np.int64)
    icp[st["perm"]] = np.arange(p.n)
    x = csc_cols(p.colptr)
    om = st["out_map"]
    assert np.array_equal(rows[om], icp[x]) and np.array_equal(cols[om], irp[p.rowind])
    # levels: a supernode after every supernode of its two structures
    first = np.asarray(st["sn_first"])
    sup = np.searchsorted(first, np.arange(p.n), side="right") - 1
    for K in range(st["nsuper"]):
        deps = np.concatenate([st["rows"][st["rows_ptr"][K]:st["rows_ptr"][K + 1]],
                               st["urows"][st["urows_ptr"][K]:st["urows_ptr"][K + 1]]])
        if deps.size:
            assert st["sn_depth"][K] == 1 + st["sn_depth"][sup[deps]].max()
        else:
            assert st["sn_depth"][K] == 0
    h.close()


def test_general_handle_refuses_split_and_grouping():
    p = gen.general_random(20, 0.1, 507)
    h = _handle(p, 0)
    with pytest.raises(ps.PselinvError) as e:
        ps.SelInv.group([h])
    assert e.value.code == -8
    with pytest.raises(ps.PselinvError):
        ps.SelInv.from_general_problem(p, symmetric=True, host_only=True)
    bad = p.meta["rperm"].copy()
    bad[0] = bad[1]
    with pytest.raises(ps.PselinvError):
        ps.SelInv.general(p.n, p.colptr, p.rowind, bad, p.meta["cperm"], host_only=True)
    h.close()
