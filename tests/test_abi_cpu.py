"""C-ABI library on the CPU: it loads, exports every declared symbol, and its
host-only symbolic analysis equals the oracle's (independent) analysis bit
for bit.  No compute call is made here."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

import gen
import oracle
import paper_1708_04539_gb300 as ps
from paper_1708_04539_gb300.binding import supernodal_coordinates
from helpers import csc_cols

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1708_04539_gb300 import build
    build.build()


def declared_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(pselinv_\w+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(ps.lib_path())
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_plan_cache_file_round_trip_host_only(tmp_path):
    """Tuned values saved to a cache file come back into another handle of
    the same structure; a file for another structure or precision, a
    malformed file and a missing file are refused without changing the
    handle's values."""
    p = gen.conv_diff_2d(24, seed=3)
    h = ps.SelInv.from_problem(p, host_only=True)
    nlev = h.structure()["nlevels"]
    triples = [(0, 0, 3), (0, 3, 1), (1, 1, 4), (nlev - 1, 4, 2), (nlev - 1, 5, 3)]
    h.plan_set(triples, ps.PREC_OZAKI_FP16)
    path = tmp_path / "plan.txt"
    h.plan_save(path, ps.PREC_OZAKI_FP16)
    h2 = ps.SelInv.from_problem(p, host_only=True)
    h2.plan_load(path, ps.PREC_OZAKI_FP16)
    assert h2.plan_get(ps.PREC_OZAKI_FP16) == sorted(triples)
    keep = [(0, 0, 1)]
    other = ps.SelInv.from_problem(gen.conv_diff_2d(20, seed=3), host_only=True)
    other.plan_set(keep, ps.PREC_OZAKI_FP16)
    bad = tmp_path / "bad.txt"
    bad.write_text("not a plan\n")
    for h3, path3, prec in [(other, path, ps.PREC_OZAKI_FP16), (h2, path, ps.PREC_FP64),
                            (other, bad, ps.PREC_OZAKI_FP16),
                            (other, tmp_path / "missing.txt", ps.PREC_OZAKI_FP16)]:
        with pytest.raises(ps.PselinvError):
            h3.plan_load(path3, prec)
    assert other.plan_get(ps.PREC_OZAKI_FP16) == keep
    # a saved value out of range is refused too
    txt = path.read_text().splitlines()
    txt[1] = "0 0 9"
    bad.write_text("\n".join(txt) + "\n")
    with pytest.raises(ps.PselinvError):
        h2.plan_load(bad, ps.PREC_OZAKI_FP16)
    assert h2.plan_get(ps.PREC_OZAKI_FP16) == sorted(triples)


def _blocks_problem(sizes):
    """Block-diagonal pattern of dense diagonal blocks of the given sizes."""
    n = sum(sizes)
    rows, cols, o = [], [], 0
    for b in sizes:
        ii, jj = np.meshgrid(np.arange(o, o + b), np.arange(o, o + b), indexing="ij")
        rows.append(ii.ravel())
        cols.append(jj.ravel())
        o += b
    r, c = np.concatenate(rows), np.concatenate(cols)
    order = np.lexsort((r, c))
    r, c = r[order], c[order]
    colptr = np.concatenate([[0], np.cumsum(np.bincount(c, minlength=n))]).astype(np.int64)
    return n, colptr, r.astype(np.int64)


def test_plan_cache_refuses_structure_with_same_counts(tmp_path):
    """Two structures with the same n, supernode count and level count but
    different supernodes: a plan saved for one is refused by the other."""
    na, cpa, ria = _blocks_problem([2, 2])
    nb, cpb, rib = _blocks_problem([3, 1])
    ha = ps.SelInv(na, cpa, ria, max_supernode=3, relax_pct=0, host_only=True)
    hb = ps.SelInv(nb, cpb, rib, max_supernode=3, relax_pct=0, host_only=True)
    sa, sb = ha.structure(), hb.structure()
    assert (sa["n"], sa["nsuper"], sa["nlevels"]) == (sb["n"], sb["nsuper"], sb["nlevels"])
    assert list(sa["sn_width"]) != list(sb["sn_width"])
    ha.plan_set([(0, 0, 3)], ps.PREC_FP64)
    path = tmp_path / "plan_a.txt"
    ha.plan_save(path, ps.PREC_FP64)
    ha2 = ps.SelInv(na, cpa, ria, max_supernode=3, relax_pct=0, host_only=True)
    ha2.plan_load(path, ps.PREC_FP64)
    assert ha2.plan_get(ps.PREC_FP64) == [(0, 0, 3)]
    with pytest.raises(ps.PselinvError):
        hb.plan_load(path, ps.PREC_FP64)
    assert hb.plan_get(ps.PREC_FP64) == []


def _header_enum(name):
    txt = open(os.path.join(ROOT, "include", "pselinv.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    body = re.search(r"enum\s+" + name + r"\s*\{(.*?)\}", txt, flags=re.S).group(1)
    return {k: int(v) for k, v in re.findall(r"(PSELINV_\w+)\s*=\s*(-?\d+)", body)}


def test_binding_names_every_step_kind():
    """The profile records name their launch kind through the binding's
    table: every kind the header declares has a name there."""
    kinds = _header_enum("pselinv_step_kind")
    assert len(kinds) >= 12
    assert sorted(kinds.values()) == sorted(ps.binding.STEP_KINDS)
    assert ps.binding.STEP_KINDS[kinds["PSELINV_STEP_SMALL_LEVEL"]] == "small_level"


def test_error_strings_and_defaults():
    lib = ps.load_library()
    for code in range(0, -9, -1):
        assert lib.pselinv_error_string(code)
    o = ps.binding.Opts()
    lib.pselinv_default_opts(ctypes.byref(o))
    assert o.max_supernode == 256 and o.relax_pct == 20 and o.use_graph == 1
    assert o.factor_precision == ps.PREC_FP64 and o.factor_split_mflops == 0


def test_factor_precision_option_is_checked():
    """opts.factor_precision takes PREC_FP64 or PREC_OZAKI_FP16 only, at
    analysis and through the setter (host-only handles: no CUDA call)."""
    p = gen.tridiagonal(5, 1)
    for bad in (2, -1):
        with pytest.raises(ps.PselinvError) as e:
            ps.SelInv.from_problem(p, host_only=True, factor_precision=bad)
        assert e.value.code == -1
        with pytest.raises(ps.PselinvError):
            ps.SelInv.from_general_problem(p, host_only=True, factor_precision=bad)
    h = ps.SelInv.from_problem(p, host_only=True, factor_precision=ps.PREC_OZAKI_FP16,
                               factor_split_mflops=-1)
    h.set_factor_precision(ps.PREC_FP64)
    with pytest.raises(ps.PselinvError):
        h.set_factor_precision(3)
    h.close()


def _compare_with_oracle(p, relax):
    h = ps.SelInv.from_problem(p, relax_pct=relax, host_only=True)
    st = h.structure()
    s = oracle.analyze(p, relax_pct=relax)
    assert st["nsuper"] == s.nsup
    assert np.array_equal(st["etree"], s.parent)
    assert np.array_equal(st["sn_first"], s.supptr[:-1])
    assert np.array_equal(st["sn_width"], np.diff(s.supptr))
    assert np.array_equal(st["sn_parent"], s.sup_parent)
    assert np.array_equal(st["sn_depth"], s.sup_depth)
    for K in range(s.nsup):
        assert np.array_equal(st["rows"][st["rows_ptr"][K]:st["rows_ptr"][K + 1]],
                              s.supernode_rows(K))
    # levels partition the supernodes by depth
    for d in range(st["nlevels"]):
        ks = st["level_sn"][st["level_ptr"][d]:st["level_ptr"][d + 1]]
        assert np.all(st["sn_depth"][ks] == d)
    # the supernodal storage covers exactly the oracle's pattern of L+U
    rows, cols = supernodal_coordinates(st)
    orows, ocols = s.lu_pattern()
    assert rows.size == orows.size
    assert np.array_equal(np.sort(rows * p.n + cols), np.sort(orows * p.n + ocols))
    # the value map sends each entry of A to its permuted position
    iperm = np.empty(p.n, dtype=np.int64)
    iperm[p.perm] = np.arange(p.n)
    vm = st["value_map"]
    assert np.array_equal(rows[vm], iperm[p.rowind])
    assert np.array_equal(cols[vm], iperm[csc_cols(p.colptr)])
    # flop counts
    w = st["sn_width"].astype(float)
    c = np.diff(st["rows_ptr"]).astype(float)
    assert np.isclose(st["flops_selinv"], np.sum(4 * c * c * w + 4 * c * w * w + 4 / 3 * w ** 3))
    h.close()


@pytest.mark.parametrize("relax", [0, 20, 60])
@pytest.mark.parametrize("maker", [
    lambda: gen.make_config(1),
    lambda: gen.upwind_3d(8, 3, max_sn=32),
    lambda: gen.stencil27_complex(5, 4, max_sn=48),
    lambda: gen.dg_blocks(3, 8, 5, max_sn=24),
    lambda: gen.random_struct_sym(150, 0.03, 6, max_sn=7),
    lambda: gen.dense(30, 7, max_sn=8),
    lambda: gen.tridiagonal(50, 8),
])
def test_host_analysis_matches_oracle(maker, relax):
    _compare_with_oracle(maker(), relax)


def test_host_analysis_config2_matches_oracle():
    _compare_with_oracle(gen.make_config(2), 20)


def test_analysis_rejects_bad_input():
    p = gen.tridiagonal(5, 1)
    bad = p.rowind.copy()
    bad[1] = 4  # breaks both sorting and symmetry
    with pytest.raises(ps.PselinvError):
        ps.SelInv(p.n, p.colptr, bad, host_only=True)
    n = 3
    with pytest.raises(ps.PselinvError) as e:
        ps.SelInv(n, np.array([0, 2, 3, 4]), np.array([0, 1, 1, 2]), host_only=True)
    assert e.value.code == -2
    with pytest.raises(ps.PselinvError):
        ps.SelInv(p.n, p.colptr, p.rowind, perm=np.zeros(5, dtype=np.int64), host_only=True)


def test_host_only_handle_refuses_compute():
    p = gen.tridiagonal(5, 1)
    h = ps.SelInv.from_problem(p, host_only=True)
    with pytest.raises(ps.PselinvError):
        h.factor(p.values)


def test_plan_cache_round_trip_host_only():
    """The tuned-plan triples set on a handle come back unchanged; a bad
    triple is refused without touching the stored ones."""
    p = gen.conv_diff_2d(24, seed=3)
    h = ps.SelInv.from_problem(p, host_only=True)
    nlev = h.structure()["nlevels"]
    assert h.plan_get(ps.PREC_OZAKI_FP16) == []
    triples = [(0, 0, 1), (0, 3, 1), (1, 1, 4), (1, 2, 16), (nlev - 1, 4, 2), (nlev - 1, 5, 0)]
    h.plan_set(triples, ps.PREC_OZAKI_FP16)
    assert h.plan_get(ps.PREC_OZAKI_FP16) == sorted(triples)
    assert h.plan_get(ps.PREC_FP64) == []
    rows = [(1, 0, 3), (1, 4, 3), (1, 5, 3)]  # row panels in the GEMM slots
    h.plan_set(triples + rows, ps.PREC_OZAKI_FP16)
    assert h.plan_get(ps.PREC_OZAKI_FP16) == sorted(triples + rows)
    h.plan_set(triples, ps.PREC_OZAKI_FP16)
    for bad in [(nlev, 0, 0), (-1, 0, 0), (0, 6, 0), (0, 1, 3), (0, 3, 2), (0, 4, 4),
                (0, 0, 4), (0, 5, -1)]:
        with pytest.raises(ps.PselinvError):
            h.plan_set(triples + [bad], ps.PREC_OZAKI_FP16)
        assert h.plan_get(ps.PREC_OZAKI_FP16) == sorted(triples)
    for bad in [(0, 3, 0), (0, 1, 4), (0, 0, 4)]:  # no precision slot in the FP64 plan
        with pytest.raises(ps.PselinvError):
            h.plan_set([bad], ps.PREC_FP64)
    h.plan_set([(0, 0, 3)], ps.PREC_FP64)
    h.plan_set([(0, 1, 2)], ps.PREC_FP64)
    assert h.plan_get(ps.PREC_FP64) == [(0, 1, 2)]
    h.plan_set([], ps.PREC_OZAKI_FP16)
    assert h.plan_get(ps.PREC_OZAKI_FP16) == []
    assert h.plan_get(ps.PREC_FP64) == [(0, 1, 2)]


def test_group_is_the_direct_sum_host_only():
    """pselinv_group through the C ABI: the grouped handle's structure is that
    of the direct sum of the members' patterns (orderings shifted), and the
    members stay usable."""
    a = gen.conv_diff_2d(7, 1, max_sn=16)
    b = gen.random_struct_sym(40, 0.1, 2, max_sn=16)
    c = gen.tridiagonal(9, 3, max_sn=16)
    members = [ps.SelInv.from_problem(q, host_only=True, max_supernode=16) for q in (a, b, c)]
    g = ps.SelInv.group(members, max_supernode=16, host_only=True)
    n_off = np.cumsum([0, a.n, b.n])
    z_off = np.cumsum([0, a.nnz, b.nnz])
    cp = np.concatenate([[0]] + [q.colptr[1:] + z for q, z in zip((a, b, c), z_off)])
    ri = np.concatenate([q.rowind + o for q, o in zip((a, b, c), n_off)])
    pm = np.concatenate([q.perm + o for q, o in zip((a, b, c), n_off)])
    d = ps.SelInv(int(n_off[-1] + c.n), cp, ri, pm, max_supernode=16, host_only=True)
    sg, sd = g.structure(), d.structure()
    for key in ("n", "nsuper", "nlevels", "storage_size", "nnz_a"):
        assert sg[key] == sd[key], key
    for key in ("perm", "sn_width", "sn_parent", "sn_depth", "rows_ptr", "rows", "value_map"):
        assert np.array_equal(sg[key], sd[key]), key
    assert members[1].structure()["n"] == b.n  # members untouched
    lib = ps.load_library()
    import ctypes
    out = ctypes.c_void_p()
    assert lib.pselinv_group(None, 0, None, ctypes.byref(out)) == -1
    for h in members + [g, d]:
        h.close()


def test_empty_and_one_by_one_analysis():
    """n = 0: an empty structure (no supernode, no level); n = 1: one
    supernode of width 1 with an empty row structure at depth 0."""
    h = ps.SelInv(0, np.array([0]), np.array([], dtype=np.int64), host_only=True)
    st = h.structure()
    assert st["nsuper"] == 0 and st["nlevels"] == 0 and st["storage_size"] == 0
    h.close()
    h = ps.SelInv(1, np.array([0, 1]), np.array([0]), host_only=True)
    st = h.structure()
    assert st["nsuper"] == 1 and st["nlevels"] == 1 and st["storage_size"] == 1
    assert np.array_equal(st["rows_ptr"], [0, 0])
    h.close()
