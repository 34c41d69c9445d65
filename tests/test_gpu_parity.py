"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
element by element on the whole pattern of L+U, for the FP64 and complex128
paths, the factorisation, the schedules, and full-size spot checks.

Tolerance: the selected-entry error of ``helpers.selected_error`` (each
entry's error relative to the largest selected entry of its row and column)
must stay below 1e-10 for the FP64 products.
"""
from __future__ import annotations

import numpy as np
import pytest

import gen
import oracle
from helpers import csc_cols, selected_error

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_04539_gb300 import build
    build.build()
    return _t


def _handle(p, **kw):
    import paper_1708_04539_gb300 as ps
    return ps.SelInv.from_problem(p, **kw)


def gpu_run(torch, p, device_values=True, **kw):
    import paper_1708_04539_gb300 as ps
    h = _handle(p, **kw)
    vals = torch.from_numpy(np.ascontiguousarray(p.values)).cuda() if device_values else \
        np.ascontiguousarray(p.values)
    h.factor(vals)
    h.selinv()
    st = h.structure()
    sn = [h.get_selected(batch=b, layout=ps.LAYOUT_SUPERNODAL) for b in range(p.nbatch)]
    pa = [h.get_selected(batch=b) for b in range(p.nbatch)]
    fac = [h.get_selected(batch=b, layout=ps.LAYOUT_FACTORS) for b in range(p.nbatch)]
    h.sync()
    return h, st, sn, pa, fac


def oracle_coo(p, b, relax):
    sel = oracle.selected_inverse(p, b=b, relax_pct=relax)
    rows, cols = sel.sym.lu_pattern()
    return sel, rows, cols, sel.values_lu_order()


def compare_full(p, st, sn_vals, b, relax, tol=TOL_FP64):
    from paper_1708_04539_gb300.binding import supernodal_coordinates
    sel, orows, ocols, ovals = oracle_coo(p, b, relax)
    grows, gcols = supernodal_coordinates(st)
    gk = grows * p.n + gcols
    ok = orows * p.n + ocols
    gi, oi = np.argsort(gk), np.argsort(ok)
    assert np.array_equal(gk[gi], ok[oi]), "structure differs from the oracle's"
    err = selected_error(sn_vals[gi], ovals[oi], orows[oi], ocols[oi], p.n)
    assert err < tol, err
    return sel, err


CASES = [
    ("cfg1", lambda: gen.make_config(1), 20),
    ("cfg1_strict", lambda: gen.make_config(1), 0),
    ("upwind12", lambda: gen.upwind_3d(12, 31, max_sn=64), 20),
    ("upwind16_wide", lambda: gen.upwind_3d(16, 32, max_sn=256), 20),
    ("stencil27_c", lambda: gen.stencil27_complex(8, 33, max_sn=64), 20),
    ("dg", lambda: gen.dg_blocks(3, 16, 34, max_sn=48), 20),
    ("random", lambda: gen.random_struct_sym(300, 0.02, 35, max_sn=24), 30),
    ("random_c", lambda: gen.random_struct_sym(250, 0.03, 36, complex_values=True, max_sn=20), 20),
    ("dense", lambda: gen.dense(150, 37, max_sn=40), 0),
    ("tridiag", lambda: gen.tridiagonal(300, 38), 0),
    ("arrow", lambda: gen.arrow(200, 39), 20),
    ("grid2d_c", lambda: gen.conv_diff_2d(25, 40, imag_diag=0.1, max_sn=32), 20),
]


@pytest.mark.parametrize("name,maker,relax", CASES, ids=[c[0] for c in CASES])
def test_selinv_matches_oracle(torch, name, maker, relax):
    p = maker()
    h, st, sn, pa, fac = gpu_run(torch, p, relax_pct=relax)
    sel, _ = compare_full(p, st, sn[0], 0, relax)
    # pattern-of-A extraction (Theorem 2) against the oracle's extraction
    ref = oracle.extract(sel, p.colptr, p.rowind)
    err = selected_error(pa[0], ref, p.rowind, csc_cols(p.colptr), p.n)
    assert err < TOL_FP64
    h.close()


@pytest.mark.parametrize("name,maker,relax", CASES[:6], ids=[c[0] for c in CASES[:6]])
def test_factor_matches_oracle(torch, name, maker, relax):
    from paper_1708_04539_gb300.binding import supernodal_coordinates
    p = maker()
    h, st, sn, pa, fac = gpu_run(torch, p, relax_pct=relax)
    s = oracle.analyze(p, relax_pct=relax)
    f = oracle.lu(s, p.colptr, p.rowind, p.values)
    orows, ocols = s.lu_pattern()
    # oracle order: diag (U_kk), lower (L), upper (U); GPU storage holds the same entries
    ovals = np.concatenate([f.diag, f.low, f.up])
    grows, gcols = supernodal_coordinates(st)
    gk, ok = grows * p.n + gcols, orows * p.n + ocols
    gi, oi = np.argsort(gk), np.argsort(ok)
    assert np.array_equal(gk[gi], ok[oi])
    err = selected_error(fac[0][gi], ovals[oi], orows[oi], ocols[oi], p.n)
    assert err < 1e-12, err
    h.close()


def test_batched_shifts_match_oracle(torch):
    p = gen.shifted_family(6, 41, nshift=3, max_sn=48)
    h, st, sn, pa, fac = gpu_run(torch, p, relax_pct=20)
    for b in range(p.nbatch):
        compare_full(p, st, sn[b], b, 20)
    h.close()


def test_schedules_graph_and_host_buffers_agree(torch):
    import paper_1708_04539_gb300 as ps
    p = gen.upwind_3d(10, 42, max_sn=64)
    _, _, sn_lvl, pa_lvl, _ = gpu_run(torch, p)
    _, _, sn_sn, _, _ = gpu_run(torch, p, schedule=ps.SCHED_PER_SUPERNODE)
    _, _, sn_ng, _, _ = gpu_run(torch, p, use_graph=False)
    _, _, sn_host, pa_host, _ = gpu_run(torch, p, device_values=False)
    _, _, sn_chk, _, _ = gpu_run(torch, p, check_level=1)
    scale = np.abs(sn_lvl[0]).max()
    for other in (sn_sn, sn_ng, sn_host, sn_chk):
        assert np.abs(other[0] - sn_lvl[0]).max() <= 1e-13 * scale
    assert np.abs(pa_host[0] - pa_lvl[0]).max() <= 1e-13 * scale


def test_repeated_selinv_is_stable(torch):
    import paper_1708_04539_gb300 as ps
    p = gen.upwind_3d(9, 43, max_sn=64)
    h = _handle(p)
    h.factor(torch.from_numpy(p.values).cuda())
    outs = []
    for _ in range(3):
        h.selinv()
        outs.append(h.get_selected(layout=ps.LAYOUT_SUPERNODAL))
    assert np.abs(outs[1] - outs[0]).max() <= 1e-13 * np.abs(outs[0]).max()
    assert np.abs(outs[2] - outs[0]).max() <= 1e-13 * np.abs(outs[0]).max()
    # a second factorisation with other values reuses the handle
    q = gen.upwind_3d(9, 44, max_sn=64)
    h.factor(torch.from_numpy(q.values).cuda())
    h.selinv()
    st = h.structure()
    compare_full(q, st, h.get_selected(layout=ps.LAYOUT_SUPERNODAL), 0, 20)
    h.close()


def test_zero_pivot_reported(torch):
    import paper_1708_04539_gb300 as ps
    p = gen.tridiagonal(40, 45)
    v = p.values.copy()
    v[0] = 0.0  # A_00 with the identity ordering
    h = _handle(p, relax_pct=0)
    with pytest.raises(ps.PselinvError) as e:
        h.factor(torch.from_numpy(v).cuda())
    assert e.value.code == -3 and e.value.info == 0
    # the handle stays usable
    h.factor(torch.from_numpy(p.values).cuda())
    h.selinv()
    h.sync()
    h.close()


def test_empty_and_single_entry(torch):
    import paper_1708_04539_gb300 as ps
    p = gen.Problem("one", 1, np.array([0, 1]), np.array([0]), np.array([4.0]), np.array([0]), 8)
    h = _handle(p)
    h.factor(torch.tensor([4.0], dtype=torch.float64, device="cuda"))
    h.selinv()
    assert np.allclose(h.get_selected(), [0.25])
    h.close()
    # diagonal matrix: every supernode a root, no panels
    n = 70
    idx = np.arange(n, dtype=np.int64)
    vals = np.linspace(1.0, 2.0, n)
    d = gen.Problem("diag", n, np.arange(n + 1), idx, vals, idx, 8)
    h = _handle(d)
    h.factor(torch.from_numpy(vals).cuda())
    h.selinv()
    assert np.allclose(h.get_selected(), 1.0 / vals, rtol=1e-15)
    h.close()


@pytest.mark.slow
def test_config2_full_size_sampled(torch):
    """The bench workload at full size: sampled columns and rows of A^{-1}
    from sparse triangular solves, and the row/column identities."""
    import paper_1708_04539_gb300 as ps
    from oracle.sampled import SampledInverse
    from paper_1708_04539_gb300.binding import supernodal_coordinates
    p = gen.make_config(2)
    h, st, sn, pa, fac = gpu_run(torch, p)
    rng = np.random.default_rng(7)
    cols = np.r_[rng.choice(p.n, 6, replace=False), p.perm[-1], p.perm[0]]
    samp = SampledInverse(p)
    X = samp.columns(cols)
    grows, gcols = supernodal_coordinates(st)
    orow, ocol = p.perm[grows], p.perm[gcols]
    for k, j in enumerate(cols):
        m = ocol == j
        ref = X[orow[m], k]
        assert np.abs(sn[0][m] - ref).max() <= TOL_FP64 * np.abs(X[:, k]).max()
    Y = samp.rows(cols)
    for k, i in enumerate(cols):
        m = orow == i
        ref = Y[ocol[m], k]
        assert np.abs(sn[0][m] - ref).max() <= TOL_FP64 * np.abs(Y[:, k]).max()
    # row identities sum_j A_ij (A^{-1})_ji = 1 from the pattern-of-A output
    B = pa[0]
    c = csc_cols(p.colptr)
    key = c * p.n + p.rowind
    order = np.argsort(key)
    tpos = order[np.searchsorted(key[order], p.rowind * p.n + c)]
    rowsum = np.zeros(p.n)
    np.add.at(rowsum, p.rowind, p.values * B[tpos])
    assert np.abs(rowsum - 1).max() < 1e-11
    h.close()


def test_uneven_instances_in_one_sweep(torch):
    """Matrices of different sizes (the uneven 2D grids of the pole-expansion
    workload, at reduced sizes) grouped as a direct sum: one factorisation and
    one selected inversion; every instance matches its own oracle result."""
    import paper_1708_04539_gb300 as ps
    probs = gen.make_config(4, size=12, instances=6)[1:]   # 6 complex 2D grids, sides 6..12
    g = ps.InstanceGroup([(q.n, q.colptr, q.rowind, q.perm) for q in probs], max_supernode=64)
    vals = g.values([q.values for q in probs])
    g.handle.factor(torch.from_numpy(vals).cuda())
    for prec, tol in ((ps.PREC_FP64, 1e-10), (ps.PREC_OZAKI_FP16, 1e-9)):
        g.handle.selinv(precision=prec)
        parts = g.split(g.handle.get_selected())
        for q, got in zip(probs, parts):
            ref = oracle.extract(oracle.selected_inverse(q), q.colptr, q.rowind)
            assert selected_error(got, ref, q.rowind, csc_cols(q.colptr), q.n) < tol
    st = g.handle.structure()
    roots = np.sum(st["sn_parent"] == -1)
    assert roots >= len(probs)   # a forest: at least one root per instance
    g.handle.close()


def test_bounded_wait_reports_timeout(torch):
    """A device wait that can never complete gives up within its budget and
    the host sees PSELINV_ERR_TIMEOUT; the context stays usable."""
    import time
    from paper_1708_04539_gb300.binding import wait_selftest
    t0 = time.perf_counter()
    assert wait_selftest(20000) == -6
    assert time.perf_counter() - t0 < 10.0
    # the device still works afterwards
    p = gen.make_config(1)
    h, st, sn, pa, fac = gpu_run(torch, p)
    compare_full(p, st, sn[0], 0, 20)
    h.close()
