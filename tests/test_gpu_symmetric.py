"""The symmetric variant (A = A^T): the sweep that skips U's normalisation,
step 5's product and the column slicing of G must give the same selected
inverse as the general sweep and as the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import gen
from test_gpu_parity import compare_full, TOL_FP64
from test_gpu_ozaki import force_split, TOL_SPLIT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_04539_gb300 import build
    build.build()
    return _t


CASES = [
    ("diffusion10", lambda: gen.sym_diffusion_3d(10, 81, max_sn=64)),
    ("diffusion14_wide", lambda: gen.sym_diffusion_3d(14, 82, max_sn=256)),
    ("complex27_sym", lambda: gen.stencil27_complex(7, 83, eps=0.0, max_sn=64)),
    ("random_sym", lambda: gen.random_struct_sym(300, 0.03, 84, symmetric_values=True, max_sn=24)),
]


def run(torch, p, prec, symmetric, all_split=False, **kw):
    import paper_1708_04539_gb300 as ps
    h = ps.SelInv.from_problem(p, symmetric=symmetric, **kw)
    h.factor(torch.from_numpy(np.ascontiguousarray(p.values)).cuda())
    if all_split:
        force_split(h)
    h.selinv(precision=prec)
    st = h.structure()
    sn = h.get_selected(layout=ps.LAYOUT_SUPERNODAL)
    h.sync()
    h.close()
    return st, sn


@pytest.mark.parametrize("name,maker", CASES, ids=[c[0] for c in CASES])
def test_symmetric_sweep_matches_oracle_and_general_sweep(torch, name, maker):
    import paper_1708_04539_gb300 as ps
    p = maker()
    st, sym64 = run(torch, p, ps.PREC_FP64, True)
    compare_full(p, st, sym64, 0, 20, tol=TOL_FP64)
    _, gen64 = run(torch, p, ps.PREC_FP64, False)
    assert np.abs(sym64 - gen64).max() <= 1e-12 * np.abs(gen64).max()
    st, symsp = run(torch, p, ps.PREC_OZAKI_FP16, True, all_split=True)
    compare_full(p, st, symsp, 0, 20, tol=TOL_SPLIT)
    st, symspn = run(torch, p, ps.PREC_OZAKI_FP16, True, all_split=True, split_normalise=True)
    compare_full(p, st, symspn, 0, 20, tol=TOL_SPLIT)


@pytest.mark.parametrize("name,maker", CASES, ids=[c[0] for c in CASES])
def test_symmetric_factorisation(torch, name, maker):
    """For A = A^T the factorisation updates only the lower triangle (the
    Schur complements are symmetric; U's panels are solved from L's, the
    diagonal blocks mirrored before their LU): the factors equal the general
    factorisation's, FP64 and with split Schur products, and the symmetric
    plan runs half the Schur-product work."""
    import paper_1708_04539_gb300 as ps
    p = maker()
    vals = torch.from_numpy(np.ascontiguousarray(p.values)).cuda()
    g = ps.SelInv.from_problem(p)
    g.factor(vals)
    ref = g.get_selected(layout=ps.LAYOUT_FACTORS)
    gflops = sum(s["flops"] for s in g.profile(1) if s["kind"] == "gemm")
    g.close()
    scale = np.abs(ref).max()
    for fprec, tol in ((ps.PREC_FP64, 1e-12), (ps.PREC_OZAKI_FP16, 1e-10)):
        h = ps.SelInv.from_problem(p, symmetric=True, factor_precision=fprec,
                                   factor_split_mflops=-1)
        h.factor(vals)
        fac = h.get_selected(layout=ps.LAYOUT_FACTORS)
        prof = h.profile(1)
        h.close()
        assert np.abs(fac - ref).max() <= tol * scale, (fprec, np.abs(fac - ref).max() / scale)
        if fprec == ps.PREC_FP64:
            sflops = sum(s["flops"] for s in prof if s["kind"] == "gemm")
            assert sflops < 0.9 * gflops, (sflops, gflops)
