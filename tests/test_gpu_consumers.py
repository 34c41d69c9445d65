"""Pole-expansion consumers of a batch of selected inverses (the use that
motivates selected inversion, Section 1): the weighted sum over shifts on
pattern(A) and sum_l w_l Tr[B A_l^{-1}], against the oracle's per-instance
selected inverses combined on the CPU."""
from __future__ import annotations

import numpy as np
import pytest

import gen
import oracle
from helpers import csc_cols

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_04539_gb300 import build
    build.build()
    return _t


def transpose_positions(p):
    c = csc_cols(p.colptr)
    key = c * p.n + p.rowind
    order = np.argsort(key)
    return order[np.searchsorted(key[order], p.rowind * p.n + c)]


def oracle_pattern_values(p, b):
    return oracle.extract(oracle.selected_inverse(p, b=b), p.colptr, p.rowind)


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_pole_expansion_sum_and_trace(torch, prec):
    import paper_1708_04539_gb300 as ps
    p = gen.shifted_family(6, 91, nshift=5, max_sn=48)
    rng = np.random.default_rng(5)
    w = rng.standard_normal(p.nbatch) + 1j * rng.standard_normal(p.nbatch)
    B = rng.standard_normal(p.nnz) + 1j * rng.standard_normal(p.nnz)
    h = ps.SelInv.from_problem(p)
    h.factor(torch.from_numpy(p.values).cuda())
    h.selinv(precision=ps.PREC_FP64 if prec == "fp64" else ps.PREC_OZAKI_FP16)
    got = h.weighted_sum(w)
    tr = h.trace(w, B)
    tr_dev = h.trace(w, torch.from_numpy(B).cuda())     # B on the device
    h.close()
    per = [oracle_pattern_values(p, b) for b in range(p.nbatch)]
    ref = sum(wl * x for wl, x in zip(w, per))
    tol = 1e-10 if prec == "fp64" else 1e-9
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    tpos = transpose_positions(p)
    ref_tr = sum(wl * np.sum(B * x[tpos]) for wl, x in zip(w, per))
    scale = sum(abs(wl) * np.sum(np.abs(B * x[tpos])) for wl, x in zip(w, per))
    assert abs(tr - ref_tr) <= tol * scale
    assert tr_dev == tr                                  # fixed reduction order


def test_real_single_instance_trace_is_sum_of_identity(torch):
    """With B = A, Tr[B A^{-1}] = sum_ij A_ij (A^{-1})_ji = Tr[A A^{-1}] = n."""
    import paper_1708_04539_gb300 as ps
    p = gen.upwind_3d(8, 92, max_sn=64)
    h = ps.SelInv.from_problem(p)
    h.factor(torch.from_numpy(p.values).cuda())
    h.selinv(precision=ps.PREC_FP64)
    tr = h.trace(np.array([1.0]), p.values)
    assert abs(tr - p.n) <= 1e-10 * p.n
    ws = h.weighted_sum(np.array([2.0]))
    assert np.abs(ws - 2.0 * h.get_selected()).max() == 0.0
    h.close()
