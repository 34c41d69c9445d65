"""Pins of the two auxiliary oracle parts that the Theorem-1 pins do not reach.

* ``oracle/sampled.py`` computes whole columns and rows of A^{-1} with sparse
  LU solves; it is the checker of the full-size parity tests.  Here it is
  pinned, on small real and complex matrices with a random symmetric
  ordering and non-symmetric values, to the double-double Gauss-Jordan
  inverse (itself pinned to exact rationals and LAPACK in
  test_oracle_pins.py).  A wrong permutation, a transposed solve or rows
  and columns swapped all fail it.
* ``oracle/mlp.py`` is the float64 reference of the launch-shape cost model
  (not from the paper; its definition is the comment of
  ``pselinv_model_create`` in include/pselinv.h).  Its forward pass, loss
  and gradient are pinned to values worked out by hand on a two-unit
  network, and its input encoding to literal vectors written from that
  definition.

Nothing here calls the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import gen
import oracle
from oracle import mlp
from oracle.sampled import SampledInverse
from helpers import dense_inverse_ref


# ---------------------------------------------------------------------------
# sampled columns and rows
# ---------------------------------------------------------------------------
SAMPLED_CASES = [
    ("random_real", lambda: gen.random_struct_sym(70, 0.07, 301, permute=True)),
    ("random_complex", lambda: gen.random_struct_sym(60, 0.08, 302, complex_values=True,
                                                     permute=True)),
    ("grid_nd_real", lambda: gen.conv_diff_2d(9, 303, sigma=0.1, max_sn=16)),
    ("grid_nd_complex", lambda: gen.conv_diff_2d(8, 304, sigma=0.1, imag_diag=0.1, max_sn=16)),
]


@pytest.mark.parametrize("name,make", SAMPLED_CASES, ids=[c[0] for c in SAMPLED_CASES])
def test_sampled_inverse_matches_double_double(name, make, oracle_lib):
    p = make()
    assert not np.array_equal(p.perm, np.arange(p.n)), "the case must exercise the ordering"
    a = p.dense()
    assert np.max(np.abs(a - a.T)) > 0.1, "values must be non-symmetric"
    ref = dense_inverse_ref(p)
    scale = np.max(np.abs(ref))
    samp = SampledInverse(p)
    rng = np.random.default_rng(7)
    idx = np.unique(np.concatenate([[0, p.n - 1], rng.choice(p.n, 12, replace=False)]))
    cols = samp.columns(idx)            # A^{-1}[:, idx]
    rows = samp.rows(idx)               # A^{-1}[idx, :] transposed
    assert cols.shape == (p.n, idx.size) and rows.shape == (p.n, idx.size)
    assert np.max(np.abs(cols - ref[:, idx])) <= 1e-13 * scale
    assert np.max(np.abs(rows - ref[idx, :].T)) <= 1e-13 * scale


def test_sampled_inverse_of_instance_b(oracle_lib):
    """Instance b of a batch is the matrix that is inverted."""
    fam = gen.shifted_family(4, 305, nshift=3, max_sn=16)
    for b in range(fam.nbatch):
        ref = dense_inverse_ref(fam, b)
        got = SampledInverse(fam, b).columns(np.arange(fam.n))
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


# ---------------------------------------------------------------------------
# cost-model reference: a forward, loss and gradient worked out by hand
# ---------------------------------------------------------------------------
# tanh(ln(a) / 2) = (a - 1) / (a + 1): pre-activations ln(3)/2 and ln(9)/2
# give the activations 1/2 and 4/5 exactly.
T3 = 0.5 * math.log(3.0)   # tanh -> 0.5
T9 = 0.5 * math.log(9.0)   # tanh -> 0.8
H = 2


def hand_params():
    """Two hidden units, inputs x = (1, 2, 0, ..., 0).

    Layer 1: W1 rows (1/4, 1/2, 0...) and (-1/2, 1, 0...): W1 x = (5/4, 3/2);
             b1 = (T3 - 5/4, T9 - 3/2)               -> h1 = (1/2, 4/5)
    Layer 2: W2 = [[1, 1/2], [1/4, -1]]: W2 h1 = (9/10, -27/40);
             b2 = (T3 - 9/10, -T9 + 27/40)           -> h2 = (1/2, -4/5)
    Output:  w3 = (2, -1), b3 = 1/4                  -> 1 + 4/5 + 1/4 = 41/20
    """
    W1 = np.zeros((H, mlp.N_IN))
    W1[0, :2] = [0.25, 0.5]
    W1[1, :2] = [-0.5, 1.0]
    b1 = np.array([T3 - 1.25, T9 - 1.5])
    W2 = np.array([[1.0, 0.5], [0.25, -1.0]])
    b2 = np.array([T3 - 0.9, -T9 + 0.675])
    w3 = np.array([2.0, -1.0])
    b3 = 0.25
    p = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, [b3]])
    x = np.zeros((1, mlp.N_IN))
    x[0, :2] = [1.0, 2.0]
    return p, x


def test_mlp_forward_by_hand():
    p, x = hand_params()
    out, (h1, h2) = mlp.forward(p, H, x)
    assert np.allclose(h1, [[0.5, 0.8]], rtol=0, atol=1e-15)
    assert np.allclose(h2, [[0.5, -0.8]], rtol=0, atol=1e-15)
    assert abs(out[0] - 41.0 / 20.0) <= 1e-14


def test_mlp_loss_and_gradient_by_hand():
    """Target y = 2: error e = 1/20, loss e^2 = 1/400, dL/dout = 2e = 1/10.

    gw3 = h2 / 10 = (1/20, -2/25);  gb3 = 1/10
    d2  = (1/10) w3 * (1 - h2^2) = (1/10)(2, -1) * (3/4, 9/25) = (3/20, -9/250)
    gW2 = d2 h1^T = [[3/40, 3/25], [-9/500, -18/625]];  gb2 = d2
    d1  = (W2^T d2) * (1 - h1^2) = (141/1000, 111/1000) * (3/4, 9/25)
        = (423/4000, 999/25000)
    gW1 = d1 x^T (columns 0 and 1 only);  gb1 = d1
    """
    p, x = hand_params()
    loss, g = mlp.loss_and_grad(p, H, x, np.array([2.0]))
    assert abs(loss - 1.0 / 400.0) <= 1e-15
    d1 = np.array([423 / 4000, 999 / 25000])
    gW1 = np.zeros((H, mlp.N_IN))
    gW1[:, 0] = d1
    gW1[:, 1] = 2 * d1
    d2 = np.array([3 / 20, -9 / 250])
    gW2 = np.array([[3 / 40, 3 / 25], [-9 / 500, -18 / 625]])
    expect = np.concatenate([gW1.ravel(), d1, gW2.ravel(), d2, [1 / 20, -2 / 25], [1 / 10]])
    assert g.shape == expect.shape
    assert np.max(np.abs(g - expect)) <= 1e-14


def test_mlp_loss_is_a_mean_over_records():
    """Two copies of the same record: the same loss and the same gradient."""
    p, x = hand_params()
    l1, g1 = mlp.loss_and_grad(p, H, x, np.array([2.0]))
    l2, g2 = mlp.loss_and_grad(p, H, np.vstack([x, x]), np.array([2.0, 2.0]))
    assert abs(l1 - l2) <= 1e-16 and np.max(np.abs(g1 - g2)) <= 1e-16


class Rec:
    def __init__(self, kind, param, slot, precision, feat):
        self.kind, self.param, self.slot, self.precision, self.feat = kind, param, slot, precision, feat


# Records and their network inputs, written from the definition: x[0..7] =
# feat / 32; x[8] = kind is GEMM (0); x[9] = kind is OZAKI_GEMM (9);
# x[10..12] one-hot GEMM tile config 0..2 (none for config 3, the row
# panels); x[13] = log2(K split) / 4 (OZAKI_GEMM); x[14] = slot / 2;
# x[15] = precision.
ENCODE_CASES = [
    (Rec(0, 1, 2, 0, [32, 64, 0, 16, 8, 4, 2, 1]),
     [1, 2, 0, 0.5, 0.25, 0.125, 0.0625, 0.03125, 1, 0, 0, 1, 0, 0, 1, 0]),
    (Rec(9, 8, 1, 1, [0, 0, 0, 0, 0, 0, 0, 96]),
     [0, 0, 0, 0, 0, 0, 0, 3, 0, 1, 0, 0, 0, 0.75, 0.5, 1]),
    (Rec(0, 3, 0, 1, [16, 16, 16, 16, 16, 16, 16, 16]),
     [0.5] * 8 + [1, 0, 0, 0, 0, 0, 0, 1]),
    (Rec(0, 0, 1, 0, [1, 0, 0, 0, 0, 0, 0, 0]),
     [1 / 32, 0, 0, 0, 0, 0, 0, 0, 1, 0, 1, 0, 0, 0, 0.5, 0]),
    (Rec(9, 1, 2, 1, [2, 2, 2, 2, 2, 2, 2, 2]),
     [1 / 16] * 8 + [0, 1, 0, 0, 0, 0, 1, 1]),
]


def test_mlp_encoding_literal_vectors():
    recs = [c[0] for c in ENCODE_CASES]
    want = np.array([c[1] for c in ENCODE_CASES], dtype=np.float64)
    assert np.array_equal(mlp.encode(recs), want)


def test_library_encoding_literal_vectors():
    """The library's host encoding gives the same literal vectors."""
    from paper_1708_04539_gb300 import build
    build.build()
    from paper_1708_04539_gb300.binding import encode_records, make_record
    recs = [make_record(kind=r.kind, param=r.param, slot=r.slot, precision=r.precision,
                        feat=r.feat) for r, _ in ENCODE_CASES]
    want = np.array([c[1] for c in ENCODE_CASES], dtype=np.float32)
    assert np.array_equal(encode_records(recs), want)


# ---------------------------------------------------------------------------
# the oracle's level-parallel driver (CPU baseline timing) = its serial sweep
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("make", [
    lambda: gen.conv_diff_2d(20, 311, sigma=0.1, max_sn=16),
    lambda: gen.random_struct_sym(150, 0.03, 312, complex_values=True, permute=True),
    lambda: gen.upwind_3d(9, 313, max_sn=32),
])
def test_parallel_oracle_is_bitwise_serial(make, oracle_lib):
    p = make()
    for relax in (0, 20):
        sym = oracle.analyze(p, relax_pct=relax)
        fac = oracle.lu(sym, p.colptr, p.rowind, p.values)
        a = oracle.selinv(fac)
        for nt in (1, 3, 8):
            b = oracle.selinv_parallel(fac, nt)
            assert np.array_equal(a.low, b.low) and np.array_equal(a.up, b.up)
            assert np.array_equal(a.diag, b.diag)
