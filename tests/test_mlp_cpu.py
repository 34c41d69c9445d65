"""Cost-model reference on the CPU: its gradient against finite differences,
and the library's host-side input encoding against the reference's."""
import numpy as np
import pytest

from oracle import mlp


class Rec:
    def __init__(self, kind, param, slot, prec, feat):
        self.kind, self.param, self.slot, self.precision, self.feat = kind, param, slot, prec, feat


def random_records(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        kind = int(rng.integers(0, 2)) * 9  # 0 = GEMM, 9 = OZAKI_GEMM
        param = int(rng.integers(0, 3)) if kind == 0 else int(2 ** rng.integers(0, 5))
        out.append(Rec(kind, param, int(rng.integers(0, 3)), int(rng.integers(0, 2)),
                       list(rng.uniform(0, 30, 8))))
    return out


def test_reference_gradient_matches_finite_differences():
    H = 7
    rng = np.random.default_rng(0)
    npar = H * 16 + H + H * H + H + H + 1
    p = rng.normal(0, 0.4, npar)
    X = mlp.encode(random_records(25, 1))
    y = rng.normal(0, 1, 25)
    loss, g = mlp.loss_and_grad(p, H, X, y)
    fd = np.zeros_like(p)
    h = 1e-6
    for i in range(npar):
        q = p.copy(); q[i] += h
        lp, _ = mlp.loss_and_grad(q, H, X, y)
        q[i] -= 2 * h
        lm, _ = mlp.loss_and_grad(q, H, X, y)
        fd[i] = (lp - lm) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))


def test_library_encoding_matches_reference():
    from paper_1708_04539_gb300 import build
    build.build()
    from paper_1708_04539_gb300.binding import encode_records, make_record
    recs = random_records(40, 2)
    lib_recs = [make_record(kind=r.kind, param=r.param, slot=r.slot, precision=r.precision,
                            feat=r.feat) for r in recs]
    x_lib = encode_records(lib_recs)
    x_ref = mlp.encode(recs)
    assert np.allclose(x_lib, x_ref, atol=1e-6)
