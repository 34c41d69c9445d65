"""Input generators: determinism, structure and the recipe's stated properties."""
import numpy as np
import pytest

import gen
from helpers import csc_cols


def _check_csc(p):
    assert p.colptr[0] == 0 and p.colptr[-1] == p.rowind.size
    cols = csc_cols(p.colptr)
    for j in range(p.n):
        r = p.rowind[p.colptr[j]:p.colptr[j + 1]]
        assert np.all(np.diff(r) > 0) and j in r
    key = set(zip(p.rowind.tolist(), cols.tolist()))
    assert all((c, r) in key for r, c in key)  # structurally symmetric
    assert np.array_equal(np.sort(p.perm), np.arange(p.n))


@pytest.mark.parametrize("maker", [
    lambda s: gen.conv_diff_2d(7, s),
    lambda s: gen.upwind_3d(5, s),
    lambda s: gen.stencil27_complex(4, s),
    lambda s: gen.dg_blocks(2, 5, s),
    lambda s: gen.shifted_family(4, s, nshift=3),
    lambda s: gen.random_struct_sym(40, 0.1, s),
    lambda s: gen.sym_diffusion_3d(4, s),
])
def test_generators_valid_and_deterministic(maker):
    a, b, c = maker(5), maker(5), maker(6)
    _check_csc(a)
    assert np.array_equal(a.values, b.values) and np.array_equal(a.rowind, b.rowind)
    assert not np.array_equal(a.values, c.values)
    for k in range(a.nbatch):
        d = a.dense(k)
        off = np.abs(d).sum(axis=1) - np.abs(np.diag(d))
        assert np.all(np.abs(np.diag(d)) > off - 1e-12)  # diagonally dominant by rows


def test_symmetric_generators_are_symmetric():
    for p in (gen.sym_diffusion_3d(5, 3), gen.stencil27_complex(4, 3, eps=0.0),
              gen.random_struct_sym(50, 0.1, 3, symmetric_values=True)):
        d = p.dense(0)
        assert np.array_equal(d, d.T)


def test_conv_diff_values_follow_recipe():
    p = gen.conv_diff_2d(6, 1)
    d = p.dense()
    assert np.allclose(np.diag(d), 4.1)
    # a_{i,i+e} + a_{i,i-e} = -2 on an interior row, per axis
    i = 2 + 6 * 2
    assert np.isclose(d[i, i + 1] + d[i, i - 1], -2.0) and np.isclose(d[i, i + 6] + d[i, i - 6], -2.0)
    assert not np.allclose(d, d.T)


def test_nd_perm_separator_property():
    """The last plane of the ordering separates the two halves of the grid."""
    m = 9
    perm = gen.nd_perm((m, m), 8)
    sep = perm[-m:]
    x = sep % m
    assert np.all(x == x[0])  # a plane x = const
    left = perm[: perm.size - m]
    lx = left % m
    assert np.all(lx != x[0])


def test_config_sizes():
    assert gen.make_config(1).n == 961
    assert gen.make_config(2, size=10).n == 1000
    c4 = gen.make_config(4, size=6, instances=3)
    assert c4[0].nbatch == 3 and len(c4) == 4
