"""Seeded synthetic inputs for the selected-inversion path.

This module only builds input matrices (sparsity pattern + values in CSC
form) and the fill-reducing ordering that Algorithm 1 takes as given
("permutation matrices P, Q" are inputs of the algorithm).  It contains none
of the method's arithmetic: no factorisation, no inversion.  Both the CPU
oracle (``oracle/``) and the CUDA path (``paper_1708_04539_gb300``) consume
what it produces; neither side imports the other.

The matrices stand in for the paper's test set (SIESTA / DGDFT / UF
collection matrices of the numerical-results section, which are not
available here): 2D/3D stencil sparsity, non-symmetric values on a
structurally symmetric pattern, complex shifts z from a pole expansion, and
DG-like dense element blocks.
"""
from .problems import (  # noqa: F401
    Problem,
    SEED_BASE,
    nd_perm,
    conv_diff_2d,
    sym_diffusion_3d,
    upwind_3d,
    stencil27_complex,
    shifted_family,
    dg_blocks,
    random_struct_sym,
    tridiagonal,
    arrow,
    dense,
    general_random,
    upwind_oneway_2d,
    make_config,
    CONFIG_NAMES,
)
