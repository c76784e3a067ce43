"""The roofline arithmetic of bench.py, counted independently on CPU.

* Algorithmic bytes of one apply: the stored scalars of every quadrature point,
  the du read and y write of every DoF, the int32 element map, the Dirichlet
  byte per node, counted from an oracle space of the same shape.
* Algorithmic flops: a sum-factorised apply written as a sequence of 1-D
  contractions on tensors of explicit shape, each contraction counting
  (outputs x length) multiply-adds, plus the pointwise flops per point.
"""
import os
import sys

import numpy as np
import pytest

from oracle import fem
from paper_2204_01722_b300 import inputs

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


@pytest.mark.parametrize("p,n", [(2, 3), (3, 2), (4, 2)])
@pytest.mark.parametrize("S,w", [(17, 8), (17, 4), (27, 8)])
def test_apply_bytes_counted_from_a_space(p, n, S, w):
    sp = fem.Space(n, n, n, inputs.box_vertices(n, n, n), p, p + 1)
    qpts = sp.ne * sp.wq.size
    expect = qpts * S * w + 2 * sp.n_dof * w + sp.elem_nodes.size * 4 + sp.n_nodes
    assert bench.apply_bytes(p, n, w, S) == expect
    assert bench.apply_bytes(p, n, w, S, bc_byte=False) == expect - sp.n_nodes
    assert bench.n_dof_of(p, n) == sp.n_dof


def contraction_fmas(shape, axis, length_out):
    """Multiply-adds of one 1-D contraction along `axis` to `length_out` outputs."""
    out = list(shape)
    out[axis] = length_out
    return int(np.prod(out)) * shape[axis], tuple(out)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_apply_flops_counted_by_contractions(p):
    P = Q = p + 1
    fma = 0
    for _ in range(3):                      # components
        s = (P, P, P)                       # interpolation to the points, x then y then z
        for ax in range(3):
            f, s = contraction_fmas(s, ax, Q)
            fma += f
        for ax in range(3):                 # collocated derivative along each direction
            f, _ = contraction_fmas((Q, Q, Q), ax, Q)
            fma += f
        for ax in range(3):                 # transposes back to the nodes
            f, _ = contraction_fmas((Q, Q, Q), ax, Q)
            fma += f
        s = (Q, Q, Q)
        for ax in range(3):
            f, s = contraction_fmas(s, ax, P)
            fma += f
    n = 2
    assert bench.apply_flops(p, n) == n ** 3 * (2 * fma + 168 * Q ** 3)


def test_headline_figures():
    assert abs(bench.apply_bytes(3, 48, 8) / 1e9 - 1.140) < 1e-3
    assert abs(bench.apply_bytes(3, 48, 4, bc_byte=False) / 1e9 - 0.583) < 1e-3
    assert abs(bench.apply_flops(3, 48) / 1e9 - 3.23) < 5e-3
