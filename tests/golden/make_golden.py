"""Writes the oracle regression fixtures of this folder.  Calls only the oracle and
the seeded input generators:

    python tests/golden/make_golden.py

Case: Q2 (q = 3) on a 2 x 1 x 1 box with vertices perturbed by 10% of h (seed 0),
E = 1, nu = 0.3, displacement from the smooth-field recipe (amplitude 0.05, seed 1),
du ~ N(0, 1) (seed 2), uniaxial Dirichlet mask.  Stored: the residual F(u) with
g = 0 on the constrained rows, and J du in the current-configuration (A) and
initial-configuration (B) linearisations, 17 significant digits each.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import fem  # noqa: E402
from paper_2204_01722_b300 import inputs  # noqa: E402

CASE = dict(n=(2, 1, 1), p=2, q=3, perturb=0.1, amp=0.05, E=1.0, nu=0.3)


def case():
    n, p, q = CASE["n"], CASE["p"], CASE["q"]
    V = inputs.box_vertices(*n, perturb=CASE["perturb"], seed=0)
    sp = fem.Space(*n, V, p, q)
    mat = fem.Material(CASE["E"], CASE["nu"], sp.ne)
    u = inputs.smooth_field(sp.node_coords(), CASE["amp"], seed=1).ravel()
    du = inputs.normal_vector(sp.n_dof, seed=2)
    mask = inputs.uniaxial_mask(sp.node_dims)
    return sp, mat, u, du, mask


def values():
    sp, mat, u, du, mask = case()
    st = fem.qp_state(sp, mat, u)
    return {"residual": fem.residual(sp, mat, u, mask),
            "jacobian_apply_A": fem.jacobian_apply(sp, st, du, mask, form="A"),
            "jacobian_apply_B": fem.jacobian_apply(sp, st, du, mask, form="B")}


def path(name):
    return os.path.join(HERE, f"oracle_q2_2x1x1_{name}.txt")


def main():
    for name, v in values().items():
        hdr = (f"oracle {name}, case {CASE} (written by tests/golden/make_golden.py from the oracle;"
               f" a regression pin of the oracle's arithmetic)")
        np.savetxt(path(name), v, fmt="%.17e", header=hdr)


if __name__ == "__main__":
    main()
