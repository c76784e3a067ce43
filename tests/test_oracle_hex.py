"""Pins of the oracle's unstructured hexahedral space (Sec. II-B: the element
restriction of a general mesh), CPU only.

* The box mesh written as an unstructured mesh, with every element's local frame
  a random cube rotation and vertex ids and element order shuffled, is the same
  discrete problem: after matching nodes by position, residual, Jacobian (both
  linearisations), diagonal and transfers equal the box space's.  Rotating an
  element permutes its Gauss points (the rule is symmetric), so this pins the
  coordinate-matched numbering and the orientation handling of the geometry.
* Patch test on an L-shaped (non-box) mesh: a linear displacement gives a
  constant stress, so the residual vanishes at every node off the boundary.
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from oracle import fem
from paper_2204_01722_b300 import inputs


def node_map(a, b):
    """perm with b.node_coords()[perm[i]] == a.node_coords()[i]."""
    d, idx = cKDTree(b.node_coords()).query(a.node_coords())
    assert d.max() < 1e-12
    assert len(np.unique(idx)) == len(idx)
    return idx


def dof_perm(perm):
    return (3 * perm[:, None] + np.arange(3)[None, :]).ravel()


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_rotated_shuffled_box_is_the_box(p):
    n = (3, 2, 2)
    V = inputs.box_vertices(*n, perturb=0.1, seed=p)
    box = fem.Space(*n, V, p, p + 1)
    Vh, H = inputs.hex_mesh_from_box(*n, V, seed=10 + p)
    hs = fem.HexSpace(Vh, H, p, p + 1)
    assert hs.n_nodes == box.n_nodes
    perm = node_map(box, hs)                       # box node i is hex node perm[i]
    dp = dof_perm(perm)
    mat_b = fem.Material(1.0, 0.3, box.ne)
    mat_h = fem.Material(1.0, 0.3, hs.ne)
    u = inputs.smooth_field(box.node_coords(), 0.05, seed=1).ravel()
    du = inputs.normal_vector(box.n_dof, seed=2)
    mask = inputs.uniaxial_mask(box.node_dims)
    uh, duh, mh = np.empty_like(u), np.empty_like(du), np.empty_like(mask)
    uh[dp], duh[dp], mh[dp] = u, du, mask
    sb, sh = fem.qp_state(box, mat_b, u), fem.qp_state(hs, mat_h, uh)
    for form in ("A", "B"):
        yb = fem.jacobian_apply(box, sb, du, mask, form=form)
        yh = fem.jacobian_apply(hs, sh, duh, mh, form=form)
        assert np.linalg.norm(yh[dp] - yb) <= 1e-12 * np.linalg.norm(yb)
    rb, rh = fem.residual(box, mat_b, u, mask), fem.residual(hs, mat_h, uh, mh)
    assert np.linalg.norm(rh[dp] - rb) <= 1e-12 * np.linalg.norm(rb)
    db, dh = fem.diagonal(box, sb, mask), fem.diagonal(hs, sh, mh)
    assert np.linalg.norm(dh[dp] - db) <= 1e-12 * np.linalg.norm(db)
    if p > 1:
        cb, ch = fem.Space(*n, V, 1, p + 1), fem.HexSpace(Vh, H, 1, p + 1)
        pc = dof_perm(node_map(cb, ch))
        uc = inputs.normal_vector(cb.n_dof, seed=3)
        uch = np.empty_like(uc)
        uch[pc] = uc
        assert np.allclose(fem.prolong(ch, hs, uch)[dp], fem.prolong(cb, box, uc), atol=1e-13)
        assert np.allclose(fem.restrict(hs, ch, duh)[pc], fem.restrict(box, cb, du), atol=1e-12)


def boundary_nodes(space):
    """Nodes on faces that only one element uses."""
    faces = {}
    P, p = space.P, space.p
    lat = np.arange(P ** 3)
    i, j, k = lat % P, (lat // P) % P, lat // (P * P)
    sel = {(0, 0): i == 0, (0, 1): i == p, (1, 0): j == 0, (1, 1): j == p, (2, 0): k == 0, (2, 1): k == p}
    corner = {(0, 0): [0, 2, 4, 6], (0, 1): [1, 3, 5, 7], (1, 0): [0, 1, 4, 5], (1, 1): [2, 3, 6, 7],
              (2, 0): [0, 1, 2, 3], (2, 1): [4, 5, 6, 7]}
    for e in range(space.ne):
        for f, m in sel.items():
            key = tuple(sorted(space.elem_verts[e, corner[f]]))
            faces.setdefault(key, []).append(space.elem_nodes[e, m])
    out = np.zeros(space.n_nodes, dtype=bool)
    for nodes in faces.values():
        if len(nodes) == 1:
            out[nodes[0]] = True
    return out


@pytest.mark.parametrize("p", [1, 2, 3])
def test_patch_test_on_l_shaped_mesh(p):
    n = (3, 3, 2)
    ez, ey, ex = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    keep = ~((ex.ravel() >= 1) & (ey.ravel() >= 2))          # an L in x-y, extruded in z
    Vh, H = inputs.hex_mesh_from_box(*n, inputs.box_vertices(*n, perturb=0.1, seed=7), seed=8, keep=keep)
    hs = fem.HexSpace(Vh, H, p, p + 1)
    X = hs.node_coords()
    A = np.array([[0.02, -0.01, 0.015], [0.01, -0.03, 0.0], [-0.02, 0.01, 0.025]])
    u = (X @ A.T + np.array([0.1, -0.2, 0.05])).ravel()
    r = fem.residual(hs, fem.Material(1.0, 0.3, hs.ne), u).reshape(-1, 3)
    inner = ~boundary_nodes(hs)
    assert inner.sum() > 0
    scale = np.abs(r).max()
    assert np.abs(r[inner]).max() <= 1e-12 * max(scale, 1.0)
