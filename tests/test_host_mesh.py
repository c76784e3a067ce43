"""Host logic of the library on the CPU (no GPU needed): the unstructured-mesh
numbering behind nh_space_hex and the symbolic phase of the Q1 COO assembly.

* Numbering: on rotated/shuffled boxes and L-shaped meshes, p = 1..4, the
  library's topological numbering and the oracle's coordinate-matched one
  (tests/test_oracle_hex.py pins it) describe the same nodes: one-to-one node
  correspondence, equal element maps after relabelling, equal coordinates.
* Invalid meshes are refused with the reason.
* Block pattern: equals the set of node pairs that share an element.
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from oracle import fem
from paper_2204_01722_b300 import inputs

nh = pytest.importorskip("paper_2204_01722_b300.nh")


def mesh(kind, n, seed):
    V = inputs.box_vertices(*n, perturb=0.1, seed=seed)
    keep = None
    if kind == "L":
        ez, ey, ex = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
        keep = ~((ex.ravel() >= 1) & (ey.ravel() >= n[1] - 1))
    return inputs.hex_mesh_from_box(*n, V, seed=seed + 1, keep=keep)


@pytest.mark.parametrize("kind", ["rotated", "L"])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_numbering_matches_oracle(kind, p):
    Vh, H = mesh(kind, (4, 3, 2), seed=p)
    emap, X = nh.nh_hex_mesh_numbering(Vh, H, p)
    hs = fem.HexSpace(Vh, H, p, p + 1)
    assert X.shape[0] == hs.n_nodes
    d, perm = cKDTree(hs.node_coords()).query(X)
    assert d.max() < 1e-13 and len(np.unique(perm)) == len(perm)
    assert np.array_equal(perm[emap], hs.elem_nodes)


def test_invalid_meshes_are_refused():
    Vh, H = inputs.hex_mesh_from_box(2, 1, 1, inputs.box_vertices(2, 1, 1), reorient=False, permute=False)
    cases = {"inverted": H.copy(), "outside": H.copy(), "repeats": H.copy(),
             "more than two": np.vstack([H, H[:1]])}
    cases["inverted"][0, [0, 1]] = cases["inverted"][0, [1, 0]]
    cases["outside"][1, 3] = len(Vh)
    cases["repeats"][1, 0] = cases["repeats"][1, 1]
    for word, bad in cases.items():
        with pytest.raises(nh.NhError) as e:
            nh.nh_hex_mesh_numbering(Vh, bad, 2)
        assert e.value.status == nh.NH_ERR_ARG and word in str(e.value)
    with pytest.raises(nh.NhError) as e:
        nh.nh_hex_mesh_numbering(Vh, H, 5)
    assert e.value.status == nh.NH_ERR_UNSUPPORTED


@pytest.mark.parametrize("kind", ["rotated", "L"])
def test_q1_block_pattern(kind):
    Vh, H = mesh(kind, (4, 3, 3), seed=9)
    emap, X = nh.nh_hex_mesh_numbering(Vh, H, 1)
    rp, cl = nh.nh_q1_block_pattern(emap, X.shape[0])
    got = {(r, int(c)) for r in range(X.shape[0]) for c in cl[rp[r]:rp[r + 1]]}
    ref = {(int(a), int(b)) for e in emap for a in e for b in e}
    assert got == ref and len(got) == len(cl)
    for r in range(X.shape[0]):
        assert np.all(np.diff(cl[rp[r]:rp[r + 1]]) > 0)


def test_morton_order_restores_locality():
    """A shuffled mesh reordered along the Z-order curve: perm is a permutation, and
    with first-touch numbering an element's nodes span a small id range again."""
    Vh, H = inputs.hex_mesh_from_box(12, 12, 12, inputs.box_vertices(12, 12, 12, perturb=0.1, seed=1), seed=2)
    perm = nh.nh_hex_morton_order(Vh, H)
    assert np.array_equal(np.sort(perm), np.arange(len(H)))

    def spread(hh):
        emap, _ = nh.nh_hex_mesh_numbering(Vh, hh, 2)
        return np.median(emap.max(axis=1) - emap.min(axis=1))
    s_shuffled, s_morton = spread(H), spread(H[perm])
    assert s_morton * 5 < s_shuffled, (s_morton, s_shuffled)
