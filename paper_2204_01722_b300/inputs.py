"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module holds no finite-element arithmetic: it only draws meshes,
displacement fields, vectors, boundary masks and material layouts from
seeded numpy generators.  Recipes:

* ``box_vertices``: unit-cube vertex lattice, interior vertices shifted by
  U(-f h, f h) per coordinate (boundary vertices stay put so faces stay planar).
* ``smooth_field``: u_i(X) = sum_m a_im sin(pi k_m . X + phi_m), m = 1..8,
  k_m in {1,2}^3, a and phi seeded, rescaled so max_nodes |u| = amplitude.
* ``normal_vector``: N(0, 1) entries.
* ``uniaxial_mask`` / ``uniaxial_bc``: x = 0 face clamped (all components),
  x = 1 face has its x-component prescribed to -delta, the rest free.
* ``hex_mesh_from_box``: the box mesh as vertex/connectivity arrays, with each
  element's local frame a random cube rotation, shuffled vertex ids and element
  order, and optionally a subset of the elements (an unstructured mesh).
* ``inclusion_modulus``: per-element Young's modulus from seeded spheres
  (centres uniform in the box, radius U(rmin, rmax) elements) added until the
  element-centroid volume fraction reaches ``vf``; E = contrast inside, 1 outside.
  With ``gap=None`` spheres may overlap (clusters form; at vf = 0.3 the stiff
  phase is near percolation).  With ``gap=g`` the spheres are disjoint with at
  least g elements between surfaces: radii are drawn up front, sorted
  largest first, and each is placed at the first of up to 2000 uniform centre
  draws that keeps the gap (``inclusion_spheres`` returns the centres and radii).
"""
import numpy as np


def box_vertices(nx, ny, nz, perturb=0.0, seed=0):
    x = np.linspace(0.0, 1.0, nx + 1)
    y = np.linspace(0.0, 1.0, ny + 1)
    z = np.linspace(0.0, 1.0, nz + 1)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    V = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    if perturb > 0.0:
        rng = np.random.default_rng(seed)
        h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
        vi = np.tile(np.arange(nx + 1), (ny + 1) * (nz + 1))
        vj = np.tile(np.repeat(np.arange(ny + 1), nx + 1), nz + 1)
        vk = np.repeat(np.arange(nz + 1), (nx + 1) * (ny + 1))
        interior = (vi > 0) & (vi < nx) & (vj > 0) & (vj < ny) & (vk > 0) & (vk < nz)
        d = rng.uniform(-perturb, perturb, size=V.shape) * h[None, :]
        V[interior] += d[interior]
    return V


def smooth_field(xyz, amplitude=0.05, seed=0, modes=8):
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    rng = np.random.default_rng(seed)
    k = rng.integers(1, 3, size=(modes, 3)).astype(np.float64)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=(modes,))
    a = rng.normal(size=(3, modes))
    arg = np.pi * (xyz @ k.T) + phi[None, :]          # [n, modes]
    u = np.sin(arg) @ a.T                              # [n, 3]
    u *= amplitude / np.max(np.linalg.norm(u, axis=1))
    return u


def normal_vector(n, seed=0):
    return np.random.default_rng(seed).standard_normal(n)


def uniform_vector(n, seed=0):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=n)


def splitmix_uniform(n, seed):
    """Counter-based uniform(-1, 1) vector: splitmix64 (Steele, Lea, Flood 2014)
    of seed * 0x100000001b3 + i, top 53 bits scaled.  The CUDA library draws the
    rough Lanczos start vector with its own implementation of the same generator."""
    M = np.uint64(0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) * np.uint64(0x100000001b3) + np.arange(n, dtype=np.uint64)
        z = z + np.uint64(0x9e3779b97f4a7c15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xbf58476d1ce4e5b9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94d049bb133111eb)
        z = z ^ (z >> np.uint64(31))
    del M
    return 2.0 * ((z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)) - 1.0


def lattice_index(node_dims):
    Nx, Ny, Nz = node_dims
    I = np.tile(np.arange(Nx), Ny * Nz)
    J = np.tile(np.repeat(np.arange(Ny), Nx), Nz)
    K = np.repeat(np.arange(Nz), Nx * Ny)
    return I, J, K


def uniaxial_mask(node_dims):
    """Boolean DoF mask [3 n_nodes]: x = 0 face all components, x = 1 face x-component."""
    Nx = node_dims[0]
    I, _, _ = lattice_index(node_dims)
    m = np.zeros((I.size, 3), dtype=bool)
    m[I == 0, :] = True
    m[I == Nx - 1, 0] = True
    return m.ravel()


def uniaxial_bc(node_dims, delta):
    """Prescribed displacement [3 n_nodes]: u_x = -delta on x = 1, zero elsewhere."""
    Nx = node_dims[0]
    I, _, _ = lattice_index(node_dims)
    g = np.zeros((I.size, 3))
    g[I == Nx - 1, 0] = -delta
    return g.ravel()


def all_faces_mask(node_dims):
    Nx, Ny, Nz = node_dims
    I, J, K = lattice_index(node_dims)
    b = (I == 0) | (I == Nx - 1) | (J == 0) | (J == Ny - 1) | (K == 0) | (K == Nz - 1)
    return np.repeat(b, 3)


def _proper_rotations():
    """The 24 rotations of the reference cube as (axis permutation, flips) with determinant +1."""
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        sgn = np.linalg.det(np.eye(3)[list(perm)])
        for flips in itertools.product((0, 1), repeat=3):
            if sgn * (-1) ** sum(flips) > 0:
                out.append((perm, flips))
    return out


def hex_mesh_from_box(nx, ny, nz, vertices=None, seed=0, reorient=True, permute=True, keep=None):
    """The box mesh as an unstructured hexahedral mesh: (vertices [nv, 3], hex8 [ne, 8]).

    hex8 rows are in tensor corner order (corner v at (v & 1, (v >> 1) & 1, v >> 2)).
    ``reorient``: each element's local frame is a random one of the 24 cube
    rotations, so shared edges and faces are seen in every relative orientation;
    ``permute``: vertex ids and element order are shuffled; ``keep`` (bool [ne],
    lexicographic box order): elements to keep, e.g. an L-shaped subset.
    """
    rng = np.random.default_rng(seed)
    V = box_vertices(nx, ny, nz) if vertices is None else np.asarray(vertices, dtype=np.float64).reshape(-1, 3)
    ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()
    corners = [(v & 1, (v >> 1) & 1, v >> 2) for v in range(8)]
    H = np.stack([(ex + c[0]) + (nx + 1) * ((ey + c[1]) + (ny + 1) * (ez + c[2])) for c in corners], axis=1)
    if keep is not None:
        H = H[np.asarray(keep, dtype=bool)]
    if reorient:
        table = []
        for perm, flips in _proper_rotations():
            row = []
            for cn in corners:                 # new local corner cn <- old corner c
                c = [0, 0, 0]
                for d in range(3):
                    c[perm[d]] = cn[d] ^ flips[d]
                row.append(c[0] + 2 * c[1] + 4 * c[2])
            table.append(row)
        table = np.array(table)
        pick = rng.integers(len(table), size=H.shape[0])
        H = np.take_along_axis(H, table[pick], axis=1)
    if permute:
        pv = rng.permutation(V.shape[0])     # old vertex i -> new id pv[i]
        Vn = np.empty_like(V)
        Vn[pv] = V
        V, H = Vn, pv[H]
        H = H[rng.permutation(H.shape[0])]
    return V, H


def _element_centroids(nx, ny, nz):
    cx = (np.arange(nx) + 0.5) / nx
    cy = (np.arange(ny) + 0.5) / ny
    cz = (np.arange(nz) + 0.5) / nz
    Z, Y, X = np.meshgrid(cz, cy, cx, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def inclusion_spheres(nx, ny, nz, seed=0, vf=0.3, rmin=2.0, rmax=6.0, gap=None):
    """Returns (centres [m, 3], radii [m], inside [ne] bool) in unit-box units."""
    rng = np.random.default_rng(seed)
    C = _element_centroids(nx, ny, nz)
    h = 1.0 / max(nx, ny, nz)
    inside = np.zeros(C.shape[0], dtype=bool)
    cs, rs = [], []
    if gap is None:
        for _ in range(100000):
            if inside.mean() >= vf:
                break
            c = rng.uniform(0.0, 1.0, size=3)
            r = rng.uniform(rmin, rmax) * h
            inside |= np.sum((C - c) ** 2, axis=1) <= r * r
            cs.append(c)
            rs.append(r)
        return np.array(cs).reshape(-1, 3), np.array(rs), inside
    radii, vol = [], 0.0
    while vol < 2.0 * vf:
        radii.append(rng.uniform(rmin, rmax) * h)
        vol += 4.0 / 3.0 * np.pi * radii[-1] ** 3
    for r in sorted(radii, reverse=True):
        if inside.mean() >= vf:
            break
        for _ in range(2000):
            c = rng.uniform(0.0, 1.0, size=3)
            if cs and np.any(np.linalg.norm(np.array(cs) - c, axis=1) < np.array(rs) + r + gap * h):
                continue
            cs.append(c)
            rs.append(r)
            inside |= np.sum((C - c) ** 2, axis=1) <= r * r
            break
    return np.array(cs).reshape(-1, 3), np.array(rs), inside


def inclusion_modulus(nx, ny, nz, seed=0, vf=0.3, rmin=2.0, rmax=6.0, contrast=1e3, gap=None):
    _, _, inside = inclusion_spheres(nx, ny, nz, seed=seed, vf=vf, rmin=rmin, rmax=rmax, gap=gap)
    return np.where(inside, contrast, 1.0)
