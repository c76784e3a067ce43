// Element restriction of a conforming unstructured hexahedral mesh (host code).
//
// The Q_p nodes of an element are the tensor lattice (i, j, k) in [0, p]^3.  Each
// lattice node lies on exactly one mesh entity: a vertex (all three indices at
// 0 or p), the interior of an edge (two), of a face (one) or of the element
// (none).  Entities are identified by their global vertex ids, so two elements
// that share an edge or a face find the same entity whatever their local
// orientation:
//   * edge {a, b}: its p - 1 interior nodes are numbered from the smaller vertex id;
//   * face {a, b, c, d}: its (p - 1)^2 interior nodes are numbered in a frame
//     whose origin is the corner with the smallest id and whose first axis
//     points to that corner's face neighbour with the smaller id.
// Global node ids are handed out in order of first touch while the elements are
// walked in order (interior nodes of element e follow its first new boundary
// nodes), which keeps each element's nodes close together in the L-vector.
// Node coordinates are the trilinear image of the GLL lattice (linear
// geometry, as on the box); a node shared by several elements must get the same
// coordinates from each of them, which the builder checks.
#include <math.h>

#include <algorithm>
#include <array>
#include <string>
#include <unordered_map>
#include <vector>

#include "nh_internal.cuh"

namespace {

uint64_t mix(uint64_t h, uint64_t v) {  // splitmix64-style combine
  h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
  h ^= h >> 31;
  h *= 0xbf58476d1ce4e5b9ull;
  return h ^ (h >> 29);
}

struct EdgeHash {
  size_t operator()(const std::pair<int64_t, int64_t>& k) const { return (size_t)mix(mix(0, k.first), k.second); }
};

struct FaceHash {
  size_t operator()(const std::array<int64_t, 4>& k) const {
    return (size_t)mix(mix(mix(mix(0, k[0]), k[1]), k[2]), k[3]);
  }
};

// per face (sorted corner ids): elements using it, and the id of its first interior node
struct FaceInfo {
  int uses = 0;
  int64_t base = -1;
};

// det of d X / d xi of the trilinear map at the corner (ci, cj, ck) in {0,1}^3
double corner_det(const double V[8][3], int ci, int cj, int ck) {
  double J[3][3];
  for (int d = 0; d < 3; d++) {  // column d: derivative along local axis d
    const int c[3] = {ci, cj, ck};
    int lo[3] = {c[0], c[1], c[2]}, hi[3] = {c[0], c[1], c[2]};
    lo[d] = 0;
    hi[d] = 1;
    const int vl = lo[0] + 2 * lo[1] + 4 * lo[2], vh = hi[0] + 2 * hi[1] + 4 * hi[2];
    for (int r = 0; r < 3; r++) J[r][d] = V[vh][r] - V[vl][r];
  }
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

}  // namespace

std::string nh_hex_numbering(int64_t nv, const double* xyz, int64_t ne, const int64_t* hex8, int p,
                             std::vector<int>& emap, std::vector<double>& coords, int64_t& n_nodes) {
  const int P = p + 1, P3 = P * P * P;
  for (int64_t e = 0; e < ne; e++)
    for (int v = 0; v < 8; v++) {
      const int64_t id = hex8[8 * e + v];
      if (id < 0 || id >= nv) return "element " + std::to_string(e) + " names vertex " + std::to_string(id) +
                                     ", outside [0, nv)";
      for (int w = 0; w < v; w++)
        if (hex8[8 * e + w] == id) return "element " + std::to_string(e) + " repeats vertex " + std::to_string(id);
    }
  // orientation: the trilinear map must have a positive Jacobian determinant at every corner
  for (int64_t e = 0; e < ne; e++) {
    double V[8][3];
    for (int v = 0; v < 8; v++)
      for (int d = 0; d < 3; d++) V[v][d] = xyz[3 * hex8[8 * e + v] + d];
    for (int c = 0; c < 8; c++)
      if (!(corner_det(V, c & 1, (c >> 1) & 1, (c >> 2) & 1) > 0.0))
        return "element " + std::to_string(e) + " is inverted or degenerate in the given vertex order "
               "(vertex v of an element sits at corner (v & 1, (v >> 1) & 1, v >> 2))";
  }
  // faces used by more than two elements make the mesh non-manifold
  std::unordered_map<std::array<int64_t, 4>, FaceInfo, FaceHash> faces;
  faces.reserve((size_t)(3.5 * ne) + 16);
  static const int kFace[6][4] = {{0, 2, 4, 6}, {1, 3, 5, 7}, {0, 1, 4, 5}, {2, 3, 6, 7}, {0, 1, 2, 3}, {4, 5, 6, 7}};
  for (int64_t e = 0; e < ne; e++)
    for (int f = 0; f < 6; f++) {
      std::array<int64_t, 4> k;
      for (int t = 0; t < 4; t++) k[t] = hex8[8 * e + kFace[f][t]];
      std::sort(k.begin(), k.end());
      if (++faces[k].uses > 2) return "a face is shared by more than two elements (element " + std::to_string(e) + ")";
    }

  std::vector<int64_t> vnode((size_t)nv, -1);
  std::unordered_map<std::pair<int64_t, int64_t>, int64_t, EdgeHash> edge_base;
  edge_base.reserve((size_t)(3.5 * ne) + 16);
  int64_t next = 0;
  emap.assign((size_t)ne * P3, 0);
  std::vector<int64_t> ids((size_t)P3);
  // per element, each edge and face is looked up once: edge cache by (axis, the
  // two fixed coordinates), face cache by (fixed axis, side) with its frame
  int64_t ebase[12], fbase[6];
  int fos[6], fot[6];
  bool falong[6];
  for (int64_t e = 0; e < ne; e++) {
    const int64_t* hv = hex8 + 8 * e;
    int64_t interior = -1;
    for (int c = 0; c < 12; c++) ebase[c] = -1;
    for (int c = 0; c < 6; c++) fbase[c] = -1;
    for (int k = 0; k < P; k++)
      for (int j = 0; j < P; j++)
        for (int i = 0; i < P; i++) {
          const int L[3] = {i, j, k};
          bool bd[3];
          int nb = 0;
          for (int d = 0; d < 3; d++) nb += (bd[d] = (L[d] == 0 || L[d] == p));
          // local corner with the given lattice coordinates at the boundary axes
          auto corner = [&](const int (&c)[3]) { return hv[(c[0] == p) + 2 * (c[1] == p) + 4 * (c[2] == p)]; };
          int64_t id;
          if (nb == 3) {
            const int64_t v = corner(L);
            if (vnode[v] < 0) vnode[v] = next++;
            id = vnode[v];
          } else if (nb == 2) {
            const int ax = !bd[0] ? 0 : !bd[1] ? 1 : 2;  // the edge's direction
            int c0[3] = {L[0], L[1], L[2]}, c1[3] = {L[0], L[1], L[2]};
            c0[ax] = 0;
            c1[ax] = p;
            const int64_t a = corner(c0), b = corner(c1);
            const int o1 = ax == 0 ? 1 : 0, o2 = ax == 2 ? 1 : 2;
            const int slot = ax * 4 + (L[o1] == p) + 2 * (L[o2] == p);
            if (ebase[slot] < 0) {
              const auto key = std::make_pair(std::min(a, b), std::max(a, b));
              auto it = edge_base.find(key);
              if (it == edge_base.end()) {
                it = edge_base.emplace(key, next).first;
                next += p - 1;
              }
              ebase[slot] = it->second;
            }
            const int t = L[ax];  // 1 .. p-1 from local corner a
            id = ebase[slot] + (a < b ? t - 1 : p - 1 - t);
          } else if (nb == 1) {
            const int fx = bd[0] ? 0 : bd[1] ? 1 : 2;  // fixed axis
            const int sa = fx == 0 ? 1 : 0, ta = fx == 2 ? 1 : 2;  // free axes, increasing
            const int slot = fx * 2 + (L[fx] == p);
            if (fbase[slot] < 0) {
              int64_t cid[2][2];  // corner ids at (s, t) in {0, p}^2
              for (int cs = 0; cs < 2; cs++)
                for (int ct = 0; ct < 2; ct++) {
                  int c[3] = {L[0], L[1], L[2]};
                  c[sa] = cs * p;
                  c[ta] = ct * p;
                  cid[cs][ct] = corner(c);
                }
              std::array<int64_t, 4> key = {cid[0][0], cid[1][0], cid[0][1], cid[1][1]};
              std::sort(key.begin(), key.end());
              FaceInfo& fi = faces[key];
              if (fi.base < 0) {
                fi.base = next;
                next += (int64_t)(p - 1) * (p - 1);
              }
              int os = 0, ot = 0;  // origin: smallest corner id
              for (int cs = 0; cs < 2; cs++)
                for (int ct = 0; ct < 2; ct++)
                  if (cid[cs][ct] < cid[os][ot]) {
                    os = cs;
                    ot = ct;
                  }
              fbase[slot] = fi.base;
              fos[slot] = os;
              fot[slot] = ot;
              falong[slot] = cid[1 - os][ot] < cid[os][1 - ot];  // neighbour with the smaller id
            }
            const int os = fos[slot], ot = fot[slot];
            const bool first_along_s = falong[slot];
            const int ds = os ? p - L[sa] : L[sa], dt = ot ? p - L[ta] : L[ta];
            const int s1 = first_along_s ? ds : dt, t1 = first_along_s ? dt : ds;
            id = fbase[slot] + (s1 - 1) + (int64_t)(p - 1) * (t1 - 1);
          } else {
            if (interior < 0) {
              interior = next;
              next += (int64_t)(p - 1) * (p - 1) * (p - 1);
            }
            id = interior + (i - 1) + (int64_t)(p - 1) * ((j - 1) + (int64_t)(p - 1) * (k - 1));
          }
          ids[(k * P + j) * P + i] = id;
        }
    if (next >= ((int64_t)1 << 29)) return "mesh too large (node ids must fit 29 bits)";
    for (int l = 0; l < P3; l++) emap[(size_t)e * P3 + l] = (int)ids[l];
  }
  n_nodes = next;

  // coordinates, with the conformity check on shared nodes
  double xn[NH_MAXP];
  nh_lobatto(P, xn);
  coords.assign((size_t)3 * n_nodes, 0.0);
  std::vector<char> seen((size_t)n_nodes, 0);
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t v = 0; v < nv; v++)
    for (int d = 0; d < 3; d++) {
      lo[d] = std::min(lo[d], xyz[3 * v + d]);
      hi[d] = std::max(hi[d], xyz[3 * v + d]);
    }
  const double tol = 1e-10 * std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-300});
  for (int64_t e = 0; e < ne; e++) {
    for (int k = 0; k < P; k++)
      for (int j = 0; j < P; j++)
        for (int i = 0; i < P; i++) {
          const double f[3][2] = {{0.5 * (1 - xn[i]), 0.5 * (1 + xn[i])},
                                  {0.5 * (1 - xn[j]), 0.5 * (1 + xn[j])},
                                  {0.5 * (1 - xn[k]), 0.5 * (1 + xn[k])}};
          double X[3] = {0, 0, 0};
          for (int v = 0; v < 8; v++) {
            const double w = f[0][v & 1] * f[1][(v >> 1) & 1] * f[2][(v >> 2) & 1];
            for (int d = 0; d < 3; d++) X[d] += w * xyz[3 * hex8[8 * e + v] + d];
          }
          const int64_t n = emap[(size_t)e * P3 + (k * P + j) * P + i];
          if (seen[n]) {
            for (int d = 0; d < 3; d++)
              if (fabs(coords[3 * n + d] - X[d]) > tol)
                return "elements disagree on the position of a shared node (element " + std::to_string(e) +
                       "): the mesh is not conforming";
          } else {
            seen[n] = 1;
            for (int d = 0; d < 3; d++) coords[3 * n + d] = X[d];
          }
        }
  }
  return std::string();
}

// Z-order (Morton) ordering of the elements by centroid: centroids scaled to the
// bounding box, 21 bits per axis interleaved into a 63-bit key, stable sort.
// Elements close in space become close in order, and with first-touch numbering
// so do their nodes.
void nh_hex_morton(int64_t nv, const double* xyz, int64_t ne, const int64_t* hex8, int64_t* perm) {
  (void)nv;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  std::vector<double> cen((size_t)3 * ne);
  for (int64_t e = 0; e < ne; e++)
    for (int d = 0; d < 3; d++) {
      double s = 0.0;
      for (int v = 0; v < 8; v++) s += xyz[3 * hex8[8 * e + v] + d];
      cen[3 * e + d] = s / 8.0;
      lo[d] = std::min(lo[d], s / 8.0);
      hi[d] = std::max(hi[d], s / 8.0);
    }
  auto spread = [](uint64_t x) {  // 21 bits -> every third bit
    x &= 0x1fffffull;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
  };
  std::vector<std::pair<uint64_t, int64_t>> key((size_t)ne);
  for (int64_t e = 0; e < ne; e++) {
    uint64_t k = 0;
    for (int d = 0; d < 3; d++) {
      const double w = hi[d] > lo[d] ? (cen[3 * e + d] - lo[d]) / (hi[d] - lo[d]) : 0.0;
      k |= spread((uint64_t)std::min(2097151.0, std::max(0.0, w * 2097151.0))) << d;
    }
    key[e] = {k, e};
  }
  std::stable_sort(key.begin(), key.end());
  for (int64_t i = 0; i < ne; i++) perm[i] = key[i].second;
}
