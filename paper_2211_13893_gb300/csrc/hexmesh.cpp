// Structured numbering of a general hexahedron list (msgfem_mesh.kind = 1),
// element-to-part maps and Dirichlet node flags (host only, no CUDA call).
//
// The local stage factorises every oversampling domain layer by layer through
// the thickness (Sec. 5.1: one element per ply), so it needs the (i, j, k)
// index space of a structured hexahedral mesh.  A hexahedron list given in any
// node and element order is mapped onto that space here: the elements' local
// node orders fix three directions (the standard order: nodes 0-3 around the
// face zeta = 0, nodes 4-7 above them), and a mesh that is topologically an
// nx x ny x nz block whose elements all use one orientation is numbered from
// the node that precedes no other.  Anything else is refused with a message
// that names the reason.
#include <string>
#include <vector>

#include "internal.h"

namespace {

// local node a of the standard order -> (di, dj, dk)
const int kHexOff[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0}, {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
// the four edges of every direction (from, to) in local node numbers
const int kEdges[3][4][2] = {{{0, 1}, {3, 2}, {4, 5}, {7, 6}},
                             {{0, 3}, {1, 2}, {4, 7}, {5, 6}},
                             {{0, 4}, {1, 5}, {2, 6}, {3, 7}}};

}  // namespace

bool recover_structure(int n_nodes, int n_elems, const int* hex8, HexNumbering& out, std::string& err) {
  if (n_nodes < 8 || n_elems < 1 || hex8 == nullptr) {
    err = "hexahedron list: needs at least one element and its eight nodes";
    return false;
  }
  for (long long e = 0; e < n_elems; ++e)
    for (int a = 0; a < 8; ++a) {
      const int v = hex8[8 * e + a];
      if (v < 0 || v >= n_nodes) {
        err = "hexahedron list: element " + std::to_string(e) + " names node " + std::to_string(v) +
              " outside 0.." + std::to_string(n_nodes - 1);
        return false;
      }
      for (int b = 0; b < a; ++b)
        if (hex8[8 * e + b] == v) {
          err = "hexahedron list: element " + std::to_string(e) + " repeats node " + std::to_string(v);
          return false;
        }
    }
  // successor and predecessor of every node along each local direction
  std::vector<int> succ(3 * (size_t)n_nodes, -1), pred(3 * (size_t)n_nodes, -1);
  for (long long e = 0; e < n_elems; ++e)
    for (int d = 0; d < 3; ++d)
      for (int t = 0; t < 4; ++t) {
        const int a = hex8[8 * e + kEdges[d][t][0]], b = hex8[8 * e + kEdges[d][t][1]];
        int& s = succ[3 * (size_t)a + d];
        int& p = pred[3 * (size_t)b + d];
        if ((s != -1 && s != b) || (p != -1 && p != a)) {
          err = "hexahedron list: the elements do not share one orientation or do not form a structured block "
                "(node " + std::to_string(a) + " has two neighbours along local direction " + std::to_string(d) +
                "); the layer-block factorisation needs an (i, j, k) numbering";
          return false;
        }
        s = b;
        p = a;
      }
  int origin = -1;
  for (int v = 0; v < n_nodes; ++v)
    if (pred[3 * (size_t)v] < 0 && pred[3 * (size_t)v + 1] < 0 && pred[3 * (size_t)v + 2] < 0) {
      if (origin >= 0) {
        err = "hexahedron list: more than one corner node precedes no other (not one structured block, or "
              "nodes used by no element)";
        return false;
      }
      origin = v;
    }
  if (origin < 0) {
    err = "hexahedron list: no corner node (the elements close on themselves)";
    return false;
  }
  auto walk = [&](int v, int d) {
    int n = 0;
    for (int u = v; u >= 0 && n <= n_nodes; u = succ[3 * (size_t)u + d]) ++n;
    return n;
  };
  const int nxn = walk(origin, 0), nyn = walk(origin, 1), nzn = walk(origin, 2);
  if ((long long)nxn * nyn * nzn != n_nodes || nxn < 2 || nyn < 2 || nzn < 2) {
    err = "hexahedron list: the node count is not that of an nx x ny x nz block (" + std::to_string(n_nodes) +
          " nodes, block of " + std::to_string(nxn) + " x " + std::to_string(nyn) + " x " + std::to_string(nzn) + ")";
    return false;
  }
  out.nx = nxn - 1;
  out.ny = nyn - 1;
  out.nz = nzn - 1;
  if ((long long)out.nx * out.ny * out.nz != n_elems) {
    err = "hexahedron list: the element count is not nx * ny * nz";
    return false;
  }
  out.node_of_user.assign(n_nodes, -1);
  int vi = origin;
  for (int i = 0; i < nxn; ++i, vi = succ[3 * (size_t)vi]) {
    int vj = vi;
    for (int j = 0; j < nyn; ++j, vj = vj >= 0 ? succ[3 * (size_t)vj + 1] : -1) {
      int vk = vj;
      for (int k = 0; k < nzn; ++k, vk = vk >= 0 ? succ[3 * (size_t)vk + 2] : -1) {
        if (vk < 0 || out.node_of_user[vk] != -1) {
          err = "hexahedron list: the nodes do not form an (i, j, k) block (a line ends early or a node repeats)";
          return false;
        }
        out.node_of_user[vk] = (i * nyn + j) * nzn + k;
      }
    }
  }
  out.elem_of_user.assign(n_elems, -1);
  std::vector<char> used((size_t)n_elems, 0);
  for (long long e = 0; e < n_elems; ++e) {
    const int s0 = out.node_of_user[hex8[8 * e]];
    const int k0 = s0 % nzn, j0 = (s0 / nzn) % nyn, i0 = s0 / nzn / nyn;
    if (i0 >= out.nx || j0 >= out.ny || k0 >= out.nz) {
      err = "hexahedron list: element " + std::to_string(e) + " starts on the far face of the block";
      return false;
    }
    for (int a = 1; a < 8; ++a)
      if (out.node_of_user[hex8[8 * e + a]] !=
          ((i0 + kHexOff[a][0]) * nyn + j0 + kHexOff[a][1]) * nzn + k0 + kHexOff[a][2]) {
        err = "hexahedron list: element " + std::to_string(e) + " is not one cell of the recovered block";
        return false;
      }
    const int idx = (i0 * out.ny + j0) * out.nz + k0;
    if (used[idx]) {
      err = "hexahedron list: two elements occupy one cell";
      return false;
    }
    used[idx] = 1;
    out.elem_of_user[e] = idx;
  }
  return true;
}

bool parts_to_boxes(int NX, int NY, int NZ, const int* elem_part, std::vector<int>& boxes, std::string& err) {
  const long long nel = (long long)NX * NY * NZ;
  int P = 0;
  for (long long e = 0; e < nel; ++e) {
    if (elem_part[e] < 0) {
      err = "elem_part: negative part id";
      return false;
    }
    P = std::max(P, elem_part[e] + 1);
  }
  std::vector<int> bx(4 * (size_t)P), cnt(P, 0);
  for (int p = 0; p < P; ++p) {
    bx[4 * p] = NX;
    bx[4 * p + 1] = -1;
    bx[4 * p + 2] = NY;
    bx[4 * p + 3] = -1;
  }
  for (int i = 0; i < NX; ++i)
    for (int j = 0; j < NY; ++j)
      for (int k = 0; k < NZ; ++k) {
        const int p = elem_part[((long long)i * NY + j) * NZ + k];
        bx[4 * p] = std::min(bx[4 * p], i);
        bx[4 * p + 1] = std::max(bx[4 * p + 1], i);
        bx[4 * p + 2] = std::min(bx[4 * p + 2], j);
        bx[4 * p + 3] = std::max(bx[4 * p + 3], j);
        ++cnt[p];
      }
  boxes.assign(4 * (size_t)P, 0);
  for (int p = 0; p < P; ++p) {
    if (cnt[p] == 0) {
      err = "elem_part: part " + std::to_string(p) + " has no element (part ids must run from 0 without gaps)";
      return false;
    }
    const int x0 = bx[4 * p], x1 = bx[4 * p + 1] + 1, y0 = bx[4 * p + 2], y1 = bx[4 * p + 3] + 1;
    if ((long long)(x1 - x0) * (y1 - y0) * NZ != cnt[p]) {
      err = "elem_part: part " + std::to_string(p) + " is not an (i, j) box through the full thickness (each " +
            "subdomain's layer blocks span whole node layers)";
      return false;
    }
    for (int i = x0; i < x1; ++i)
      for (int j = y0; j < y1; ++j)
        for (int k = 0; k < NZ; ++k)
          if (elem_part[((long long)i * NY + j) * NZ + k] != p) {
            err = "elem_part: part " + std::to_string(p) + " is not an (i, j) box through the full thickness";
            return false;
          }
    boxes[4 * p] = x0;
    boxes[4 * p + 1] = x1;
    boxes[4 * p + 2] = y0;
    boxes[4 * p + 3] = y1;
  }
  return true;
}

bool dirichlet_is_clamped_face(int NX, int NY, int NZ, const unsigned char* flags, std::string& err) {
  (void)NX;
  const long long nn = (long long)(NX + 1) * (NY + 1) * (NZ + 1), face = (long long)(NY + 1) * (NZ + 1);
  for (long long n = 0; n < nn; ++n)
    if ((flags[n] != 0) != (n < face)) {
      err = "dirichlet_node: the flagged nodes must be exactly the face i = 0 (in a hexahedron list: the face "
            "where the elements' local direction 0 -> 1 starts); the DoF classes and rigid-mode pins of the local "
            "stage assume that clamped face";
      return false;
    }
  return true;
}
