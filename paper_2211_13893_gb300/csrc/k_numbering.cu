// General mesh input (msgfem_mesh.kind = 1, msgfem_mesh.dirichlet_node,
// msgfem_partition.elem_part) mapped onto the structured problem, and the
// node permutation of solution vectors between the caller's numbering and the
// structured one (Sec. 3.1, Sec. 4.1: the paper's meshes are general
// hexahedron lists partitioned by ParMETIS).
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace {

// dir 0: out[user u] = in[structured node_of_user[u]]; dir 1: the inverse
__global__ void k_permute_nodes(double* __restrict__ out, const double* __restrict__ in,
                                const int* __restrict__ node_of_user, int nnode, int dir) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 3 * nnode; e += gridDim.x * blockDim.x) {
    const int u = e / 3, c = e % 3, s = 3 * node_of_user[u] + c;
    if (dir == 0) out[e] = in[s];
    else out[s] = in[e];
  }
}

bool is_dev(const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// host copy of n doubles from a host or device pointer
bool fetch(const double* src, size_t n, std::vector<double>& dst) {
  dst.resize(n);
  if (is_dev(src)) return cudaMemcpy(dst.data(), src, n * sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess;
  std::memcpy(dst.data(), src, n * sizeof(double));
  return true;
}

msgfem_status fail(msgfem_h* out, const std::string& msg) {
  msgfem* h = new msgfem();
  h->err = msg;
  *out = h;
  return MSGFEM_EINVAL;
}

}  // namespace

msgfem_status vec_in(msgfem* h, const double* user, double* d_struct) {
  const int nnode = (h->NX + 1) * (h->NY + 1) * (h->NZ + 1);
  cudaStream_t st = h->stream;
  if (h->node_of_user.empty()) {
    CK(cudaMemcpyAsync(d_struct, user, 3 * (size_t)nnode * sizeof(double), cudaMemcpyDefault, st));
    return MSGFEM_OK;
  }
  CK(cudaMemcpyAsync(h->d_perm_tmp, user, 3 * (size_t)nnode * sizeof(double), cudaMemcpyDefault, st));
  k_permute_nodes<<<(3 * nnode + 255) / 256, 256, 0, st>>>(d_struct, h->d_perm_tmp, h->d_node_of_user, nnode, 1);
  ++g_launch_count;
  CK_LAUNCH();
  return MSGFEM_OK;
}

msgfem_status vec_out(msgfem* h, const double* d_struct, double* user) {
  const int nnode = (h->NX + 1) * (h->NY + 1) * (h->NZ + 1);
  cudaStream_t st = h->stream;
  if (h->node_of_user.empty()) {
    CK(cudaMemcpyAsync(user, d_struct, 3 * (size_t)nnode * sizeof(double), cudaMemcpyDefault, st));
    return MSGFEM_OK;
  }
  k_permute_nodes<<<(3 * nnode + 255) / 256, 256, 0, st>>>(h->d_perm_tmp, d_struct, h->d_node_of_user, nnode, 0);
  ++g_launch_count;
  CK_LAUNCH();
  CK(cudaMemcpyAsync(user, h->d_perm_tmp, 3 * (size_t)nnode * sizeof(double), cudaMemcpyDefault, st));
  return MSGFEM_OK;
}

msgfem_status angles_in(msgfem* h, const double* user, std::vector<double>& out) {
  const size_t nel = (size_t)h->NX * h->NY * h->NZ;
  std::vector<double> a;
  if (!fetch(user, nel * h->S, a)) {
    h->err = "element angles: copy failed";
    return MSGFEM_ECUDA;
  }
  out.assign(a.size(), 0.0);
  for (int i = 0; i < h->S; ++i)
    for (size_t e = 0; e < nel; ++e) out[i * nel + h->elem_of_user[e]] = a[i * nel + e];
  return MSGFEM_OK;
}

// msgfem_setup for the general descriptors: recover the structured numbering
// of a hexahedron list, check the Dirichlet flags, turn an element -> part
// map into boxes, permute every per-node and per-element input into the
// structured order and set up the structured problem; the handle keeps the
// permutation for the solution vectors.
msgfem_status setup_general(const msgfem_mesh* mesh, const msgfem_plies* plies, const msgfem_partition* part,
                            int overlap, int oversampling, const msgfem_options* opt, msgfem_h* out) {
  msgfem_mesh m = *mesh;
  msgfem_plies pl = *plies;
  msgfem_partition pt = *part;
  HexNumbering hn;
  std::string err;
  std::vector<double> xyz, load, ang, frame;
  const int S = (opt && opt->instances > 1) ? opt->instances : 1;
  if (mesh->kind != 0 && mesh->kind != 1) return fail(out, "unknown mesh kind");
  if (mesh->kind == 1) {
    if (mesh->node_xyz == nullptr || mesh->hex8 == nullptr) return fail(out, "hexahedron list: node_xyz and hex8 are required");
    if (!recover_structure(mesh->n_nodes, mesh->n_elems, mesh->hex8, hn, err)) return fail(out, err);
    const int nyn = hn.ny + 1, nzn = hn.nz + 1;
    xyz.assign(3 * (size_t)mesh->n_nodes, 0.0);
    for (int u = 0; u < mesh->n_nodes; ++u)
      for (int c = 0; c < 3; ++c) {
        const double v = mesh->node_xyz[3 * (size_t)u + c];
        if (!std::isfinite(v)) return fail(out, "hexahedron list: non-finite node coordinate");
        xyz[3 * (size_t)hn.node_of_user[u] + c] = v;
      }
    // every element right-handed: the Jacobian of its trilinear map at the centre
    for (int i = 0; i < hn.nx; ++i)
      for (int j = 0; j < hn.ny; ++j)
        for (int k = 0; k < hn.nz; ++k) {
          double d[3][3] = {{0}};
          for (int a = 0; a < 8; ++a) {
            const int di = a & 1, dj = (a >> 1) & 1, dk = a >> 2;
            const double* X = &xyz[3 * (((size_t)(i + di) * nyn + j + dj) * nzn + k + dk)];
            for (int c = 0; c < 3; ++c) {
              d[0][c] += (di ? 0.25 : -0.25) * X[c];
              d[1][c] += (dj ? 0.25 : -0.25) * X[c];
              d[2][c] += (dk ? 0.25 : -0.25) * X[c];
            }
          }
          const double det = d[0][0] * (d[1][1] * d[2][2] - d[1][2] * d[2][1]) -
                             d[0][1] * (d[1][0] * d[2][2] - d[1][2] * d[2][0]) +
                             d[0][2] * (d[1][0] * d[2][1] - d[1][1] * d[2][0]);
          if (!(det > 0.0))
            return fail(out, "hexahedron list: an element is inverted or degenerate (local nodes 0-3 must run "
                             "counterclockwise seen from node 4)");
        }
    m.kind = 0;
    m.nx = hn.nx;
    m.ny = hn.ny;
    m.nz = hn.nz;
    m.hx = m.hy = m.hz = 1.0;   // unused with node coordinates
    m.xyz = xyz.data();
    m.node_xyz = nullptr;
    m.hex8 = nullptr;
    if (mesh->load) {
      std::vector<double> l;
      if (!fetch(mesh->load, 3 * (size_t)mesh->n_nodes, l)) return fail(out, "nodal loads: copy failed");
      load.assign(l.size(), 0.0);
      for (int u = 0; u < mesh->n_nodes; ++u)
        for (int c = 0; c < 3; ++c) load[3 * (size_t)hn.node_of_user[u] + c] = l[3 * (size_t)u + c];
      m.load = load.data();
    }
    const size_t nel = (size_t)mesh->n_elems;
    std::vector<double> a;
    if (!fetch(plies->elem_angle_deg, nel * S, a)) return fail(out, "element angles: copy failed");
    ang.assign(a.size(), 0.0);
    for (int i = 0; i < S; ++i)
      for (size_t e = 0; e < nel; ++e) ang[i * nel + hn.elem_of_user[e]] = a[i * nel + e];
    pl.elem_angle_deg = ang.data();
    if (plies->elem_frame) {
      std::vector<double> f;
      if (!fetch(plies->elem_frame, 9 * nel, f)) return fail(out, "ply frames: copy failed");
      frame.assign(f.size(), 0.0);
      for (size_t e = 0; e < nel; ++e)
        for (int c = 0; c < 9; ++c) frame[9 * (size_t)hn.elem_of_user[e] + c] = f[9 * e + c];
      pl.elem_frame = frame.data();
    }
  }
  const int NX = m.nx, NY = m.ny, NZ = m.nz;
  if (NX <= 0 || NY <= 0 || NZ <= 0) return MSGFEM_EINVAL;
  const size_t nn = (size_t)(NX + 1) * (NY + 1) * (NZ + 1), nel = (size_t)NX * NY * NZ;
  if (mesh->dirichlet_node) {
    std::vector<unsigned char> dn(nn);
    for (size_t u = 0; u < nn; ++u) dn[hn.node_of_user.empty() ? u : hn.node_of_user[u]] = mesh->dirichlet_node[u];
    if (!dirichlet_is_clamped_face(NX, NY, NZ, dn.data(), err)) return fail(out, err);
  }
  m.dirichlet_node = nullptr;
  std::vector<int> boxes;
  if (part->elem_part) {
    std::vector<int> ep(nel);
    for (size_t e = 0; e < nel; ++e) ep[hn.elem_of_user.empty() ? e : hn.elem_of_user[e]] = part->elem_part[e];
    if (!parts_to_boxes(NX, NY, NZ, ep.data(), boxes, err)) return fail(out, err);
    pt.n_boxes = (int)(boxes.size() / 4);
    pt.boxes = boxes.data();
    pt.elem_part = nullptr;
  }
  msgfem_status st = msgfem_setup(&m, &pl, &pt, overlap, oversampling, opt, out);
  if (st != MSGFEM_OK || mesh->kind != 1 || *out == nullptr) return st;
  msgfem* h = *out;
  h->node_of_user = hn.node_of_user;
  h->elem_of_user = hn.elem_of_user;
  std::vector<int> user_of_node(nn);
  for (size_t u = 0; u < nn; ++u) user_of_node[hn.node_of_user[u]] = (int)u;
  void* p = nullptr;
  TRY(dev_alloc_bytes(h, &p, nn * sizeof(int)));
  h->d_node_of_user = static_cast<int*>(p);
  TRY(dev_alloc_bytes(h, &p, nn * sizeof(int)));
  h->d_user_of_node = static_cast<int*>(p);
  TRY(dev_alloc_bytes(h, &p, 3 * nn * sizeof(double)));
  h->d_perm_tmp = static_cast<double*>(p);
  CK(cudaMemcpy(h->d_node_of_user, hn.node_of_user.data(), nn * sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->d_user_of_node, user_of_node.data(), nn * sizeof(int), cudaMemcpyHostToDevice));
  return MSGFEM_OK;
}

extern "C" msgfem_status msgfem_get_numbering(msgfem_h h, int* dims, int* node_of_user, int* elem_of_user) {
  if (!h) return MSGFEM_EINVAL;
  const int nn = (h->NX + 1) * (h->NY + 1) * (h->NZ + 1), nel = h->NX * h->NY * h->NZ;
  if (dims) {
    dims[0] = h->NX;
    dims[1] = h->NY;
    dims[2] = h->NZ;
  }
  for (int u = 0; node_of_user && u < nn; ++u) node_of_user[u] = h->node_of_user.empty() ? u : h->node_of_user[u];
  for (int e = 0; elem_of_user && e < nel; ++e) elem_of_user[e] = h->elem_of_user.empty() ? e : h->elem_of_user[e];
  return MSGFEM_OK;
}
