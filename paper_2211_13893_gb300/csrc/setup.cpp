// Host-side set-up: box decomposition, DoF classes, partition of unity, the
// compact layer numberings and the static task schedules of the layer-block
// factorisation and solves.
//
// Decomposition (Secs. 3.1, 3.3): subdomain (a, b) owns the element box
// [a NX / sx, (a+1) NX / sx) x [b NY / sy, (b+1) NY / sy) x [0, NZ), or
// subdomain j owns the j-th given box; Omega and Omega* grow it by o and o*
// element layers, clipped to the mesh.
// DoF classes on Omega* (Sec. 4.3): class 3 (B3) = nodes on the clamped face
// x = 0; class 2 (B2) = other nodes on the closure of the part of dOmega*
// inside Omega; class 1 (B1) = the rest.
// Partition of unity (Sec. 4.2): weights start at 0 on the closure of the
// part of dOmega inside Omega and 2o elsewhere in Omega, then 2o - 1 Jacobi
// sweeps of w_p <- min(w_p, min_q w_q + 1, 2o) over nodes q sharing an
// element with p; mu_{j,p} = w_{j,p} / sum_i w_{i,p}.
#include <cmath>
#include <cstring>
#include <functional>
#include <limits>
#include <map>
#include <queue>
#include <tuple>
#include <type_traits>
#include <unordered_map>
#include <string>

#include "internal.h"

namespace {

struct Box { int x0, x1, y0, y1; };   // element box [x0, x1) x [y0, y1)

Box grow(const Box& b, int m, int NX, int NY) {
  return {std::max(0, b.x0 - m), std::min(NX, b.x1 + m), std::max(0, b.y0 - m), std::min(NY, b.y1 + m)};
}

// relaxed PoU weights on the node box of Omega (3-D array, k fastest)
std::vector<double> pou_weights(const Box& om, int NX, int NY, int NZ, int o) {
  const int nx = om.x1 - om.x0 + 1, ny = om.y1 - om.y0 + 1, nz = NZ + 1;
  std::vector<double> w((size_t)nx * ny * nz), nw;
  auto idx = [&](int i, int j, int k) { return ((size_t)i * ny + j) * nz + k; };
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < ny; ++j) {
      const int gi = om.x0 + i, gj = om.y0 + j;
      const bool cut = (gi == om.x0 && om.x0 > 0) || (gi == om.x1 && om.x1 < NX) ||
                       (gj == om.y0 && om.y0 > 0) || (gj == om.y1 && om.y1 < NY);
      for (int k = 0; k < nz; ++k) w[idx(i, j, k)] = cut ? 0.0 : 2.0 * o;
    }
  for (int sweep = 0; sweep < 2 * o - 1; ++sweep) {
    nw = w;
    for (int i = 0; i < nx; ++i)
      for (int j = 0; j < ny; ++j)
        for (int k = 0; k < nz; ++k) {
          double best = w[idx(i, j, k)];
          for (int di = -1; di <= 1; ++di)
            for (int dj = -1; dj <= 1; ++dj)
              for (int dk = -1; dk <= 1; ++dk) {
                const int a = i + di, b = j + dj, c = k + dk;
                if (a < 0 || a >= nx || b < 0 || b >= ny || c < 0 || c >= nz) continue;
                best = std::min(best, w[idx(a, b, c)] + 1.0);
              }
          nw[idx(i, j, k)] = std::min(best, 2.0 * o);
        }
    w.swap(nw);
  }
  return w;
}

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Consistent nodal load of the traction (-p, 0, 0) on the i = NX face: for
// every face quad, int N_a dA over its bilinear map X(s, r), with 2x2 Gauss
// points (exact on a planar quad, whose area element is linear in s and r).
// Returns the x component per face node (j, k), index j (NZ + 1) + k.
std::vector<double> end_face_load(const msgfem* h) {
  const int NY = h->NY, NZ = h->NZ;
  std::vector<double> f((size_t)(NY + 1) * (NZ + 1), 0.0);
  const double gp = 0.57735026918962576451;
  const int cj[4] = {0, 1, 1, 0}, ck[4] = {0, 0, 1, 1};
  for (int j = 0; j < NY; ++j)
    for (int k = 0; k < NZ; ++k) {
      double X[4][3];
      for (int a = 0; a < 4; ++a) node_xyz(h, h->NX, j + cj[a], k + ck[a], X[a]);
      for (int g = 0; g < 4; ++g) {
        const double s = (g & 1) ? gp : -gp, r = (g & 2) ? gp : -gp;
        double Xs[3] = {0, 0, 0}, Xr[3] = {0, 0, 0}, N[4];
        for (int a = 0; a < 4; ++a) {
          const double sa = cj[a] ? 1.0 : -1.0, ra = ck[a] ? 1.0 : -1.0;
          N[a] = 0.25 * (1.0 + sa * s) * (1.0 + ra * r);
          for (int d = 0; d < 3; ++d) {
            Xs[d] += 0.25 * sa * (1.0 + ra * r) * X[a][d];
            Xr[d] += 0.25 * (1.0 + sa * s) * ra * X[a][d];
          }
        }
        const double cx = Xs[1] * Xr[2] - Xs[2] * Xr[1], cy = Xs[2] * Xr[0] - Xs[0] * Xr[2],
                     cz = Xs[0] * Xr[1] - Xs[1] * Xr[0];
        const double dA = std::sqrt(cx * cx + cy * cy + cz * cz);
        for (int a = 0; a < 4; ++a) f[(size_t)(j + cj[a]) * (NZ + 1) + k + ck[a]] += N[a] * dA;
      }
    }
  for (double& v : f) v *= -h->traction;
  return f;
}

}  // namespace

// The load vector b of Eq. fe_matrix_system on all DoFs (node-major, 3 per
// node): the given nodal loads, or the consistent nodal load of the traction
// on the i = NX face; zero on the clamped face i = 0.
std::vector<double> global_load(const msgfem* h) {
  const int NX = h->NX, NY = h->NY, NZ = h->NZ;
  const size_t nn = (size_t)(NX + 1) * (NY + 1) * (NZ + 1);
  std::vector<double> b(3 * nn, 0.0);
  if (!h->h_load.empty()) {
    b = h->h_load;
  } else {
    const std::vector<double> face = end_face_load(h);
    for (int j = 0; j <= NY; ++j)
      for (int k = 0; k <= NZ; ++k) b[3 * (((size_t)NX * (NY + 1) + j) * (NZ + 1) + k)] = face[(size_t)j * (NZ + 1) + k];
  }
  for (size_t n = 0; n < (size_t)(NY + 1) * (NZ + 1); ++n)
    for (int c = 0; c < 3; ++c) b[3 * n + c] = 0.0;   // i = 0: the first (NY+1)(NZ+1) nodes
  return b;
}

void node_xyz(const msgfem* h, int i, int j, int k, double X[3]) {
  if (!h->h_xyz.empty()) {
    const size_t n = ((size_t)i * (h->NY + 1) + j) * (h->NZ + 1) + k;
    X[0] = h->h_xyz[3 * n]; X[1] = h->h_xyz[3 * n + 1]; X[2] = h->h_xyz[3 * n + 2];
  } else {
    X[0] = i * h->hx; X[1] = j * h->hy; X[2] = k * h->hz;
  }
}

msgfem_status build_problem(msgfem* h) {
  const int NX = h->NX, NY = h->NY, NZ = h->NZ;
  std::vector<Box> hats;
  if (!h->boxes.empty()) {
    // explicit boxes: each element of the NX x NY grid in exactly one box
    std::vector<int> cover((size_t)NX * NY, 0);
    for (size_t b = 0; b + 3 < h->boxes.size(); b += 4) {
      Box hat{h->boxes[b], h->boxes[b + 1], h->boxes[b + 2], h->boxes[b + 3]};
      if (hat.x0 < 0 || hat.x1 > NX || hat.y0 < 0 || hat.y1 > NY || hat.x1 <= hat.x0 || hat.y1 <= hat.y0) {
        h->err = "partition box empty or outside the mesh";
        return MSGFEM_EINVAL;
      }
      for (int x = hat.x0; x < hat.x1; ++x)
        for (int y = hat.y0; y < hat.y1; ++y) cover[(size_t)x * NY + y]++;
      hats.push_back(hat);
    }
    for (int c : cover)
      if (c != 1) {
        h->err = "partition boxes do not tile the mesh";
        return MSGFEM_EINVAL;
      }
  } else {
    for (int a = 0; a < h->sx; ++a)
      for (int b = 0; b < h->sy; ++b)
        hats.push_back({(a * NX) / h->sx, ((a + 1) * NX) / h->sx, (b * NY) / h->sy, ((b + 1) * NY) / h->sy});
  }
  h->N = (int)hats.size();
  h->sub.assign(h->N, SubDev{});
  h->hsub.assign(h->N, HostSub{});
  h->n1.assign(h->N, 0);
  h->n2.assign(h->N, 0);
  h->n3.assign(h->N, 0);
  std::vector<Box> omega(h->N), star(h->N);
  for (int j = 0; j < h->N; ++j) {
    const Box& hat = hats[j];
    if (hat.x1 <= hat.x0 || hat.y1 <= hat.y0) {
      h->err = "partition has an empty subdomain";
      return MSGFEM_EINVAL;
    }
    omega[j] = grow(hat, h->o, NX, NY);
    star[j] = grow(hat, h->os, NX, NY);
  }
  const std::vector<double> face = end_face_load(h);
  // partition of unity: global weight sums
  const size_t nnodes = (size_t)(NX + 1) * (NY + 1) * (NZ + 1);
  std::vector<double> total(nnodes, 0.0);
  std::vector<std::vector<double>> wts(h->N);
  for (int j = 0; j < h->N; ++j) {
    const Box& om = omega[j];
    wts[j] = pou_weights(om, NX, NY, NZ, h->o);
    const int nx = om.x1 - om.x0 + 1, ny = om.y1 - om.y0 + 1;
    for (int i = 0; i < nx; ++i)
      for (int jj = 0; jj < ny; ++jj)
        for (int k = 0; k <= NZ; ++k)
          total[((size_t)(om.x0 + i) * (NY + 1) + om.y0 + jj) * (NZ + 1) + k] +=
              wts[j][((size_t)i * ny + jj) * (NZ + 1) + k];
  }
  for (size_t n = 0; n < nnodes; ++n)
    if (!(total[n] > 0.0)) {
      h->err = "partition of unity: a node has zero total weight";
      return MSGFEM_EINVAL;
    }
  for (int j = 0; j < h->N; ++j) {
    SubDev& s = h->sub[j];
    HostSub& hs = h->hsub[j];
    const Box& st = star[j];
    const Box& om = omega[j];
    s.inst = 0;
    s.I0 = st.x0; s.I1 = st.x1; s.J0 = st.y0; s.J1 = st.y1;
    s.oI0 = om.x0; s.oI1 = om.x1; s.oJ0 = om.y0; s.oJ1 = om.y1;
    s.nxn = st.x1 - st.x0 + 1;
    s.nyn = st.y1 - st.y0 + 1;
    s.nzn = NZ + 1;
    s.npl = s.nxn * s.nyn;
    s.nnode = s.npl * s.nzn;
    s.nfull = 3 * s.nnode;
    s.floating = st.x0 > 0 ? 1 : 0;
    s.loaded = st.x1 == NX ? 1 : 0;
    hs.cls.assign(s.npl, 1);
    int c1 = 0, c2 = 0, c3 = 0;
    for (int q = 0; q < s.npl; ++q) {
      const int gi = s.I0 + q / s.nyn, gj = s.J0 + q % s.nyn;
      signed char c = 1;
      if (gi == 0) c = 3;
      else if ((gi == st.x0 && st.x0 > 0) || (gi == st.x1 && st.x1 < NX) || (gj == st.y0 && st.y0 > 0) ||
               (gj == st.y1 && st.y1 < NY))
        c = 2;
      hs.cls[q] = c;
      (c == 1 ? c1 : c == 2 ? c2 : c3)++;
    }
    h->n1[j] = 3 * c1 * s.nzn;
    h->n2[j] = 3 * c2 * s.nzn;
    h->n3[j] = 3 * c3 * s.nzn;
    s.nK = 3 * (c1 + c2);
    s.nA = 3 * c1;
    s.bK = round_up(std::max(s.nK, 1), TILE);
    s.bA = round_up(std::max(s.nA, 1), TILE);
    hs.mapK.assign(s.bK, -1);
    hs.mapA.assign(s.bA, -1);
    hs.invK.assign(3 * s.npl, -1);
    hs.invA.assign(3 * s.npl, -1);
    int ck = 0, ca = 0;
    for (int q = 0; q < s.npl; ++q)
      for (int c = 0; c < 3; ++c) {
        if (hs.cls[q] != 3) { hs.mapK[ck] = 3 * q + c; hs.invK[3 * q + c] = ck++; }
        if (hs.cls[q] == 1) { hs.mapA[ca] = 3 * q + c; hs.invA[3 * q + c] = ca++; }
      }
    for (int i = 0; i < 6; ++i) s.pin[i] = -1;
    if (s.floating) {
      // 3-2-1 pins on three bottom corners A, B, C of the Omega* node box: all
      // components at A; at B the two components least aligned with AB (they
      // stop the rotations about the axes normal to AB); at C the component
      // that the remaining rotation about AB moves most, max |(AB x AC)_c|
      // (on the box beam: y, z at B and z at C)
      const int qa = 0, qb = (s.nxn - 1) * s.nyn, qc = s.nyn - 1;
      double A[3], B[3], Cc[3];
      node_xyz(h, s.I0, s.J0, 0, A);
      node_xyz(h, s.I1, s.J0, 0, B);
      node_xyz(h, s.I0, s.J1, 0, Cc);
      const double ab[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
      const double ac[3] = {Cc[0] - A[0], Cc[1] - A[1], Cc[2] - A[2]};
      int skip = 0;
      for (int d = 1; d < 3; ++d)
        if (std::fabs(ab[d]) > std::fabs(ab[skip])) skip = d;
      const double nrm[3] = {ab[1] * ac[2] - ab[2] * ac[1], ab[2] * ac[0] - ab[0] * ac[2],
                             ab[0] * ac[1] - ab[1] * ac[0]};
      int cpin = 0;
      for (int d = 1; d < 3; ++d)
        if (std::fabs(nrm[d]) > std::fabs(nrm[cpin])) cpin = d;
      s.pin[0] = 3 * qa; s.pin[1] = 3 * qa + 1; s.pin[2] = 3 * qa + 2;
      int np = 3;
      for (int d = 0; d < 3; ++d)
        if (d != skip) s.pin[np++] = 3 * qb + d;
      s.pin[5] = 3 * qc + cpin;
    }
    // mu on Omega* nodes (zero outside Omega)
    hs.mu.assign(s.nnode, 0.0);
    const int onx = om.x1 - om.x0 + 1, ony = om.y1 - om.y0 + 1;
    for (int k = 0; k <= NZ; ++k)
      for (int q = 0; q < s.npl; ++q) {
        const int gi = s.I0 + q / s.nyn, gj = s.J0 + q % s.nyn;
        if (gi < om.x0 || gi > om.x1 || gj < om.y0 || gj > om.y1) continue;
        const double w = wts[j][((size_t)(gi - om.x0) * ony + (gj - om.y0)) * (NZ + 1) + k];
        (void)onx;
        hs.mu[(size_t)k * s.npl + q] = w / total[((size_t)gi * (NY + 1) + gj) * (NZ + 1) + k];
      }
    // the given nodal loads on the Omega* nodes (a particular function when
    // they touch B1), or the consistent nodal load of the traction (-p, 0, 0)
    // on the x = L face
    hs.bload.assign(s.nfull, 0.0);
    if (!h->h_load.empty()) {
      bool b1 = false;
      for (int k = 0; k <= NZ; ++k)
        for (int q = 0; q < s.npl; ++q) {
          const int gi = s.I0 + q / s.nyn, gj = s.J0 + q % s.nyn;
          const size_t gn = ((size_t)gi * (NY + 1) + gj) * (NZ + 1) + k;
          for (int c = 0; c < 3; ++c) {
            const double v = h->h_load[3 * gn + c];
            hs.bload[((size_t)k * s.npl + q) * 3 + c] = v;
            b1 = b1 || (v != 0.0 && hs.cls[q] == 1);
          }
        }
      s.loaded = b1 ? 1 : 0;
    } else if (s.loaded)
      for (int k = 0; k <= NZ; ++k)
        for (int q = 0; q < s.npl; ++q) {
          const int gi = s.I0 + q / s.nyn, gj = s.J0 + q % s.nyn;
          if (gi != NX) continue;
          hs.bload[((size_t)k * s.npl + q) * 3] = face[(size_t)gj * (NZ + 1) + k];
        }
  }
  // batched instances: subdomain j of instance i is subdomain i N0 + j
  h->N0 = h->N;
  if (h->S > 1) {
    for (int i = 1; i < h->S; ++i)
      for (int j = 0; j < h->N0; ++j) {
        SubDev c = h->sub[j];
        c.inst = i;
        h->sub.push_back(c);
        h->hsub.push_back(h->hsub[j]);
        h->n1.push_back(h->n1[j]);
        h->n2.push_back(h->n2[j]);
        h->n3.push_back(h->n3[j]);
      }
    h->N = h->S * h->N0;
  }
  // coarse pairs: Omega_s node box intersected with Omega*_t node box
  // (within one instance; the coarse problem exists for unbatched handles)
  h->pairs.clear();
  for (int s = 0; s < h->N0; ++s)
    for (int t = 0; t < h->N0; ++t) {
      const SubDev& S = h->sub[s];
      const SubDev& T = h->sub[t];
      const int x0 = std::max(S.oI0, T.I0), x1 = std::min(S.oI1, T.I1);
      const int y0 = std::max(S.oJ0, T.J0), y1 = std::min(S.oJ1, T.J1);
      if (x0 <= x1 && y0 <= y1) h->pairs.push_back({s, t, x0, x1, y0, y1});
    }
  return MSGFEM_OK;
}

// Element types of the angle field in h->h_angles (one field per instance):
// one per ply (and instance) when the angle depends on the layer only and the
// mesh is the box with default frames (layered); on a curved mesh, elements
// with the same shape (corners up to a translation, compared bit for bit),
// ply frame and angle share one type, etype maps every element
// (instance-major) to its type and trep gives a type's first element; else one
// type per element.  types holds each type's angle.
void element_types(const msgfem* h, bool& layered, std::vector<double>& types, std::vector<int>& etype,
                   std::vector<int>& trep) {
  const size_t nel = (size_t)h->NX * h->NY * h->NZ;
  const size_t ntot = nel * h->S;
  const bool geometric = !h->h_xyz.empty() || !h->h_frame.empty();
  layered = !geometric;
  for (size_t e = 0; e < ntot && layered; ++e)
    layered = h->h_angles[e] == h->h_angles[(e / nel) * nel + e % h->NZ];
  types.clear();
  etype.clear();
  trep.clear();
  if (layered) {
    for (int i = 0; i < h->S; ++i)
      types.insert(types.end(), h->h_angles.begin() + (size_t)i * nel, h->h_angles.begin() + (size_t)i * nel + h->NZ);
  } else if (geometric) {
    etype.resize(ntot);
    std::unordered_map<std::string, int> seen;
    std::string key;
    for (size_t g = 0; g < ntot; ++g) {
      const size_t e = g % nel;
      const int ie = (int)(e / ((size_t)h->NY * h->NZ)), je = (int)((e / h->NZ) % h->NY), ke = (int)(e % h->NZ);
      double v[34];
      double X0[3];
      node_xyz(h, ie, je, ke, X0);
      for (int a = 0; a < 8; ++a) {
        double X[3];
        node_xyz(h, ie + (a & 1), je + ((a >> 1) & 1), ke + (a >> 2), X);
        for (int d = 0; d < 3; ++d) v[3 * a + d] = X[d] - X0[d];
      }
      for (int q = 0; q < 9; ++q) v[24 + q] = h->h_frame.empty() ? 0.0 : h->h_frame[e * 9 + q];
      v[33] = h->h_angles[g];
      key.assign(reinterpret_cast<const char*>(v), sizeof(v));
      auto it = seen.find(key);
      if (it == seen.end()) {
        it = seen.emplace(key, (int)types.size()).first;
        types.push_back(h->h_angles[g]);
        trep.push_back((int)e);
      }
      etype[g] = it->second;
    }
  } else {
    types = h->h_angles;
  }
}

// ---------------------------------------------------------------------------
// Device storage of the layer blocks (D, E, Linv of K and A11), their factors
// and the compact solve buffers of one subdomain, in the factor's precision;
// the parts are laid out in this order, each aligned to 256 bytes.
namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

template <typename T>
size_t place_blocks(SubDev& s, char* base, bool assign) {
  const size_t bK2 = (size_t)s.bK * s.bK, bA2 = (size_t)s.bA * s.bA;
  const size_t parts[12] = {bK2 * (2 * s.nzn - 1), bK2 * s.nzn, bA2 * (2 * s.nzn - 1), bA2 * s.nzn,
                            (size_t)s.nzn * s.bK * PST, (size_t)s.nzn * s.bA * PST, (size_t)s.bK * PST,
                            (size_t)s.bA * PST, (size_t)s.nzn * s.bK * KB, (size_t)s.nzn * s.bA * KB,
                            (size_t)s.bK * KB, (size_t)s.bA * KB};
  size_t off = 0;
  T* p[12];
  for (int i = 0; i < 12; ++i) {
    p[i] = reinterpret_cast<T*>(base + off);
    off = align_up(off + parts[i] * sizeof(T), 256);
  }
  if (assign) {
    if constexpr (std::is_same<T, float>::value) {
      s.DKf = p[0]; s.EKf = p[0] + bK2 * s.nzn; s.LKf = p[1];
      s.DAf = p[2]; s.EAf = p[2] + bA2 * s.nzn; s.LAf = p[3];
      s.ycKf = p[4]; s.ycAf = p[5]; s.rcKf = p[6]; s.rcAf = p[7];
      s.ycK8f = p[8]; s.ycA8f = p[9]; s.rcK8f = p[10]; s.rcA8f = p[11];
    } else {
      s.DK = p[0]; s.EK = p[0] + bK2 * s.nzn; s.LK = p[1];
      s.DA = p[2]; s.EA = p[2] + bA2 * s.nzn; s.LA = p[3];
      s.ycK = p[4]; s.ycA = p[5]; s.rcK = p[6]; s.rcA = p[7];
      s.ycK8 = p[8]; s.ycA8 = p[9]; s.rcK8 = p[10]; s.rcA8 = p[11];
    }
  }
  return off;
}

}  // namespace

size_t sub_block_bytes(msgfem* h, int j) {
  SubDev& s = h->sub[j];
  return h->mixed ? place_blocks<float>(s, nullptr, false) : place_blocks<double>(s, nullptr, false);
}

size_t place_sub_blocks(msgfem* h, int j, char* base) {
  SubDev& s = h->sub[j];
  return h->mixed ? place_blocks<float>(s, base, true) : place_blocks<double>(s, base, true);
}

// Subdomains are taken largest first and a wave is closed when the next one no
// longer fits (waves of similar sizes); members are kept in index order.  When
// everything fits: one wave of all subdomains.
msgfem_status plan_waves(msgfem* h, size_t budget) {
  std::vector<size_t> bytes(h->N);
  size_t total = 0;
  for (int j = 0; j < h->N; ++j) total += (bytes[j] = sub_block_bytes(h, j));
  h->waves.clear();
  h->wave_of.assign(h->N, 0);
  if (total <= budget) {
    h->waves.emplace_back();
    for (int j = 0; j < h->N; ++j) h->waves[0].members.push_back(j);
  } else {
    std::vector<int> order(h->N);
    for (int j = 0; j < h->N; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return bytes[a] > bytes[b]; });
    size_t used = 0;
    for (int j : order) {
      if (bytes[j] > budget) {
        h->waves.clear();
        h->err = "a subdomain's factor storage exceeds the wave budget (msgfem_options.wave_mb)";
        return MSGFEM_ENOMEM;
      }
      if (h->waves.empty() || used + bytes[j] > budget) {
        h->waves.emplace_back();
        used = 0;
      }
      h->waves.back().members.push_back(j);
      used += bytes[j];
    }
    for (auto& w : h->waves) std::sort(w.members.begin(), w.members.end());
  }
  size_t pool = 0;
  for (size_t w = 0; w < h->waves.size(); ++w) {
    size_t sum = 0;
    for (int j : h->waves[w].members) {
      sum += bytes[j];
      h->wave_of[j] = (int)w;
    }
    pool = std::max(pool, sum);
  }
  h->pool_bytes = pool;
  return MSGFEM_OK;
}

// ---------------------------------------------------------------------------
// Factorisation schedule: per layer, SYRK; per tile column k either
// right-looking (POTRF, TRMM, UPDATE of the whole trailing matrix by column k,
// inner dimension 64) or left-looking (UPDATE of column k by the finished
// columns 0..k-1, inner dimension 64 k, then POTRF, TRMM): the same work in
// fewer, longer tasks.  The block inverse of layer l (TRTRI rows 1..T-1, each row depending
// on the previous one) needs only L_l, so row i is issued together with the
// (i-1)-th step of layer l + 1: it fills the SMs that the narrow POTRF and
// TRMM steps leave idle.  Tasks of all subdomains (and of K and A11) with the
// same key are launched together; within a step the longest tasks go first.
namespace {

template <typename T>
using FactorKeysT = std::map<long long, std::vector<TileTaskT<T>>>;
using FactorKeys = FactorKeysT<double>;

// Split of the block inverse's long row tasks (the coarse matrix: one dense
// block of up to ~65 tiles): a task of block row i, column k sums i - k tile
// products on one CTA, so the row's critical path grows with the matrix size.
// With split > 0, a task of more than `split` tiles becomes partial sums of at
// most `split` tiles each (one step, into scratch tiles) and a final task that
// adds them through an identity strip [I I ... I] and post-multiplies (the next
// step).  ident is 64 x (64 * maxc) row-major with maxc = ceil((T - 1) / split).
struct InverseSplit {
  int split = 0;
  void* scratch = nullptr;   // tiles of 64 x 64, contiguous
  const void* ident = nullptr;
  int ident_ld = 0;
};

template <typename Sc>
void add_matrix_tasks(FactorKeysT<Sc>& fk, Sc* D, Sc* E, Sc* L, int b, int nL, int sub, int Tmax, bool left = false,
                      long long skew = 0, const InverseSplit& isp = InverseSplit()) {
  const int T = b / TILE;
  const long long per_layer = 3LL * Tmax + 1;
  auto tileD = [&](int l, int i, int j) { return D + (size_t)l * b * b + (size_t)i * TILE * b + (size_t)j * TILE; };
  auto tileE = [&](int l, int i, int j) { return E + (size_t)l * b * b + (size_t)i * TILE * b + (size_t)j * TILE; };
  auto tileL = [&](int l, int i, int j) { return L + (size_t)l * b * b + (size_t)i * TILE * b + (size_t)j * TILE; };
  for (int l = 0; l < nL; ++l) {
    const long long base = l * per_layer + skew;
    if (l > 0)
      for (int i = 0; i < T; ++i)
        for (int j = 0; j <= i; ++j)
          fk[base].push_back({tileE(l - 1, i, 0), tileE(l - 1, j, 0), tileD(l, i, j), nullptr, b, b, b, b,
                              G_TRANSB | G_ACC | G_NEG | (i == j ? G_SYMC : 0), sub});
    for (int k = 0; k < T && left; ++k) {
      // left-looking: update of tile column k with all finished columns 0..k-1
      // (one GEMM of inner dimension 64 k per tile instead of k GEMMs of 64)
      auto& upd = fk[base + 1 + 3 * k];
      if (k > 0) {
        for (int i = k; i < T; ++i)
          upd.push_back({tileD(l, i, 0), tileD(l, k, 0), tileD(l, i, k), nullptr, b, b, b, k * TILE,
                         G_TRANSB | G_ACC | G_NEG | (i == k ? G_SYMC : 0), sub});
        if (l + 1 < nL)
          for (int i = 0; i < T; ++i)
            upd.push_back({tileE(l, i, 0), tileD(l, k, 0), tileE(l, i, k), nullptr, b, b, b, k * TILE,
                           G_TRANSB | G_ACC | G_NEG, sub});
      }
      fk[base + 2 + 3 * k].push_back({nullptr, nullptr, tileD(l, k, k), tileL(l, k, k), 0, 0, b, 0, G_POTRF, sub});
      auto& trmm = fk[base + 3 + 3 * k];
      for (int i = k + 1; i < T; ++i)
        trmm.push_back({tileD(l, i, k), tileL(l, k, k), tileD(l, i, k), nullptr, b, b, b, TILE, G_TRANSB | G_TRIB, sub});
      if (l + 1 < nL)
        for (int i = 0; i < T; ++i)
          trmm.push_back({tileE(l, i, k), tileL(l, k, k), tileE(l, i, k), nullptr, b, b, b, TILE, G_TRANSB | G_TRIB, sub});
    }
    for (int k = 0; k < T && !left; ++k) {
      // right-looking: POTRF, TRMM, then the update of the whole trailing matrix
      fk[base + 1 + 3 * k].push_back({nullptr, nullptr, tileD(l, k, k), tileL(l, k, k), 0, 0, b, 0, G_POTRF, sub});
      auto& trmm = fk[base + 2 + 3 * k];
      for (int i = k + 1; i < T; ++i)
        trmm.push_back({tileD(l, i, k), tileL(l, k, k), tileD(l, i, k), nullptr, b, b, b, TILE, G_TRANSB | G_TRIB, sub});
      if (l + 1 < nL)
        for (int i = 0; i < T; ++i)
          trmm.push_back({tileE(l, i, k), tileL(l, k, k), tileE(l, i, k), nullptr, b, b, b, TILE, G_TRANSB | G_TRIB, sub});
      auto& upd = fk[base + 3 + 3 * k];
      for (int j = k + 1; j < T; ++j) {
        for (int i = j; i < T; ++i)
          upd.push_back({tileD(l, i, k), tileD(l, j, k), tileD(l, i, j), nullptr, b, b, b, TILE,
                         G_TRANSB | G_ACC | G_NEG | (i == j ? G_SYMC : 0), sub});
        if (l + 1 < nL)
          for (int i = 0; i < T; ++i)
            upd.push_back({tileE(l, i, k), tileD(l, j, k), tileE(l, i, j), nullptr, b, b, b, TILE,
                           G_TRANSB | G_ACC | G_NEG, sub});
      }
    }
    // block inverse rows, deferred into the steps of the next layer
    const long long next = (l + 1) * per_layer + skew;
    for (int i = 1; i < T && isp.split <= 0; ++i) {
      auto& tr = fk[next + (i - 1)];
      for (int k = 0; k < i; ++k)
        tr.push_back({tileD(l, i, k), tileL(l, k, k), tileL(l, i, k), tileL(l, i, i), b, b, b, (i - k) * TILE,
                      G_POSTMUL | G_NEG, sub});
    }
    for (int i = 1; i < T && isp.split > 0; ++i) {
      auto& part = fk[next + 2 * (i - 1)];
      auto& fin = fk[next + 2 * (i - 1) + 1];
      size_t off = 0;   // scratch tiles of row i
      for (int k = 0; k < i; ++k) {
        if (i - k <= isp.split) {
          fin.push_back({tileD(l, i, k), tileL(l, k, k), tileL(l, i, k), tileL(l, i, i), b, b, b, (i - k) * TILE,
                         G_POSTMUL | G_NEG, sub});
          continue;
        }
        const int nc = (i - k + isp.split - 1) / isp.split;
        Sc* s0 = static_cast<Sc*>(isp.scratch) + off * TILE * TILE;
        for (int c = 0; c < nc; ++c) {
          const int m0 = k + c * isp.split, nm = std::min(isp.split, i - m0);
          part.push_back({tileD(l, i, m0), tileL(l, m0, k), s0 + (size_t)c * TILE * TILE, nullptr, b, b, TILE,
                          nm * TILE, 0, sub});
        }
        fin.push_back({static_cast<const Sc*>(isp.ident), s0, tileL(l, i, k), tileL(l, i, i), isp.ident_ld, TILE, b,
                       nc * TILE, G_POSTMUL | G_NEG, sub});
        off += nc;
      }
    }
  }
}

template <typename T>
void flatten(FactorKeysT<T>& fk, ScheduleT<T>& sch, bool append = false) {
  if (!append) {
    sch.steps.clear();
    sch.gemm.clear();
    sch.k32 = true;
  }
  sch.steps.emplace_back();
  for (auto& kv : fk) {
    auto& v = kv.second;
    if (v.empty()) continue;
    for (const auto& t : v)
      if (!(t.flags & G_POTRF) && t.K % 32 != 0) sch.k32 = false;
    // POTRF tasks (short critical path) and then the longest GEMM tasks first
    std::stable_sort(v.begin(), v.end(), [](const TileTaskT<T>& x, const TileTaskT<T>& y) {
      const int px = (x.flags & G_POTRF) ? 1 : 0, py = (y.flags & G_POTRF) ? 1 : 0;
      if (px != py) return px > py;
      return x.K > y.K;
    });
    sch.steps.back().push_back({(int)sch.gemm.size(), (int)v.size()});
    sch.gemm.insert(sch.gemm.end(), v.begin(), v.end());
  }
}

// Solve schedule of one matrix kind over all subdomains.
template <typename Sc>
void add_solve_tasks(std::map<long long, std::vector<SolveTaskT<Sc>>>& keys, Sc* E, Sc* L, Sc* yc, Sc* rc,
                     const int* map, int b, int nL, int npl, int sub, int PW, long long skew = 0) {
  const int T = b / TILE;
  for (int l = 0; l < nL; ++l) {
    const int row_off = l * 3 * npl;
    for (int i = 0; i < T; ++i) {
      SolveTaskT<Sc> f1{};
      f1.C = rc + (size_t)i * TILE * PW;
      f1.gmap = map + i * TILE;
      f1.row_off = row_off;
      f1.sub = sub;
      f1.flags = S_INIT_GATHER;
      if (l > 0) {
        f1.A = E + (size_t)(l - 1) * b * b + (size_t)i * TILE * b;
        f1.B = yc + (size_t)(l - 1) * b * PW;
        f1.lda = b;
        f1.K = b;
        f1.flags |= S_NEG;
      }
      keys[2LL * l + skew].push_back(f1);
      SolveTaskT<Sc> f2{};
      f2.C = yc + (size_t)l * b * PW + (size_t)i * TILE * PW;
      f2.A = L + (size_t)l * b * b + (size_t)i * TILE * b;
      f2.B = rc;
      f2.lda = b;
      f2.K = (i + 1) * TILE;
      f2.sub = sub;
      keys[2LL * l + 1 + skew].push_back(f2);
    }
  }
  for (int l = nL - 1; l >= 0; --l) {
    const long long kb = 2LL * nL + 1 + 2LL * (nL - 1 - l) + skew;
    const int row_off = l * 3 * npl;
    for (int i = 0; i < T; ++i) {
      SolveTaskT<Sc> b1{};
      b1.C = rc + (size_t)i * TILE * PW;
      b1.init = yc + (size_t)l * b * PW + (size_t)i * TILE * PW;
      b1.flags = S_INIT_TILE;
      b1.sub = sub;
      if (l + 1 < nL) {
        b1.A = E + (size_t)l * b * b + (size_t)i * TILE;
        b1.B = yc + (size_t)(l + 1) * b * PW;
        b1.lda = b;
        b1.K = b;
        b1.flags |= S_TRANSA | S_NEG;
      }
      keys[kb].push_back(b1);
      SolveTaskT<Sc> b2{};
      b2.C = yc + (size_t)l * b * PW + (size_t)i * TILE * PW;
      b2.A = L + (size_t)l * b * b + (size_t)i * TILE * b + (size_t)i * TILE;
      b2.B = rc + (size_t)i * TILE * PW;
      b2.lda = b;
      b2.K = b - i * TILE;
      b2.flags = S_TRANSA | S_SCATTER;
      b2.smap = map + i * TILE;
      b2.row_off = row_off;
      b2.sub = sub;
      keys[kb + 1].push_back(b2);
    }
  }
}

template <typename T>
void flatten_solve(std::map<long long, std::vector<SolveTaskT<T>>>& keys, SolveScheduleT<T>& sch,
                   bool append = false) {
  if (!append) {
    sch.steps.clear();
    sch.tasks.clear();
    sch.kmax = 0;
    sch.k64 = true;
  }
  sch.steps.emplace_back();
  for (auto& kv : keys) {
    if (kv.second.empty()) continue;
    // longest tasks first: CTAs are dispatched in launch order (LPT balance)
    std::stable_sort(kv.second.begin(), kv.second.end(),
                     [](const SolveTaskT<T>& x, const SolveTaskT<T>& y) { return x.K > y.K; });
    sch.steps.back().push_back({(int)sch.tasks.size(), (int)kv.second.size()});
    for (const auto& t : kv.second) {
      sch.kmax = std::max(sch.kmax, t.K);
      if (t.K % 64 != 0) sch.k64 = false;
    }
    sch.tasks.insert(sch.tasks.end(), kv.second.begin(), kv.second.end());
  }
}

}  // namespace

// The 2N factorisations of a wave are independent chains; they are dealt into
// NGROUP groups, each launched on its own stream, so that a group's narrow
// steps (POTRF, TRMM, late UPDATEs) overlap the wide steps of the others
// instead of waiting at a common launch boundary.
// Ticket order of the persistent factorisation: the start order of a list
// schedule of the tasks on `workers` resident CTAs, simulated on the host with
// estimated task times (a tile Cholesky ~12 units, a GEMM task 2 + K / 64, one
// more with the post-multiplication), always starting a task of the chain with
// the longest remaining path.  A task starts in the simulation only after the
// previous step of its chain has finished, so the order is topological.
void build_persistent_meta(const ScheduleT<float>& s, std::vector<int4>& meta, int& pcount, int workers) {
  const int ng = (int)s.steps.size();
  std::vector<int> base(ng + 1, 0);
  for (int g = 0; g < ng; ++g) base[g + 1] = base[g] + (int)s.steps[g].size();
  pcount = base[ng];
  auto cost = [&](const TileTaskT<float>& t) {
    if (t.flags & G_POTRF) return 12.0;
    return 2.0 + t.K / 64.0 + ((t.flags & G_POSTMUL) ? 1.0 : 0.0);
  };
  // remaining path of each chain from each step (the slowest task of every later step)
  std::vector<std::vector<double>> rem(ng);
  for (int g = 0; g < ng; ++g) {
    const auto& st = s.steps[g];
    rem[g].assign(st.size() + 1, 0.0);
    for (int k = (int)st.size() - 1; k >= 0; --k) {
      double mx = 0.0;
      for (int i = st[k].first; i < st[k].first + st[k].count; ++i) mx = std::max(mx, cost(s.gemm[i]));
      rem[g][k] = rem[g][k + 1] + mx;
    }
  }
  std::vector<int> cur(ng, 0), started(ng, 0), done(ng, 0);
  std::priority_queue<std::pair<double, int>> ready;   // (remaining path, chain)
  for (int g = 0; g < ng; ++g)
    if (!s.steps[g].empty()) ready.push({rem[g][0], g});
  using Ev = std::pair<double, int>;   // (finish time, chain)
  std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> running;
  meta.clear();
  meta.reserve(s.gemm.size());
  double now = 0.0;
  int free_workers = std::max(1, workers);
  while (!ready.empty() || !running.empty()) {
    while (free_workers > 0 && !ready.empty()) {
      const int g = ready.top().second;
      ready.pop();
      const int k = cur[g];
      const SchedStep& st = s.steps[g][k];
      const int i = st.first + started[g]++;
      const int self = base[g] + k;
      meta.push_back(make_int4(self, k > 0 ? self - 1 : -1, k > 0 ? s.steps[g][k - 1].count : 0, i));
      running.push({now + cost(s.gemm[i]), g});
      --free_workers;
      if (started[g] < st.count) ready.push({rem[g][k], g});
    }
    if (running.empty()) break;
    const Ev e = running.top();
    running.pop();
    now = e.first;
    ++free_workers;
    const int g = e.second;
    if (++done[g] == s.steps[g][cur[g]].count) {   // the chain's step is complete: its next step is ready
      ++cur[g];
      started[g] = done[g] = 0;
      if (cur[g] < (int)s.steps[g].size()) ready.push({rem[g][cur[g]], g});
    }
  }
}

int factor_groups(const msgfem* h, const WaveSched& w) {
  return (h->mixed && h->factor_persistent) ? std::max(1, 2 * (int)w.members.size()) : h->ngroup_factor;
}

void build_wave_factor_schedule(msgfem* h, WaveSched& w) {
  int Tmax = 1;
  for (const auto& s : h->sub) Tmax = std::max(Tmax, std::max(s.bK, s.bA) / TILE);
  const int ng = factor_groups(h, w);
  const bool left = h->factor_left != 0;
  if (h->mixed) {
    std::vector<FactorKeysT<float>> fk(ng);
    int chain = 0;
    for (int j : w.members) {
      SubDev& s = h->sub[j];
      add_matrix_tasks(fk[chain++ % ng], s.DKf, s.EKf, s.LKf, s.bK, s.nzn, j, Tmax, left);
      add_matrix_tasks(fk[chain++ % ng], s.DAf, s.EAf, s.LAf, s.bA, s.nzn, j, Tmax, left);
    }
    w.factf.steps.clear();
    w.factf.gemm.clear();
    for (int g = 0; g < ng; ++g) flatten(fk[g], w.factf, true);
    if (h->factor_persistent) build_persistent_meta(w.factf, w.pmeta, w.pcount, 3 * 152);
    else w.pmeta.clear();
    return;
  }
  std::vector<FactorKeys> fk(ng);
  int chain = 0;
  for (int j : w.members) {
    SubDev& s = h->sub[j];
    add_matrix_tasks(fk[chain++ % ng], s.DK, s.EK, s.LK, s.bK, s.nzn, j, Tmax, left);
    add_matrix_tasks(fk[chain++ % ng], s.DA, s.EA, s.LA, s.bA, s.nzn, j, Tmax, left);
  }
  w.fact.steps.clear();
  w.fact.gemm.clear();
  for (int g = 0; g < ng; ++g) flatten(fk[g], w.fact, true);
}

void build_factor_schedule(msgfem* h) {
  for (WaveSched& w : h->waves) build_wave_factor_schedule(h, w);
}

namespace {
template <typename T>
void build_solves_t(msgfem* h, const std::vector<int>& members, SolveScheduleT<T>& sK, SolveScheduleT<T>& sA,
                    SolveScheduleT<T>& sK8, SolveScheduleT<T>& sA8, bool f32) {
  const int ng = h->ngroup;
  using Keys = std::map<long long, std::vector<SolveTaskT<T>>>;
  std::vector<Keys> kk(ng), ka(ng), kk8(ng), ka8(ng);
  for (size_t m = 0; m < members.size(); ++m) {
    const int j = members[m];
    SubDev& s = h->sub[j];
    const int g = (int)(m % ng);
    T* EK = f32 ? (T*)s.EKf : (T*)s.EK;
    T* LK = f32 ? (T*)s.LKf : (T*)s.LK;
    T* EA = f32 ? (T*)s.EAf : (T*)s.EA;
    T* LA = f32 ? (T*)s.LAf : (T*)s.LA;
    add_solve_tasks(kk[g], EK, LK, f32 ? (T*)s.ycKf : (T*)s.ycK, f32 ? (T*)s.rcKf : (T*)s.rcK, s.mapK, s.bK, s.nzn,
                    s.npl, j, PST);
    add_solve_tasks(ka[g], EA, LA, f32 ? (T*)s.ycAf : (T*)s.ycA, f32 ? (T*)s.rcAf : (T*)s.rcA, s.mapA, s.bA, s.nzn,
                    s.npl, j, PST);
    add_solve_tasks(kk8[g], EK, LK, f32 ? (T*)s.ycK8f : (T*)s.ycK8, f32 ? (T*)s.rcK8f : (T*)s.rcK8, s.mapK, s.bK,
                    s.nzn, s.npl, j, KB);
    add_solve_tasks(ka8[g], EA, LA, f32 ? (T*)s.ycA8f : (T*)s.ycA8, f32 ? (T*)s.rcA8f : (T*)s.rcA8, s.mapA, s.bA,
                    s.nzn, s.npl, j, KB);
  }
  for (SolveScheduleT<T>* ss : {&sK, &sA, &sK8, &sA8}) {
    ss->steps.clear();
    ss->tasks.clear();
    ss->kmax = 0;
    ss->k64 = true;
  }
  for (int g = 0; g < ng; ++g) {
    flatten_solve(kk[g], sK, true);
    flatten_solve(ka[g], sA, true);
    flatten_solve(kk8[g], sK8, true);
    flatten_solve(ka8[g], sA8, true);
  }
}
}  // namespace

// Subdomains are dealt into the stream groups as well (per wave).
void build_wave_solve_schedules(msgfem* h, WaveSched& w) {
  if (h->mixed)
    build_solves_t<float>(h, w.members, w.solveKf, w.solveAf, w.solveK8f, w.solveA8f, true);
  else
    build_solves_t<double>(h, w.members, w.solveK, w.solveA, w.solveK8, w.solveA8, false);
}

void build_solve_schedules(msgfem* h) {
  for (WaveSched& w : h->waves) build_wave_solve_schedules(h, w);
}

// Coarse matrix: one dense block of size NcPad, factorised by the same tile
// tasks (subdomain index N is the always-active coarse slot), and solved
// with one forward and one backward sweep.
void build_coarse_schedules(msgfem* h) {
  FactorKeys fk;
  const int b = h->NcPad;
  InverseSplit isp;
  if (h->d_cscr != nullptr && h->d_cid != nullptr) {
    size_t tiles = 0;
    int maxc = 1;
    coarse_inverse_split_sizes(b / TILE, COARSE_INV_SPLIT, &tiles, &maxc);
    isp.split = COARSE_INV_SPLIT;
    isp.scratch = h->d_cscr;
    isp.ident = h->d_cid;
    isp.ident_ld = maxc * TILE;
  }
  add_matrix_tasks<double>(fk, h->d_AH, nullptr, h->d_AHinv, b, 1, h->N, b / TILE, false, 0, isp);
  flatten(fk, h->cfact);
  const int T = b / TILE;
  std::map<long long, std::vector<SolveTask>> keys;
  for (int i = 0; i < T; ++i) {
    SolveTask f1{};
    f1.C = h->d_rH + (size_t)i * TILE * PST;
    f1.init = h->d_bH + (size_t)i * TILE * PST;
    f1.flags = S_INIT_TILE;
    f1.sub = h->N;
    keys[0].push_back(f1);
    SolveTask f2{};
    f2.C = h->d_yH + (size_t)i * TILE * PST;
    f2.A = h->d_AHinv + (size_t)i * TILE * b;
    f2.B = h->d_rH;
    f2.lda = b;
    f2.K = (i + 1) * TILE;
    f2.sub = h->N;
    keys[1].push_back(f2);
    SolveTask b2{};
    b2.C = h->d_cH + (size_t)i * TILE * PST;
    b2.A = h->d_AHinv + (size_t)i * TILE * b + (size_t)i * TILE;
    b2.B = h->d_yH + (size_t)i * TILE * PST;
    b2.lda = b;
    b2.K = b - i * TILE;
    b2.flags = S_TRANSA;
    b2.sub = h->N;
    keys[2].push_back(b2);
  }
  flatten_solve(keys, h->csolve);
}

// Memory plan of a problem on the host (no handle, no CUDA call): the same
// decomposition as msgfem_setup, the storage of every subdomain and the waves.
extern "C" msgfem_status msgfem_plan(const msgfem_mesh* mesh, const msgfem_partition* part, int overlap,
                                     int oversampling, const msgfem_options* opt, msgfem_plan_info* info) {
  if (!mesh || !part || !info) return MSGFEM_EINVAL;
  if (mesh->kind == 1 || part->elem_part != nullptr) {
    // hexahedron list (host coordinates) or element -> part map: the structured problem
    msgfem_mesh m = *mesh;
    msgfem_partition pt = *part;
    HexNumbering hn;
    std::string err;
    std::vector<double> xyz;
    std::vector<int> boxes;
    if (mesh->kind == 1) {
      if (mesh->node_xyz == nullptr || !recover_structure(mesh->n_nodes, mesh->n_elems, mesh->hex8, hn, err))
        return MSGFEM_EINVAL;
      xyz.assign(3 * (size_t)mesh->n_nodes, 0.0);
      for (int u = 0; u < mesh->n_nodes; ++u)
        for (int c = 0; c < 3; ++c) xyz[3 * (size_t)hn.node_of_user[u] + c] = mesh->node_xyz[3 * (size_t)u + c];
      m.kind = 0;
      m.nx = hn.nx;
      m.ny = hn.ny;
      m.nz = hn.nz;
      m.xyz = xyz.data();
    }
    if (part->elem_part != nullptr) {
      const size_t nel = (size_t)m.nx * m.ny * m.nz;
      std::vector<int> ep(nel);
      for (size_t e = 0; e < nel; ++e) ep[hn.elem_of_user.empty() ? e : hn.elem_of_user[e]] = part->elem_part[e];
      if (!parts_to_boxes(m.nx, m.ny, m.nz, ep.data(), boxes, err)) return MSGFEM_EINVAL;
      pt.n_boxes = (int)(boxes.size() / 4);
      pt.boxes = boxes.data();
      pt.elem_part = nullptr;
    }
    return msgfem_plan(&m, &pt, overlap, oversampling, opt, info);
  }
  if (mesh->nx <= 0 || mesh->ny <= 0 || mesh->nz <= 0) return MSGFEM_EINVAL;
  if (mesh->xyz == nullptr && (!(mesh->hx > 0) || !(mesh->hy > 0) || !(mesh->hz > 0))) return MSGFEM_EINVAL;
  if (part->n_boxes < 0 || (part->n_boxes > 0 && part->boxes == nullptr)) return MSGFEM_EINVAL;
  if (part->n_boxes == 0 && (part->sx <= 0 || part->sy <= 0 || part->sx > mesh->nx || part->sy > mesh->ny))
    return MSGFEM_EINVAL;
  if (overlap < 1 || oversampling < overlap) return MSGFEM_EINVAL;
  if (opt && opt->precision != MSGFEM_FP64 && opt->precision != MSGFEM_MIXED) return MSGFEM_EINVAL;
  msgfem h{};   // value-initialised: the options and material stay zero
  h.NX = mesh->nx; h.NY = mesh->ny; h.NZ = mesh->nz;
  h.hx = mesh->hx; h.hy = mesh->hy; h.hz = mesh->hz; h.traction = mesh->traction;
  h.sx = part->sx; h.sy = part->sy; h.o = overlap; h.os = oversampling;
  if (part->n_boxes > 0) {
    h.boxes.assign(part->boxes, part->boxes + 4 * (size_t)part->n_boxes);
    h.sx = part->n_boxes;
    h.sy = 1;
  }
  const size_t nnodes = (size_t)(h.NX + 1) * (h.NY + 1) * (h.NZ + 1);
  if (mesh->xyz != nullptr) {
    h.h_xyz.assign(mesh->xyz, mesh->xyz + 3 * nnodes);
    for (double v : h.h_xyz)
      if (!std::isfinite(v)) return MSGFEM_EINVAL;
  }
  h.S = (opt && opt->instances > 1) ? opt->instances : 1;
  h.mixed = (opt && opt->precision == MSGFEM_MIXED) ? 1 : 0;
  memset(info, 0, sizeof(*info));
  msgfem_status st = build_problem(&h);
  if (st != MSGFEM_OK) return st;
  size_t total = 0, largest = 0;
  int max_star = 0;
  for (int j = 0; j < h.N; ++j) {
    const size_t b = sub_block_bytes(&h, j);
    total += b;
    largest = std::max(largest, b);
    max_star = std::max(max_star, h.sub[j].nfull);
  }
  const double mib = 1048576.0;
  info->n_subdomains = h.N;
  info->blocks_mb = (double)total / mib;
  info->largest_mb = (double)largest / mib;
  info->n_dof = 3 * (long long)nnodes;
  info->max_star_dof = max_star;
  const size_t budget = (opt && opt->wave_mb > 0) ? (size_t)(opt->wave_mb * mib) : std::numeric_limits<size_t>::max();
  st = plan_waves(&h, budget);
  if (st != MSGFEM_OK) return st;
  info->waves = (int)h.waves.size();
  info->pool_mb = (double)h.pool_bytes / mib;
  return MSGFEM_OK;
}

// Scratch tiles and identity-strip width (tiles) of the split coarse inverse.
void coarse_inverse_split_sizes(int T, int split, size_t* scratch_tiles, int* maxc) {
  size_t most = 0;
  for (int i = 1; i < T; ++i) {
    size_t tiles = 0;
    for (int k = 0; k < i; ++k)
      if (i - k > split) tiles += (size_t)((i - k + split - 1) / split);
    most = std::max(most, tiles);
  }
  *scratch_tiles = most;
  *maxc = std::max(1, (T - 1 + split - 1) / split);
}
