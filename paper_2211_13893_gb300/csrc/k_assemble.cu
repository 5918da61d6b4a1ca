// Local assembly on the GPU: ply tensors, element stiffness, node stencils of
// a_{Omega*_j} and the dense z-layer blocks of K and A11.
//
// Material (Sec. 2, Eq. eq-hooke; Sec. 5.1): the orthotropic ply stiffness
// in its axes is the inverse of the engineering compliance; it is rotated to
// the global frame with the Voigt strain transformation M of the ply axes
// (rows of Q: fibre cos t a0 + sin t a1, transverse -sin t a0 + cos t a1,
// normal a2 of the element's frame; a0, a1, a2 = x, y, z on the box beam),
// C = M^T C_ply M, so that eps:C:eps is invariant.
// Element (Eq. element_stiffness): K_e = sum_g B_g^T C B_g det J_g over the
// 2x2x2 Gauss points (weights 1) of the trilinear map of the element's eight
// nodes (a brick on the box beam), with the 6x24 Voigt B matrix, three
// non-zeros per column.
// GPU node order inside an element: a = ax + 2 ay + 4 az, (ax, ay, az) in
// {0,1}^3; element DoF 3 a + c.
#include <type_traits>

#include "internal.h"

namespace {

__device__ void ply_stiffness(const double* E9, double theta_deg, const double* frame, double C[6][6]) {
  const double E1 = E9[0], E2 = E9[1], E3 = E9[2], G12 = E9[3], G13 = E9[4], G23 = E9[5];
  const double n12 = E9[6], n13 = E9[7], n23 = E9[8];
  // normal compliance block and its inverse (cofactors)
  const double s11 = 1.0 / E1, s22 = 1.0 / E2, s33 = 1.0 / E3;
  const double s12 = -n12 / E1, s13 = -n13 / E1, s23 = -n23 / E2;
  const double c11 = s22 * s33 - s23 * s23, c12 = s13 * s23 - s12 * s33, c13 = s12 * s23 - s13 * s22;
  const double c22 = s11 * s33 - s13 * s13, c23 = s12 * s13 - s11 * s23, c33 = s11 * s22 - s12 * s12;
  const double det = s11 * c11 + s12 * c12 + s13 * c13;
  double Cm[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) Cm[i][j] = 0.0;
  Cm[0][0] = c11 / det; Cm[0][1] = Cm[1][0] = c12 / det; Cm[0][2] = Cm[2][0] = c13 / det;
  Cm[1][1] = c22 / det; Cm[1][2] = Cm[2][1] = c23 / det; Cm[2][2] = c33 / det;
  Cm[3][3] = G23; Cm[4][4] = G13; Cm[5][5] = G12;
  // ply axes (rows of Q) in global coordinates
  double th = theta_deg * (3.14159265358979323846 / 180.0);
  const double c = cos(th), s = sin(th);
  double a[3][3] = {{1.0, 0.0, 0.0}, {0.0, 1.0, 0.0}, {0.0, 0.0, 1.0}};
  if (frame != nullptr)
    for (int r = 0; r < 3; ++r)
      for (int d = 0; d < 3; ++d) a[r][d] = frame[3 * r + d];
  double Q[3][3];
  for (int d = 0; d < 3; ++d) {
    Q[0][d] = c * a[0][d] + s * a[1][d];
    Q[1][d] = -s * a[0][d] + c * a[1][d];
    Q[2][d] = a[2][d];
  }
  // eps_ply = M eps_global (Voigt 11 22 33 23 13 12, engineering shear):
  // M[(i,j)][(p,q)] = (i == j ? 1 : 2) * (p == q ? Q_ip Q_jp : (Q_ip Q_jq + Q_iq Q_jp) / 2)
  const int vi[6] = {0, 1, 2, 1, 0, 0}, vj[6] = {0, 1, 2, 2, 2, 1};
  double M[6][6];
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J) {
      const int i = vi[I], j = vj[I], p = vi[J], q = vj[J];
      const double f = (i == j) ? 1.0 : 2.0;
      M[I][J] = (p == q) ? f * Q[i][p] * Q[j][p] : 0.5 * f * (Q[i][p] * Q[j][q] + Q[i][q] * Q[j][p]);
    }
  double CM[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 6; ++k) acc += Cm[i][k] * M[k][j];
      CM[i][j] = acc;
    }
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 6; ++k) acc += M[k][i] * CM[k][j];
      C[i][j] = acc;
    }
}

// One block per element type; thread (r, c) computes K_e[r][c].
//   layered: type = instance * NZ + ply k (box beam, angle per ply);
//   curved mesh (node coordinates or ply frames): one type per distinct
//   (shape up to translation, frame, angle), trep[type] its first element;
//   otherwise type = instance * nel + element.
__global__ void __launch_bounds__(576)
k_element_stiffness(const double* __restrict__ angles, const double* __restrict__ E9, int layered,
                    int NX, int NY, int NZ, double hx, double hy, double hz, const double* __restrict__ xyz,
                    const double* __restrict__ frame, const int* __restrict__ trep, double* __restrict__ Ke) {
  const int type = blockIdx.x;
  const int nel = NX * NY * NZ;
  // element of the first instance whose corners and frame the type has
  const int e = trep ? trep[type] : (layered ? type % NZ : type % nel);
  const int ie = layered ? 0 : e / (NY * NZ), je = layered ? 0 : (e / NZ) % NY, ke = e % NZ;
  __shared__ double C[6][6];
  __shared__ double X[8][3];        // corner coordinates
  __shared__ double Jinv[8][3][3];  // [gauss][r][d] = d xi_r / d x_d
  __shared__ double detJ[8];
  __shared__ double dN[8][8][3];    // [gauss][node][d/dx, d/dy, d/dz]
  const int tid = threadIdx.x;
  if (tid == 0) {
    double Cl[6][6];
    ply_stiffness(E9, angles[type], frame != nullptr ? frame + (size_t)e * 9 : nullptr, Cl);
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) C[i][j] = Cl[i][j];
  }
  if (tid < 24) {
    const int a = tid / 3, d = tid % 3;
    const int ax = a & 1, ay = (a >> 1) & 1, az = a >> 2;
    if (xyz != nullptr) {
      const size_t node = ((size_t)(ie + ax) * (NY + 1) + (je + ay)) * (NZ + 1) + (ke + az);
      X[a][d] = xyz[3 * node + d];
    } else {
      X[a][d] = d == 0 ? ax * hx : (d == 1 ? ay * hy : az * hz);
    }
  }
  __syncthreads();
  const double gp = 0.57735026918962576451;   // 1/sqrt(3)
  if (tid < 8) {
    // Jacobian J[d][r] = dx_d / dxi_r at Gauss point g, its determinant and inverse
    const int g = tid;
    const double xi[3] = {(g & 1) ? gp : -gp, (g & 2) ? gp : -gp, (g & 4) ? gp : -gp};
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < 8; ++a) {
      const double sa[3] = {(a & 1) ? 1.0 : -1.0, (a & 2) ? 1.0 : -1.0, (a & 4) ? 1.0 : -1.0};
      const double f0 = 1.0 + sa[0] * xi[0], f1 = 1.0 + sa[1] * xi[1], f2 = 1.0 + sa[2] * xi[2];
      const double dr[3] = {0.125 * sa[0] * f1 * f2, 0.125 * f0 * sa[1] * f2, 0.125 * f0 * f1 * sa[2]};
      for (int d = 0; d < 3; ++d)
        for (int r = 0; r < 3; ++r) J[d][r] += X[a][d] * dr[r];
    }
    const double m00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double m01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double m02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double dt = J[0][0] * m00 + J[0][1] * m01 + J[0][2] * m02;
    const double inv = 1.0 / dt;
    // (J^{-1})[r][d] = cofactor(J)[d][r] / det
    Jinv[g][0][0] = m00 * inv;
    Jinv[g][1][0] = m01 * inv;
    Jinv[g][2][0] = m02 * inv;
    Jinv[g][0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * inv;
    Jinv[g][1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * inv;
    Jinv[g][2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * inv;
    Jinv[g][0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * inv;
    Jinv[g][1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * inv;
    Jinv[g][2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * inv;
    detJ[g] = dt;
  }
  __syncthreads();
  if (tid < 64) {
    const int g = tid >> 3, a = tid & 7;
    const double xi[3] = {(g & 1) ? gp : -gp, (g & 2) ? gp : -gp, (g & 4) ? gp : -gp};
    const double sa[3] = {(a & 1) ? 1.0 : -1.0, (a & 2) ? 1.0 : -1.0, (a & 4) ? 1.0 : -1.0};
    const double f0 = 1.0 + sa[0] * xi[0], f1 = 1.0 + sa[1] * xi[1], f2 = 1.0 + sa[2] * xi[2];
    const double dr[3] = {0.125 * sa[0] * f1 * f2, 0.125 * f0 * sa[1] * f2, 0.125 * f0 * f1 * sa[2]};
    for (int d = 0; d < 3; ++d) dN[g][a][d] = dr[0] * Jinv[g][0][d] + dr[1] * Jinv[g][1][d] + dr[2] * Jinv[g][2][d];
  }
  __syncthreads();
  // B column of DoF (a, c): row c holds dN/dx_c, two shear rows the other derivatives
  const int ROW[3][3] = {{0, 4, 5}, {1, 3, 5}, {2, 3, 4}};
  const int DER[3][3] = {{0, 2, 1}, {1, 2, 0}, {2, 1, 0}};
  const int r = tid / 24, c = tid % 24;
  const int ar = r / 3, cr = r % 3, ac = c / 3, cc = c % 3;
  double acc = 0.0;
  for (int g = 0; g < 8; ++g) {
    const double* dr = dN[g][ar];
    const double* dc = dN[g][ac];
    double t = 0.0;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      double u = 0.0;
#pragma unroll
      for (int n = 0; n < 3; ++n) u += C[ROW[cr][m]][ROW[cc][n]] * dc[DER[cc][n]];
      t += dr[DER[cr][m]] * u;
    }
    acc += t * detJ[g];
  }
  Ke[(size_t)type * 576 + tid] = acc;
}

// Node stencil of a_{Omega*}: thread per (node, neighbour slot); slot
// (di, dj, dk) = ((s/9)-1, ((s/3)%3)-1, (s%3)-1).  Only elements inside the
// Omega* box contribute (Eq. restricted_bilinear_form).
__global__ void __launch_bounds__(216)
k_stencil(const SubDev* __restrict__ subs, const double* __restrict__ Ke, int layered, const int* __restrict__ etype,
          int NY, int NZ, int nel) {
  const SubDev s = subs[blockIdx.y];
  const int tid = threadIdx.x;
  const int node = blockIdx.x * 8 + tid / 27, slot = tid % 27;
  if (node >= s.nnode) return;
  const int k = node / s.npl, q = node % s.npl;
  const int gi = s.I0 + q / s.nyn, gj = s.J0 + q % s.nyn;
  const int di = slot / 9 - 1, dj = (slot / 3) % 3 - 1, dk = slot % 3 - 1;
  double acc[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) acc[e] = 0.0;
  for (int ez = 0; ez < 2; ++ez)
    for (int ey = 0; ey < 2; ++ey)
      for (int ex = 0; ex < 2; ++ex) {
        const int ie = gi - 1 + ex, je = gj - 1 + ey, ke = k - 1 + ez;
        if (ie < s.I0 || ie >= s.I1 || je < s.J0 || je >= s.J1 || ke < 0 || ke >= NZ) continue;
        const int ax = gi - ie, ay = gj - je, az = k - ke;              // node position in element
        const int bx = ax + di, by = ay + dj, bz = az + dk;            // neighbour position
        if (bx < 0 || bx > 1 || by < 0 || by > 1 || bz < 0 || bz > 1) continue;
        const int a = ax + 2 * ay + 4 * az, b = bx + 2 * by + 4 * bz;
        const int el = s.inst * nel + (ie * NY + je) * NZ + ke;
        const int type = etype ? etype[el] : (layered ? s.inst * NZ + ke : el);
        const double* K = Ke + (size_t)type * 576;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) acc[c * 3 + cc] += K[(3 * a + c) * 24 + 3 * b + cc];
      }
  double* out = s.stencil + ((size_t)node * 27 + slot) * 9;
#pragma unroll
  for (int e = 0; e < 9; ++e) out[e] = acc[e];
}

__device__ __forceinline__ bool is_pinned(const SubDev& s, int row) {
#pragma unroll
  for (int i = 0; i < 6; ++i)
    if (s.pin[i] == row) return true;
  return false;
}

template <typename T> struct Blocks;
template <> struct Blocks<double> {
  __device__ static double* D(const SubDev& s, int mat) { return mat == 0 ? s.DK : s.DA; }
  __device__ static double* E(const SubDev& s, int mat) { return mat == 0 ? s.EK : s.EA; }
};
template <> struct Blocks<float> {
  __device__ static float* D(const SubDev& s, int mat) { return mat == 0 ? s.DKf : s.DAf; }
  __device__ static float* E(const SubDev& s, int mat) { return mat == 0 ? s.EKf : s.EAf; }
};

// Scatter the stencil into the layer blocks of K (mat 0) and A11 (mat 1).
// Thread per (node, slot); slots with dk = 0 go to D_k, dk = -1 to E_{k-1}.
template <typename T>
__global__ void __launch_bounds__(216)
k_layer_blocks(const SubDev* __restrict__ subs, const int* __restrict__ active) {
  if (!active[blockIdx.y]) return;
  const SubDev s = subs[blockIdx.y];
  const int tid = threadIdx.x;
  const int node = blockIdx.x * 8 + tid / 27, slot = tid % 27;
  if (node >= s.nnode) return;
  const int dk = slot % 3 - 1;
  if (dk == 1) return;
  const int k = node / s.npl, q = node % s.npl;
  if (dk == -1 && k == 0) return;
  const int di = slot / 9 - 1, dj = (slot / 3) % 3 - 1;
  const int qi = q / s.nyn + di, qj = q % s.nyn + dj;
  if (qi < 0 || qi >= s.nxn || qj < 0 || qj >= s.nyn) return;
  const int q2 = qi * s.nyn + qj;
  const double* st = s.stencil + ((size_t)node * 27 + slot) * 9;
  for (int mat = 0; mat < 2; ++mat) {
    const int* inv = mat == 0 ? s.invK : s.invA;
    const int b = mat == 0 ? s.bK : s.bA;
    T* blk = (dk == 0) ? (Blocks<T>::D(s, mat) + (size_t)k * b * b) : (Blocks<T>::E(s, mat) + (size_t)(k - 1) * b * b);
    for (int c = 0; c < 3; ++c) {
      const int rr = inv[3 * q + c];
      if (rr < 0) continue;
      if (mat == 0 && s.floating && is_pinned(s, (k * s.npl + q) * 3 + c)) continue;
      for (int cc = 0; cc < 3; ++cc) {
        const int col = inv[3 * q2 + cc];
        if (col < 0) continue;
        if (mat == 0 && s.floating && is_pinned(s, ((k + dk) * s.npl + q2) * 3 + cc)) continue;
        blk[(size_t)rr * b + col] = (T)st[c * 3 + cc];
      }
    }
  }
}

// Identity on padding rows and pinned DoFs.
template <typename T>
__global__ void k_block_identity(const SubDev* __restrict__ subs, const int* __restrict__ active) {
  if (!active[blockIdx.y]) return;
  const SubDev s = subs[blockIdx.y];
  const int k = blockIdx.x;
  if (k >= s.nzn) return;
  T* DK = Blocks<T>::D(s, 0);
  T* DA = Blocks<T>::D(s, 1);
  for (int c = s.nK + threadIdx.x; c < s.bK; c += blockDim.x) DK[(size_t)k * s.bK * s.bK + (size_t)c * s.bK + c] = (T)1;
  for (int c = s.nA + threadIdx.x; c < s.bA; c += blockDim.x) DA[(size_t)k * s.bA * s.bA + (size_t)c * s.bA + c] = (T)1;
  if (s.floating && threadIdx.x < 6 && s.pin[threadIdx.x] >= 0) {
    const int row = s.pin[threadIdx.x];
    const int layer = row / (3 * s.npl), r = s.invK[row % (3 * s.npl)];
    if (layer == k && r >= 0) DK[(size_t)k * s.bK * s.bK + (size_t)r * s.bK + r] = (T)1;
  }
}

}  // namespace

void launch_element_stiffness(msgfem* h) {
  k_element_stiffness<<<h->ntypes, 576, 0, h->stream>>>(h->d_angles_type, h->d_E9, h->layered, h->NX, h->NY,
                                                        h->NZ, h->hx, h->hy, h->hz, h->d_xyz, h->d_frame,
                                                        h->typed ? h->d_trep : nullptr, h->d_Ke); ++g_launch_count;
}

void launch_stencil(msgfem* h) {
  int maxn = 0;
  for (const auto& s : h->sub) maxn = std::max(maxn, s.nnode);
  dim3 grid((maxn + 7) / 8, h->N);
  k_stencil<<<grid, 216, 0, h->stream>>>(h->d_sub, h->d_Ke, h->layered, h->typed ? h->d_etype : nullptr, h->NY, h->NZ,
                                         h->NX * h->NY * h->NZ);
  ++g_launch_count;
}

// Layer blocks of the subdomains of the current wave (the active ones).
template <typename T>
static void layer_blocks_t(msgfem* h) {
  for (int j = 0; j < h->N; ++j) {
    if (j < (int)h->act_host.size() && !h->act_host[j]) continue;
    const SubDev& s = h->sub[j];
    T* DK = std::is_same<T, float>::value ? (T*)s.DKf : (T*)s.DK;
    T* DA = std::is_same<T, float>::value ? (T*)s.DAf : (T*)s.DA;
    cudaMemsetAsync(DK, 0, sizeof(T) * (size_t)s.bK * s.bK * (2 * s.nzn - 1), h->stream);
    cudaMemsetAsync(DA, 0, sizeof(T) * (size_t)s.bA * s.bA * (2 * s.nzn - 1), h->stream);
  }
  int maxn = 0, maxz = 0;
  for (const auto& s : h->sub) { maxn = std::max(maxn, s.nnode); maxz = std::max(maxz, s.nzn); }
  dim3 grid((maxn + 7) / 8, h->N);
  k_layer_blocks<T><<<grid, 216, 0, h->stream>>>(h->d_sub, h->d_flags); ++g_launch_count;
  dim3 g2(maxz, h->N);
  k_block_identity<T><<<g2, 128, 0, h->stream>>>(h->d_sub, h->d_flags); ++g_launch_count;
}

void launch_layer_blocks(msgfem* h) { layer_blocks_t<double>(h); }
void launch_layer_blocks_f32(msgfem* h) { layer_blocks_t<float>(h); }
