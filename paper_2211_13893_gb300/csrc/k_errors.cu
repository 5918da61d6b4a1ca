// Relative L2 errors of the displacement and strain fields of the coarse
// solution (Sec. 5.4, e_d and e_eps): for v = u_ref - u^G and v = u_ref, the
// integrals of |v|^2 and eps(v) : eps(v) over every element by 2x2x2
// Gauss-Legendre quadrature through the trilinear map of its corners (the box
// or the given node coordinates).  One pass over the elements; each block
// writes its four partial sums and the host adds them in a fixed order.
//
// Element corner a (a = ax + 2 ay + 4 az) of element (ie, je, ke) is node
// (ie + ax, je + ay, ke + az); its shape function is
// N_a = (1 + s_x xi)(1 + s_y eta)(1 + s_z zeta) / 8 with s = -1 for a 0 bit
// and +1 for a 1 bit.
#include <cmath>

#include "internal.h"

namespace {

constexpr int ERR_THREADS = 256;
constexpr int ERR_MAX_BLOCKS = 1024;

struct FieldSums {
  double disp, strain;
};

// |v|^2 and eps(v):eps(v) at one quadrature point for nodal values v[8][3]
// with shape values N and physical gradients dNx[a][j] = dN_a / dx_j.
__device__ __forceinline__ FieldSums point_sums(const double (&v)[8][3], const double (&N)[8],
                                                const double (&dNx)[8][3]) {
  double u[3] = {0.0, 0.0, 0.0}, G[3][3] = {};
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      u[c] = fma(N[a], v[a][c], u[c]);
#pragma unroll
      for (int j = 0; j < 3; ++j) G[c][j] = fma(v[a][c], dNx[a][j], G[c][j]);
    }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double e = 0.5 * (G[i][j] + G[j][i]);
      s = fma(e, e, s);
    }
  return {u[0] * u[0] + u[1] * u[1] + u[2] * u[2], s};
}

__global__ void __launch_bounds__(ERR_THREADS)
k_l2_errors(const double* __restrict__ ref, const double* __restrict__ u, int NX, int NY, int NZ, double hx,
            double hy, double hz, const double* __restrict__ xyz, double* __restrict__ part) {
  __shared__ double red[4][ERR_THREADS];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const long long nel = (long long)NX * NY * NZ;
  const double g = 1.0 / sqrt(3.0);
  for (long long el = (long long)blockIdx.x * ERR_THREADS + threadIdx.x; el < nel;
       el += (long long)gridDim.x * ERR_THREADS) {
    const int ke = (int)(el % NZ);
    const long long ij = el / NZ;
    const int je = (int)(ij % NY), ie = (int)(ij / NY);
    double X[8][3], vd[8][3], vr[8][3];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int ax = a & 1, ay = (a >> 1) & 1, az = a >> 2;
      const size_t node = ((size_t)(ie + ax) * (NY + 1) + (je + ay)) * (NZ + 1) + (ke + az);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        X[a][d] = xyz != nullptr ? xyz[3 * node + d] : (d == 0 ? (ie + ax) * hx : d == 1 ? (je + ay) * hy : (ke + az) * hz);
        vr[a][d] = ref[3 * node + d];
        vd[a][d] = vr[a][d] - u[3 * node + d];
      }
    }
    for (int q = 0; q < 8; ++q) {
      const double xi[3] = {(q & 1) ? g : -g, ((q >> 1) & 1) ? g : -g, (q >> 2) ? g : -g};
      double N[8], dNr[8][3];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const double sx = (a & 1) ? 1.0 : -1.0, sy = ((a >> 1) & 1) ? 1.0 : -1.0, sz = (a >> 2) ? 1.0 : -1.0;
        const double f0 = 1.0 + sx * xi[0], f1 = 1.0 + sy * xi[1], f2 = 1.0 + sz * xi[2];
        N[a] = 0.125 * f0 * f1 * f2;
        dNr[a][0] = 0.125 * sx * f1 * f2;
        dNr[a][1] = 0.125 * f0 * sy * f2;
        dNr[a][2] = 0.125 * f0 * f1 * sz;
      }
      double J[3][3] = {};   // J[i][r] = dx_i / dxi_r
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int r = 0; r < 3; ++r) J[i][r] = fma(X[a][i], dNr[a][r], J[i][r]);
      const double m00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
      const double m01 = J[1][0] * J[2][2] - J[1][2] * J[2][0];
      const double m02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
      const double det = J[0][0] * m00 - J[0][1] * m01 + J[0][2] * m02;
      const double id = 1.0 / det;
      double Ji[3][3];       // Ji[r][j] = dxi_r / dx_j
      Ji[0][0] = m00 * id;
      Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
      Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
      Ji[1][0] = -m01 * id;
      Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
      Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
      Ji[2][0] = m02 * id;
      Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
      Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
      double dNx[8][3];
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          dNx[a][j] = dNr[a][0] * Ji[0][j] + dNr[a][1] * Ji[1][j] + dNr[a][2] * Ji[2][j];
      const FieldSums d = point_sums(vd, N, dNx);
      const FieldSums r = point_sums(vr, N, dNx);
      acc[0] = fma(det, d.disp, acc[0]);      // unit Gauss weights
      acc[1] = fma(det, d.strain, acc[1]);
      acc[2] = fma(det, r.disp, acc[2]);
      acc[3] = fma(det, r.strain, acc[3]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) red[i][threadIdx.x] = acc[i];
  __syncthreads();
  for (int st = ERR_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      for (int i = 0; i < 4; ++i) red[i][threadIdx.x] += red[i][threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < 4; ++i) part[4 * blockIdx.x + i] = red[i][0];
  }
}

int l2_error_blocks(const msgfem* h) {
  const long long nel = (long long)h->NX * h->NY * h->NZ;
  return (int)std::min<long long>(ERR_MAX_BLOCKS, std::max<long long>(1, (nel + ERR_THREADS - 1) / ERR_THREADS));
}

}  // namespace

extern "C" msgfem_status msgfem_solution_errors(msgfem_h h, const double* u_ref, double* errors_out) {
  if (!h || !u_ref || !errors_out) return MSGFEM_EINVAL;
  if (h->stage < 4) {
    h->err = "msgfem_solution_errors needs the coarse solution of msgfem_solve";
    return MSGFEM_ESTATE;
  }
  cudaStream_t st = h->stream;
  const size_t ndof = 3 * (size_t)(h->NX + 1) * (h->NY + 1) * (h->NZ + 1);
  (void)ndof;
  TRY(vec_in(h, u_ref, h->d_ref));
  const int nb = l2_error_blocks(h);
  k_l2_errors<<<nb, ERR_THREADS, 0, st>>>(h->d_ref, h->d_u, h->NX, h->NY, h->NZ, h->hx, h->hy, h->hz, h->d_xyz,
                                          h->d_l2);
  ++g_launch_count;
  CK_LAUNCH();
  std::vector<double> part(4 * (size_t)nb);
  CK(cudaMemcpyAsync(part.data(), h->d_l2, part.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = 0; b < nb; ++b)
    for (int i = 0; i < 4; ++i) s[i] += part[4 * (size_t)b + i];
  errors_out[0] = s[2] > 0.0 ? std::sqrt(std::max(s[0], 0.0) / s[2]) : 0.0;
  errors_out[1] = s[3] > 0.0 ? std::sqrt(std::max(s[1], 0.0) / s[3]) : 0.0;
  return MSGFEM_OK;
}
