// Coarse level: Galerkin blocks A^H_{st} = V_s^T A V_t (Eq.
// GFEM_coarse_approximation), load b^H_s = V_s^T b, prolongation
// u^G = sum_s R_s^T V_s c_s and the energy norm a(v, v) = sum_e v_e^T K_e v_e
// (Theorem 1).  V_s = D_mu [phi, psi_hat] is zero outside Omega_s, and
// A V_s equals the Omega*_s stencil product of V_s on Omega*_s.
#include "internal.h"

namespace {

constexpr int CROWS = 512;

// Partial G_st over a chunk of rows of the pair's node box (all layers, 3 comps).
__global__ void __launch_bounds__(256)
k_pair_partial(const SubDev* __restrict__ subs, const CoarsePair* __restrict__ pairs, double* __restrict__ part,
               int nchunk) {
  const CoarsePair pr = pairs[blockIdx.y];
  const SubDev& S = subs[pr.s];
  const SubDev& T = subs[pr.t];
  const int nx = pr.x1 - pr.x0 + 1, ny = pr.y1 - pr.y0 + 1;
  const int nrows = nx * ny * S.nzn * 3;
  const int tid = threadIdx.x, a = tid >> 3, b = (tid & 7) * 4;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  __shared__ double Xs[32][PST];
  __shared__ double Ys[32][PST];
  const int r0 = blockIdx.x * CROWS;
  const int r1 = min(r0 + CROWS, nrows);
  for (int rb = r0; rb < r1; rb += 32) {
    for (int e = tid; e < 32 * PST; e += 256) {
      const int rr = rb + e / PST, col = e % PST;
      double xv = 0.0, yv = 0.0;
      if (rr < r1) {
        const int c = rr % 3, node = rr / 3;
        const int k = node / (nx * ny), ij = node % (nx * ny);
        const int gi = pr.x0 + ij / ny, gj = pr.y0 + ij % ny;
        const int rs = ((k * S.npl + (gi - S.I0) * S.nyn + (gj - S.J0)) * 3 + c);
        const int rt = ((k * T.npl + (gi - T.I0) * T.nyn + (gj - T.J0)) * 3 + c);
        xv = S.CB[(size_t)rs * PST + col];
        yv = T.CW[(size_t)rt * PST + col];
      }
      Xs[e / PST][col] = xv;
      Ys[e / PST][col] = yv;
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < 32; ++r) {
      const double xa = Xs[r][a];
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[j] = fma(xa, Ys[r][b + j], acc[j]);
    }
    __syncthreads();
  }
  double* out = part + ((size_t)blockIdx.y * nchunk + blockIdx.x) * PST * PST;
#pragma unroll
  for (int j = 0; j < 4; ++j) out[a * PST + b + j] = acc[j];
}

__global__ void k_pair_reduce(const SubDev* __restrict__ subs, const CoarsePair* __restrict__ pairs,
                              const double* __restrict__ part, int nchunk, const int* __restrict__ coff,
                              const int* __restrict__ msz, double* __restrict__ AH, int ld) {
  const CoarsePair pr = pairs[blockIdx.x];
  const SubDev& S = subs[pr.s];
  const int nrows = (pr.x1 - pr.x0 + 1) * (pr.y1 - pr.y0 + 1) * S.nzn * 3;
  const int nc = (nrows + CROWS - 1) / CROWS;
  const int ms = msz[pr.s], mt = msz[pr.t];
  for (int e = threadIdx.x; e < PST * PST; e += blockDim.x) {
    const int a = e / PST, b = e % PST;
    if (a >= ms || b >= mt) continue;
    double acc = 0.0;
    for (int c = 0; c < nc; ++c) acc += part[((size_t)blockIdx.x * nchunk + c) * PST * PST + e];
    AH[(size_t)(coff[pr.s] + a) * ld + coff[pr.t] + b] = acc;
  }
}

// AH <- (AH + AH^T) / 2 on the leading Nc block; identity on the padding.
__global__ void k_symmetrize(double* AH, int Nc, int ld) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)ld * ld; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / ld), c = (int)(e % ld);
    if (r < Nc && c < Nc) {
      if (r < c) {
        const double v = 0.5 * (AH[(size_t)r * ld + c] + AH[(size_t)c * ld + r]);
        AH[(size_t)r * ld + c] = v;
        AH[(size_t)c * ld + r] = v;
      }
    } else {
      AH[e] = (r == c) ? 1.0 : 0.0;
    }
  }
}

// b^H rows of subdomain s: sum_r CB[r][a] b[r]; one block per subdomain.
__global__ void k_coarse_rhs(const SubDev* __restrict__ subs, const int* __restrict__ coff,
                             const int* __restrict__ msz, double* __restrict__ bH) {
  const SubDev& s = subs[blockIdx.x];
  __shared__ double red[8][PST];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double acc = 0.0;
  for (int r = w; r < s.nfull; r += 8) acc = fma(s.CB[(size_t)r * PST + lane], s.bload[r], acc);
  red[w][lane] = acc;
  __syncthreads();
  if (w == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i][lane];
    if (lane < msz[blockIdx.x]) bH[(size_t)(coff[blockIdx.x] + lane) * PST] = t;
  }
}

// u^G on global DoFs: sum over subdomains whose Omega box holds the node.
__global__ void k_prolong(const SubDev* __restrict__ subs, int N, const int* __restrict__ coff,
                          const int* __restrict__ msz, const double* __restrict__ cH, double* __restrict__ u,
                          int NY, int NZ, int ndof) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ndof; g += gridDim.x * blockDim.x) {
    const int node = g / 3, c = g % 3;
    const int k = node % (NZ + 1), ij = node / (NZ + 1);
    const int gi = ij / (NY + 1), gj = ij % (NY + 1);
    double acc = 0.0;
    for (int sidx = 0; sidx < N; ++sidx) {
      const SubDev& s = subs[sidx];
      if (gi < s.oI0 || gi > s.oI1 || gj < s.oJ0 || gj > s.oJ1) continue;
      const int row = (k * s.npl + (gi - s.I0) * s.nyn + (gj - s.J0)) * 3 + c;
      const double* v = s.CB + (size_t)row * PST;
      const double* cc = cH + (size_t)coff[sidx] * PST;
      for (int a = 0; a < msz[sidx]; ++a) acc = fma(v[a], cc[(size_t)a * PST], acc);
    }
    u[g] = acc;
  }
}

// Energy sums over elements: out[2 b] = sum d^T K_e d with d = ref - u,
// out[2 b + 1] = sum ref^T K_e ref.
__global__ void __launch_bounds__(256)
k_energy(const double* __restrict__ Ke, int layered, const int* __restrict__ etype, const double* __restrict__ ref,
         const double* __restrict__ u, int NX, int NY, int NZ, double* __restrict__ out) {
  __shared__ double red[2][256];
  double e0 = 0.0, e1 = 0.0;
  const int nel = NX * NY * NZ;
  for (int el = blockIdx.x * blockDim.x + threadIdx.x; el < nel; el += gridDim.x * blockDim.x) {
    const int ke = el % NZ, ij = el / NZ, je = ij % NY, ie = ij / NY;
    double d[24], r[24];
    for (int a = 0; a < 8; ++a) {
      const int ax = a & 1, ay = (a >> 1) & 1, az = a >> 2;
      const int node = ((ie + ax) * (NY + 1) + je + ay) * (NZ + 1) + ke + az;
      for (int c = 0; c < 3; ++c) {
        r[3 * a + c] = ref[3 * node + c];
        d[3 * a + c] = r[3 * a + c] - (u ? u[3 * node + c] : 0.0);
      }
    }
    const double* K = Ke + (size_t)(etype ? etype[el] : (layered ? ke : el)) * 576;
    for (int i = 0; i < 24; ++i) {
      double kd = 0.0, kr = 0.0;
      for (int j = 0; j < 24; ++j) {
        kd = fma(K[i * 24 + j], d[j], kd);
        kr = fma(K[i * 24 + j], r[j], kr);
      }
      e0 = fma(d[i], kd, e0);
      e1 = fma(r[i], kr, e1);
    }
  }
  red[0][threadIdx.x] = e0;
  red[1][threadIdx.x] = e1;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      red[0][threadIdx.x] += red[0][threadIdx.x + st];
      red[1][threadIdx.x] += red[1][threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = red[0][0];
    out[2 * blockIdx.x + 1] = red[1][0];
  }
}

// Eigenvectors of subdomain j to the output layout ((i-I0) nyn + (j-J0)) nzn + k.
__global__ void k_basis_out(const SubDev* __restrict__ subs, int j, double* __restrict__ out, int ncols) {
  const SubDev& s = subs[j];
  const size_t total = (size_t)s.nfull * ncols;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int col = (int)(e / s.nfull), orow = (int)(e % s.nfull);
    const int onode = orow / 3, c = orow % 3;
    const int k = onode % s.nzn, q = onode / s.nzn;
    const int row = (k * s.npl + q) * 3 + c;
    out[e] = s.EV[(size_t)row * PST + col];
  }
}

// One vector of subdomain j between the internal full layout (row
// (k npl + q) 3 + c, stride sstride / dstride between rows) and the layout of
// msgfem_get_basis (row (q nzn + k) 3 + c, q = (i - I0) nyn + (j - J0)).
__global__ void k_vec_layout(const SubDev* __restrict__ subs, int j, const double* __restrict__ src, int sstride,
                             double* __restrict__ dst, int dstride, int to_output) {
  const SubDev& s = subs[j];
  for (int orow = blockIdx.x * blockDim.x + threadIdx.x; orow < s.nfull; orow += gridDim.x * blockDim.x) {
    const int onode = orow / 3, c = orow % 3;
    const int k = onode % s.nzn, q = onode / s.nzn;
    const int row = (k * s.npl + q) * 3 + c;
    if (to_output) dst[(size_t)orow * dstride] = src[(size_t)row * sstride];
    else dst[(size_t)row * dstride] = src[(size_t)orow * sstride];
  }
}

}  // namespace

void launch_vec_layout(msgfem* h, int j, const double* src, int sstride, double* dst, int dstride, int to_output) {
  k_vec_layout<<<64, 256, 0, h->stream>>>(h->d_sub, j, src, sstride, dst, dstride, to_output); ++g_launch_count;
}

void launch_coarse_blocks(msgfem* h) {
  int maxrows = 0;
  for (const auto& p : h->pairs)
    maxrows = std::max(maxrows, (p.x1 - p.x0 + 1) * (p.y1 - p.y0 + 1) * (h->NZ + 1) * 3);
  const int nchunk = (maxrows + CROWS - 1) / CROWS;
  dim3 grid(nchunk, (unsigned)h->pairs.size());
  k_pair_partial<<<grid, 256, 0, h->stream>>>(h->d_sub, h->d_pairs, h->d_pair_part, nchunk); ++g_launch_count;
  k_pair_reduce<<<(unsigned)h->pairs.size(), 256, 0, h->stream>>>(h->d_sub, h->d_pairs, h->d_pair_part, nchunk,
                                                                  h->d_coff, h->d_m, h->d_AH, h->NcPad); ++g_launch_count;
  k_symmetrize<<<256, 256, 0, h->stream>>>(h->d_AH, h->Nc, h->NcPad); ++g_launch_count;
}

void launch_coarse_rhs(msgfem* h) {
  cudaMemsetAsync(h->d_bH, 0, sizeof(double) * (size_t)h->NcPad * PST, h->stream);
  k_coarse_rhs<<<h->N, 256, 0, h->stream>>>(h->d_sub, h->d_coff, h->d_m, h->d_bH); ++g_launch_count;
}

void launch_prolong(msgfem* h) {
  const int ndof = 3 * (h->NX + 1) * (h->NY + 1) * (h->NZ + 1);
  k_prolong<<<(ndof + 255) / 256, 256, 0, h->stream>>>(h->d_sub, h->N, h->d_coff, h->d_m, h->d_cH, h->d_u, h->NY,
                                                       h->NZ, ndof); ++g_launch_count;
}

int energy_blocks(msgfem* h) {
  const int nel = h->NX * h->NY * h->NZ;
  return std::min(1024, (nel + 255) / 256);
}

void launch_energy(msgfem* h, const double* d_ref, const double* d_u, double* d_out) {
  k_energy<<<energy_blocks(h), 256, 0, h->stream>>>(h->d_Ke, h->layered, h->typed ? h->d_etype : nullptr, d_ref, d_u,
                                                    h->NX, h->NY, h->NZ, d_out); ++g_launch_count;
}

void launch_basis_out(msgfem* h, int j, double* d_out, int ncols) {
  k_basis_out<<<256, 256, 0, h->stream>>>(h->d_sub, j, d_out, ncols); ++g_launch_count;
}
