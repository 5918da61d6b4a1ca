// Warm-start plumbing on an MS-GFEM handle: network features from the
// ply-angle perturbation field, training targets from the converged local
// eigenvectors (B2 rows, Procrustes-aligned) and the start block of the block
// Krylov eigensolver.
#include "internal.h"
#include "msgfem_warm.h"

namespace {

// features of subdomain j: dtheta on the elements of the Omega* box, (i, j, k) order, k fastest
__global__ void k_warm_features(const SubDev* __restrict__ subs, const double* __restrict__ dtheta, int NY, int NZ,
                                long long nel, float scale, float* __restrict__ feat, int ld) {
  const SubDev& s = subs[blockIdx.y];
  dtheta += (size_t)s.inst * nel;   // the instance's field
  const int ex = s.I1 - s.I0, ey = s.J1 - s.J0;
  const int ne = ex * ey * NZ;
  float* f = feat + (size_t)blockIdx.y * ld;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ld; e += gridDim.x * blockDim.x) {
    float v = 0.f;
    if (e < ne) {
      const int k = e % NZ, b = (e / NZ) % ey, a = e / (NZ * ey);
      v = scale * (float)dtheta[((size_t)(s.I0 + a) * NY + (s.J0 + b)) * NZ + k];
    }
    f[e] = v;
  }
}

// eigen-decomposition of a symmetric n x n matrix (n <= 8) by cyclic Jacobi
// rotations (Golub and Van Loan, Sec. 8.5); A is overwritten by diag(lambda),
// V receives the eigenvectors as columns.  One thread.
__device__ void jacobi_small(double (*A)[8], double (*V)[8], int n) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i][j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += A[i][j] * A[i][j];
        if (i != j) off += A[i][j] * A[i][j];
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (A[p][q] == 0.0) continue;
        const double th = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < n; ++k) {   // A <- A J
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - sn * akq;
          A[k][q] = sn * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {   // A <- J^T A
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - sn * aqk;
          A[q][k] = sn * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {   // V <- V J
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - sn * vkq;
          V[k][q] = sn * vkp + c * vkq;
        }
      }
  }
}

// out [n2][ld] = X Q with X = EV columns nr .. nr + nw - 1 on the B2 rows and
// Q the orthogonal polar factor of M = X^T ref (identity without ref).
// One CTA of 256 threads.
__global__ void __launch_bounds__(256)
k_warm_targets(const double* __restrict__ EV, const int* __restrict__ b2rows, int n2, int nr, int nw,
               const float* __restrict__ ref, float* __restrict__ out, int ld) {
  __shared__ double M[8][8];
  __shared__ double G[8][8];
  __shared__ double V[8][8];
  __shared__ double Q[8][8];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (ref != nullptr) {
    for (int idx = w; idx < 64; idx += 8) {
      const int a = idx / 8, b = idx % 8;
      double sacc = 0.0;
      if (a < nw && b < nw)
        for (int r = lane; r < n2; r += 32) sacc += EV[(size_t)b2rows[r] * PST + nr + a] * (double)ref[(size_t)r * ld + b];
      for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
      if (lane == 0) M[a][b] = sacc;
    }
  }
  __syncthreads();
  if (tid == 0) {
    for (int i = 0; i < 8; ++i)
      for (int j = 0; j < 8; ++j) Q[i][j] = i == j ? 1.0 : 0.0;
    if (ref != nullptr) {
      // Q = M (M^T M)^{-1/2} = M V diag(lambda^{-1/2}) V^T
      for (int i = 0; i < nw; ++i)
        for (int j = 0; j < nw; ++j) {
          double g = 0.0;
          for (int k = 0; k < nw; ++k) g += M[k][i] * M[k][j];
          G[i][j] = g;
        }
      jacobi_small(G, V, nw);
      double lmax = 0.0;
      for (int i = 0; i < nw; ++i) lmax = fmax(lmax, G[i][i]);
      double MV[8][8];
      for (int i = 0; i < nw; ++i)
        for (int k = 0; k < nw; ++k) {
          double acc = 0.0;
          for (int l = 0; l < nw; ++l) acc += M[i][l] * V[l][k];
          MV[i][k] = G[k][k] > 1e-28 * lmax && G[k][k] > 0.0 ? acc / sqrt(G[k][k]) : 0.0;
        }
      for (int i = 0; i < nw; ++i)
        for (int j = 0; j < nw; ++j) {
          double acc = 0.0;
          for (int k = 0; k < nw; ++k) acc += MV[i][k] * V[j][k];
          Q[i][j] = acc;
        }
    }
  }
  __syncthreads();
  for (size_t e = tid; e < (size_t)n2 * ld; e += 256) {
    const int r = (int)(e / ld), c = (int)(e % ld);
    double v = 0.0;
    if (c < nw) {
      const double* x = EV + (size_t)b2rows[r] * PST + nr;
      for (int a = 0; a < nw; ++a) v += x[a] * Q[a][c];
    }
    out[e] = (float)v;
  }
}

struct WarmDev { const float* X0; int ld, ncols, n2; const int* b2rows; };

// start block rows on B2 from the registered X0 (first ncols columns)
__global__ void k_load_start(const SubDev* __restrict__ subs, const int* __restrict__ active,
                             const WarmDev* __restrict__ warm, int which) {
  if (active != nullptr && !active[blockIdx.y]) return;
  const WarmDev wd = warm[blockIdx.y];
  if (wd.X0 == nullptr) return;
  double* X = mv_ptr(subs[blockIdx.y], which);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < wd.n2 * wd.ncols; e += gridDim.x * blockDim.x) {
    const int r = e / wd.ncols, c = e % wd.ncols;
    X[(size_t)wd.b2rows[r] * KB + c] = (double)wd.X0[(size_t)r * wd.ld + c];
  }
}

// bad[j] = 1 when the registered start block of subdomain j holds a non-finite
// value (its first ncols columns)
__global__ void k_check_start(const WarmDev* __restrict__ warm, int* __restrict__ bad) {
  const WarmDev wd = warm[blockIdx.x];
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  if (wd.X0 != nullptr)
    for (int e = threadIdx.x; e < wd.n2 * wd.ncols; e += blockDim.x)
      if (!isfinite(wd.X0[(size_t)(e / wd.ncols) * wd.ld + e % wd.ncols])) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) bad[blockIdx.x] = any;
}

}  // namespace

// Registered start blocks with a non-finite entry (a network that produced
// NaN): bad[j] = 1 for those subdomains.  Uses d_ncols as scratch.
msgfem_status warm_check(msgfem* h, std::vector<int>& bad) {
  bad.assign(h->N, 0);
  k_check_start<<<h->N, 256, 0, h->stream>>>(static_cast<const WarmDev*>(h->d_warm), h->d_ncols);
  ++g_launch_count;
  CK_LAUNCH();
  CK(cudaMemcpyAsync(bad.data(), h->d_ncols, h->N * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return MSGFEM_OK;
}

// B2 row lists (ascending full-layout rows of the interface DoFs), built once
msgfem_status warm_rows(msgfem* h) {
  if ((int)h->d_b2rows.size() == h->N) return MSGFEM_OK;
  h->d_b2rows.assign(h->N, nullptr);
  for (int j = 0; j < h->N; ++j) {
    const SubDev& s = h->sub[j];
    std::vector<int> rows;
    for (int n = 0; n < s.nnode; ++n)
      if (h->hsub[j].cls[n % s.npl] == 2)
        for (int c = 0; c < 3; ++c) rows.push_back(3 * n + c);
    if ((int)rows.size() != h->n2[j]) {
      h->err = "interface row count does not match the DoF classes";
      return MSGFEM_ESTATE;
    }
    void* buf = nullptr;
    TRY(dev_alloc_bytes(h, &buf, std::max<size_t>(1, rows.size()) * sizeof(int)));
    int* d = static_cast<int*>(buf);
    if (!rows.empty()) CK(cudaMemcpy(d, rows.data(), rows.size() * sizeof(int), cudaMemcpyHostToDevice));
    h->d_b2rows[j] = d;
  }
  return MSGFEM_OK;
}

// upload the start-block descriptors; true when any subdomain has one
bool warm_upload(msgfem* h) {
  bool any = false;
  for (const auto& w : h->warm) any = any || w.X0 != nullptr;
  if (!any) return false;
  std::vector<WarmDev> wd(h->N);
  for (int j = 0; j < h->N; ++j)
    wd[j] = {h->warm[j].X0, h->warm[j].ld, h->warm[j].ncols, h->n2[j], h->d_b2rows[j]};
  if (h->d_warm == nullptr && dev_alloc_bytes(h, &h->d_warm, h->N * sizeof(WarmDev)) != MSGFEM_OK) return false;
  cudaMemcpyAsync(h->d_warm, wd.data(), h->N * sizeof(WarmDev), cudaMemcpyHostToDevice, h->stream);
  cudaStreamSynchronize(h->stream);
  return true;
}

void launch_load_start(msgfem* h, int which) {
  dim3 grid(16, h->N);
  k_load_start<<<grid, 256, 0, h->stream>>>(h->d_sub, h->d_flags, static_cast<const WarmDev*>(h->d_warm), which);
  ++g_launch_count;
}

extern "C" {

msgfem_status msgfem_warm_features(msgfem_h h, const double* dtheta, float scale, float* feat, int ld,
                                   int* nfeat_out) {
  if (!h) return MSGFEM_EINVAL;
  int nmax = 0;
  for (const auto& s : h->sub) nmax = std::max(nmax, (s.I1 - s.I0) * (s.J1 - s.J0) * h->NZ);
  if (nfeat_out) *nfeat_out = nmax;
  if (feat == nullptr) return MSGFEM_OK;   // size query
  if (dtheta == nullptr) return MSGFEM_EINVAL;
  if (ld < nmax) {
    h->err = "feature row length below the largest Omega* element count";
    return MSGFEM_EINVAL;
  }
  dim3 grid((ld + 255) / 256, h->N);
  k_warm_features<<<grid, 256, 0, h->stream>>>(h->d_sub, dtheta, h->NY, h->NZ, (long long)h->NX * h->NY * h->NZ, scale,
                                               feat, ld);
  ++g_launch_count;
  CK(cudaGetLastError());
  return MSGFEM_OK;
}

msgfem_status msgfem_warm_sizes(msgfem_h h, int j, int n_loc, int* n2_out, int* nw_out) {
  if (!h || j < 0 || j >= h->N) return MSGFEM_EINVAL;
  const int nl = n_loc > 0 ? n_loc : (j < (int)h->nloc_j.size() ? h->nloc_j[j] : h->n_loc);
  if (n2_out) *n2_out = h->n2[j];
  if (nw_out) *nw_out = nl - (h->sub[j].floating ? std::min(6, nl) : 0);
  return MSGFEM_OK;
}

msgfem_status msgfem_warm_targets(msgfem_h h, int j, const float* ref, float* out, int ld) {
  if (!h || !out || j < 0 || j >= h->N || ld < KB) return MSGFEM_EINVAL;
  if (h->stage < 2) return MSGFEM_ESTATE;
  TRY(warm_rows(h));
  const SubDev& s = h->sub[j];
  const int nl = h->nloc_j[j];
  const int nr = s.floating ? std::min(6, nl) : 0;
  const int nw = std::min(KB, nl - nr);
  k_warm_targets<<<1, 256, 0, h->stream>>>(s.EV, h->d_b2rows[j], h->n2[j], nr, nw, ref, out, ld);
  ++g_launch_count;
  CK(cudaGetLastError());
  return MSGFEM_OK;
}

msgfem_status msgfem_set_start_block(msgfem_h h, int j, const float* X0, int ld, int ncols) {
  if (!h || j < 0 || j >= h->N) return MSGFEM_EINVAL;
  if (X0 != nullptr && (ncols < 1 || ncols > KB || ld < ncols)) return MSGFEM_EINVAL;
  if (X0 != nullptr && h->geneo) {
    h->err = "start blocks are B2 blocks of the A-harmonic eigenproblem; a GenEO handle takes none";
    return MSGFEM_EINVAL;
  }
  TRY(warm_rows(h));
  if ((int)h->warm.size() != h->N) h->warm.assign(h->N, WarmStart{});
  h->warm[j] = X0 ? WarmStart{X0, ld, ncols} : WarmStart{};
  return MSGFEM_OK;
}

}  // extern "C"
