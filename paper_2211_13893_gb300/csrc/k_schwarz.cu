// Two-level additive Schwarz preconditioned conjugate gradients for the fine
// problem A u = b on the free DoFs (msgfem_schwarz_solve): the solver that a
// coarse space of the local stage preconditions (Sec. 2.3, Eq.
// condition_bound) and the paper's reference solver for u_h (Sec. 5.3-5.4).
//
//   M^{-1} r = sum_j R_j^T A_j^{-1} R_j r + V A_0^{-1} V^T r
//
// R_j restricts to the DoFs of V_{h,0}(Omega_j) (nodes of Omega_j off its cut
// boundary and off the clamped face): on a handle whose oversampling equals
// its overlap these are the B1 DoFs, and A_j is that handle's A11, whose
// layer-block factors do the local solves.  V and A_0 = V^T A V are the coarse
// basis and coarse matrix of a handle after msgfem_coarse_assemble (MS-GFEM or
// GenEO), whose coarse Cholesky factor does the coarse solve.  The products
// with A are element by element from the element stiffness matrices, one
// thread per node gathering the (at most eight) elements around it, so the
// result does not depend on the launch order.
#include <cmath>
#include <string>

#include "internal.h"

namespace {

constexpr int DOT_BLOCKS = 304;   // 2 per SM: partial sums of the dot products

// y = A x on all DoFs (rows of the clamped face i = 0 zero; x is zero there)
__global__ void __launch_bounds__(128)
k_apply_A(const double* __restrict__ Ke, int layered, const int* __restrict__ etype, const double* __restrict__ x,
          double* __restrict__ y, int NX, int NY, int NZ) {
  const int nnode = (NX + 1) * (NY + 1) * (NZ + 1);
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < nnode; n += gridDim.x * blockDim.x) {
    const int k = n % (NZ + 1), ij = n / (NZ + 1), j = ij % (NY + 1), i = ij / (NY + 1);
    double y0 = 0.0, y1 = 0.0, y2 = 0.0;
    if (i > 0) {
      for (int ie = max(i - 1, 0); ie <= min(i, NX - 1); ++ie)
        for (int je = max(j - 1, 0); je <= min(j, NY - 1); ++je)
          for (int ke = max(k - 1, 0); ke <= min(k, NZ - 1); ++ke) {
            const int el = (ie * NY + je) * NZ + ke;
            const int a = (i - ie) | ((j - je) << 1) | ((k - ke) << 2);   // this node in the element
            const double* K = Ke + (size_t)(etype ? etype[el] : (layered ? ke : el)) * 576 + (size_t)(3 * a) * 24;
            for (int b = 0; b < 8; ++b) {
              const int nb = ((ie + (b & 1)) * (NY + 1) + je + ((b >> 1) & 1)) * (NZ + 1) + ke + (b >> 2);
              const double x0 = x[3 * nb], x1 = x[3 * nb + 1], x2 = x[3 * nb + 2];
              y0 = fma(K[3 * b], x0, fma(K[3 * b + 1], x1, fma(K[3 * b + 2], x2, y0)));
              y1 = fma(K[24 + 3 * b], x0, fma(K[24 + 3 * b + 1], x1, fma(K[24 + 3 * b + 2], x2, y1)));
              y2 = fma(K[48 + 3 * b], x0, fma(K[48 + 3 * b + 1], x1, fma(K[48 + 3 * b + 2], x2, y2)));
            }
          }
    }
    y[3 * n] = y0;
    y[3 * n + 1] = y1;
    y[3 * n + 2] = y2;
  }
}

__device__ __forceinline__ int global_node(const SubDev& s, int k, int q, int NY, int NZ) {
  const int gi = s.I0 + q / s.nyn, gj = s.J0 + q % s.nyn;
  return (gi * (NY + 1) + gj) * (NZ + 1) + k;
}

// R_j r: column 0 of the KB-wide block `which` of every subdomain holds r on
// its B1 rows, everything else zero
__global__ void k_local_gather(const SubDev* __restrict__ subs, const double* __restrict__ r, int which, int NY,
                               int NZ) {
  const SubDev& s = subs[blockIdx.y];
  double* X = mv_ptr(s, which);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)s.nfull * KB;
       e += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / KB), col = (int)(e % KB);
    const int n = row / 3, c = row % 3, k = n / s.npl, q = n % s.npl;
    double v = 0.0;
    if (col == 0 && s.cls[q] == 1) v = r[3 * (size_t)global_node(s, k, q, NY, NZ) + c];
    X[e] = v;
  }
}

// z = sum_j R_j^T w_j (column 0 of block `which`, B1 rows), subdomains summed
// in index order for every DoF
__global__ void k_local_scatter(const SubDev* __restrict__ subs, int N, int which, double* __restrict__ z, int NY,
                                int NZ, int ndof) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ndof; g += gridDim.x * blockDim.x) {
    const int node = g / 3, c = g % 3;
    const int k = node % (NZ + 1), ij = node / (NZ + 1), gi = ij / (NY + 1), gj = ij % (NY + 1);
    double acc = 0.0;
    for (int sidx = 0; sidx < N; ++sidx) {
      const SubDev& s = subs[sidx];
      if (gi < s.I0 || gi > s.I1 || gj < s.J0 || gj > s.J1) continue;
      const int q = (gi - s.I0) * s.nyn + (gj - s.J0);
      if (s.cls[q] != 1) continue;
      acc += mv_ptr(s, which)[(size_t)((k * s.npl + q) * 3 + c) * KB];
    }
    z[g] = acc;
  }
}

// r_H = V^T r into column 0 of bH (the coarse handle's weighted basis CB)
__global__ void k_coarse_restrict(const SubDev* __restrict__ subs, const int* __restrict__ coff,
                                  const int* __restrict__ msz, const double* __restrict__ r, double* __restrict__ bH,
                                  int NY, int NZ) {
  const SubDev& s = subs[blockIdx.x];
  __shared__ double red[8][PST];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double acc = 0.0;
  for (int row = w; row < s.nfull; row += 8) {
    const int n = row / 3, c = row % 3;
    const double rv = r[3 * (size_t)global_node(s, n / s.npl, n % s.npl, NY, NZ) + c];
    acc = fma(s.CB[(size_t)row * PST + lane], rv, acc);
  }
  red[w][lane] = acc;
  __syncthreads();
  if (w == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i][lane];
    if (lane < msz[blockIdx.x]) bH[(size_t)(coff[blockIdx.x] + lane) * PST] = t;
  }
}

// z += V c (column 0 of cH), subdomains summed in index order
__global__ void k_prolong_add(const SubDev* __restrict__ subs, int N, const int* __restrict__ coff,
                              const int* __restrict__ msz, const double* __restrict__ cH, double* __restrict__ z,
                              int NY, int NZ, int ndof) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ndof; g += gridDim.x * blockDim.x) {
    const int node = g / 3, c = g % 3;
    const int k = node % (NZ + 1), ij = node / (NZ + 1), gi = ij / (NY + 1), gj = ij % (NY + 1);
    double acc = 0.0;
    for (int sidx = 0; sidx < N; ++sidx) {
      const SubDev& s = subs[sidx];
      if (gi < s.oI0 || gi > s.oI1 || gj < s.oJ0 || gj > s.oJ1) continue;
      const int row = (k * s.npl + (gi - s.I0) * s.nyn + (gj - s.J0)) * 3 + c;
      const double* v = s.CB + (size_t)row * PST;
      const double* cc = cH + (size_t)coff[sidx] * PST;
      for (int a = 0; a < msz[sidx]; ++a) acc = fma(v[a], cc[(size_t)a * PST], acc);
    }
    z[g] += acc;
  }
}

// partial sums of a . b (and, with c, of a . c as well), one per block
__global__ void __launch_bounds__(256)
k_dot_partial(const double* __restrict__ a, const double* __restrict__ b, const double* __restrict__ c, int n,
              double* __restrict__ part) {
  __shared__ double red[2][256];
  double s0 = 0.0, s1 = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    s0 = fma(a[i], b[i], s0);
    if (c) s1 = fma(a[i], c[i], s1);
  }
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      red[0][threadIdx.x] += red[0][threadIdx.x + st];
      red[1][threadIdx.x] += red[1][threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = red[0][0];
    part[2 * blockIdx.x + 1] = red[1][0];
  }
}

// x += alpha p, r -= alpha q
__global__ void k_cg_step(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                          const double* __restrict__ q, double alpha, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    r[i] = fma(-alpha, q[i], r[i]);
  }
}

// p = z + beta p; r = b - y (mode 1); plain copy (mode 2)
__global__ void k_cg_axpy(double* __restrict__ out, const double* __restrict__ u, const double* __restrict__ v,
                          double beta, int n, int mode) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (mode == 0) out[i] = fma(beta, out[i], u[i]);
    else if (mode == 1) out[i] = u[i] - v[i];
    else out[i] = u[i];
  }
}

// zero the clamped face (the first (NY+1)(NZ+1) nodes)
__global__ void k_zero_clamped(double* __restrict__ x, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = 0.0;
}

bool dev_ptr(const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Extreme eigenvalues of the symmetric tridiagonal matrix (d, e) by bisection
// on the Sturm sequence count (Lanczos matrix of the CG coefficients).
double tridiag_extreme(const std::vector<double>& d, const std::vector<double>& e, bool largest) {
  const int n = (int)d.size();
  double lo = d[0], hi = d[0];
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(e[i]) : 0.0);
    lo = std::min(lo, d[i] - r);
    hi = std::max(hi, d[i] + r);
  }
  // count of eigenvalues below x
  auto below = [&](double x) {
    int c = 0;
    double q = d[0] - x;
    if (q < 0) ++c;
    for (int i = 1; i < n; ++i) {
      const double qq = q != 0.0 ? q : 1e-300;
      q = d[i] - x - e[i - 1] * e[i - 1] / qq;
      if (q < 0) ++c;
    }
    return c;
  };
  const int target = largest ? n - 1 : 0;   // find x with below(x) crossing target + 1
  for (int it = 0; it < 200 && hi - lo > 1e-14 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (below(mid) > target) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

msgfem_status schwarz_run(msgfem_h hl, msgfem_h hc, const double* b_in, const double* u0, double rtol,
                          int max_iter, double* u_out, msgfem_pcg_info* info);

}  // namespace

extern "C" msgfem_status msgfem_schwarz_solve(msgfem_h hl, msgfem_h hc, const double* b_in, const double* u0,
                                              double rtol, int max_iter, double* u_out, msgfem_pcg_info* info) {
  if (!hl || !u_out) return MSGFEM_EINVAL;
  const msgfem_status st = schwarz_run(hl, hc, b_in, u0, rtol, max_iter, u_out, info);
  const msgfem_status ke = check_stage_error(hl);   // the local solves' TMA stages
  return ke != MSGFEM_OK ? ke : st;
}

namespace {

msgfem_status schwarz_run(msgfem_h hl, msgfem_h hc, const double* b_in, const double* u0, double rtol,
                          int max_iter, double* u_out, msgfem_pcg_info* info) {
  if (!hl || !u_out) return MSGFEM_EINVAL;
  msgfem* h = hl;
  if (h->stage < 1) return MSGFEM_ESTATE;
  if (h->S > 1 || h->os != h->o) {
    h->err = "the local handle of msgfem_schwarz_solve needs one instance and oversampling equal to overlap "
             "(its A11 factors are the Dirichlet problems on Omega_j)";
    return MSGFEM_EINVAL;
  }
  if (hc) {
    if (hc->NX != h->NX || hc->NY != h->NY || hc->NZ != h->NZ || hc->S > 1) {
      h->err = "the coarse handle must hold the same mesh";
      return MSGFEM_EINVAL;
    }
    if (hc->stage < 3) {
      h->err = "the coarse handle has no coarse problem (msgfem_coarse_assemble)";
      return MSGFEM_ESTATE;
    }
  }
  if (!(rtol > 0.0)) rtol = 1e-10;
  if (max_iter <= 0) max_iter = 2000;
  cudaStream_t st = h->stream;
  const int NX = h->NX, NY = h->NY, NZ = h->NZ;
  const int nnode = (NX + 1) * (NY + 1) * (NZ + 1);
  const int ndof = 3 * nnode;
  const int nclamp = 3 * (NY + 1) * (NZ + 1);
  if (hc) CK(cudaStreamSynchronize(hc->stream));   // the coarse handle's own work is complete
  TRY(schwarz_factors(h));
  if (h->d_pcg_vec == nullptr) {
    void* p = nullptr;
    TRY(dev_alloc_bytes(h, &p, (size_t)6 * ndof * sizeof(double)));
    h->d_pcg_vec = static_cast<double*>(p);
    TRY(dev_alloc_bytes(h, &p, (size_t)2 * DOT_BLOCKS * sizeof(double)));
    h->d_pcg_part = static_cast<double*>(p);
  }
  double* x = h->d_pcg_vec;
  double* r = x + ndof;
  double* z = r + ndof;
  double* p = z + ndof;
  double* q = p + ndof;
  double* bv = q + ndof;
  // right-hand side and start
  if (b_in) {
    TRY(vec_in(h, b_in, bv));
  } else {
    const std::vector<double> b = global_load(h);
    CK(cudaMemcpyAsync(bv, b.data(), (size_t)ndof * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  }
  if (u0) TRY(vec_in(h, u0, x));
  else CK(cudaMemsetAsync(x, 0, (size_t)ndof * sizeof(double), st));
  const int gs = 2 * 152;
  k_zero_clamped<<<gs, 256, 0, st>>>(bv, nclamp);
  k_zero_clamped<<<gs, 256, 0, st>>>(x, nclamp);
  g_launch_count += 2;
  const int* et = h->typed ? h->d_etype : nullptr;
  auto apply_A = [&](const double* in, double* out) {
    k_apply_A<<<(nnode + 127) / 128, 128, 0, st>>>(h->d_Ke, h->layered, et, in, out, NX, NY, NZ);
    ++g_launch_count;
  };
  std::vector<double> part(2 * DOT_BLOCKS);
  auto dots = [&](const double* a, const double* bb, const double* c, double& s0, double& s1) -> msgfem_status {
    k_dot_partial<<<DOT_BLOCKS, 256, 0, st>>>(a, bb, c, ndof, h->d_pcg_part);
    ++g_launch_count;
    CK(cudaMemcpyAsync(part.data(), h->d_pcg_part, part.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    s0 = s1 = 0.0;
    for (int i = 0; i < DOT_BLOCKS; ++i) {
      s0 += part[2 * i];
      s1 += part[2 * i + 1];
    }
    return MSGFEM_OK;
  };
  // z = M^{-1} r
  auto precond = [&]() -> msgfem_status {
    set_dense_context(h->d_flags, h->d_notspd, h->d_sub);
    dim3 grid(64, h->N);
    k_local_gather<<<grid, 256, 0, st>>>(h->d_sub, r, MV_TB, NY, NZ);
    ++g_launch_count;
    schwarz_local_solve(h);
    k_local_scatter<<<(ndof + 255) / 256, 256, 0, st>>>(h->d_sub, h->N, MV_WB, z, NY, NZ, ndof);
    ++g_launch_count;
    if (hc) {
      set_dense_context(hc->d_flags, hc->d_notspd, hc->d_sub);
      k_coarse_restrict<<<hc->N, 256, 0, st>>>(hc->d_sub, hc->d_coff, hc->d_m, r, hc->d_bH, NY, NZ);
      ++g_launch_count;
      run_solve_mv(hc->csolve, st, 0, 0, 0);
      k_prolong_add<<<(ndof + 255) / 256, 256, 0, st>>>(hc->d_sub, hc->N, hc->d_coff, hc->d_m, hc->d_cH, z, NY, NZ,
                                                         ndof);
      ++g_launch_count;
      set_dense_context(h->d_flags, h->d_notspd, h->d_sub);
    }
    CK_LAUNCH();
    return MSGFEM_OK;
  };
  // r = b - A x
  apply_A(x, q);
  k_cg_axpy<<<gs, 256, 0, st>>>(r, bv, q, 0.0, ndof, 1);
  ++g_launch_count;
  double bb = 0.0, dummy = 0.0, rr = 0.0;
  TRY(dots(bv, bv, nullptr, bb, dummy));
  TRY(dots(r, r, nullptr, rr, dummy));
  const double nb = std::sqrt(bb) > 0.0 ? std::sqrt(bb) : 1.0;
  TRY(precond());
  k_cg_axpy<<<gs, 256, 0, st>>>(p, z, nullptr, 0.0, ndof, 2);
  ++g_launch_count;
  double rz = 0.0;
  TRY(dots(r, z, nullptr, rz, dummy));
  std::vector<double> alphas, betas;
  int it = 0;
  double res = std::sqrt(rr) / nb;
  bool broke = false;
  while (res > rtol && it < max_iter) {
    apply_A(p, q);
    double pq = 0.0;
    TRY(dots(p, q, nullptr, pq, dummy));
    if (!(pq > 0.0) || !std::isfinite(pq)) { broke = true; break; }
    const double alpha = rz / pq;
    k_cg_step<<<gs, 256, 0, st>>>(x, r, p, q, alpha, ndof);
    ++g_launch_count;
    TRY(precond());
    double rz_new = 0.0;
    TRY(dots(r, z, r, rz_new, rr));   // r . z and r . r
    const double beta = rz_new / rz;
    rz = rz_new;
    k_cg_axpy<<<gs, 256, 0, st>>>(p, z, nullptr, beta, ndof, 0);
    ++g_launch_count;
    alphas.push_back(alpha);
    betas.push_back(beta);
    ++it;
    res = std::sqrt(std::max(rr, 0.0)) / nb;
    if (!std::isfinite(res)) { broke = true; break; }
  }
  TRY(vec_out(h, x, u_out));
  CK(cudaStreamSynchronize(st));
  if (hc) {
    // the coarse handle's own right-hand side b^H is restored for its msgfem_solve
    launch_coarse_rhs(hc);
    CK(cudaStreamSynchronize(hc->stream));
  }
  if (info) {
    info->iterations = it;
    info->residual = res;
    info->lambda_min = info->lambda_max = info->kappa = 1.0;
    const int k = (int)alphas.size();
    if (k > 0) {
      // Lanczos matrix of M^{-1} A from the CG coefficients
      std::vector<double> d(k), e(std::max(k - 1, 0));
      d[0] = 1.0 / alphas[0];
      for (int i = 1; i < k; ++i) d[i] = 1.0 / alphas[i] + betas[i - 1] / alphas[i - 1];
      for (int i = 0; i + 1 < k; ++i) e[i] = std::sqrt(std::max(betas[i], 0.0)) / alphas[i];
      info->lambda_min = tridiag_extreme(d, e, false);
      info->lambda_max = tridiag_extreme(d, e, true);
      info->kappa = info->lambda_max / info->lambda_min;
    }
  }
  if (broke) {
    h->err = "Schwarz PCG broke down (non-positive curvature or non-finite residual)";
    return MSGFEM_ENOTSPD;
  }
  if (res > rtol) {
    h->err = "Schwarz PCG reached max_iter at relative residual " + std::to_string(res);
    return MSGFEM_ENOCONV;
  }
  return MSGFEM_OK;
}
}  // namespace
