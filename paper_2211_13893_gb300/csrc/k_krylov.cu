// Block Krylov (block Lanczos with full re-orthogonalisation) for the
// A-harmonic local eigenproblem S x = lambda T x, run on the shift-invert
// operator M = S^{-1} T, which is self-adjoint in the T inner product.
//
// Vectors are kept in their A-harmonic extension phi = E x (full Omega*
// layout); M phi = E [K^{-1} B phi]_2 with B = D_mu K D_mu (one K solve and one
// A11 solve per block).  M is self-adjoint in the inner product
// N = S + sigma T, <phi_a, phi_b>_N = phi_a^T (K + sigma B) phi_b, which is
// definite on the rigid modes (where S vanishes) and on the near-null space of
// T (vectors living where mu ~ 0, which T alone cannot see), so rounding noise
// is never normalised into the basis.  With Q_m N-orthonormal,
// M Q_m = Q_m H_m + Q_{m+1} R_{m+1} E_m^T; a Ritz pair (mu, y) of H_m gives
// lambda = 1/mu and the relative residual ||M x - mu x||_N / (mu ||x||_N) =
// ||R_{m+1} y_last|| / mu without extra solves; x^T T x = 1 / (lambda + sigma)
// gives the B-normalised eigenvector.
#include "internal.h"

namespace {

constexpr double KSIGMA = 1e-2;   // N = S + KSIGMA T

// y = alpha [D_mu] K [D_mu] x on KB-wide blocks: 4 nodes per warp, lane % 8 = column.
__global__ void __launch_bounds__(256)
k_stencil_kb(const SubDev* __restrict__ subs, const int* __restrict__ active, int src, int dst, int mode,
             double alpha) {
  const int sidx = blockIdx.y;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  const int lane = threadIdx.x & 31, col = lane & (KB - 1);
  const int node = (blockIdx.x * 8 + (threadIdx.x >> 5)) * (32 / KB) + (lane / KB);
  if (node >= s.nnode) return;
  const double* x = mv_ptr(s, src);
  double* y = mv_ptr(s, dst);
  const int k = node / s.npl, q = node % s.npl;
  const int qi = q / s.nyn, qj = q % s.nyn;
  const double* st = s.stencil + (size_t)node * 243;
  double y0 = 0.0, y1 = 0.0, y2 = 0.0, z0 = 0.0, z1 = 0.0, z2 = 0.0;
  for (int slot = 0; slot < 27; ++slot) {
    const int di = slot / 9 - 1, dj = (slot / 3) % 3 - 1, dk = slot % 3 - 1;
    const int ni = qi + di, nj = qj + dj, nk = k + dk;
    if (ni < 0 || ni >= s.nxn || nj < 0 || nj >= s.nyn || nk < 0 || nk >= s.nzn) continue;
    const int nb = nk * s.npl + ni * s.nyn + nj;
    const double* xr = x + (size_t)nb * 3 * KB + col;
    const double* c = st + slot * 9;
    if (mode == 4) {
      // N x = K x + sigma D_mu K D_mu x in one pass (sigma = alpha)
      const double x0 = xr[0], x1 = xr[KB], x2 = xr[2 * KB], m = s.mu[nb];
      const double k0 = fma(c[0], x0, fma(c[1], x1, c[2] * x2));
      const double k1 = fma(c[3], x0, fma(c[4], x1, c[5] * x2));
      const double k2 = fma(c[6], x0, fma(c[7], x1, c[8] * x2));
      y0 += k0; y1 += k1; y2 += k2;
      z0 = fma(m, k0, z0); z1 = fma(m, k1, z1); z2 = fma(m, k2, z2);
      continue;
    }
    const double sc = (mode & 1) ? s.mu[nb] : 1.0;
    const double x0 = sc * xr[0], x1 = sc * xr[KB], x2 = sc * xr[2 * KB];
    y0 = fma(c[0], x0, fma(c[1], x1, fma(c[2], x2, y0)));
    y1 = fma(c[3], x0, fma(c[4], x1, fma(c[5], x2, y1)));
    y2 = fma(c[6], x0, fma(c[7], x1, fma(c[8], x2, y2)));
  }
  double* yr = y + (size_t)node * 3 * KB + col;
  if (mode == 4) {
    const double sm = alpha * s.mu[node];
    yr[0] = fma(sm, z0, y0);
    yr[KB] = fma(sm, z1, y1);
    yr[2 * KB] = fma(sm, z2, y2);
    return;
  }
  const double post = alpha * ((mode & 2) ? s.mu[node] : 1.0);
  yr[0] = post * y0;
  yr[KB] = post * y1;
  yr[2 * KB] = post * y2;
}

constexpr int KROWS = 512;

// Partial sums of G[a][b] = sum_r X[r][a] Y[r][b], a < nx (X of stride xs),
// b < KB (Y of stride KB).
__global__ void __launch_bounds__(256)
k_gram_kb_partial(const SubDev* __restrict__ subs, const int* __restrict__ active, int wx, int xs, int nx, int wy,
                  int only_floating, double* __restrict__ part, int nchunk) {
  const int sidx = blockIdx.y;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  if (only_floating && !s.floating) return;
  __shared__ double Xs[32][MQ + 1];
  __shared__ double Ys[32][KB];
  const double* X = mv_ptr(s, wx);
  const double* Yv = mv_ptr(s, wy);
  const int tid = threadIdx.x;
  const int nout = nx * KB;
  double acc[3] = {0.0, 0.0, 0.0};
  const int r0 = blockIdx.x * KROWS;
  const int r1 = min(r0 + KROWS, s.nfull);
  for (int rb = r0; rb < r1; rb += 32) {
    for (int e = tid; e < 32 * nx; e += 256) {
      const int rr = rb + e / nx;
      Xs[e / nx][e % nx] = rr < r1 ? X[(size_t)rr * xs + e % nx] : 0.0;
    }
    for (int e = tid; e < 32 * KB; e += 256) {
      const int rr = rb + e / KB;
      Ys[e / KB][e % KB] = rr < r1 ? Yv[(size_t)rr * KB + e % KB] : 0.0;
    }
    __syncthreads();
    for (int i = 0; i < 3; ++i) {
      const int o = tid + 256 * i;
      if (o >= nout) break;
      const int a = o / KB, b = o % KB;
      double v = acc[i];
#pragma unroll 8
      for (int r = 0; r < 32; ++r) v = fma(Xs[r][a], Ys[r][b], v);
      acc[i] = v;
    }
    __syncthreads();
  }
  double* out = part + ((size_t)sidx * nchunk + blockIdx.x) * MQ * KB;
  for (int i = 0; i < 3; ++i) {
    const int o = tid + 256 * i;
    if (o < nout) out[o] = r0 < s.nfull ? acc[i] : 0.0;
  }
}

__global__ void k_gram_kb_reduce(const SubDev* __restrict__ subs, const int* __restrict__ active, int nx,
                                 int only_floating, const double* __restrict__ part, int nchunk) {
  const int sidx = blockIdx.x;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  if (only_floating && !s.floating) return;
  const int nc = (s.nfull + KROWS - 1) / KROWS;
  for (int o = threadIdx.x; o < nx * KB; o += blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < nc; ++c) acc += part[((size_t)sidx * nchunk + c) * MQ * KB + o];
    s.Hc[o] = acc;
  }
}

// Y -= X Hc with X of stride xs and nx columns, Y a KB-wide block.
__global__ void __launch_bounds__(256)
k_update_kb(const SubDev* __restrict__ subs, const int* __restrict__ active, int wx, int xs, int nx, int wy,
            int only_floating) {
  const int sidx = blockIdx.y;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  if (only_floating && !s.floating) return;
  __shared__ double C[MQ][KB];
  for (int e = threadIdx.x; e < nx * KB; e += 256) C[e / KB][e % KB] = s.Hc[e];
  __syncthreads();
  const double* X = mv_ptr(s, wx);
  double* Y = mv_ptr(s, wy);
  const int col = threadIdx.x % KB;
  for (int r = blockIdx.x * (256 / KB) + threadIdx.x / KB; r < s.nfull; r += gridDim.x * (256 / KB)) {
    const double* xr = X + (size_t)r * xs;
    double acc = Y[(size_t)r * KB + col];
    for (int a = 0; a < nx; ++a) acc = fma(-xr[a], C[a][col], acc);
    Y[(size_t)r * KB + col] = acc;
  }
}

// H[a][j KB + c] (+)= Hc[a][c], a < m.
__global__ void k_h_accum(const SubDev* __restrict__ subs, const int* __restrict__ active, int m, int j, int add) {
  const int sidx = blockIdx.x;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  for (int e = threadIdx.x; e < m * KB; e += blockDim.x) {
    const int a = e / KB, c = e % KB;
    double* h = s.H + (size_t)a * MQ + j * KB + c;
    *h = add ? *h + s.Hc[e] : s.Hc[e];
  }
}

// One pass of CholeskyQR2 of a KB-wide block in the N inner product:
// Hc = W^T N W = L L^T and Y[0:KB][0:KB] = L^{-T}.  Pass 1 drops columns that
// are rounding noise -- a pivot below 1e-12 of the column's own squared norm
// (dependent inside the block) or below 1e-20 of its squared norm before
// Gram-Schmidt (the Krylov space is exhausted) -- and keeps R1 = L^T in
// Y[KB:2KB][0:KB].  Pass 2 re-orthonormalises the surviving columns and, for
// j >= 0, stores R_{j+1} = L2^T R1 in H[(j+1) KB + r][j KB + c].
__global__ void k_cholqr_kb(const SubDev* __restrict__ subs, const int* __restrict__ active, int j, int pass) {
  const int sidx = blockIdx.x;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  if (threadIdx.x != 0) return;
  double G[KB][KB], L[KB][KB], U[KB][KB], n0[KB];
  for (int a = 0; a < KB; ++a)
    for (int b = 0; b < KB; ++b) { G[a][b] = 0.5 * (s.Hc[a * KB + b] + s.Hc[b * KB + a]); L[a][b] = 0.0; U[a][b] = 0.0; }
  for (int c = 0; c < KB; ++c) {
    n0[c] = G[c][c];
    if (pass == 1 && j >= 0)
      for (int a = 0; a < (j + 1) * KB; ++a) {
        const double hc = s.H[(size_t)a * MQ + j * KB + c];
        n0[c] += hc * hc;
      }
  }
  bool dead[KB];
  for (int c = 0; c < KB; ++c) {
    double v = G[c][c];
    for (int k = 0; k < c; ++k) v -= L[c][k] * L[c][k];
    dead[c] = !(G[c][c] > 0.0) || !(v > 1e-12 * G[c][c]) || !(v > 1e-20 * n0[c]);
    if (dead[c]) {
      s.status[3] = 1;
      continue;
    }
    L[c][c] = sqrt(v);
    for (int r = c + 1; r < KB; ++r) {
      double w = G[r][c];
      for (int k = 0; k < c; ++k) w -= L[r][k] * L[c][k];
      L[r][c] = w / L[c][c];
    }
  }
  for (int c = 0; c < KB; ++c) {
    if (dead[c]) continue;
    for (int i = c; i >= 0; --i) {
      if (dead[i]) continue;
      double v = (i == c) ? 1.0 : 0.0;
      for (int k = i + 1; k <= c; ++k) v -= L[k][i] * U[k][c];
      U[i][c] = v / L[i][i];
    }
  }
  for (int a = 0; a < KB; ++a)
    for (int b = 0; b < KB; ++b) s.Y[a * PST + b] = U[a][b];
  if (pass == 1) {
    for (int r = 0; r < KB; ++r)
      for (int c = 0; c < KB; ++c) s.Y[(KB + r) * PST + c] = L[c][r];
  } else if (j >= 0) {
    for (int r = 0; r < KB; ++r)
      for (int c = 0; c < KB; ++c) {
        double v = 0.0;
        for (int k = 0; k < KB; ++k) v += L[k][r] * s.Y[(KB + k) * PST + c];   // (L2^T R1)[r][c]
        s.H[(size_t)((j + 1) * KB + r) * MQ + j * KB + c] = v;
      }
  }
}

// X <- X Y[0:KB][0:KB] on a KB-wide block.
__global__ void __launch_bounds__(256)
k_rotate_kb(const SubDev* __restrict__ subs, const int* __restrict__ active, int which) {
  const int sidx = blockIdx.y;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  __shared__ double Ys[KB][KB];
  if (threadIdx.x < KB * KB) Ys[threadIdx.x / KB][threadIdx.x % KB] = s.Y[(threadIdx.x / KB) * PST + threadIdx.x % KB];
  __syncthreads();
  double* X = mv_ptr(s, which);
  const int col = threadIdx.x % KB;
  for (int r = blockIdx.x * (256 / KB) + threadIdx.x / KB; r < s.nfull; r += gridDim.x * (256 / KB)) {
    double xr[KB];
#pragma unroll
    for (int a = 0; a < KB; ++a) xr[a] = X[(size_t)r * KB + a];
    __syncwarp();
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < KB; ++a) acc = fma(xr[a], Ys[a][col], acc);
    X[(size_t)r * KB + col] = acc;
  }
}

// dst[:, j KB + c] = src[:, c] (dst = QB or NQ)
__global__ void k_store_block(const SubDev* __restrict__ subs, const int* __restrict__ active, int src, int j,
                              int dst) {
  const int sidx = blockIdx.y;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  const double* X = mv_ptr(s, src);
  double* D = mv_ptr(s, dst);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)s.nfull * KB;
       e += (size_t)gridDim.x * blockDim.x)
    D[(e / KB) * MQ + j * KB + e % KB] = X[e];
}

__global__ void k_zero_kb(const SubDev* __restrict__ subs, const int* __restrict__ active, int which, int col0_only) {
  if (active != nullptr && !active[blockIdx.y]) return;
  const SubDev& s = subs[blockIdx.y];
  double* X = mv_ptr(s, which);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)s.nfull * KB;
       e += (size_t)gridDim.x * blockDim.x)
    X[e] = 0.0;
  (void)col0_only;
}

// Start block on the rows of DoF class fill_cls (counter-based uniform(-1, 1)),
// zero elsewhere: B2 for the A-harmonic problem, B1 for GenEO.
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void k_random_kb(const SubDev* __restrict__ subs, const int* __restrict__ active, int which,
                            unsigned long long seed, int fill_cls) {
  const int sidx = blockIdx.y;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  double* X = mv_ptr(s, which);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)s.nfull * KB;
       e += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / KB), col = (int)(e % KB);
    const int q = (row / 3) % s.npl;
    double v = 0.0;
    if (s.cls[q] == fill_cls) {
      const uint64_t key = mix64(seed ^ mix64(((uint64_t)sidx << 40) ^ ((uint64_t)row << 8) ^ col));
      v = (double)(key >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
    X[e] = v;
  }
}

__global__ void k_mask_kb(const SubDev* __restrict__ subs, const int* __restrict__ active, int which, int keep) {
  const int sidx = blockIdx.y;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  double* X = mv_ptr(s, which);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)s.nfull * KB;
       e += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(e / KB / 3) % s.npl;
    if (!((keep >> s.cls[q]) & 1)) X[e] = 0.0;
  }
}

__global__ void k_zero_pins_kb(const SubDev* __restrict__ subs, const int* __restrict__ active, int which) {
  if (active != nullptr && !active[blockIdx.x]) return;
  const SubDev& s = subs[blockIdx.x];
  if (!s.floating) return;
  double* X = mv_ptr(s, which);
  const int i = threadIdx.x / KB, c = threadIdx.x % KB;
  if (i < 6 && s.pin[i] >= 0) X[(size_t)s.pin[i] * KB + c] = 0.0;
}

// dst[:, 0] = sign * bload, other columns zero (KB-wide block)
__global__ void k_load_col_kb(const SubDev* __restrict__ subs, const int* __restrict__ active, int which, double sign) {
  if (active != nullptr && !active[blockIdx.y]) return;
  const SubDev& s = subs[blockIdx.y];
  double* X = mv_ptr(s, which);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)s.nfull * KB;
       e += (size_t)gridDim.x * blockDim.x)
    X[e] = (e % KB == 0) ? sign * s.bload[e / KB] : 0.0;
}

__global__ void k_take_col_kb(const SubDev* __restrict__ subs, const int* __restrict__ active, int which) {
  if (active != nullptr && !active[blockIdx.y]) return;
  const SubDev& s = subs[blockIdx.y];
  const double* X = mv_ptr(s, which);
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < s.nfull; r += gridDim.x * blockDim.x)
    s.psi[r] = X[(size_t)r * KB];
}

// Rayleigh-Ritz on the leading m x m block of H (symmetrised): parallel cyclic
// Jacobi in dynamic shared memory; the nw largest mu give theta = 1/mu
// ascending, Yk[:, i] their coefficient vectors, resid[i] = theta_i
// ||R_{m+1} y_last||.
__global__ void __launch_bounds__(256)
k_rr_krylov(const SubDev* __restrict__ subs, const int* __restrict__ active, const int* __restrict__ mvec,
            const int* __restrict__ nwvec) {
  const int sidx = blockIdx.x;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  const int m = mvec[sidx], nw = nwvec[sidx];
  if (m <= 0 || nw <= 0) return;
  extern __shared__ double sh[];
  double (*A)[MQ + 1] = reinterpret_cast<double (*)[MQ + 1]>(sh);
  double (*V)[MQ + 1] = reinterpret_cast<double (*)[MQ + 1]>(sh + MQ * (MQ + 1));
  __shared__ double cs[MQ / 2], sn[MQ / 2];
  __shared__ int pa[MQ / 2], pb[MQ / 2], perm[MQ];
  __shared__ int again;
  const int tid = threadIdx.x;
  for (int e = tid; e < m * m; e += 256) {
    const int r = e / m, c = e % m;
    A[r][c] = 0.5 * (s.H[(size_t)r * MQ + c] + s.H[(size_t)c * MQ + r]);
    V[r][c] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int mm = (m + 1) & ~1;
  __shared__ double red_off[8], red_tot[8];
  for (int sweep = 0; sweep < 30; ++sweep) {
    {
      // off-diagonal and total Frobenius mass, reduced over the block
      double off = 0.0, tot = 0.0;
      for (int e = tid; e < m * m; e += 256) {
        const int i = e / m, j = e % m;
        const double v = A[i][j] * A[i][j];
        tot += v;
        if (i != j) off += v;
      }
      for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
      }
      if ((tid & 31) == 0) {
        red_off[tid >> 5] = off;
        red_tot[tid >> 5] = tot;
      }
      __syncthreads();
      if (tid == 0) {
        double so = 0.0, st = 0.0;
        for (int w = 0; w < 8; ++w) { so += red_off[w]; st += red_tot[w]; }
        again = so > 1e-30 * st;
      }
      __syncthreads();
    }
    if (!again) break;
    for (int round = 0; round < mm - 1; ++round) {
      if (tid < mm / 2) {
        int a = (tid == 0) ? 0 : ((round + tid - 1) % (mm - 1)) + 1;
        int b = ((round + mm - 2 - tid) % (mm - 1)) + 1;
        if (a > b) { const int t = a; a = b; b = t; }
        pa[tid] = a;
        pb[tid] = b;
        double c = 1.0, sv = 0.0;
        if (b < m) {
          const double apq = A[a][b];
          if (fabs(apq) > 1e-300) {
            const double tau = (A[b][b] - A[a][a]) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            sv = t * c;
          }
        }
        cs[tid] = c;
        sn[tid] = sv;
      }
      __syncthreads();
      for (int e = tid; e < (mm / 2) * m; e += 256) {
        const int k = e / m, col = e % m;
        const int a = pa[k], b = pb[k];
        if (b >= m) continue;
        const double x = A[a][col], y = A[b][col];
        A[a][col] = cs[k] * x - sn[k] * y;
        A[b][col] = sn[k] * x + cs[k] * y;
      }
      __syncthreads();
      for (int e = tid; e < (mm / 2) * m; e += 256) {
        const int k = e / m, row = e % m;
        const int a = pa[k], b = pb[k];
        if (b >= m) continue;
        const double x = A[row][a], y = A[row][b];
        A[row][a] = cs[k] * x - sn[k] * y;
        A[row][b] = sn[k] * x + cs[k] * y;
        const double vx = V[row][a], vy = V[row][b];
        V[row][a] = cs[k] * vx - sn[k] * vy;
        V[row][b] = sn[k] * vx + cs[k] * vy;
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    for (int i = 0; i < m; ++i) perm[i] = i;
    for (int i = 0; i < m; ++i)   // descending mu
      for (int j = i + 1; j < m; ++j)
        if (A[perm[j]][perm[j]] > A[perm[i]][perm[i]]) { const int t = perm[i]; perm[i] = perm[j]; perm[j] = t; }
  }
  __syncthreads();
  for (int e = tid; e < MQ * PST; e += 256) {
    const int a = e / PST, i = e % PST;
    s.Yk[e] = (a < m && i < nw) ? V[a][perm[i]] : 0.0;
  }
  if (tid < nw) {
    // Ritz values of M in the N = S + sigma T inner product lie in [0, 1 / sigma];
    // a wanted one below 1e-14 (lambda above 1e14) comes from a basis that broke down
    const double mu = A[perm[tid]][perm[tid]];
    const bool valid = mu > 1e-14;
    const double th = valid ? 1.0 / mu : 1e300;
    double r2 = 0.0;
    if (m + KB <= MQ + KB)
      for (int r = 0; r < KB; ++r) {
        double v = 0.0;
        for (int c = 0; c < KB; ++c) v += s.H[(size_t)(m + r) * MQ + (m - KB + c)] * V[m - KB + c][perm[tid]];
        r2 += v * v;
      }
    s.theta[tid] = th;
    // no positive Ritz value (a basis that broke down, e.g. from a non-finite
    // start block whose columns were all dropped): never converged
    s.resid[tid] = valid ? th * sqrt(r2) : INFINITY;
  }
}

// dst[:, i] = src[:, 0:m] Yk[:, i] for i < nw, zero for i >= nw (src = QB:
// Ritz vectors; src = NQ: their N products); with scale = 1 the columns are
// B-normalised (factor sqrt(theta_i + sigma)).
__global__ void __launch_bounds__(256)
k_ritz(const SubDev* __restrict__ subs, const int* __restrict__ active, const int* __restrict__ mvec,
       const int* __restrict__ nwvec, int scale, int src, int dst) {
  const int sidx = blockIdx.y;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  const int m = mvec[sidx], nw = nwvec[sidx];
  __shared__ double Ys[MQ][PST];
  for (int e = threadIdx.x; e < MQ * PST; e += 256) Ys[e / PST][e % PST] = s.Yk[e];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int r = blockIdx.x * 8 + (threadIdx.x >> 5); r < s.nfull; r += gridDim.x * 8) {
    const double* q = mv_ptr(s, src) + (size_t)r * MQ;
    double acc = 0.0;
    for (int a0 = 0; a0 < m; a0 += 32) {
      const double qv = (a0 + lane < m) ? q[a0 + lane] : 0.0;
      const int na = min(32, m - a0);
      for (int a = 0; a < na; ++a) acc = fma(__shfl_sync(0xffffffffu, qv, a), Ys[a0 + a][lane], acc);
    }
    mv_ptr(s, dst)[(size_t)r * PST + lane] = (lane < nw) ? (scale ? acc * sqrt(s.theta[lane] + KSIGMA) : acc) : 0.0;
  }
}

// Thick restart, basis part: dst[:, 0:k] = ritz[:, 0:k] (Ritz vectors),
// dst[:, k:k+KB] = block (the residual block Q_{m+1}); run for QB and for NQ.
__global__ void k_restart_basis(const SubDev* __restrict__ subs, const int* __restrict__ active, int k, int ritz,
                                int block, int dst) {
  const int sidx = blockIdx.y;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  const double* R = mv_ptr(s, ritz);
  const double* B = mv_ptr(s, block);
  double* D = mv_ptr(s, dst);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)s.nfull * (k + KB);
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t r = e / (k + KB);
    const int c = (int)(e % (k + KB));
    D[r * MQ + c] = c < k ? R[r * PST + c] : B[r * KB + (c - k)];
  }
}

// H = 0 for the active subdomains before a Krylov run: the Lanczos steps write
// only the block upper Hessenberg part, and a thick restart of an earlier run
// leaves its arrow rows below it.
__global__ void k_zero_h(const SubDev* __restrict__ subs, const int* __restrict__ active) {
  const int sidx = blockIdx.x;
  if (active != nullptr && !active[sidx]) return;
  double* H = subs[sidx].H;
  for (int e = threadIdx.x; e < (MQ + KB) * MQ; e += blockDim.x) H[e] = 0.0;
}

// Thick restart, projected operator: H = [diag(mu) ; R_{m+1} Y_last] in the
// first k columns, zero elsewhere (the next block's coefficients are filled by
// Gram-Schmidt).  One block per subdomain.
__global__ void k_restart_h(const SubDev* __restrict__ subs, const int* __restrict__ active, int m, int k) {
  const int sidx = blockIdx.x;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  __shared__ double RY[KB][PST];
  __shared__ double mu[PST];
  for (int e = threadIdx.x; e < KB * k; e += blockDim.x) {
    const int r = e / k, i = e % k;
    double v = 0.0;
    for (int c = 0; c < KB; ++c) v += s.H[(size_t)(m + r) * MQ + (m - KB + c)] * s.Yk[(size_t)(m - KB + c) * PST + i];
    RY[r][i] = v;
  }
  if (threadIdx.x < k) mu[threadIdx.x] = 1.0 / s.theta[threadIdx.x];
  __syncthreads();
  for (size_t e = threadIdx.x; e < (size_t)(MQ + KB) * MQ; e += blockDim.x) {
    const int r = (int)(e / MQ), c = (int)(e % MQ);
    double v = 0.0;
    if (c < k) {
      if (r == c) v = mu[c];
      else if (r >= k && r < k + KB) v = RY[r - k][c];
    }
    s.H[e] = v;
  }
}

}  // namespace

static int max_nnode_k(msgfem* h) {
  int m = 0;
  for (const auto& s : h->sub) m = std::max(m, s.nnode);
  return m;
}

void launch_stencil_kb(msgfem* h, int src, int dst, int mode, double alpha) {
  dim3 grid((max_nnode_k(h) + 31) / 32, h->N);
  k_stencil_kb<<<grid, 256, 0, h->stream>>>(h->d_sub, h->d_flags, src, dst, mode, alpha); ++g_launch_count;
}

// Hc[0:nx][0:KB] = X[:, 0:nx]^T Y
void launch_gram_kb(msgfem* h, int wx, int xs, int nx, int wy, int only_floating) {
  const int nchunk = (3 * max_nnode_k(h) + KROWS - 1) / KROWS;
  dim3 grid(nchunk, h->N);
  k_gram_kb_partial<<<grid, 256, 0, h->stream>>>(h->d_sub, h->d_flags, wx, xs, nx, wy, only_floating,
                                                 h->d_gram_part, nchunk); ++g_launch_count;
  k_gram_kb_reduce<<<h->N, 256, 0, h->stream>>>(h->d_sub, h->d_flags, nx, only_floating, h->d_gram_part, nchunk); ++g_launch_count;
}

void launch_update_kb(msgfem* h, int wx, int xs, int nx, int wy, int only_floating) {
  dim3 grid(std::max(1, (3 * max_nnode_k(h) + 255) / 256), h->N);
  k_update_kb<<<grid, 256, 0, h->stream>>>(h->d_sub, h->d_flags, wx, xs, nx, wy, only_floating); ++g_launch_count;
}

void launch_h_accum(msgfem* h, int m, int j, int add) {
  k_h_accum<<<h->N, 256, 0, h->stream>>>(h->d_sub, h->d_flags, m, j, add); ++g_launch_count;
}

void launch_cholqr_kb(msgfem* h, int j, int pass) { k_cholqr_kb<<<h->N, 32, 0, h->stream>>>(h->d_sub, h->d_flags, j, pass); ++g_launch_count; }

void launch_rotate_kb(msgfem* h, int which) {
  dim3 grid(std::max(1, (3 * max_nnode_k(h) + 255) / 256), h->N);
  k_rotate_kb<<<grid, 256, 0, h->stream>>>(h->d_sub, h->d_flags, which); ++g_launch_count;
}

void launch_store_block(msgfem* h, int src, int j, int dst) {
  dim3 grid(256, h->N);
  k_store_block<<<grid, 256, 0, h->stream>>>(h->d_sub, h->d_flags, src, j, dst); ++g_launch_count;
}

void launch_random_kb(msgfem* h, int which, unsigned long long seed) {
  dim3 grid(256, h->N);
  k_random_kb<<<grid, 256, 0, h->stream>>>(h->d_sub, h->d_flags, which, seed, h->geneo ? 1 : 2); ++g_launch_count;
}

void launch_mask_kb(msgfem* h, int which, int keep) {
  dim3 grid(256, h->N);
  k_mask_kb<<<grid, 256, 0, h->stream>>>(h->d_sub, h->d_flags, which, keep); ++g_launch_count;
}

void launch_zero_pins_kb(msgfem* h, int which) { k_zero_pins_kb<<<h->N, 6 * KB, 0, h->stream>>>(h->d_sub, h->d_flags, which); ++g_launch_count; }

void launch_load_col_kb(msgfem* h, int which, double sign) {
  dim3 grid(256, h->N);
  k_load_col_kb<<<grid, 256, 0, h->stream>>>(h->d_sub, h->d_flags, which, sign); ++g_launch_count;
}

void launch_take_col_kb(msgfem* h, int which) {
  dim3 grid(64, h->N);
  k_take_col_kb<<<grid, 256, 0, h->stream>>>(h->d_sub, h->d_flags, which); ++g_launch_count;
}

void launch_zero_kb(msgfem* h, int which) {
  dim3 grid(256, h->N);
  k_zero_kb<<<grid, 256, 0, h->stream>>>(h->d_sub, h->d_flags, which, 0); ++g_launch_count;
}

void launch_rr_krylov(msgfem* h, const int* d_m, const int* d_nw) {
  static bool attr = false;
  const int smem = 2 * MQ * (MQ + 1) * (int)sizeof(double);
  if (!attr) {
    cudaFuncSetAttribute(k_rr_krylov, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  k_rr_krylov<<<h->N, 256, smem, h->stream>>>(h->d_sub, h->d_flags, d_m, d_nw); ++g_launch_count;
}

void launch_ritz(msgfem* h, const int* d_m, const int* d_nw, int scale, bool masked, int src, int dst) {
  dim3 grid(std::max(1, (3 * max_nnode_k(h) + 8 * 16 - 1) / (8 * 16)), h->N);
  k_ritz<<<grid, 256, 0, h->stream>>>(h->d_sub, masked ? h->d_flags : nullptr, d_m, d_nw, scale, src, dst);
  ++g_launch_count;
}

void launch_zero_h(msgfem* h) {
  k_zero_h<<<h->N, 256, 0, h->stream>>>(h->d_sub, h->d_flags);
  ++g_launch_count;
}

// Thick restart: QB = [Ritz vectors (PHI) | W], NQ = [their N products (CW) | N W (ZB)]
void launch_restart(msgfem* h, int m, int k) {
  dim3 grid(256, h->N);
  k_restart_basis<<<grid, 256, 0, h->stream>>>(h->d_sub, h->d_flags, k, MV_PHI, MV_WB, MV_QB); ++g_launch_count;
  k_restart_basis<<<grid, 256, 0, h->stream>>>(h->d_sub, h->d_flags, k, MV_CW, MV_ZB, MV_NQ); ++g_launch_count;
  k_restart_h<<<h->N, 256, 0, h->stream>>>(h->d_sub, h->d_flags, m, k); ++g_launch_count;
}
