// Kernels of the subspace iteration on [nfull][PST] multivectors: matrix-free
// stencil products (K, and B = D_mu K D_mu of Eq. algebraicAharmonic), block
// inner products, the small Rayleigh-Ritz eigenproblem, rotations, rigid-body
// modes and masks.  All FP64.
#include "internal.h"

#include <cstdio>

namespace {

// y = alpha * [D_mu] K [D_mu] x, one warp per node, lane = column.
// mode bit 0: scale x by mu (pre), bit 1: scale y by mu (post).
__global__ void __launch_bounds__(256)
k_stencil_apply(const SubDev* __restrict__ subs, const int* __restrict__ active, int src, int dst,
                int mode, double alpha) {
  const int sidx = blockIdx.y;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  const int node = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (node >= s.nnode) return;
  const double* x = mv_ptr(s, src);
  double* y = mv_ptr(s, dst);
  const int k = node / s.npl, q = node % s.npl;
  const int qi = q / s.nyn, qj = q % s.nyn;
  const double* st = s.stencil + (size_t)node * 243;
  double y0 = 0.0, y1 = 0.0, y2 = 0.0;
  for (int slot = 0; slot < 27; ++slot) {
    const int di = slot / 9 - 1, dj = (slot / 3) % 3 - 1, dk = slot % 3 - 1;
    const int ni = qi + di, nj = qj + dj, nk = k + dk;
    if (ni < 0 || ni >= s.nxn || nj < 0 || nj >= s.nyn || nk < 0 || nk >= s.nzn) continue;
    const int nb = nk * s.npl + ni * s.nyn + nj;
    const double sc = (mode & 1) ? s.mu[nb] : 1.0;
    const double* xr = x + (size_t)nb * 3 * PST + lane;
    const double x0 = sc * xr[0], x1 = sc * xr[PST], x2 = sc * xr[2 * PST];
    const double* c = st + slot * 9;
    y0 = fma(c[0], x0, fma(c[1], x1, fma(c[2], x2, y0)));
    y1 = fma(c[3], x0, fma(c[4], x1, fma(c[5], x2, y1)));
    y2 = fma(c[6], x0, fma(c[7], x1, fma(c[8], x2, y2)));
  }
  const double post = alpha * ((mode & 2) ? s.mu[node] : 1.0);
  double* yr = y + (size_t)node * 3 * PST + lane;
  yr[0] = post * y0;
  yr[PST] = post * y1;
  yr[2 * PST] = post * y2;
}

constexpr int GRAM_ROWS = 512;

// Partial Gram sums G = X^T Y over row chunks; thread owns G[a][b..b+3].
__global__ void __launch_bounds__(256)
k_gram_partial(const SubDev* __restrict__ subs, const int* __restrict__ active, int wx, int wy,
               double* __restrict__ part, int nchunk) {
  const int sidx = blockIdx.y;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  const int r0 = blockIdx.x * GRAM_ROWS;
  double* out = part + ((size_t)sidx * nchunk + blockIdx.x) * PST * PST;
  const int tid = threadIdx.x, a = tid >> 3, b = (tid & 7) * 4;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  if (r0 < s.nfull) {
    __shared__ double Xs[32][PST];
    __shared__ double Ys[32][PST];
    const double* X = mv_ptr(s, wx);
    const double* Yv = mv_ptr(s, wy);
    const int r1 = min(r0 + GRAM_ROWS, s.nfull);
    for (int rb = r0; rb < r1; rb += 32) {
      for (int e = tid; e < 32 * PST; e += 256) {
        const int rr = rb + e / PST;
        Xs[e / PST][e % PST] = rr < r1 ? X[(size_t)rr * PST + e % PST] : 0.0;
        Ys[e / PST][e % PST] = rr < r1 ? Yv[(size_t)rr * PST + e % PST] : 0.0;
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
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) out[a * PST + b + j] = acc[j];
}

__global__ void k_gram_reduce(const SubDev* __restrict__ subs, const int* __restrict__ active,
                              const double* __restrict__ part, int nchunk, int wg) {
  const int sidx = blockIdx.x;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  const int nc = (s.nfull + GRAM_ROWS - 1) / GRAM_ROWS;
  double* G = gm_ptr(s, wg);
  for (int e = threadIdx.x; e < PST * PST; e += blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < nc; ++c) acc += part[((size_t)sidx * nchunk + c) * PST * PST + e];
    G[e] = acc;
  }
}

// X <- X Y (first ncols columns of Y used, result columns ncols.. zero),
// one warp per row, in place.
__global__ void __launch_bounds__(256)
k_rotate(const SubDev* __restrict__ subs, const int* __restrict__ active, int which, int wy, int ncols) {
  const int sidx = blockIdx.y;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  __shared__ double Ys[PST][PST];
  const double* Y = gm_ptr(s, wy);
  for (int e = threadIdx.x; e < PST * PST; e += 256) Ys[e / PST][e % PST] = Y[e];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  double* X = mv_ptr(s, which);
  for (int row = blockIdx.x * 8 + (threadIdx.x >> 5); row < s.nfull; row += gridDim.x * 8) {
    const double xv = X[(size_t)row * PST + lane];
    double acc = 0.0;
    for (int k = 0; k < ncols; ++k) acc = fma(__shfl_sync(0xffffffffu, xv, k), Ys[k][lane], acc);
    X[(size_t)row * PST + lane] = lane < ncols ? acc : 0.0;
  }
}

// out <- out - R C with C = G[0:nr][:] (rows 0..nr-1 of a PST x PST matrix).
__global__ void __launch_bounds__(256)
k_sub_rc(const SubDev* __restrict__ subs, const int* __restrict__ active, int wout, int wr, int wc, int nr) {
  const int sidx = blockIdx.y;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  if (!s.floating) return;
  __shared__ double Cs[8][PST];
  const double* C = gm_ptr(s, wc);
  for (int e = threadIdx.x; e < nr * PST; e += 256) Cs[e / PST][e % PST] = C[e];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  double* O = mv_ptr(s, wout);
  const double* R = mv_ptr(s, wr);
  for (int row = blockIdx.x * 8 + (threadIdx.x >> 5); row < s.nfull; row += gridDim.x * 8) {
    const double rv = R[(size_t)row * PST + lane];
    double acc = O[(size_t)row * PST + lane];
    for (int k = 0; k < nr; ++k) acc = fma(-__shfl_sync(0xffffffffu, rv, k), Cs[k][lane], acc);
    O[(size_t)row * PST + lane] = acc;
  }
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Start block: uniform(-1, 1) from a counter-based generator on B2 rows,
// columns < p; zero elsewhere.
__global__ void k_random_b2(const SubDev* __restrict__ subs, int which, int p, unsigned long long seed) {
  const int sidx = blockIdx.y;
  const SubDev& s = subs[sidx];
  double* X = mv_ptr(s, which);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)s.nfull * PST;
       e += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / PST), col = (int)(e % PST);
    const int q = (row / 3) % s.npl;
    double v = 0.0;
    if (col < p && s.cls[q] == 2) {
      const uint64_t key = splitmix64(seed ^ splitmix64(((uint64_t)sidx << 40) ^ ((uint64_t)row << 8) ^ col));
      v = (double)(key >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
    X[e] = v;
  }
}

// Zero rows whose node class c has bit c of keep clear.
__global__ void k_mask_rows(const SubDev* __restrict__ subs, const int* __restrict__ active, int which, int keep) {
  const int sidx = blockIdx.y;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  double* X = mv_ptr(s, which);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)s.nfull * PST;
       e += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(e / PST / 3) % s.npl;
    if (!((keep >> s.cls[q]) & 1)) X[e] = 0.0;
  }
}

__global__ void k_zero_pins(const SubDev* __restrict__ subs, int which) {
  const SubDev& s = subs[blockIdx.x];
  if (!s.floating) return;
  double* X = mv_ptr(s, which);
  const int i = threadIdx.x / PST, c = threadIdx.x % PST;
  if (i < 6 && s.pin[i] >= 0) X[(size_t)s.pin[i] * PST + c] = 0.0;
}

// dst[:, dcol] = sign * (src vector or multivector column)
__global__ void k_copy_col(const SubDev* __restrict__ subs, int wsrc, int scol, int wdst, int dcol, double sign) {
  const SubDev& s = subs[blockIdx.y];
  const double* src;
  int sstride;
  if (wsrc == -1) { src = s.bload; sstride = 1; scol = 0; }
  else if (wsrc == -2) { src = s.psi; sstride = 1; scol = 0; }
  else { src = mv_ptr(s, wsrc); sstride = PST; }
  double* dst;
  int dstride;
  if (wdst == -2) { dst = s.psi; dstride = 1; dcol = 0; }
  else { dst = mv_ptr(s, wdst); dstride = PST; }
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < s.nfull; r += gridDim.x * blockDim.x)
    dst[(size_t)r * dstride + dcol] = sign * src[(size_t)r * sstride + scol];
}

__global__ void k_copy_mv(const SubDev* __restrict__ subs, const int* __restrict__ active, int wsrc, int wdst) {
  const int sidx = blockIdx.y;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  const double* a = mv_ptr(s, wsrc);
  double* b = mv_ptr(s, wdst);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)s.nfull * PST;
       e += (size_t)gridDim.x * blockDim.x)
    b[e] = a[e];
}

// Rigid-body modes of Omega* (floating subdomains): translations and
// rotations about the middle of two opposite corners of the node box, in
// columns 0..5.  Node coordinates come from xyz (general mesh) or the box.
__device__ __forceinline__ void node_pos(const double* xyz, int NY, int NZ, double hx, double hy, double hz, int i,
                                         int j, int k, double P[3]) {
  if (xyz != nullptr) {
    const size_t n = ((size_t)i * (NY + 1) + j) * (NZ + 1) + k;
    P[0] = xyz[3 * n]; P[1] = xyz[3 * n + 1]; P[2] = xyz[3 * n + 2];
  } else {
    P[0] = i * hx; P[1] = j * hy; P[2] = k * hz;
  }
}

__global__ void k_rigid(const SubDev* __restrict__ subs, double hx, double hy, double hz,
                        const double* __restrict__ xyz, int NY, int NZ) {
  const SubDev& s = subs[blockIdx.y];
  if (!s.floating) return;
  double P0[3], P1[3];
  node_pos(xyz, NY, NZ, hx, hy, hz, s.I0, s.J0, 0, P0);
  node_pos(xyz, NY, NZ, hx, hy, hz, s.I1, s.J1, s.nzn - 1, P1);
  const double cx = 0.5 * (P0[0] + P1[0]), cy = 0.5 * (P0[1] + P1[1]), cz = 0.5 * (P0[2] + P1[2]);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)s.nfull * PST;
       e += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / PST), col = (int)(e % PST);
    const int node = row / 3, comp = row % 3;
    const int k = node / s.npl, q = node % s.npl;
    double P[3];
    node_pos(xyz, NY, NZ, hx, hy, hz, s.I0 + q / s.nyn, s.J0 + q % s.nyn, k, P);
    const double x = P[0] - cx, y = P[1] - cy, z = P[2] - cz;
    double v = 0.0;
    if (col < 3) v = (comp == col) ? 1.0 : 0.0;
    else if (col == 3) v = comp == 1 ? -z : (comp == 2 ? y : 0.0);    // e_x x r
    else if (col == 4) v = comp == 0 ? z : (comp == 2 ? -x : 0.0);    // e_y x r
    else if (col == 5) v = comp == 0 ? -y : (comp == 1 ? x : 0.0);    // e_z x r
    s.R[e] = v;
  }
}

// Y = L^{-T} with L L^T = G[0:n, 0:n] (G scaled to unit diagonal first);
// columns >= n of Y are zero.  One block per subdomain.  If drop_last and
// the last pivot is tiny relative to its diagonal, that column is dropped
// (reported through s.status[2] = n - 1).
__global__ void k_chol_inv_small(const SubDev* __restrict__ subs, const int* __restrict__ active, int wg,
                                 const int* __restrict__ ncol_sub, int nfixed, int drop_last) {
  const int sidx = blockIdx.x;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  const int n = ncol_sub ? ncol_sub[sidx] : nfixed;
  if (n <= 0) return;
  __shared__ double L[PST][PST + 1];
  __shared__ double U[PST][PST + 1];
  __shared__ double d[PST];
  __shared__ int nn;
  const double* G = gm_ptr(s, wg);
  const int tid = threadIdx.x;
  for (int e = tid; e < PST * PST; e += blockDim.x) {
    const int r = e / PST, c = e % PST;
    L[r][c] = (r < n && c < n) ? G[e] : 0.0;
    U[r][c] = 0.0;
  }
  if (tid == 0) nn = n;
  __syncthreads();
  if (tid < n) d[tid] = L[tid][tid] > 0.0 ? 1.0 / sqrt(L[tid][tid]) : 0.0;
  __syncthreads();
  for (int e = tid; e < n * n; e += blockDim.x) L[e / n][e % n] *= d[e / n] * d[e % n];
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      double v = L[j][j];
      if (drop_last && j == n - 1 && !(v > 1e-20)) { nn = n - 1; v = 1.0; }
      L[j][j] = sqrt(v > 1e-300 ? v : 1e-300);
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < n; i += blockDim.x) L[i][j] /= L[j][j];
    __syncthreads();
    for (int e = tid; e < n * n; e += blockDim.x) {
      const int i = e / n, k = e % n;
      if (i > j && k > j && k <= i) L[i][k] -= L[i][j] * L[k][j];
    }
    __syncthreads();
  }
  // U = L^{-T}: solve L^T U = I column by column (thread per column)
  if (tid < n) {
    const int c = tid;
    for (int i = n - 1; i >= 0; --i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int m = i + 1; m < n; ++m) v -= L[m][i] * U[m][c];
      U[i][c] = v / L[i][i];
    }
  }
  __syncthreads();
  double* Y = s.Y;
  const int nk = nn;
  for (int e = tid; e < PST * PST; e += blockDim.x) {
    const int r = e / PST, c = e % PST;
    Y[e] = (r < nk && c < nk) ? d[r] * U[r][c] : 0.0;
  }
  if (tid == 0) s.status[2] = nk;
}

// Rayleigh-Ritz on the p x p pencil (GK = Phi^T K Phi, GT = Phi^T B Phi):
// D GT D = L L^T, C = L^{-1} D GK D L^{-T}, Jacobi eigen-decomposition
// C V = V diag(theta), Y = D L^{-T} V sorted by ascending theta.
__global__ void __launch_bounds__(256)
k_small_eig(const SubDev* __restrict__ subs, const int* __restrict__ active, int p) {
  const int sidx = blockIdx.x;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  __shared__ double T[PST][PST + 1], C[PST][PST + 1], V[PST][PST + 1];
  __shared__ double d[PST], cs[PST / 2], sn[PST / 2];
  __shared__ int perm[PST], pi_[PST / 2], pj_[PST / 2];
  __shared__ double offn;
  const int tid = threadIdx.x;
  const double* GT = s.G1;
  const double* GK = s.G2;
  for (int e = tid; e < PST * PST; e += 256) {
    const int r = e / PST, c = e % PST;
    T[r][c] = (r < p && c < p) ? 0.5 * (GT[r * PST + c] + GT[c * PST + r]) : 0.0;
    C[r][c] = (r < p && c < p) ? 0.5 * (GK[r * PST + c] + GK[c * PST + r]) : 0.0;
    V[r][c] = 0.0;
  }
  __syncthreads();
  if (tid < p) d[tid] = T[tid][tid] > 0.0 ? 1.0 / sqrt(T[tid][tid]) : 1.0;
  __syncthreads();
  for (int e = tid; e < p * p; e += 256) {
    const int r = e / p, c = e % p;
    T[r][c] *= d[r] * d[c];
    C[r][c] *= d[r] * d[c];
  }
  __syncthreads();
  // Cholesky of T (lower, in place)
  for (int j = 0; j < p; ++j) {
    if (tid == 0) {
      const double v = T[j][j];
      T[j][j] = sqrt(v > 1e-28 ? v : 1e-28);
      if (!(v > 1e-28)) s.status[1] = 1;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < p; i += 256) T[i][j] /= T[j][j];
    __syncthreads();
    for (int e = tid; e < p * p; e += 256) {
      const int i = e / p, k = e % p;
      if (i > j && k > j && k <= i) T[i][k] -= T[i][j] * T[k][j];
    }
    __syncthreads();
  }
  // C <- L^{-1} C (columns independent), then C <- C L^{-T} (rows independent)
  if (tid < p) {
    const int c = tid;
    for (int i = 0; i < p; ++i) {
      double v = C[i][c];
      for (int m = 0; m < i; ++m) v -= T[i][m] * C[m][c];
      C[i][c] = v / T[i][i];
    }
  }
  __syncthreads();
  if (tid < p) {
    const int r = tid;
    for (int i = 0; i < p; ++i) {
      double v = C[r][i];
      for (int m = 0; m < i; ++m) v -= T[i][m] * C[r][m];
      C[r][i] = v / T[i][i];
    }
  }
  __syncthreads();
  for (int e = tid; e < p * p; e += 256) {
    const int r = e / p, c = e % p;
    if (r < c) {
      const double a = 0.5 * (C[r][c] + C[c][r]);
      C[r][c] = a;
      C[c][r] = a;
    }
    V[r][c] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  // parallel cyclic Jacobi (round-robin pairing over an even number of slots)
  const int m = (p + 1) & ~1;
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (tid == 0) {
      double off = 0.0, tot = 0.0;
      for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j) {
          const double v = C[i][j] * C[i][j];
          tot += v;
          if (i != j) off += v;
        }
      offn = (off <= 1e-30 * tot) ? 0.0 : 1.0;
    }
    __syncthreads();
    if (offn == 0.0) break;
    for (int round = 0; round < m - 1; ++round) {
      if (tid < m / 2) {
        // slots: 0 fixed, others rotate
        int a = (tid == 0) ? 0 : ((round + tid - 1) % (m - 1)) + 1;
        int b = ((round + m - 2 - tid) % (m - 1)) + 1;
        if (a > b) { const int t = a; a = b; b = t; }
        pi_[tid] = a;
        pj_[tid] = b;
        double c = 1.0, sv = 0.0;
        if (b < p && a < p) {
          const double apq = C[a][b];
          if (fabs(apq) > 1e-300) {
            const double app = C[a][a], aqq = C[b][b];
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            sv = t * c;
          }
        }
        cs[tid] = c;
        sn[tid] = sv;
      }
      __syncthreads();
      // rows: C <- J^T C
      for (int e = tid; e < (m / 2) * p; e += 256) {
        const int k = e / p, col = e % p;
        const int a = pi_[k], b = pj_[k];
        if (b >= p) continue;
        const double c = cs[k], sv = sn[k];
        const double x = C[a][col], y = C[b][col];
        C[a][col] = c * x - sv * y;
        C[b][col] = sv * x + c * y;
      }
      __syncthreads();
      // columns: C <- C J, V <- V J
      for (int e = tid; e < (m / 2) * p; e += 256) {
        const int k = e / p, row = e % p;
        const int a = pi_[k], b = pj_[k];
        if (b >= p) continue;
        const double c = cs[k], sv = sn[k];
        const double x = C[row][a], y = C[row][b];
        C[row][a] = c * x - sv * y;
        C[row][b] = sv * x + c * y;
        const double vx = V[row][a], vy = V[row][b];
        V[row][a] = c * vx - sv * vy;
        V[row][b] = sv * vx + c * vy;
      }
      __syncthreads();
    }
  }
  // U = L^{-T} V (back substitution per column)
  if (tid < p) {
    const int c = tid;
    for (int i = p - 1; i >= 0; --i) {
      double v = V[i][c];
      for (int k = i + 1; k < p; ++k) v -= T[k][i] * V[k][c];
      V[i][c] = v / T[i][i];
    }
  }
  if (tid == 0) {
    for (int i = 0; i < p; ++i) perm[i] = i;
    for (int i = 0; i < p; ++i)
      for (int j = i + 1; j < p; ++j)
        if (C[perm[j]][perm[j]] < C[perm[i]][perm[i]]) { const int t = perm[i]; perm[i] = perm[j]; perm[j] = t; }
  }
  __syncthreads();
  for (int e = tid; e < PST * PST; e += 256) {
    const int r = e / PST, c = e % PST;
    s.Y[e] = (r < p && c < p) ? d[r] * V[r][perm[c]] : 0.0;
  }
  if (tid < PST) s.theta[tid] = tid < p ? C[perm[tid]][perm[tid]] : 0.0;
}

// Per-column sums over rows whose node class is 2 (B2):
// out[0][c] = ||A_c + alpha_c B_c||^2, out[1][c] = ||A_c||^2, out[2][c] = ||B_c||^2,
// alpha_c = theta[c].  Partial per chunk; reduced by k_colnorm_reduce.
__global__ void __launch_bounds__(256)
k_colnorm_partial(const SubDev* __restrict__ subs, const int* __restrict__ active, int wa, int wb,
                  double* __restrict__ part, int nchunk, int keep, double sgn) {
  const int sidx = blockIdx.y;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __shared__ double red[8][3][32];
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  const int r0 = blockIdx.x * GRAM_ROWS;
  const double* A = mv_ptr(s, wa);
  const double* B = mv_ptr(s, wb);
  const double th = s.theta[lane];
  for (int r = r0 + w; r < min(r0 + GRAM_ROWS, s.nfull); r += 8) {
    const int q = (r / 3) % s.npl;
    if (!((keep >> s.cls[q]) & 1)) continue;
    const double a = A[(size_t)r * PST + lane], b = B[(size_t)r * PST + lane];
    const double v = a + sgn * th * b;
    a0 += v * v;
    a1 += a * a;
    a2 += b * b;
  }
  red[w][0][lane] = a0;
  red[w][1][lane] = a1;
  red[w][2][lane] = a2;
  __syncthreads();
  if (w < 3) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i][w][lane];
    part[(((size_t)sidx * nchunk + blockIdx.x) * 3 + w) * 32 + lane] = t;
  }
}

__global__ void k_colnorm_reduce(const SubDev* __restrict__ subs, const int* __restrict__ active,
                                 const double* __restrict__ part, int nchunk, int p) {
  const int sidx = blockIdx.x;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  const int nc = (s.nfull + GRAM_ROWS - 1) / GRAM_ROWS;
  const int lane = threadIdx.x;
  if (lane >= 32) return;
  double t[3] = {0.0, 0.0, 0.0};
  for (int c = 0; c < nc; ++c)
    for (int w = 0; w < 3; ++w) t[w] += part[(((size_t)sidx * nchunk + c) * 3 + w) * 32 + lane];
  const double th = s.theta[lane];
  const double den = sqrt(t[1]) + fabs(th) * sqrt(t[2]);
  s.resid[lane] = (lane < p && den > 0.0) ? sqrt(t[0]) / den : 0.0;
}

// D = diag(theta) X - Y on columns < p (zero elsewhere).
__global__ void k_theta_axpy(const SubDev* __restrict__ subs, const int* __restrict__ active, int wx, int wy,
                             int wd, int p) {
  const int sidx = blockIdx.y;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  const double* X = mv_ptr(s, wx);
  const double* Yv = mv_ptr(s, wy);
  double* D = mv_ptr(s, wd);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)s.nfull * PST;
       e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % PST);
    D[e] = c < p ? s.theta[c] * X[e] - Yv[e] : 0.0;
  }
}

__global__ void k_scale_rows_mu(const SubDev* __restrict__ subs, int which) {
  const SubDev& s = subs[blockIdx.y];
  double* X = mv_ptr(s, which);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)s.nfull * PST;
       e += (size_t)gridDim.x * blockDim.x)
    X[e] *= s.mu[e / PST / 3];
}

}  // namespace

static const int* act(msgfem* h) { return h->d_flags; }

static int max_nnode(msgfem* h) {
  int m = 0;
  for (const auto& s : h->sub) m = std::max(m, s.nnode);
  return m;
}

void launch_stencil_apply(msgfem* h, int src, int dst, int mode, double alpha) {
  dim3 grid((max_nnode(h) + 7) / 8, h->N);
  k_stencil_apply<<<grid, 256, 0, h->stream>>>(h->d_sub, act(h), src, dst, mode, alpha); ++g_launch_count;
}

void launch_gram(msgfem* h, int wx, int wy, int wg) {
  const int nchunk = (3 * max_nnode(h) + GRAM_ROWS - 1) / GRAM_ROWS;
  dim3 grid(nchunk, h->N);
  k_gram_partial<<<grid, 256, 0, h->stream>>>(h->d_sub, act(h), wx, wy, h->d_gram_part, nchunk); ++g_launch_count;
  k_gram_reduce<<<h->N, 256, 0, h->stream>>>(h->d_sub, act(h), h->d_gram_part, nchunk, wg); ++g_launch_count;
}

void launch_small_eig(msgfem* h, int p) { k_small_eig<<<h->N, 256, 0, h->stream>>>(h->d_sub, act(h), p); ++g_launch_count; }

void launch_rotate(msgfem* h, int which, int wy, int ncols) {
  dim3 grid(std::max(1, (3 * max_nnode(h) + 8 * 16 - 1) / (8 * 16)), h->N);
  k_rotate<<<grid, 256, 0, h->stream>>>(h->d_sub, act(h), which, wy, ncols); ++g_launch_count;
}

void launch_sub_rc(msgfem* h, int wout, int wr, int wc, int nr) {
  dim3 grid(std::max(1, (3 * max_nnode(h) + 8 * 16 - 1) / (8 * 16)), h->N);
  k_sub_rc<<<grid, 256, 0, h->stream>>>(h->d_sub, act(h), wout, wr, wc, nr); ++g_launch_count;
}

void launch_random_b2(msgfem* h, int which, int p, unsigned long long seed) {
  dim3 grid(256, h->N);
  k_random_b2<<<grid, 256, 0, h->stream>>>(h->d_sub, which, p, seed); ++g_launch_count;
}

void launch_mask_rows(msgfem* h, int which, int keep) {
  dim3 grid(256, h->N);
  k_mask_rows<<<grid, 256, 0, h->stream>>>(h->d_sub, act(h), which, keep); ++g_launch_count;
}

void launch_zero_pins(msgfem* h, int which) { k_zero_pins<<<h->N, 6 * PST, 0, h->stream>>>(h->d_sub, which); ++g_launch_count; }

void launch_copy_col(msgfem* h, int wsrc, int scol, int wdst, int dcol, double sign) {
  dim3 grid(64, h->N);
  k_copy_col<<<grid, 256, 0, h->stream>>>(h->d_sub, wsrc, scol, wdst, dcol, sign); ++g_launch_count;
}

void launch_copy_mv(msgfem* h, int wsrc, int wdst) {
  dim3 grid(256, h->N);
  k_copy_mv<<<grid, 256, 0, h->stream>>>(h->d_sub, act(h), wsrc, wdst); ++g_launch_count;
}

void launch_rigid_modes(msgfem* h) {
  dim3 grid(256, h->N);
  k_rigid<<<grid, 256, 0, h->stream>>>(h->d_sub, h->hx, h->hy, h->hz, h->d_xyz, h->NY, h->NZ); ++g_launch_count;
}

void launch_chol_inv_small(msgfem* h, int wg, const int* d_ncols, int nfixed, int drop_last) {
  k_chol_inv_small<<<h->N, 256, 0, h->stream>>>(h->d_sub, act(h), wg, d_ncols, nfixed, drop_last); ++g_launch_count;
}

void launch_colnorms(msgfem* h, int wa, int wb, int p, int keep, double sgn) {
  const int nchunk = (3 * max_nnode(h) + GRAM_ROWS - 1) / GRAM_ROWS;
  dim3 grid(nchunk, h->N);
  k_colnorm_partial<<<grid, 256, 0, h->stream>>>(h->d_sub, act(h), wa, wb, h->d_gram_part, nchunk, keep, sgn);
  ++g_launch_count;
  k_colnorm_reduce<<<h->N, 32, 0, h->stream>>>(h->d_sub, act(h), h->d_gram_part, nchunk, p); ++g_launch_count;
}

void launch_scale_rows_mu(msgfem* h, int which) {
  dim3 grid(256, h->N);
  k_scale_rows_mu<<<grid, 256, 0, h->stream>>>(h->d_sub, which); ++g_launch_count;
}

void launch_theta_axpy(msgfem* h, int wx, int wy, int wd, int p) {
  dim3 grid(256, h->N);
  k_theta_axpy<<<grid, 256, 0, h->stream>>>(h->d_sub, act(h), wx, wy, wd, p); ++g_launch_count;
}

namespace {
// D = X - Y on multivectors of the same stride (rows of all subdomains)
__global__ void k_x_minus_y(const SubDev* __restrict__ subs, const int* __restrict__ active, int wx, int wy,
                            int wd, int stride) {
  const int sidx = blockIdx.y;
  if (active != nullptr && !active[sidx]) return;
  const SubDev& s = subs[sidx];
  const double* X = mv_ptr(s, wx);
  const double* Yv = mv_ptr(s, wy);
  double* D = mv_ptr(s, wd);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)s.nfull * stride;
       e += (size_t)gridDim.x * blockDim.x)
    D[e] = X[e] - Yv[e];
}

// Adaptive iterative refinement of the FP32 solves.  Per active subdomain and
// column, the residual norm of the KB-wide block R over the rows of the DoF
// classes in keep (bit c for class c: B1 and B2 for K, B1 for A11; the rows
// the solve acts on) is compared with a reference norm: the column of the right-hand side
// block Ref, or, when Ref is absent, the residual recorded at step -1.  A
// column is done when its relative residual is below tol or fell by less than
// 10 % since the previous step (the FP64 rounding floor of the residual); a
// subdomain whose columns are all done leaves the remaining refinement steps:
// its active flag is cleared and the caller restores the flags afterwards.
// Columns with a zero reference (unused columns) count as done.
__global__ void __launch_bounds__(256)
k_refine_check(const SubDev* __restrict__ subs, int* __restrict__ flags, int wr, int wref, int keep, int step,
               double tol, double* __restrict__ prev, double* __restrict__ refn) {
  const int sidx = blockIdx.x;
  if (!flags[sidx]) return;
  const SubDev& s = subs[sidx];
  const double* R = mv_ptr(s, wr);
  const double* F = wref >= 0 ? mv_ptr(s, wref) : nullptr;
  // thread t handles column t % KB of rows t / KB, t / KB + 32, ...
  const int c = threadIdx.x % KB;
  double r2 = 0.0, f2 = 0.0;
  for (int row = threadIdx.x / KB; row < s.nfull; row += blockDim.x / KB) {
    if (!((keep >> s.cls[(row / 3) % s.npl]) & 1)) continue;
    const double rv = R[(size_t)row * KB + c];
    r2 += rv * rv;
    if (F) {
      const double fv = F[(size_t)row * KB + c];
      f2 += fv * fv;
    }
  }
  // lanes with equal column are KB apart within a warp
  for (int o = 16; o >= KB; o >>= 1) {
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    f2 += __shfl_xor_sync(0xffffffffu, f2, o);
  }
  __shared__ double sr[8][KB], sf[8][KB];
  if ((threadIdx.x & 31) < KB) {
    sr[threadIdx.x >> 5][c] = r2;
    sf[threadIdx.x >> 5][c] = f2;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double* pv = prev + (size_t)sidx * KB;
  double* rf = refn + (size_t)sidx * KB;
  bool all_done = true;
  for (int cc = 0; cc < KB; ++cc) {
    double rt = 0.0, ft = 0.0;
    for (int w = 0; w < 8; ++w) { rt += sr[w][cc]; ft += sf[w][cc]; }
    const double rn = sqrt(rt);
    if (step < 0) {   // record the reference only
      rf[cc] = rn;
      pv[cc] = rn;
      continue;
    }
    const double ref = F ? sqrt(ft) : rf[cc];
    const bool done = ref == 0.0 || rn <= tol * ref || (step > 0 && rn > 0.9 * pv[cc]);
    pv[cc] = rn;
    all_done = all_done && done;
  }
  if (step >= 0 && all_done) flags[sidx] = 0;
}

// X[:, 0] -= bload (KB-wide block)
__global__ void k_sub_load_kb(const SubDev* __restrict__ subs, const int* __restrict__ active, int which) {
  if (active != nullptr && !active[blockIdx.y]) return;
  const SubDev& s = subs[blockIdx.y];
  double* X = mv_ptr(s, which);
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < s.nfull; r += gridDim.x * blockDim.x)
    X[(size_t)r * KB] -= s.bload[r];
}
}  // namespace

void launch_x_minus_y(msgfem* h, int wx, int wy, int wd, int stride) {
  dim3 grid(256, h->N);
  k_x_minus_y<<<grid, 256, 0, h->stream>>>(h->d_sub, act(h), wx, wy, wd, stride); ++g_launch_count;
}

void launch_refine_check(msgfem* h, int wr, int wref, int keep, int step) {
  launch_refine_check_tol(h, wr, wref, keep, step, REFINE_TOL);
}

void launch_refine_check_tol(msgfem* h, int wr, int wref, int keep, int step, double tol) {
  k_refine_check<<<h->N, 256, 0, h->stream>>>(h->d_sub, h->d_flags, wr, wref, keep, step, tol, h->d_rprev,
                                               h->d_rref);
  ++g_launch_count;
}

namespace {
// d[slot][c] = sum over rows of the DoF classes in `keep` of X[r][c] Y[r][c]
// (KB-wide blocks): COLDOT_CH blocks per active subdomain write partial sums,
// then one thread per (subdomain, column) adds them in a fixed order.
constexpr int COLDOT_CH = 16;

__global__ void __launch_bounds__(256)
k_coldot_kb_partial(const SubDev* __restrict__ subs, const int* __restrict__ flags, int wx, int wy, int keep,
                    double* __restrict__ part) {
  const int sidx = blockIdx.y;
  if (!flags[sidx]) return;
  const SubDev& s = subs[sidx];
  const double* X = mv_ptr(s, wx);
  const double* Y = mv_ptr(s, wy);
  const int per = (s.nfull + COLDOT_CH - 1) / COLDOT_CH;
  const int r0 = blockIdx.x * per, r1 = min(r0 + per, s.nfull);
  const int c = threadIdx.x % KB;
  double acc = 0.0;
  for (int row = r0 + threadIdx.x / KB; row < r1; row += blockDim.x / KB) {
    if (!((keep >> s.cls[(row / 3) % s.npl]) & 1)) continue;
    acc += X[(size_t)row * KB + c] * Y[(size_t)row * KB + c];
  }
  for (int o = 16; o >= KB; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double sa[8][KB];
  if ((threadIdx.x & 31) < KB) sa[threadIdx.x >> 5][c] = acc;
  __syncthreads();
  if (threadIdx.x < KB) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sa[w][threadIdx.x];
    part[((size_t)sidx * COLDOT_CH + blockIdx.x) * KB + threadIdx.x] = t;
  }
}

__global__ void k_coldot_kb_reduce(const int* __restrict__ flags, const double* __restrict__ part,
                                   double* __restrict__ pcg, int slot, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * KB) return;
  const int sidx = i / KB, c = i % KB;
  if (!flags[sidx]) return;
  double t = 0.0;
  for (int b = 0; b < COLDOT_CH; ++b) t += part[((size_t)sidx * COLDOT_CH + b) * KB + c];
  pcg[((size_t)sidx * 4 + slot) * KB + c] = t;
}

// CG updates per column (scalars from d_pcg slots 0: r.z, 1: p.q, 2: new r.z):
//   PCG_STEP: alpha = rz / pq; x += alpha p; r -= alpha q
//   PCG_DIR:  beta = rz_new / rz; p = z + beta p
//   PCG_DIR0: p = z
// A non-positive or non-finite ratio gives a zero step (the column then stalls
// and its refinement check stops it).
__global__ void __launch_bounds__(256)
k_pcg_update(const SubDev* __restrict__ subs, const int* __restrict__ flags, const double* __restrict__ pcg,
             int mode, int wx, int wr, int wz, int wp, int wq) {
  const int sidx = blockIdx.y;
  if (!flags[sidx]) return;
  const SubDev& s = subs[sidx];
  const double* d = pcg + (size_t)sidx * 4 * KB;
  double* X = mv_ptr(s, wx);
  double* R = mv_ptr(s, wr);
  const double* Z = mv_ptr(s, wz);
  double* P = mv_ptr(s, wp);
  const double* Q = mv_ptr(s, wq);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)s.nfull * KB;
       e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % KB);
    if (mode == PCG_STEP) {
      const double rz = d[c], pq = d[KB + c];
      double a = rz / pq;
      if (!(pq > 0.0) || !(rz > 0.0) || !isfinite(a)) a = 0.0;
      X[e] += a * P[e];
      R[e] -= a * Q[e];
    } else if (mode == PCG_DIR) {
      const double rz = d[c], rzn = d[2 * KB + c];
      double b = rzn / rz;
      if (!(rz > 0.0) || !isfinite(b)) b = 0.0;
      P[e] = Z[e] + b * P[e];
    } else {
      P[e] = Z[e];
    }
  }
}

// slot 0 <- slot 2 (r.z of the new residual becomes the current one)
__global__ void k_pcg_shift(const int* __restrict__ flags, double* __restrict__ pcg, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * KB) return;
  const int sidx = i / KB, c = i % KB;
  if (!flags[sidx]) return;
  pcg[(size_t)sidx * 4 * KB + c] = pcg[((size_t)sidx * 4 + 2) * KB + c];
}
}  // namespace

// (partial sums in the Gram scratch: N * COLDOT_CH * KB doubles, far below its size)
void launch_coldot_kb(msgfem* h, int wx, int wy, int keep, int slot) {
  dim3 grid(COLDOT_CH, h->N);
  k_coldot_kb_partial<<<grid, 256, 0, h->stream>>>(h->d_sub, h->d_flags, wx, wy, keep, h->d_gram_part);
  ++g_launch_count;
  k_coldot_kb_reduce<<<(h->N * KB + 255) / 256, 256, 0, h->stream>>>(h->d_flags, h->d_gram_part, h->d_pcg, slot, h->N);
  ++g_launch_count;
}

void launch_pcg_update(msgfem* h, int mode, int wx, int wr, int wz, int wp, int wq) {
  dim3 grid(64, h->N);
  k_pcg_update<<<grid, 256, 0, h->stream>>>(h->d_sub, h->d_flags, h->d_pcg, mode, wx, wr, wz, wp, wq);
  ++g_launch_count;
  if (mode == PCG_DIR) {
    k_pcg_shift<<<(h->N * KB + 255) / 256, 256, 0, h->stream>>>(h->d_flags, h->d_pcg, h->N);
    ++g_launch_count;
  }
}

void launch_sub_load_kb(msgfem* h, int which) {
  dim3 grid(64, h->N);
  k_sub_load_kb<<<grid, 256, 0, h->stream>>>(h->d_sub, h->d_flags, which); ++g_launch_count;
}
