// Dense tile kernels behind the layer-block Cholesky factorisation and the
// block triangular solves of the local shift-invert operator, for FP64 (plain
// path) and FP32 (mixed path) block storage.
//
// The factorisation of a block-tridiagonal SPD matrix (z-layer blocks, see
// internal.h) is expressed as a static list of 64x64 tile tasks grouped into
// steps (built once by the host scheduler in setup.cpp):
//   SYRK    D_l -= L_{l,l-1} L_{l,l-1}^T
//   POTRF   L_kk = chol(D_kk), Li_kk = L_kk^{-1}          (one CTA per tile)
//   TRMM    L_ik = D_ik Li_kk^T   (panel below, and the E_l panel)
//   UPDATE  D_ij -= L_ik L_jk^T   (trailing tiles of the panel)
//   TRTRI   Linv_ik = -Li_ii sum_m L_im Linv_mk             (block inverse)
// POTRF and GEMM tasks share one kernel, so independent work of different
// phases (the block inverse of layer l and the factorisation of layer l + 1)
// can fill the same launch.  FP64 arithmetic runs at ~2 DFMA/clk/SM on this
// part, so the FP64 kernels are bound by the FP64 pipe and only need enough
// independent tasks in flight.  The FP32 factorisation's tile Cholesky runs
// in FP64 by default and in FP32 on request (msgfem_options.tile_chol): in
// FP64 one 64 x 64 tile takes ~90k DFMA on one SM, and every tile column of
// every layer waits for one.
#include "internal.h"

#include <cooperative_groups.h>
#include <type_traits>

#include "tc_gemm.cuh"

namespace cg = cooperative_groups;

// compile-time tunables of the streaming solve
#ifndef SOLVE_CLUSTER
#define SOLVE_CLUSTER 1   // CTAs (one cluster) per 64-row task, splitting its inner dimension
#endif
#ifndef SOLVE_PDL
#define SOLVE_PDL 1       // solve steps use programmatic dependent launch
#endif
#ifndef SOLVE_ASYNC
#define SOLVE_ASYNC 1     // FP32 solves through the cp.async pipeline (k_solve_async)
#endif
#ifndef SOLVE_MIN_BLOCKS
#define SOLVE_MIN_BLOCKS 2   // resident CTAs per SM the register budget is sized for
#endif
#ifndef SOLVE_ROWS_F32
#define SOLVE_ROWS_F32 4  // rows per warp pass of the FP32 plain-A variant (4 or 8)
#endif

namespace {

constexpr int KC = 16;   // K chunk of the tile GEMM
constexpr int TILE_SMEM = 2 * 64 * 65 * (int)sizeof(double);   // dynamic shared memory per CTA

// Global loads of tile operands: plain, or (L2) at the L2 only, for operands
// that other SMs write during the same launch (the persistent factorisation).
template <bool L2, typename T>
__device__ __forceinline__ T ldg_op(const T* p) {
  if constexpr (L2) return __ldcg(p);
  else return *p;
}

// Cholesky and inverse of one 64x64 SPD tile in shared memory, computed in Tc
// (FP64; FP32 on request in the mixed path).  L occupies the lower triangle of
// A; X = L^{-1} is kept transposed in the strict upper triangle shifted by one
// column (X[i][c] at A[c][i + 1], the pad column).  The tile Cholesky sits on
// the critical path of every tile column of the factorisation, and FP64 runs
// at 2 DFMA/clk/SM here, so the dependent chains are kept short: one
// reciprocal square root per pivot (the column is scaled by it), the trailing
// update on a 16 x 16 thread grid over the lower triangle, and the inverse by
// forward substitution per column with four lanes per column (partial sums
// over m mod 4, joined by two shuffles) and the pivots' reciprocals.
template <typename T, typename Tc = double, bool L2 = false>
__device__ void tile_potrf_inv(const TileTaskT<T>& t, Tc (*A)[65], int* notspd) {
  __shared__ int bad;
  __shared__ Tc rdiag[64];
  const int tid = threadIdx.x;
  const Tc zero = (Tc)0, tiny = (Tc)(sizeof(Tc) == 4 ? 1e-30 : 1e-300);
  if (tid == 0) bad = 0;
  for (int e = tid; e < 64 * 64; e += 256) {
    const int r = e >> 6, c = e & 63;
    A[r][c] = (c <= r) ? (Tc)ldg_op<L2>(t.C + (size_t)r * t.ldc + c) : zero;
  }
  if (tid < 64) A[tid][64] = zero;
  __syncthreads();
  for (int j = 0; j < 64; ++j) {
    if (tid == 0) {
      Tc d = A[j][j];
      if (!(d > zero)) { bad = 1; d = tiny; }
      const Tc r = rsqrt(d);
      A[j][j] = d * r;
      rdiag[j] = r;
    }
    __syncthreads();
    const Tc rj = rdiag[j];
    for (int i = j + 1 + tid; i < 64; i += 256) A[i][j] *= rj;
    __syncthreads();
    for (int ii = j + 1 + (tid >> 4); ii < 64; ii += 16) {
      const Tc lij = A[ii][j];
      for (int kk = j + 1 + (tid & 15); kk <= ii; kk += 16) A[ii][kk] = fma(-lij, A[kk][j], A[ii][kk]);
    }
    __syncthreads();
  }
  // X = L^{-1} by columns: X[i][c] = -(sum_{m=c}^{i-1} L[i][m] X[m][c]) / L[i][i];
  // lanes 4c .. 4c + 3 own column c (a warp holds 8 columns and runs the rows
  // from its first column on, so that every lane meets the shuffles)
  if (tid < 64) rdiag[tid] = (Tc)1 / A[tid][tid];
  __syncthreads();
  {
    const int c = tid >> 2, q = tid & 3, c0 = (tid >> 5) * 8;
    if (q == 0) A[c][c + 1] = rdiag[c];
    __syncwarp();
    for (int i = c0 + 1; i < 64; ++i) {
      Tc s = zero;
      for (int m = c + q; m < i; m += 4) s = fma(A[i][m], A[c][m + 1], s);
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      if (q == 0 && i > c) A[c][i + 1] = -s * rdiag[i];
      __syncwarp();
    }
  }
  __syncthreads();
  T* Li = const_cast<T*>(t.P);
  for (int e = tid; e < 64 * 64; e += 256) {
    const int r = e >> 6, c = e & 63;
    t.C[(size_t)r * t.ldc + c] = (T)((c <= r) ? A[r][c] : zero);
    Li[(size_t)r * t.ldc + c] = (T)((c <= r) ? A[c][r + 1] : zero);
  }
  if (tid == 0 && bad && notspd != nullptr) atomicExch(&notspd[t.sub >= 0 ? t.sub : 0], 1);
}

// The products of one K chunk: 4 x 4 outputs per thread (rows ty + 16 i,
// columns tx + 16 j), output column groups j >= JLO (the others meet only
// zeros of a triangular B in this chunk); with SYM only the blocks j <= i.
template <typename T, int JLO, bool SYM>
__device__ __forceinline__ void tile_chunk(T (*As)[65], T (*Bs)[65], T (&acc)[4][4], int tx, int ty) {
#pragma unroll
  for (int kk = 0; kk < KC; ++kk) {
    T a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
    for (int j = JLO; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = JLO; j < 4; ++j)
        if (!SYM || j <= i) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
}

// One tile task per CTA: a 64x64 GEMM tile (4x4 outputs per thread, operands
// staged through shared memory in K chunks of 16) or a tile POTRF.
template <typename T>
__global__ void __launch_bounds__(256)
k_tile_task(const TileTaskT<T>* __restrict__ tasks, const int* __restrict__ active, int* __restrict__ notspd) {
  const TileTaskT<T> t = tasks[blockIdx.x];
  if (t.sub >= 0 && active != nullptr && !active[t.sub]) return;
  extern __shared__ double smem_d[];
  if (t.flags & G_POTRF) {
    tile_potrf_inv(t, reinterpret_cast<double (*)[65]>(smem_d), notspd);
    return;
  }
  T* smem = reinterpret_cast<T*>(smem_d);
  T (*As)[65] = reinterpret_cast<T (*)[65]>(smem);                 // [KC][65]: As[k][m]
  T (*Bs)[65] = reinterpret_cast<T (*)[65]>(smem + KC * 65);      // [KC][65]: Bs[k][n]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
  const bool transB = (t.flags & G_TRANSB) != 0;
  for (int k0 = 0; k0 < t.K; k0 += KC) {
    {
      const int r = tid >> 2, c = (tid & 3) * 4;
      const T* a = t.A + (size_t)r * t.lda + k0 + c;
#pragma unroll
      for (int i = 0; i < 4; ++i) As[c + i][r] = a[i];
    }
    if (transB) {
      const int n = tid >> 2, c = (tid & 3) * 4;
      const T* b = t.B + (size_t)n * t.ldb + k0 + c;
#pragma unroll
      for (int i = 0; i < 4; ++i) Bs[c + i][n] = b[i];
    } else {
      const int k = tid >> 4, n = (tid & 15) * 4;
      const T* b = t.B + (size_t)(k0 + k) * t.ldb + n;
#pragma unroll
      for (int i = 0; i < 4; ++i) Bs[k][n + i] = b[i];
    }
    __syncthreads();
    // triangular B (G_TRIB): in the chunk at k0 the output columns below k0,
    // tx + 16 j with j < k0 / 16, meet only zeros of B; those products are skipped
    // and a diagonal output tile (G_SYMC) forms only its blocks on or below the diagonal
    const int jlo = (t.flags & G_TRIB) ? (k0 >> 4) : 0;
    if (t.flags & G_SYMC) tile_chunk<T, 0, true>(As, Bs, acc, tx, ty);
    else if (jlo == 0) tile_chunk<T, 0, false>(As, Bs, acc, tx, ty);
    else if (jlo == 1) tile_chunk<T, 1, false>(As, Bs, acc, tx, ty);
    else if (jlo == 2) tile_chunk<T, 2, false>(As, Bs, acc, tx, ty);
    else tile_chunk<T, 3, false>(As, Bs, acc, tx, ty);
    __syncthreads();
  }
  if (t.flags & G_POSTMUL) {
    // C = P * (A op(B)): product and P both staged in shared memory.  P is a
    // diagonal block inverse (lower triangular): rows 16 i .. 16 i + 15 meet
    // only zeros of P beyond column 16 i + 15, so chunk c of m feeds row groups i >= c
    T (*Cs)[65] = reinterpret_cast<T (*)[65]>(smem);
    T (*Ps)[65] = reinterpret_cast<T (*)[65]>(smem + 64 * 65);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) Cs[ty + 16 * i][tx + 16 * j] = acc[i][j];
    for (int e = tid; e < 64 * 64; e += 256) Ps[e >> 6][e & 63] = t.P[(size_t)(e >> 6) * t.ldc + (e & 63)];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
#pragma unroll
    for (int c = 0; c < 4; ++c)
      for (int m = 16 * c; m < 16 * c + 16; ++m) {
        T b[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Cs[m][tx + 16 * j];
#pragma unroll
        for (int i = c; i < 4; ++i) {
          const T pv = Ps[ty + 16 * i][m];
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(pv, b[j], acc[i][j]);
        }
      }
  }
  const T sgn = (t.flags & G_NEG) ? (T)-1 : (T)1;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      T* c = t.C + (size_t)(ty + 16 * i) * t.ldc + tx + 16 * j;
      const T v = sgn * acc[i][j];
      *c = (t.flags & G_ACC) ? *c + v : v;
    }
}

// One step of a block triangular solve: C(64 x PC) = init + sign op(A) B,
// with PC right-hand sides.  Compact buffers have scalar type T; the
// full-layout multivectors gathered from / scattered to are FP64 with row
// stride PC (scatter_add accumulates instead of overwriting).
constexpr int SKC = 32;
// FP32 tile task (mixed path): the same task semantics as k_tile_task with an
// FP32-specific inner loop.  32-deep k chunks, the next chunk's global loads
// held in registers while the current one is multiplied, and a 4 x 4 register
// tile of contiguous rows and columns so that both operands come from shared
// memory as 16-byte vectors (2 vector loads per 16 FMA).  POTRF tasks run the
// tile Cholesky of k_tile_task in FP32 or FP64 (f32_tile_potrf).
constexpr int KC32 = 32;
constexpr int LDS32 = 68;   // shared row stride (floats): 16-byte aligned rows

template <bool L2 = false>
__device__ __forceinline__ void f32_tile_gemm(const TileTaskT<float>& t, double* smem_d) {
  float* smem = reinterpret_cast<float*>(smem_d);
  float (*As)[LDS32] = reinterpret_cast<float (*)[LDS32]>(smem);                  // [KC32][LDS32]: As[k][m]
  float (*Bs)[LDS32] = reinterpret_cast<float (*)[LDS32]>(smem + KC32 * LDS32);   // [KC32][LDS32]: Bs[k][n]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const bool transB = (t.flags & G_TRANSB) != 0;
  // global -> register mapping of one chunk: A (and B^T) rows m = tid & 63,
  // columns kc = (tid >> 6) * 8 .. + 7; B rows k = tid >> 3, columns (tid & 7) * 8 .. + 7
  const int lm = tid & 63, lk = (tid >> 6) * 8;
  const int bk = tid >> 3, bn = (tid & 7) * 8;
  float4 ra[2], rb[2];
  auto load = [&](int k0) {
    const float4* a = reinterpret_cast<const float4*>(t.A + (size_t)lm * t.lda + k0 + lk);
    ra[0] = ldg_op<L2>(a);
    ra[1] = ldg_op<L2>(a + 1);
    if (transB) {
      const float4* b = reinterpret_cast<const float4*>(t.B + (size_t)lm * t.ldb + k0 + lk);
      rb[0] = ldg_op<L2>(b);
      rb[1] = ldg_op<L2>(b + 1);
    } else {
      const float4* b = reinterpret_cast<const float4*>(t.B + (size_t)(k0 + bk) * t.ldb + bn);
      rb[0] = ldg_op<L2>(b);
      rb[1] = ldg_op<L2>(b + 1);
    }
  };
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  load(0);
  for (int k0 = 0; k0 < t.K; k0 += KC32) {
    {
      const float av[8] = {ra[0].x, ra[0].y, ra[0].z, ra[0].w, ra[1].x, ra[1].y, ra[1].z, ra[1].w};
#pragma unroll
      for (int i = 0; i < 8; ++i) As[lk + i][lm] = av[i];
      if (transB) {
        const float bv[8] = {rb[0].x, rb[0].y, rb[0].z, rb[0].w, rb[1].x, rb[1].y, rb[1].z, rb[1].w};
#pragma unroll
        for (int i = 0; i < 8; ++i) Bs[lk + i][lm] = bv[i];
      } else {
        *reinterpret_cast<float4*>(&Bs[bk][bn]) = rb[0];
        *reinterpret_cast<float4*>(&Bs[bk][bn + 4]) = rb[1];
      }
    }
    __syncthreads();
    if (k0 + KC32 < t.K) load(k0 + KC32);
#pragma unroll
    for (int kk = 0; kk < KC32; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&As[kk][4 * ty]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][4 * tx]);
      const float a4[4] = {a.x, a.y, a.z, a.w}, b4[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a4[i], b4[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (t.flags & G_POSTMUL) {
    // C = P * (A op(B)): product and P both staged in shared memory
    float (*Cs)[LDS32] = reinterpret_cast<float (*)[LDS32]>(smem);
    float (*Ps)[LDS32] = reinterpret_cast<float (*)[LDS32]>(smem + 64 * LDS32);
#pragma unroll
    for (int i = 0; i < 4; ++i)
      *reinterpret_cast<float4*>(&Cs[4 * ty + i][4 * tx]) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    for (int e = tid; e < 64 * 16; e += 256) {
      const int r = e >> 4, c = (e & 15) * 4;
      *reinterpret_cast<float4*>(&Ps[r][c]) = ldg_op<L2>(reinterpret_cast<const float4*>(t.P + (size_t)r * t.ldc + c));
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int m = 0; m < 64; ++m) {
      const float4 b = *reinterpret_cast<const float4*>(&Cs[m][4 * tx]);
      const float b4[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float pv = Ps[4 * ty + i][m];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(pv, b4[j], acc[i][j]);
      }
    }
  }
  const float sgn = (t.flags & G_NEG) ? -1.f : 1.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float4* c = reinterpret_cast<float4*>(t.C + (size_t)(4 * ty + i) * t.ldc + 4 * tx);
    float4 v = make_float4(sgn * acc[i][0], sgn * acc[i][1], sgn * acc[i][2], sgn * acc[i][3]);
    if (t.flags & G_ACC) {
      const float4 o = ldg_op<L2>(c);
      v.x += o.x; v.y += o.y; v.z += o.z; v.w += o.w;
    }
    *c = v;
  }
}

// Tile Cholesky of the FP32 factorisation in FP64 or, with potrf32, in FP32.
template <bool L2 = false>
__device__ __forceinline__ void f32_tile_potrf(const TileTaskT<float>& t, double* smem_d, int* notspd,
                                               int potrf32) {
  if (potrf32) tile_potrf_inv<float, float, L2>(t, reinterpret_cast<float (*)[65]>(smem_d), notspd);
  else tile_potrf_inv<float, double, L2>(t, reinterpret_cast<double (*)[65]>(smem_d), notspd);
}

__global__ void __launch_bounds__(256)
k_tile_task_f32(const TileTaskT<float>* __restrict__ tasks, const int* __restrict__ active,
                int* __restrict__ notspd, int potrf32) {
  const TileTaskT<float> t = tasks[blockIdx.x];
  if (t.sub >= 0 && active != nullptr && !active[t.sub]) return;
  extern __shared__ double smem_d[];
  if (t.flags & G_POTRF) {
    f32_tile_potrf(t, smem_d, notspd, potrf32);
    return;
  }
  f32_tile_gemm(t, smem_d);
}

// Persistent form of the FP32 factorisation: one cooperative launch runs the
// whole task list of a wave.  Every CTA takes the next task by an atomic ticket
// (tasks are numbered step by step across all chains, a topological order),
// waits until the previous step of the task's chain has completed (thread 0
// spins on that step's completion counter with acquire loads, bounded by two
// seconds, and gives up when another CTA has reported an error), runs it with
// L2-only operand loads (operands are written by other SMs during the launch),
// and counts it complete (a device-scope fence by thread 0 after the CTA's
// barrier, then a release increment).  All CTAs are resident
// (cooperative launch), so a task's predecessors, which hold smaller tickets,
// are always running or done: the waits end.  meta[t] = (counter of the task's
// step, counter of the previous step or -1, tasks in the previous step, index
// of the task in the schedule's task list).
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__global__ void __launch_bounds__(256)
k_factor_persistent(const TileTaskT<float>* __restrict__ tasks, const int4* __restrict__ meta, int ntask,
                    int* __restrict__ counters, int* __restrict__ ticket, const int* __restrict__ active,
                    int* __restrict__ notspd, int* __restrict__ err, int potrf32) {
  extern __shared__ double smem_d[];
  __shared__ int s_t, s_ok;
  for (;;) {
    if (threadIdx.x == 0) {
      const int t = atomicAdd(ticket, 1);
      int ok = 1;
      if (t < ntask) {
        const int4 m = meta[t];
        if (m.y >= 0) {
          const uint64_t t0 = tc::gtimer();
          while (ld_acquire(counters + m.y) < m.z) {
            if (*reinterpret_cast<volatile int*>(err) != 0 || tc::gtimer() - t0 > 2000000000ull) {
              ok = 0;
              break;
            }
            __nanosleep(100);
          }
        }
      }
      s_t = t;
      s_ok = ok;
    }
    __syncthreads();
    const int t = s_t;
    if (t >= ntask) return;
    if (!s_ok) {
      if (threadIdx.x == 0) atomicExch(err, 2);
      return;
    }
    const int4 mt = meta[t];
    const TileTaskT<float> task = tasks[mt.w];
    if (!(task.sub >= 0 && active != nullptr && !active[task.sub])) {
      if (task.flags & G_POTRF) f32_tile_potrf<true>(task, smem_d, notspd, potrf32);
      else f32_tile_gemm<true>(task, smem_d);
    }
    __syncthreads();   // the task's stores are done (and the shared tiles may be reused)
    if (threadIdx.x == 0) {
      // a device-scope fence after the barrier covers the stores of the whole CTA;
      // then the release increment of the step's counter
      __threadfence();
      asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(counters + mt.x) : "memory");
    }
  }
}

// The same task semantics with the plain GEMM tasks (A op(B)^T, no
// post-multiplication) on the tensor cores (tc_gemm.cuh: TMA, tcgen05.mma in
// split TF32, TMEM accumulator); POTRF tasks and the block-inverse tasks keep
// their FP64 / FP32 SIMT paths.
__global__ void __launch_bounds__(256)
k_tile_task_tc(const TileTaskT<float>* __restrict__ tasks, const int* __restrict__ active, int* __restrict__ notspd,
               const SubDev* __restrict__ subs, const CUtensorMap* __restrict__ maps, int potrf32) {
  const TileTaskT<float> t = tasks[blockIdx.x];
  if (t.sub >= 0 && active != nullptr && !active[t.sub]) return;
  extern __shared__ double smem_d[];
  if (t.flags & G_POTRF) {
    f32_tile_potrf(t, smem_d, notspd, potrf32);
    return;
  }
  if ((t.flags & G_POSTMUL) || !(t.flags & G_TRANSB) || t.K % tc::KCH != 0 || t.sub < 0) {
    f32_tile_gemm(t, smem_d);
    return;
  }
  tc::gemm_task(t, reinterpret_cast<unsigned char*>(smem_d), subs, maps, notspd);
}

template <typename T, int PC>
__global__ void __launch_bounds__(256)
k_solve_step(const SolveTaskT<T>* __restrict__ tasks, const SubDev* __restrict__ subs,
             const int* __restrict__ active, int src, int dst, int gather_neg, int scatter_add) {
  constexpr int TXN = PC < 16 ? PC : 16;   // threads along columns
  constexpr int CPT = PC / TXN;            // columns per thread
  constexpr int TYN = 256 / TXN;           // threads along rows
  constexpr int RPT = 64 / TYN;            // rows per thread
  const SolveTaskT<T> t = tasks[blockIdx.x];
  if (t.sub >= 0 && active != nullptr && !active[t.sub]) return;
  __shared__ T As[SKC][65];
  __shared__ T Bs[SKC][PC + 1];
  const int tid = threadIdx.x, tx = tid % TXN, ty = tid / TXN;
  T acc[RPT][CPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i)
#pragma unroll
    for (int j = 0; j < CPT; ++j) acc[i][j] = (T)0;
  const bool transA = (t.flags & S_TRANSA) != 0;
  for (int k0 = 0; k0 < t.K; k0 += SKC) {
    if (!transA) {
      const int r = tid >> 2, c = (tid & 3) * 8;
      const T* a = t.A + (size_t)r * t.lda + k0 + c;
#pragma unroll
      for (int i = 0; i < 8; ++i) As[c + i][r] = a[i];
    } else {
      const int k = tid >> 3, m = (tid & 7) * 8;
      const T* a = t.A + (size_t)(k0 + k) * t.lda + m;
#pragma unroll
      for (int i = 0; i < 8; ++i) As[k][m + i] = a[i];
    }
    for (int e = tid; e < SKC * PC; e += 256) Bs[e / PC][e % PC] = t.B[(size_t)(k0 + e / PC) * PC + e % PC];
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < SKC; ++kk) {
      T a[RPT], b[CPT];
#pragma unroll
      for (int i = 0; i < RPT; ++i) a[i] = As[kk][ty + TYN * i];
#pragma unroll
      for (int j = 0; j < CPT; ++j) b[j] = Bs[kk][tx + TXN * j];
#pragma unroll
      for (int i = 0; i < RPT; ++i)
#pragma unroll
        for (int j = 0; j < CPT; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  const T sgn = (t.flags & S_NEG) ? (T)-1 : (T)1;
  const double* gfull = nullptr;
  double* sfull = nullptr;
  if (t.flags & (S_INIT_GATHER | S_SCATTER)) {
    const SubDev& s = subs[t.sub];
    if (t.flags & S_INIT_GATHER) gfull = mv_ptr(s, src) + (size_t)t.row_off * PC;
    if (t.flags & S_SCATTER) sfull = mv_ptr(s, dst) + (size_t)t.row_off * PC;
  }
  const double gs = gather_neg ? -1.0 : 1.0;
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int r = ty + TYN * i;
    const int gmr = (t.flags & S_INIT_GATHER) ? t.gmap[r] : -1;
    const int smr = (t.flags & S_SCATTER) ? t.smap[r] : -1;
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      const int c = tx + TXN * j;
      T v = sgn * acc[i][j];
      if (t.flags & S_INIT_TILE) v += t.init[r * PC + c];
      if (gmr >= 0) v += (T)(gs * gfull[(size_t)gmr * PC + c]);
      t.C[r * PC + c] = v;
      if (smr >= 0) {
        double* o = sfull + (size_t)smr * PC + c;
        *o = scatter_add ? *o + (double)v : (double)v;
      }
    }
  }
}

// Streaming variant of the solve step for KB right-hand sides.  The solves
// are bound by memory, not arithmetic: every task reads a 64-row slab of a
// factor block once.  The small B block (K x KB) is staged once in shared
// memory and every thread keeps several 16-byte loads of A in flight.
//   plain A:      lane <-> a 16-byte vector of consecutive k, each warp owns
//                 8 rows (R at a time), partial sums reduced with shuffles;
//   transposed A: thread <-> (16-byte vector of output rows, k group), the
//                 k groups are summed through shared memory.
// Staging layout: rows of B in chunks of VN rows (one A vector), each chunk
// padded by one 16-byte vector so that the chunks read by the 8 lanes of a
// 128-bit shared-memory phase fall in distinct bank groups.  The staging area
// is reused for the reduction after a barrier.
template <typename T> struct SolveVec;
template <> struct SolveVec<float> {
  using V = float4;
  static constexpr int N = 4;
  __device__ static void split(const V& v, float (&a)[4]) { a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w; }
};
template <> struct SolveVec<double> {
  using V = double2;
  static constexpr int N = 2;
  __device__ static void split(const V& v, double (&a)[2]) { a[0] = v.x; a[1] = v.y; }
};

template <typename T>
__device__ __forceinline__ void load_row_kb(const T* p, T (&b)[KB]) {
  using V = typename SolveVec<T>::V;
  constexpr int N = SolveVec<T>::N;
#pragma unroll
  for (int j = 0; j < KB / N; ++j) {
    T e[N];
    SolveVec<T>::split(reinterpret_cast<const V*>(p)[j], e);
#pragma unroll
    for (int i = 0; i < N; ++i) b[N * j + i] = e[i];
  }
}

// elements per staged chunk of VN rows (padded), and the number of k groups
// of the transposed variant
template <typename T>
__host__ __device__ constexpr int solve_cs() { return SolveVec<T>::N * (KB + 1); }
template <typename T>
__host__ __device__ constexpr int solve_kg() { return 256 / (64 / SolveVec<T>::N); }

template <typename T, int CL>
__global__ void __launch_bounds__(256, SOLVE_MIN_BLOCKS)
k_solve_stream(const SolveTaskT<T>* __restrict__ tasks, const SubDev* __restrict__ subs,
               const int* __restrict__ active, int src, int dst, int gather_neg, int scatter_add) {
  constexpr int VN = SolveVec<T>::N;
  constexpr int CS = solve_cs<T>();
  constexpr int TPR = 64 / VN;          // threads across the 64 output rows (transposed A)
  constexpr int KG = solve_kg<T>();     // k groups (transposed A)
  constexpr int R = sizeof(T) == 4 ? SOLVE_ROWS_F32 : 4;   // rows per pass (plain A)
  constexpr int NP = 8 / R;
  static_assert(8 * KB == 64, "the plain-A reduction assumes KB == 8");
  static_assert(64 % CL == 0, "cluster size must divide the tile rows");
  using V = typename SolveVec<T>::V;
  // CL consecutive CTAs (one thread-block cluster) share a task and split its
  // inner dimension; rank q takes chunks [c0, c1) of VN columns
  const int rank = blockIdx.x % CL;
  const SolveTaskT<T> t = tasks[blockIdx.x / CL];
  if (t.sub >= 0 && active != nullptr && !active[t.sub]) return;   // uniform over the cluster
  extern __shared__ double smem_s[];
  T* Out = reinterpret_cast<T*>(smem_s);   // [64][KB] partial result of this CTA
  T* Bs = Out + 64 * KB;                   // staging of B rows [k0, k1), later the reduction area
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int nch = t.K / VN, per = (nch + CL - 1) / CL;
  const int c0 = min(rank * per, nch), c1 = min(c0 + per, nch);
  const int k0 = c0 * VN, kl = (c1 - c0) * VN;
  {
    // vector loads of B (rows of KB elements are 16-byte aligned); VN-element
    // vector e covers row e / (KB / VN), columns (e % (KB / VN)) * VN ...
    const V* Bv = reinterpret_cast<const V*>(t.B + (size_t)k0 * KB);
    for (int e = tid; e < kl * (KB / VN); e += 256) {
      const int k = e / (KB / VN), c = (e % (KB / VN)) * VN;
      *reinterpret_cast<V*>(Bs + (k / VN) * CS + (k % VN) * KB + c) = Bv[e];
    }
  }
  __syncthreads();
  const bool transA = (t.flags & S_TRANSA) != 0;
  if (!transA) {
    T res[2] = {(T)0, (T)0};
#pragma unroll
    for (int g = 0; g < NP; ++g) {
      const int r0 = w * 8 + g * R;
      T acc[R][KB];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < KB; ++c) acc[r][c] = (T)0;
      const T* a0 = t.A + (size_t)r0 * t.lda;
      // the loads of the next chunk are issued before the arithmetic of the
      // current one (register double buffer)
      V nxt[R];
      if (c0 + lane < c1) {
#pragma unroll
        for (int r = 0; r < R; ++r)
          nxt[r] = *reinterpret_cast<const V*>(a0 + (size_t)r * t.lda + (size_t)(c0 + lane) * VN);
      }
#pragma unroll 1
      for (int kc = c0 + lane; kc < c1; kc += 32) {
        T a[R][VN];
#pragma unroll
        for (int r = 0; r < R; ++r) SolveVec<T>::split(nxt[r], a[r]);
        if (kc + 32 < c1) {
#pragma unroll
          for (int r = 0; r < R; ++r)
            nxt[r] = *reinterpret_cast<const V*>(a0 + (size_t)r * t.lda + (size_t)(kc + 32) * VN);
        }
        const T* bp = Bs + (size_t)(kc - c0) * CS;
#pragma unroll
        for (int v = 0; v < VN; ++v) {
          T b[KB];
          load_row_kb<T>(bp + v * KB, b);
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < KB; ++c) acc[r][c] = fma(a[r][v], b[c], acc[r][c]);
        }
      }
      // every lane holds all R x KB sums after the butterfly; lane L keeps
      // entries L and L + 32 of the 8 x KB block of its warp (rows 4j + L / KB)
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < KB; ++c) {
          T v = acc[r][c];
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
          const int idx = g * R * KB + r * KB + c;
          if (lane == idx % 32) res[idx / 32] = v;
        }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) Out[(w * 8 + 4 * j + lane / KB) * KB + lane % KB] = res[j];
  } else {
    const int mv = tid % TPR, kg = tid / TPR;
    T acc[VN][KB];
#pragma unroll
    for (int v = 0; v < VN; ++v)
#pragma unroll
      for (int c = 0; c < KB; ++c) acc[v][c] = (T)0;
    const T* a0 = t.A + mv * VN;
#pragma unroll 8
    for (int k = kg; k < kl; k += KG) {
      T a[VN];
      SolveVec<T>::split(*reinterpret_cast<const V*>(a0 + (size_t)(k0 + k) * t.lda), a);
      T b[KB];
      load_row_kb<T>(Bs + (size_t)(k / VN) * CS + (k % VN) * KB, b);
#pragma unroll
      for (int v = 0; v < VN; ++v)
#pragma unroll
        for (int c = 0; c < KB; ++c) acc[v][c] = fma(a[v], b[c], acc[v][c]);
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < VN; ++v)
#pragma unroll
      for (int c = 0; c < KB; ++c) Bs[((size_t)kg * 64 + mv * VN + v) * KB + c] = acc[v][c];
    __syncthreads();
    for (int e = tid; e < 64 * KB; e += 256) {
      T v = (T)0;
#pragma unroll
      for (int q = 0; q < KG; ++q) v += Bs[(size_t)q * 64 * KB + e];
      Out[e] = v;
    }
  }
  // sum the partial results of the cluster (distributed shared memory); rank q
  // finishes rows [q 64 / CL, (q + 1) 64 / CL)
  constexpr int RPR = 64 / CL;
  if constexpr (CL > 1) cg::this_cluster().sync();
  else __syncthreads();
  const T sgn = (t.flags & S_NEG) ? (T)-1 : (T)1;
  const double* gfull = nullptr;
  double* sfull = nullptr;
  if (t.flags & (S_INIT_GATHER | S_SCATTER)) {
    const SubDev& s = subs[t.sub];
    if (t.flags & S_INIT_GATHER) gfull = mv_ptr(s, src) + (size_t)t.row_off * KB;
    if (t.flags & S_SCATTER) sfull = mv_ptr(s, dst) + (size_t)t.row_off * KB;
  }
  const double gs = gather_neg ? -1.0 : 1.0;
  for (int e = tid; e < RPR * KB; e += 256) {
    const int ee = rank * RPR * KB + e;
    const int r = ee / KB, c = ee % KB;
    T v = (T)0;
    if constexpr (CL > 1) {
      cg::cluster_group cl = cg::this_cluster();
#pragma unroll
      for (int q = 0; q < CL; ++q) v += cl.map_shared_rank(Out, q)[ee];
    } else {
      v = Out[ee];
    }
    v = sgn * v;
    if (t.flags & S_INIT_TILE) v += t.init[r * KB + c];
    const int gmr = (t.flags & S_INIT_GATHER) ? t.gmap[r] : -1;
    if (gmr >= 0) v += (T)(gs * gfull[(size_t)gmr * KB + c]);
    t.C[r * KB + c] = v;
    const int smr = (t.flags & S_SCATTER) ? t.smap[r] : -1;
    if (smr >= 0) {
      double* o = sfull + (size_t)smr * KB + c;
      *o = scatter_add ? *o + (double)v : (double)v;
    }
  }
  // keep this CTA's partial result alive until every peer has read it
  if constexpr (CL > 1) cg::this_cluster().sync();
}

// ---------------------------------------------------------------------------
// FP32 solve step with an asynchronous-copy pipeline (the mixed-precision
// path).  Measured on the streaming kernel: one CTA pulls only ~7 GB/s, since
// each thread can keep just one register-resident chunk of the factor in
// flight.  Here the factor slab of a task (64 rows x K, or K x 64 read
// transposed) moves through a ring of ASYNC_DEPTH shared-memory stages of
// 64 x 64 floats (16 KiB) with cp.async (16 bytes per copy, 4 copies per
// thread and stage), so ASYNC_DEPTH - 1 stages (48 KiB) are in flight per CTA
// without holding registers.  Thread (g, h) of the 16 x 16 thread grid owns 4
// output rows (g) and a 4-wide k slice (h) of every stage and keeps a 4 x KB
// accumulator; the 16 k slices are summed through shared memory at the end.
constexpr int ASYNC_DEPTH = 4;
constexpr int ASYNC_STAGE = 64 * 64;             // floats per stage
constexpr int ASYNC_CS = 4 * (KB + 1);           // floats per staged chunk of 4 B rows (padded)

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// all threads: copy stage i of the slab into ring slot i % ASYNC_DEPTH
__device__ __forceinline__ void async_issue(const SolveTaskT<float>& t, bool transA, int i, float* ring, int tid) {
  float* dst0 = ring + (size_t)(i % ASYNC_DEPTH) * ASYNC_STAGE;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = tid + 256 * q, r = c >> 4, c4 = (c & 15) * 4;
    // plain: row r, columns 64 i + c4 ..; transposed: row 64 i + r, columns c4 ..
    const float* src = transA ? t.A + (size_t)(64 * i + r) * t.lda + c4 : t.A + (size_t)r * t.lda + 64 * i + c4;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst0 + r * 64 + c4)), "l"(src)
                 : "memory");
  }
}

__global__ void __launch_bounds__(256, 2)
k_solve_async(const SolveTaskT<float>* __restrict__ tasks, const SubDev* __restrict__ subs,
              const int* __restrict__ active, int src, int dst, int gather_neg, int scatter_add) {
  const SolveTaskT<float> t = tasks[blockIdx.x];
  if (t.sub >= 0 && active != nullptr && !active[t.sub]) return;
  extern __shared__ __align__(128) unsigned char smem_b[];
  float* ring = reinterpret_cast<float*>(smem_b);                     // [ASYNC_DEPTH][64][64]
  float* Bs = ring + ASYNC_DEPTH * ASYNC_STAGE;                       // [K / 4][ASYNC_CS]
  const int tid = threadIdx.x;
  const bool transA = (t.flags & S_TRANSA) != 0;
  const int nst = t.K / 64;
  // the next step may launch now; the factor slab does not depend on the
  // previous step, so its first stages are requested before waiting for it
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  for (int i = 0; i < ASYNC_DEPTH - 1; ++i) {
    if (i < nst) async_issue(t, transA, i, ring, tid);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");   // B, the gathered vectors and C follow the previous step
  {
    const float4* Bv = reinterpret_cast<const float4*>(t.B);
    for (int e = tid; e < t.K * (KB / 4); e += 256) {
      const int k = e / (KB / 4), c = (e % (KB / 4)) * 4;
      *reinterpret_cast<float4*>(Bs + (k / 4) * ASYNC_CS + (k % 4) * KB + c) = Bv[e];
    }
  }
  // thread grid: plain A: h = tid % 16 (k slice), g = tid / 16 (rows);
  //              transposed: g = tid % 16 (rows), h = tid / 16 (k slice)
  const int h = transA ? tid / 16 : tid % 16;
  const int g = transA ? tid % 16 : tid / 16;
  float acc[4][KB];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < KB; ++c) acc[r][c] = 0.f;
  for (int i = 0; i < nst; ++i) {
    // keep ASYNC_DEPTH - 1 stages in flight: issue stage i + DEPTH - 1 into the
    // slot consumed in iteration i - 1 (released by its trailing barrier)
    if (i + ASYNC_DEPTH - 1 < nst) async_issue(t, transA, i + ASYNC_DEPTH - 1, ring, tid);
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group %0;" ::"n"(ASYNC_DEPTH - 1) : "memory");
    __syncthreads();   // stage i (every thread's copies) and, at i = 0, the staged B are visible
    const float* stg = ring + (size_t)(i % ASYNC_DEPTH) * ASYNC_STAGE;
    const float* bp = Bs + (size_t)(16 * i + h) * ASYNC_CS;   // B rows 64 i + 4 h .. + 3
    float b[4][KB];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const float4 b0 = *reinterpret_cast<const float4*>(bp + v * KB);
      const float4 b1 = *reinterpret_cast<const float4*>(bp + v * KB + 4);
      b[v][0] = b0.x; b[v][1] = b0.y; b[v][2] = b0.z; b[v][3] = b0.w;
      b[v][4] = b1.x; b[v][5] = b1.y; b[v][6] = b1.z; b[v][7] = b1.w;
    }
    if (!transA) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float4 a = *reinterpret_cast<const float4*>(stg + (4 * g + r) * 64 + 4 * h);
        const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int v = 0; v < 4; ++v)
#pragma unroll
          for (int c = 0; c < KB; ++c) acc[r][c] = fmaf(av[v], b[v][c], acc[r][c]);
      }
    } else {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const float4 a = *reinterpret_cast<const float4*>(stg + (4 * h + v) * 64 + 4 * g);
        const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < KB; ++c) acc[r][c] = fmaf(av[r], b[v][c], acc[r][c]);
      }
    }
    __syncthreads();   // every warp is done with the slot
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  // sum the 16 k slices: red[h][row][c] in the (now idle) ring
  float* red = ring;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    float* o = red + ((size_t)h * 64 + 4 * g + r) * KB;
    *reinterpret_cast<float4*>(o) = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
    *reinterpret_cast<float4*>(o + 4) = make_float4(acc[r][4], acc[r][5], acc[r][6], acc[r][7]);
  }
  __syncthreads();
  const float sgn = (t.flags & S_NEG) ? -1.f : 1.f;
  const double* gfull = nullptr;
  double* sfull = nullptr;
  if (t.flags & (S_INIT_GATHER | S_SCATTER)) {
    const SubDev& s = subs[t.sub];
    if (t.flags & S_INIT_GATHER) gfull = mv_ptr(s, src) + (size_t)t.row_off * KB;
    if (t.flags & S_SCATTER) sfull = mv_ptr(s, dst) + (size_t)t.row_off * KB;
  }
  const double gsg = gather_neg ? -1.0 : 1.0;
  for (int e = tid; e < 64 * KB; e += 256) {
    const int r = e / KB, c = e % KB;
    float v = 0.f;
#pragma unroll
    for (int q = 0; q < 16; ++q) v += red[(size_t)q * 64 * KB + e];
    v = sgn * v;
    if (t.flags & S_INIT_TILE) v += t.init[r * KB + c];
    const int gmr = (t.flags & S_INIT_GATHER) ? t.gmap[r] : -1;
    if (gmr >= 0) v += (float)(gsg * gfull[(size_t)gmr * KB + c]);
    t.C[r * KB + c] = v;
    const int smr = (t.flags & S_SCATTER) ? t.smap[r] : -1;
    if (smr >= 0) {
      double* o = sfull + (size_t)smr * KB + c;
      *o = scatter_add ? *o + (double)v : (double)v;
    }
  }
}

// The same solve step with the factor slab staged by the tensor memory
// accelerator: one thread issues one cp.async.bulk.tensor.2d per 64 x 64 stage
// (16 KiB, unswizzled: the ring's row-major layout) that completes on the
// stage's mbarrier, instead of 1,024 16-byte cp.async copies from all threads.
// The tensor maps cover the subdomain's FP32 layer-block arrays on this GPU
// only (no multicast).  Before any copy the task's slab (when it has one:
// tasks with inner dimension 0 only gather or add their initial tile) is
// checked to lie in one mapped array with the array's row stride, a
// 16-byte-aligned column and every stage inside the array; waits are bounded.
// A task that fails the check or a stage that does not arrive within a second
// sets *err and the task's products are skipped.
__global__ void __launch_bounds__(256, 2)
k_solve_tma(const SolveTaskT<float>* __restrict__ tasks, const SubDev* __restrict__ subs,
            const int* __restrict__ active, int src, int dst, int gather_neg, int scatter_add,
            const CUtensorMap* __restrict__ maps, int* __restrict__ err) {
  const SolveTaskT<float> t = tasks[blockIdx.x];
  if (t.sub >= 0 && active != nullptr && !active[t.sub]) return;
  extern __shared__ __align__(128) unsigned char smem_b[];
  // the ring on a 1024-byte boundary (the launch adds 1 KiB of shared memory)
  float* ring = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_b) + 1023) & ~uintptr_t(1023));
  float* Bs = ring + ASYNC_DEPTH * ASYNC_STAGE;                       // [K / 4][ASYNC_CS]
  __shared__ __align__(8) unsigned long long full[ASYNC_DEPTH];
  __shared__ const CUtensorMap* smap;
  __shared__ int sx, sy, sbad;
  const int tid = threadIdx.x;
  const bool transA = (t.flags & S_TRANSA) != 0;
  const int nst = t.K / 64;
  const uint32_t ring_s = tc::saddr(ring), bar0 = tc::saddr(full);
  int issued = 0;   // stages issued (thread 0)
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  // stage i of the slab: plain A, rows 0..63 x columns 64 i ..; transposed, rows 64 i .. x columns 0..63
  auto issue = [&](int i) {
    const uint32_t bar = bar0 + 8 * (i % ASYNC_DEPTH);
    tc::mbar_expect_tx(bar, (uint32_t)(ASYNC_STAGE * sizeof(float)));
    tc::tma_load_2d(ring_s + (uint32_t)((i % ASYNC_DEPTH) * ASYNC_STAGE * sizeof(float)), smap,
                    sx + (transA ? 0 : 64 * i), sy + (transA ? 64 * i : 0), bar);
    issued = i + 1;
  };
  if (tid == 0) {
    for (int d = 0; d < ASYNC_DEPTH; ++d) tc::mbar_init(bar0 + 8 * d, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    int x = 0, y = 0;
    const CUtensorMap* m = (nst > 0 && t.sub >= 0) ? tc::locate(subs[t.sub], maps, t.sub, t.A, x, y) : nullptr;
    if (m != nullptr) {
      const SubDev& sd = subs[t.sub];
      const int which = (int)(m - maps) - 4 * t.sub;   // DKf, LKf, DAf, LAf
      const int b = which < 2 ? sd.bK : sd.bA;
      const int rows = (which == 0 ? 2 * sd.nzn - 1 : which == 1 ? sd.nzn : which == 2 ? 2 * sd.nzn - 1 : sd.nzn) * b;
      const int w = transA ? 64 : 64 * nst, hgt = transA ? 64 * nst : 64;
      if (t.lda != b || (x & 3) != 0 || x + w > b || y + hgt > rows) m = nullptr;
    }
    smap = m;
    sx = x;
    sy = y;
    sbad = nst > 0 && m == nullptr;
    // the factor slab does not depend on the previous step: its first stages go out first
    if (m != nullptr)
      for (int i = 0; i < ASYNC_DEPTH - 1 && i < nst; ++i) issue(i);
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");   // B, the gathered vectors and C follow the previous step
  {
    const float4* Bv = reinterpret_cast<const float4*>(t.B);
    for (int e = tid; e < t.K * (KB / 4); e += 256) {
      const int k = e / (KB / 4), c = (e % (KB / 4)) * 4;
      *reinterpret_cast<float4*>(Bs + (k / 4) * ASYNC_CS + (k % 4) * KB + c) = Bv[e];
    }
  }
  __syncthreads();
  bool ok = !sbad;
  const int h = transA ? tid / 16 : tid % 16;
  const int g = transA ? tid % 16 : tid / 16;
  float acc[4][KB];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < KB; ++c) acc[r][c] = 0.f;
  int waited = 0;   // stages whose copies have been waited for
  for (int i = 0; i < nst && ok; ++i) {
    // keep ASYNC_DEPTH - 1 stages in flight: stage i + DEPTH - 1 goes into the
    // slot released by the trailing barrier of iteration i - 1
    if (tid == 0 && i + ASYNC_DEPTH - 1 < nst) {
      tc::fence_async_smem();
      issue(i + ASYNC_DEPTH - 1);
    }
    const bool w = tc::mbar_wait(bar0 + 8 * (i % ASYNC_DEPTH), (i / ASYNC_DEPTH) & 1);
    if (!__syncthreads_and(w)) {
      ok = false;
      break;
    }
    waited = i + 1;
    const float* stg = ring + (size_t)(i % ASYNC_DEPTH) * ASYNC_STAGE;
    const float* bp = Bs + (size_t)(16 * i + h) * ASYNC_CS;   // B rows 64 i + 4 h .. + 3
    float b[4][KB];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const float4 b0 = *reinterpret_cast<const float4*>(bp + v * KB);
      const float4 b1 = *reinterpret_cast<const float4*>(bp + v * KB + 4);
      b[v][0] = b0.x; b[v][1] = b0.y; b[v][2] = b0.z; b[v][3] = b0.w;
      b[v][4] = b1.x; b[v][5] = b1.y; b[v][6] = b1.z; b[v][7] = b1.w;
    }
    if (!transA) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float4 a = *reinterpret_cast<const float4*>(stg + (4 * g + r) * 64 + 4 * h);
        const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int v = 0; v < 4; ++v)
#pragma unroll
          for (int c = 0; c < KB; ++c) acc[r][c] = fmaf(av[v], b[v][c], acc[r][c]);
      }
    } else {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const float4 a = *reinterpret_cast<const float4*>(stg + (4 * h + v) * 64 + 4 * g);
        const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < KB; ++c) acc[r][c] = fmaf(av[r], b[v][c], acc[r][c]);
      }
    }
    __syncthreads();   // every warp is done with the slot
  }
  if (!ok) {
    // a stage did not arrive: wait once more (bounded) for every copy issued, then report
    if (tid == 0) {
      for (int i = waited; i < issued; ++i) tc::mbar_wait(bar0 + 8 * (i % ASYNC_DEPTH), (i / ASYNC_DEPTH) & 1);
      if (err != nullptr) atomicExch(err, 1);
    }
    __syncthreads();
  }
  // sum the 16 k slices: red[h][row][c] in the (now idle) ring
  float* red = ring;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    float* o = red + ((size_t)h * 64 + 4 * g + r) * KB;
    *reinterpret_cast<float4*>(o) = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
    *reinterpret_cast<float4*>(o + 4) = make_float4(acc[r][4], acc[r][5], acc[r][6], acc[r][7]);
  }
  __syncthreads();
  const float sgn = (t.flags & S_NEG) ? -1.f : 1.f;
  const double* gfull = nullptr;
  double* sfull = nullptr;
  if (t.flags & (S_INIT_GATHER | S_SCATTER)) {
    const SubDev& s = subs[t.sub];
    if (t.flags & S_INIT_GATHER) gfull = mv_ptr(s, src) + (size_t)t.row_off * KB;
    if (t.flags & S_SCATTER) sfull = mv_ptr(s, dst) + (size_t)t.row_off * KB;
  }
  const double gsg = gather_neg ? -1.0 : 1.0;
  for (int e = tid; e < 64 * KB; e += 256) {
    const int r = e / KB, c = e % KB;
    float v = 0.f;
#pragma unroll
    for (int q = 0; q < 16; ++q) v += red[(size_t)q * 64 * KB + e];
    v = sgn * v;
    if (t.flags & S_INIT_TILE) v += t.init[r * KB + c];
    const int gmr = (t.flags & S_INIT_GATHER) ? t.gmap[r] : -1;
    if (gmr >= 0) v += (float)(gsg * gfull[(size_t)gmr * KB + c]);
    t.C[r * KB + c] = v;
    const int smr = (t.flags & S_SCATTER) ? t.smap[r] : -1;
    if (smr >= 0) {
      double* o = sfull + (size_t)smr * KB + c;
      *o = scatter_add ? *o + (double)v : (double)v;
    }
  }
}

size_t solve_async_smem(int kmax) {
  return (size_t)ASYNC_DEPTH * ASYNC_STAGE * sizeof(float) + (size_t)((kmax + 3) / 4) * ASYNC_CS * sizeof(float);
}


constexpr size_t SOLVE_SMEM_MAX = 110 * 1024;

constexpr int SOLVE_CL = SOLVE_CLUSTER;   // CTAs per task (cluster size) of the streaming solve

// shared memory of k_solve_stream<T, cl> for tasks with inner dimension <= kmax
template <typename T>
size_t solve_stream_smem(int kmax, int cl) {
  const int nch = (kmax + SolveVec<T>::N - 1) / SolveVec<T>::N;
  const size_t stage = (size_t)((nch + cl - 1) / cl) * solve_cs<T>();
  const size_t red = (size_t)solve_kg<T>() * 64 * KB;
  return (64 * KB + (stage > red ? stage : red)) * sizeof(T);
}

}  // namespace

long long g_launch_count = 0;

static int* g_active = nullptr;   // set by the driver before schedule runs
static int* g_notspd = nullptr;
static const SubDev* g_subs = nullptr;
static const void* g_tc_maps = nullptr;   // tensor maps of the FP32 arrays: tensor-core factorisation on
static const void* g_solve_maps = nullptr;   // tensor maps of the FP32 arrays for the TMA solve stages
static int* g_kerr = nullptr;                // error flag of the TMA solve stages
static int g_potrf32 = 0;                    // tile Cholesky of the FP32 factorisation in FP32

void set_dense_context(int* active, int* notspd, const SubDev* subs) {
  g_active = active;
  g_notspd = notspd;
  g_subs = subs;
}

void set_factor_kernel(const void* tc_maps, int potrf32) {
  g_tc_maps = tc_maps;
  g_potrf32 = potrf32;
}

void set_solve_maps(const void* maps, int* err) {
  g_solve_maps = maps;
  g_kerr = err;
}

bool encode_tc_maps(const msgfem* h, std::vector<CUtensorMap>& maps, std::string& err, int box_cols,
                    CUtensorMapSwizzle swz);

msgfem_status tc_maps_build(msgfem* h) {
  std::vector<CUtensorMap> maps;
  std::string err;
  if (!encode_tc_maps(h, maps, err, tc::KCH, CU_TENSOR_MAP_SWIZZLE_128B)) {
    h->err = err;
    return MSGFEM_ECUDA;
  }
  if (h->d_tc_maps == nullptr) TRY(dev_alloc_bytes(h, &h->d_tc_maps, maps.size() * sizeof(CUtensorMap)));
  CK(cudaMemcpy(h->d_tc_maps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
  return MSGFEM_OK;
}

// tensor maps of the TMA solve stages: boxes of 64 x 64 FP32, unswizzled (the
// ring's row-major stage layout), and the stage error flag; built on first use
msgfem_status solve_maps_build(msgfem* h) {
  if (h->d_solve_maps == nullptr) {
    std::vector<CUtensorMap> maps;
    std::string err;
    if (!encode_tc_maps(h, maps, err, 64, CU_TENSOR_MAP_SWIZZLE_NONE)) {
      h->err = err;
      return MSGFEM_ECUDA;
    }
    TRY(dev_alloc_bytes(h, &h->d_solve_maps, maps.size() * sizeof(CUtensorMap)));
    CK(cudaMemcpy(h->d_solve_maps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
  }
  TRY(kerr_ensure(h));
  set_solve_maps(h->d_solve_maps, h->d_kerr);
  return MSGFEM_OK;
}

// the device error flag of bounded waits (TMA solve stages, persistent factorisation)
msgfem_status kerr_ensure(msgfem* h) {
  if (h->d_kerr != nullptr) return MSGFEM_OK;
  void* p = nullptr;
  TRY(dev_alloc_bytes(h, &p, sizeof(int)));
  h->d_kerr = static_cast<int*>(p);
  CK(cudaMemset(h->d_kerr, 0, sizeof(int)));
  return MSGFEM_OK;
}

msgfem_status run_factor_persistent(msgfem* h, const WaveSched& w, cudaStream_t st) {
  static int nb = 0, nsm = 0;
  if (nb == 0) {
    CK(cudaFuncSetAttribute(k_factor_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, TILE_SMEM));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_factor_persistent, 256, TILE_SMEM));
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (nb < 1) {
      nb = 0;
      h->err = "the persistent factorisation kernel does not fit on an SM";
      return MSGFEM_ECUDA;
    }
  }
  if (w.d_pmeta == nullptr || w.d_pcount == nullptr) {
    h->err = "the persistent factorisation has no task order (schedule built without it)";
    return MSGFEM_ECUDA;
  }
  TRY(kerr_ensure(h));
  CK(cudaMemsetAsync(w.d_pcount, 0, ((size_t)w.pcount + 1) * sizeof(int), st));
  const TileTaskT<float>* tasks = w.factf.d_gemm;
  const int4* meta = w.d_pmeta;
  int ntask = (int)w.pmeta.size();
  int* counters = w.d_pcount;
  int* ticket = w.d_pcount + w.pcount;
  const int* active = g_active;
  int* notspd = g_notspd;
  int* err = h->d_kerr;
  int potrf32 = g_potrf32;
  void* args[] = {&tasks, &meta, &ntask, &counters, &ticket, &active, &notspd, &err, &potrf32};
  CK(cudaLaunchCooperativeKernel((const void*)k_factor_persistent, dim3(nb * nsm), dim3(256), args, TILE_SMEM, st));
  ++g_launch_count;
  return MSGFEM_OK;
}

int tile_chol_fp32(const msgfem* h) { return h->mixed && h->opt.tile_chol == 1 && !h->potrf_fp64 ? 1 : 0; }

msgfem_status select_factor_kernel(msgfem* h) {
  const int potrf32 = tile_chol_fp32(h);
  if (h->mixed && h->factor_tc) {
    if (h->d_tc_maps == nullptr) TRY(tc_maps_build(h));
    set_factor_kernel(h->d_tc_maps, potrf32);
  } else {
    set_factor_kernel(nullptr, potrf32);
  }
  if (h->mixed && h->solve_variant == SOLVE_TMA_RING) TRY(solve_maps_build(h));
  set_solve_maps(h->d_solve_maps, h->d_kerr);
  return MSGFEM_OK;
}

msgfem_status check_stage_error(msgfem* h) {
  if (h->d_kerr == nullptr) return MSGFEM_OK;
  int e = 0;
  CK(cudaMemcpy(&e, h->d_kerr, sizeof(int), cudaMemcpyDeviceToHost));
  if (e == 0) return MSGFEM_OK;
  CK(cudaMemset(h->d_kerr, 0, sizeof(int)));
  h->err = e == 2 ? "a task of the persistent factorisation waited more than two seconds for its predecessors"
                  : "a tensor-memory-accelerator solve stage failed its slab check or did not arrive within a second";
  return MSGFEM_ECUDA;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  if (fn == nullptr) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// Tensor maps of every subdomain's four FP32 arrays (layer blocks D|E and
// inverses of K, then of A11): 2-D row-major arrays of b FP32 columns, boxes of
// 64 rows x 32 columns (128 bytes, the swizzle width) with 128-byte swizzle.
// Every tile task of the factorisation starts on a 64-column tile boundary, so
// each copy's inner coordinate is a multiple of 32 elements (128 bytes).
bool encode_tc_maps(const msgfem* h, std::vector<CUtensorMap>& maps, std::string& err, int box_cols = tc::KCH,
                    CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B) {
  EncodeTiledFn enc = encode_tiled();
  if (enc == nullptr) {
    err = "cuTensorMapEncodeTiled is not available from the driver";
    return false;
  }
  maps.assign(4 * (size_t)h->N, CUtensorMap{});
  for (int j = 0; j < h->N; ++j) {
    const SubDev& s = h->sub[j];
    const float* base[4] = {s.DKf, s.LKf, s.DAf, s.LAf};
    const int b[4] = {s.bK, s.bK, s.bA, s.bA};
    const int rows[4] = {(2 * s.nzn - 1) * s.bK, s.nzn * s.bK, (2 * s.nzn - 1) * s.bA, s.nzn * s.bA};
    for (int m = 0; m < 4; ++m) {
      if (base[m] == nullptr || b[m] < TILE) {
        err = "tensor maps: a subdomain has no FP32 layer blocks";
        return false;
      }
      const cuuint64_t dim[2] = {(cuuint64_t)b[m], (cuuint64_t)rows[m]};
      const cuuint64_t stride[1] = {(cuuint64_t)b[m] * sizeof(float)};
      const cuuint32_t box[2] = {(cuuint32_t)box_cols, 64};
      const cuuint32_t estr[2] = {1, 1};
      const CUresult r = enc(&maps[4 * (size_t)j + m], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                             const_cast<float*>(base[m]), dim, stride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) {
        err = "cuTensorMapEncodeTiled failed for subdomain " + std::to_string(j);
        return false;
      }
    }
  }
  return true;
}

// Launch the steps of all groups: group g on stream gs->s[g] (forked from and
// joined back to st); without a stream set everything goes to st in order.
template <typename Sched, typename Launch>
static void run_groups(const Sched& s, cudaStream_t st, const StreamSet* gs, Launch launch) {
  const int ng = (int)s.steps.size();
  const bool multi = gs != nullptr && ng > 1;
  if (multi) {
    cudaEventRecord(gs->fork, st);
    for (int g = 0; g < ng; ++g) cudaStreamWaitEvent(gs->s[g], gs->fork, 0);
  }
  size_t maxlen = 0;
  for (const auto& v : s.steps) maxlen = std::max(maxlen, v.size());
  for (size_t k = 0; k < maxlen; ++k)
    for (int g = 0; g < ng; ++g) {
      if (k >= s.steps[g].size() || s.steps[g][k].count == 0) continue;
      launch(s.steps[g][k], multi ? gs->s[g] : st);
      ++g_launch_count;
    }
  if (multi) {
    for (int g = 0; g < ng; ++g) {
      cudaEventRecord(gs->join[g], gs->s[g]);
      cudaStreamWaitEvent(st, gs->join[g], 0);
    }
  }
}

// Dynamic shared memory above 48 KiB must be enabled before the first launch
// (and before any stream capture of one).
void prepare_tile_kernels() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(k_tile_task<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, TILE_SMEM);
  cudaFuncSetAttribute(k_tile_task<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, TILE_SMEM);
  cudaFuncSetAttribute(k_tile_task_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, TILE_SMEM);
  cudaFuncSetAttribute(k_tile_task_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, std::max(TILE_SMEM, tc::SMEM));
  cudaFuncSetAttribute(k_solve_stream<double, SOLVE_CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_SMEM_MAX);
  cudaFuncSetAttribute(k_solve_stream<float, SOLVE_CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_SMEM_MAX);
  cudaFuncSetAttribute(k_solve_stream<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_SMEM_MAX);
  cudaFuncSetAttribute(k_solve_stream<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_SMEM_MAX);
  cudaFuncSetAttribute(k_solve_stream<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_SMEM_MAX);
  cudaFuncSetAttribute(k_solve_stream<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_SMEM_MAX);
  cudaFuncSetAttribute(k_solve_async, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_SMEM_MAX);
  cudaFuncSetAttribute(k_solve_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_SMEM_MAX);
  done = true;
}

template <typename T>
void run_schedule(const ScheduleT<T>& s, cudaStream_t st, const StreamSet* gs) {
  prepare_tile_kernels();
  run_groups(s, st, gs, [&](const SchedStep& step, cudaStream_t stream) {
    if constexpr (std::is_same<T, float>::value) {
      if (s.k32 && g_tc_maps != nullptr) {
        k_tile_task_tc<<<step.count, 256, std::max(TILE_SMEM, tc::SMEM), stream>>>(
            s.d_gemm + step.first, g_active, g_notspd, g_subs, static_cast<const CUtensorMap*>(g_tc_maps),
            g_potrf32);
        return;
      }
      if (s.k32) {
        k_tile_task_f32<<<step.count, 256, TILE_SMEM, stream>>>(s.d_gemm + step.first, g_active, g_notspd,
                                                                g_potrf32);
        return;
      }
    }
    k_tile_task<T><<<step.count, 256, TILE_SMEM, stream>>>(s.d_gemm + step.first, g_active, g_notspd);
  });
}

// Launch with programmatic dependent launch: the kernel may start while its
// stream predecessor finishes; it calls griddepcontrol.wait before touching
// anything the predecessor writes.
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kernel)(KArgs...), int grid, size_t smem, cudaStream_t stream, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = SOLVE_PDL ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Cluster launch of the streaming solve: CL CTAs (one thread-block cluster) per
// 64-row task, splitting its inner dimension.
template <typename T, int CL>
static void launch_stream_cluster(const SolveScheduleT<T>& s, const SchedStep& step, size_t smem, cudaStream_t stream,
                                  int src, int dst, int gather_neg, int scatter_add) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(step.count * CL);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_solve_stream<T, CL>, (const SolveTaskT<T>*)(s.d_tasks + step.first),
                     (const SubDev*)g_subs, (const int*)g_active, src, dst, gather_neg, scatter_add);
}

// variant (KB-wide solves): SOLVE_DEFAULT = the build's choice (FP32: the
// cp.async ring when every inner dimension is a multiple of 64; FP64: register
// streaming), SOLVE_ASYNC_RING, SOLVE_STREAM (register streaming, one CTA per
// 64-row task), SOLVE_STREAM_CL2 (two-CTA cluster per task), SOLVE_TMA_RING
// (FP32: the ring filled by tensor-memory-accelerator copies; needs the tensor
// maps of set_solve_maps).  A variant that
// does not apply (ring for FP64 or ragged inner dimensions, shared memory over
// the limit) falls back to the default.
template <typename T>
void run_solve_mv(const SolveScheduleT<T>& s, cudaStream_t st, int src, int dst, int gather_neg, int width,
                  const StreamSet* gs, int scatter_add, int variant) {
  prepare_tile_kernels();
  const size_t smem = solve_stream_smem<T>(s.kmax, SOLVE_CL);
  const bool stream_ok = smem <= SOLVE_SMEM_MAX;
  const size_t smem2 = solve_stream_smem<T>(s.kmax, 2);
  // FP32: asynchronous-copy pipeline when every task's inner dimension is a multiple of 64
  const size_t asmem = solve_async_smem(s.kmax);
  const bool async_ok = std::is_same<T, float>::value && s.k64 && asmem <= SOLVE_SMEM_MAX;
  int v = variant;
  if (v == SOLVE_TMA_RING && (!async_ok || asmem + 1024 > SOLVE_SMEM_MAX || g_solve_maps == nullptr))
    v = SOLVE_DEFAULT;
  if (v == SOLVE_ASYNC_RING && !async_ok) v = SOLVE_DEFAULT;
  if (v == SOLVE_STREAM && !stream_ok) v = SOLVE_DEFAULT;
  if (v == SOLVE_STREAM_CL2 && smem2 > SOLVE_SMEM_MAX) v = SOLVE_DEFAULT;
  if (v == SOLVE_DEFAULT) v = (async_ok && SOLVE_ASYNC) ? SOLVE_ASYNC_RING : (SOLVE_CL == 2 ? SOLVE_STREAM_CL2 : SOLVE_STREAM);
  run_groups(s, st, gs, [&](const SchedStep& step, cudaStream_t stream) {
    if (width != KB) {
      k_solve_step<T, PST><<<step.count, 256, 0, stream>>>(s.d_tasks + step.first, g_subs, g_active, src, dst,
                                                           gather_neg, scatter_add);
      return;
    }
    if constexpr (std::is_same<T, float>::value) {
      if (v == SOLVE_TMA_RING) {
        launch_pdl(k_solve_tma, step.count, asmem + 1024, stream, s.d_tasks + step.first, g_subs, g_active, src, dst,
                   gather_neg, scatter_add, static_cast<const CUtensorMap*>(g_solve_maps), g_kerr);
        return;
      }
      if (v == SOLVE_ASYNC_RING) {
        launch_pdl(k_solve_async, step.count, asmem, stream, s.d_tasks + step.first, g_subs, g_active, src, dst,
                   gather_neg, scatter_add);
        return;
      }
    }
    if (v == SOLVE_STREAM && stream_ok) {
      // (programmatic launch measured slower for the FP64 steps: 707 vs 690 ms per C2 step)
      k_solve_stream<T, 1><<<step.count, 256, smem, stream>>>(s.d_tasks + step.first, g_subs, g_active, src, dst,
                                                              gather_neg, scatter_add);
    } else if (v == SOLVE_STREAM_CL2 && smem2 <= SOLVE_SMEM_MAX) {
      launch_stream_cluster<T, 2>(s, step, smem2, stream, src, dst, gather_neg, scatter_add);
    } else {
      k_solve_step<T, KB><<<step.count, 256, 0, stream>>>(s.d_tasks + step.first, g_subs, g_active, src, dst,
                                                          gather_neg, scatter_add);
    }
  });
}

template void run_schedule<double>(const ScheduleT<double>&, cudaStream_t, const StreamSet*);
template void run_schedule<float>(const ScheduleT<float>&, cudaStream_t, const StreamSet*);
template void run_solve_mv<double>(const SolveScheduleT<double>&, cudaStream_t, int, int, int, int,
                                   const StreamSet*, int, int);
template void run_solve_mv<float>(const SolveScheduleT<float>&, cudaStream_t, int, int, int, int,
                                  const StreamSet*, int, int);
