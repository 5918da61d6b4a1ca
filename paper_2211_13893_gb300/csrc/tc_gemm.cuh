// Tensor-core tile GEMM of the FP32 layer-block factorisation (mixed path):
// C(64 x 64) [+]= sign A(64 x K) B(64 x K)^T on the fifth-generation tensor
// cores with FP32 accuracy.  Every FP32 operand is split exactly into three
// TF32 parts, a = a_hi + a_mid + a_lo (11 + 11 + 2 significant bits, each part
// rounded to TF32), and the products of weight down to 2^-22 are formed:
//   a b ~ a_hi b_hi + a_hi b_mid + a_mid b_hi + a_mid b_mid + a_hi b_lo + a_lo b_hi,
// so that the dropped terms are below 2^-33 |a| |b| and the accuracy is that of
// the tensor core's FP32 accumulation (a split into two parts, the published
// 3xTF32 scheme, leaves 2^-21 and measurably slowed the conjugate-gradient
// solves that this factor preconditions).
//
// Data path per 32-deep K chunk (one CTA per tile task):
//   TMA (cp.async.bulk.tensor.2d, 128-byte swizzle) moves the 64 x 32 FP32
//   tiles of A and B from the layer-block arrays into shared memory, two chunks
//   in flight on an mbarrier ring;  the CTA splits them at the same swizzled
//   positions into the TF32 parts (the canonical K-major layout the MMA
//   reads);  one elected thread issues 4 x 6 tcgen05.mma kind::tf32 (M = 128:
//   rows 64..127 of A are zero, N = 64, K = 8) into a 64-column TMEM
//   accumulator and commits them to an mbarrier;  after the last chunk warps
//   0-1 read rows 0..63 back with tcgen05.ld and update C.
// Every mbarrier wait is bounded (a second of %globaltimer); a timeout sets
// bit 1 of the subdomain's error flag, waits once more for the work in flight
// and still frees the TMEM.
#pragma once
#include <cuda.h>
#include <cstdint>

namespace tc {

constexpr int THREADS = 256;
constexpr int KCH = 32;                       // K chunk (32 FP32 = one 128-byte swizzle row)
constexpr uint32_t TMEM_COLS = 64;
// instruction descriptor: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9, 10-12 = 2),
// both K-major, N = 64 (bits 17-22 = N / 8), M = 128 (bits 24-28 = M / 16)
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
// shared-memory layout (bytes from a 1024-aligned base)
constexpr int OFF_RAW_A = 0;          // [2][64 rows][128 B]  TMA destinations
constexpr int OFF_RAW_B = 16384;      // [2][64 rows][128 B]
constexpr int OFF_A = 32768;          // 3 parts (hi, mid, lo) x [128 rows][128 B], rows 64..127 zero
constexpr int A_PART = 16384;
constexpr int OFF_B = 81920;          // 3 parts x [64 rows][128 B]
constexpr int B_PART = 8192;
constexpr int OFF_BAR = 106496;       // full[2], mma (8 B each), TMEM address (4 B)
constexpr int SMEM = OFF_BAR + 64 + 1024;   // + alignment slack
constexpr uint32_t CHUNK_BYTES = 2 * 64 * 128;   // A and B tiles of one chunk
constexpr unsigned long long TIMEOUT_NS = 1000000000ull;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// wait for the phase of the given parity, at most TIMEOUT_NS; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_test(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (!mbar_test(bar, parity))
    if (gtimer() - t0 > TIMEOUT_NS) return false;
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)2 << 61);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(IDESC), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// round to TF32 (nearest, ties away), returned as an FP32 bit pattern
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// x = hi + mid + lo exactly: hi = tf32(x), mid = tf32(x - hi), lo = x - hi - mid
// (both differences are exact in FP32; lo keeps the last two bits of x)
__device__ __forceinline__ void split3(float x, float& hi, float& mid, float& lo) {
  hi = to_tf32(x);
  const float r = x - hi;
  mid = to_tf32(r);
  lo = to_tf32(r - mid);
}

// 16 consecutive TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Tensor map and (x, y) coordinates of the tile at p: one of the subdomain's
// four FP32 arrays (K: layer blocks D|E, inverses; A11: the same), each a
// row-major 2-D array of b columns.
__device__ __forceinline__ const CUtensorMap* locate(const SubDev& s, const CUtensorMap* maps, int sub, const float* p,
                                                     int& x, int& y) {
  const float* base[4] = {s.DKf, s.LKf, s.DAf, s.LAf};
  const int b[4] = {s.bK, s.bK, s.bA, s.bA};
  const int rows[4] = {(2 * s.nzn - 1) * s.bK, s.nzn * s.bK, (2 * s.nzn - 1) * s.bA, s.nzn * s.bA};
  for (int m = 0; m < 4; ++m) {
    if (base[m] == nullptr || p < base[m]) continue;
    const long long off = p - base[m];
    if (off >= (long long)rows[m] * b[m]) continue;
    y = (int)(off / b[m]);
    x = (int)(off % b[m]);
    return maps + 4 * (size_t)sub + m;
  }
  return nullptr;
}

// One G_TRANSB tile task (no post-multiplication) on the tensor cores.
template <typename Task>
__device__ void gemm_task(const Task& t, unsigned char* smem_raw, const SubDev* subs, const CUtensorMap* maps,
                          int* notspd) {
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t base = saddr(sm);
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t bar_full0 = base + OFF_BAR, bar_mma = base + OFF_BAR + 16;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + OFF_BAR + 32);
  __shared__ const CUtensorMap* smap[2];
  __shared__ int scoord[4];
  if (tid == 0) {
    mbar_init(bar_full0, 1);
    mbar_init(bar_full0 + 8, 1);
    mbar_init(bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    int xa = 0, ya = 0, xb = 0, yb = 0;
    smap[0] = locate(subs[t.sub], maps, t.sub, t.A, xa, ya);
    smap[1] = locate(subs[t.sub], maps, t.sub, t.B, xb, yb);
    scoord[0] = xa; scoord[1] = ya; scoord[2] = xb; scoord[3] = yb;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // zero rows 64..127 of the three A parts (M = 128 with 64 real rows)
  for (int e = tid; e < 3 * 512; e += THREADS) {
    const int part = e >> 9, i = e & 511;
    reinterpret_cast<float4*>(sm + OFF_A + A_PART * part + 8192)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const CUtensorMap* mapA = smap[0];
  const CUtensorMap* mapB = smap[1];
  bool ok = mapA != nullptr && mapB != nullptr;   // the same in every thread
  const int nch = t.K / KCH;
  if (ok && tid == 0) {
    mbar_expect_tx(bar_full0, CHUNK_BYTES);
    tma_load_2d(base + OFF_RAW_A, mapA, scoord[0], scoord[1], bar_full0);
    tma_load_2d(base + OFF_RAW_B, mapB, scoord[2], scoord[3], bar_full0);
  }
  // work in flight when a wait gives up: the copy of chunk `late_c` (-1 none)
  // and the products of chunk `late_m` (-1 none)
  int late_c = -1, late_m = -1;
  for (int c = 0; c < nch && ok; ++c) {
    const int s = c & 1;
    bool w = mbar_wait(bar_full0 + 8 * s, (c >> 1) & 1);
    if (c > 0) w = mbar_wait(bar_mma, (c - 1) & 1) && w;   // the previous products have read the operands
    if (!__syncthreads_and(w)) {                             // one decision for the whole CTA
      ok = false;
      late_c = c;
      late_m = c - 1;
      break;
    }
    if (tid == 0 && c + 1 < nch) {
      // raw buffer s ^ 1 was last read by the split of chunk c - 1, before the barrier above
      const uint32_t bar = bar_full0 + 8 * (s ^ 1);
      fence_async_smem();
      mbar_expect_tx(bar, CHUNK_BYTES);
      tma_load_2d(base + OFF_RAW_A + 8192 * (s ^ 1), mapA, scoord[0] + KCH * (c + 1), scoord[1], bar);
      tma_load_2d(base + OFF_RAW_B + 8192 * (s ^ 1), mapB, scoord[2] + KCH * (c + 1), scoord[3], bar);
    }
    // split the raw tiles at the same (swizzled) positions: 16-byte chunks
    for (int e = tid; e < 1024; e += THREADS) {
      const int isb = e >> 9, i = e & 511;
      const float4 v = reinterpret_cast<const float4*>(sm + (isb ? OFF_RAW_B : OFF_RAW_A) + 8192 * s)[i];
      float4 p0, p1, p2;
      split3(v.x, p0.x, p1.x, p2.x);
      split3(v.y, p0.y, p1.y, p2.y);
      split3(v.z, p0.z, p1.z, p2.z);
      split3(v.w, p0.w, p1.w, p2.w);
      unsigned char* dst = sm + (isb ? OFF_B : OFF_A);
      const int stride = isb ? B_PART : A_PART;
      reinterpret_cast<float4*>(dst)[i] = p0;
      reinterpret_cast<float4*>(dst + stride)[i] = p1;
      reinterpret_cast<float4*>(dst + 2 * stride)[i] = p2;
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < KCH / 8; ++ks) {
        const uint32_t o = 32 * ks;   // 8 TF32 along K
        const uint64_t ah = sdesc(base + OFF_A + o), am = sdesc(base + OFF_A + A_PART + o),
                       al = sdesc(base + OFF_A + 2 * A_PART + o);
        const uint64_t bh = sdesc(base + OFF_B + o), bm = sdesc(base + OFF_B + B_PART + o),
                       bl = sdesc(base + OFF_B + 2 * B_PART + o);
        // the smallest products first
        mma_tf32(tmem, al, bh, (c > 0 || ks > 0) ? 1u : 0u);
        mma_tf32(tmem, ah, bl, 1u);
        mma_tf32(tmem, am, bm, 1u);
        mma_tf32(tmem, am, bh, 1u);
        mma_tf32(tmem, ah, bm, 1u);
        mma_tf32(tmem, ah, bh, 1u);
      }
      mma_commit(bar_mma);
    }
  }
  if (ok && nch > 0 && !__syncthreads_and(mbar_wait(bar_mma, (nch - 1) & 1))) {
    ok = false;
    late_m = nch - 1;
  }
  if (!ok) {
    // gave up: one more bounded wait for what is still in flight, then report
    if (late_c >= 0) mbar_wait(bar_full0 + 8 * (late_c & 1), (late_c >> 1) & 1);
    if (late_m >= 0) mbar_wait(bar_mma, late_m & 1);
    if (tid == 0 && notspd != nullptr) atomicOr(&notspd[t.sub >= 0 ? t.sub : 0], 2);
  }
  fence_after();
  if (ok && warp < 2) {
    // rows 32 warp + lane of D live in TMEM lanes of the same index
    const int r = 32 * warp + (tid & 31);
    const float sgn = (t.flags & G_NEG) ? -1.f : 1.f;
    float* crow = t.C + (size_t)r * t.ldc;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + 16 * q, v);
#pragma unroll
      for (int j = 0; j < 16; j += 4) {
        float4* cp = reinterpret_cast<float4*>(crow + 16 * q + j);
        float4 o = make_float4(sgn * v[j], sgn * v[j + 1], sgn * v[j + 2], sgn * v[j + 3]);
        if (t.flags & G_ACC) {
          const float4 c = *cp;
          o.x += c.x; o.y += c.y; o.z += c.z; o.w += c.w;
        }
        *cp = o;
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

}  // namespace tc
