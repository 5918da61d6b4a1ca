// Warm-start network: a multilayer perceptron with tanh hidden layers, its
// mean-squared-error gradient and Adam, all in FP32 on the GPU.
//
// Every layer is one tiled GEMM (64x64 output tile per CTA, 16-deep K chunks
// staged in shared memory, 4x4 outputs per thread) with the bias, the tanh
// and the tanh derivative fused into the epilogue:
//   forward      Z_l = H_{l-1} W_l^T + b_l, H_l = tanh(Z_l) (linear output layer)
//   weight grad  dW_l = G_l^T H_{l-1}, db_l = column sums of G_l
//   data grad    G_{l-1} = (G_l W_l) * (1 - H_{l-1}^2)
// with G_L = 2 (Y - T) / (B d).  The network is small (a few hundred
// thousand weights) and its batches are a few hundred rows, so these GEMMs
// take microseconds; they are not on the eigensolver's critical path.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "msgfem_warm.h"

extern long long g_launch_count;   // kernel launches issued by this library

struct msgfem_net {
  std::vector<int> sizes;
  int L = 0;                       // layers (weight matrices)
  int bmax = 0;
  long long np = 0;
  std::vector<long long> woff, boff;
  float* p = nullptr;              // parameters
  float* g = nullptr;              // gradient
  float* m = nullptr;              // Adam moments
  float* v = nullptr;
  std::vector<float*> act;         // act[l], l = 1..L-1: hidden outputs [bmax][sizes[l]]; act[L]: output
  float* d1 = nullptr;             // back-propagated gradients [bmax][max width] (ping-pong)
  float* d2 = nullptr;
  double* part = nullptr;          // loss partial sums
  double* loss = nullptr;          // [1]
  int t = 0;                       // Adam step count
  cudaStream_t st = nullptr;
};

namespace {

constexpr int GT = 64;    // output tile
constexpr int GK = 16;    // K chunk
constexpr int LOSS_BLOCKS = 240;

enum { EPI_PLAIN = 0, EPI_BIAS_TANH = 1, EPI_BIAS = 2, EPI_DTANH = 3 };

// C[m][n] = sum_k A(m, k) B(k, n) with A(m, k) = A[m lda + k] (or A[k lda + m]
// when AT) and B(k, n) = B[k ldb + n] (or B[n ldb + k] when BT), followed by
// the epilogue EPI.  H (EPI_DTANH) is read with the leading dimension of C.
template <bool AT, bool BT, int EPI>
__global__ void __launch_bounds__(256)
k_gemm(int M, int N, int K, const float* __restrict__ A, int lda, const float* __restrict__ B, int ldb,
       float* __restrict__ C, int ldc, const float* __restrict__ bias, const float* __restrict__ H) {
  __shared__ float As[GK][GT + 4];
  __shared__ float Bs[GK][GT + 4];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += GK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = tid + 256 * i;
      int m, k;
      if (AT) { m = e % GT; k = e / GT; } else { m = e / GK; k = e % GK; }
      const int gm = m0 + m, gk = k0 + k;
      float a = 0.f;
      if (gm < M && gk < K) a = AT ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
      As[k][m] = a;
      int n, kb;
      if (BT) { n = e / GK; kb = e % GK; } else { n = e % GT; kb = e / GT; }
      const int gn = n0 + n, gkb = k0 + kb;
      float b = 0.f;
      if (gn < N && gkb < K) b = BT ? B[(size_t)gn * ldb + gkb] : B[(size_t)gkb * ldb + gn];
      Bs[kb][n] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      float v = acc[i][j];
      if (EPI == EPI_BIAS_TANH) v = tanhf(v + bias[gn]);
      if (EPI == EPI_BIAS) v += bias[gn];
      if (EPI == EPI_DTANH) {
        const float h = H[(size_t)gm * ldc + gn];
        v *= 1.f - h * h;
      }
      C[(size_t)gm * ldc + gn] = v;
    }
  }
}

// G = scale (Y - T) over n entries; per-block partial sums of (Y - T)^2
__global__ void k_mse_grad(const float* __restrict__ Y, const float* __restrict__ T, long long n, float scale,
                           float* __restrict__ G, double* __restrict__ part) {
  __shared__ double red[256];
  double s = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float d = Y[e] - T[e];
    G[e] = scale * d;
    s += (double)d * (double)d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// loss = sum of the partials / n (fixed order: deterministic)
__global__ void k_loss_final(const double* __restrict__ part, int np, long long n, double* __restrict__ loss) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[0] = red[0] / (double)n;
}

// gb[n] = sum_b G[b][n]
__global__ void k_colsum(const float* __restrict__ G, int B, int N, float* __restrict__ gb) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += G[(size_t)b * N + n];
  gb[n] = s;
}

// Adam (Kingma and Ba 2015, Algorithm 1); c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t)
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float ge = g[e];
    const float me = b1 * m[e] + (1.f - b1) * ge;
    const float ve = b2 * v[e] + (1.f - b2) * ge * ge;
    m[e] = me;
    v[e] = ve;
    p[e] -= lr * (me * c1) / (sqrtf(ve * c2) + eps);
  }
}

template <bool AT, bool BT, int EPI>
void gemm(cudaStream_t st, int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
          const float* bias = nullptr, const float* H = nullptr) {
  dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
  k_gemm<AT, BT, EPI><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, H);
  ++g_launch_count;
}

// forward pass; the output goes to Y (or the handle's output buffer when Y is null)
void forward(msgfem_net* n, const float* X, int B, float* Y) {
  const float* h = X;
  for (int l = 0; l < n->L; ++l) {
    const int in = n->sizes[l], out = n->sizes[l + 1];
    const float* W = n->p + n->woff[l];
    const float* b = n->p + n->boff[l];
    const bool last = l + 1 == n->L;
    float* o = last ? (Y ? Y : n->act[n->L]) : n->act[l + 1];
    if (last) gemm<false, true, EPI_BIAS>(n->st, B, out, in, h, in, W, in, o, out, b);
    else gemm<false, true, EPI_BIAS_TANH>(n->st, B, out, in, h, in, W, in, o, out, b);
    h = o;
  }
}

// forward + backward into n->g; loss into n->loss[0]
void gradient(msgfem_net* n, const float* X, const float* T, int B) {
  forward(n, X, B, nullptr);
  const int dout = n->sizes[n->L];
  const long long cnt = (long long)B * dout;
  k_mse_grad<<<LOSS_BLOCKS, 256, 0, n->st>>>(n->act[n->L], T, cnt, 2.f / (float)cnt, n->d1, n->part);
  k_loss_final<<<1, 256, 0, n->st>>>(n->part, LOSS_BLOCKS, cnt, n->loss);
  g_launch_count += 2;
  float* G = n->d1;
  float* Gn = n->d2;
  for (int l = n->L - 1; l >= 0; --l) {
    const int in = n->sizes[l], out = n->sizes[l + 1];
    const float* hin = l == 0 ? X : n->act[l];
    gemm<true, false, EPI_PLAIN>(n->st, out, in, B, G, out, hin, in, n->g + n->woff[l], in);
    k_colsum<<<(out + 255) / 256, 256, 0, n->st>>>(G, B, out, n->g + n->boff[l]);
    ++g_launch_count;
    if (l > 0) {
      gemm<false, false, EPI_DTANH>(n->st, B, in, out, G, out, n->p + n->woff[l], in, Gn, in, nullptr, n->act[l]);
      float* tmp = G;
      G = Gn;
      Gn = tmp;
    }
  }
}

bool ok(cudaError_t e) { return e == cudaSuccess; }

}  // namespace

extern "C" {

msgfem_status msgfem_net_create(int n_sizes, const int* sizes, int max_batch, const float* init_params, void* stream,
                                msgfem_net_h* out) {
  if (!out) return MSGFEM_EINVAL;
  *out = nullptr;
  if (n_sizes < 2 || !sizes || max_batch < 1) return MSGFEM_EINVAL;
  for (int i = 0; i < n_sizes; ++i)
    if (sizes[i] < 1) return MSGFEM_EINVAL;
  msgfem_net* n = new msgfem_net();
  n->sizes.assign(sizes, sizes + n_sizes);
  n->L = n_sizes - 1;
  n->bmax = max_batch;
  n->st = static_cast<cudaStream_t>(stream);
  long long off = 0;
  int wmax = 0;
  for (int l = 0; l < n->L; ++l) {
    n->woff.push_back(off);
    off += (long long)sizes[l + 1] * sizes[l];
    n->boff.push_back(off);
    off += sizes[l + 1];
  }
  for (int i = 0; i < n_sizes; ++i) wmax = sizes[i] > wmax ? sizes[i] : wmax;
  n->np = off;
  n->act.assign(n->L + 1, nullptr);
  bool good = ok(cudaMalloc(&n->p, off * sizeof(float))) && ok(cudaMalloc(&n->g, off * sizeof(float))) &&
              ok(cudaMalloc(&n->m, off * sizeof(float))) && ok(cudaMalloc(&n->v, off * sizeof(float))) &&
              ok(cudaMalloc(&n->d1, (size_t)max_batch * wmax * sizeof(float))) &&
              ok(cudaMalloc(&n->d2, (size_t)max_batch * wmax * sizeof(float))) &&
              ok(cudaMalloc(&n->part, LOSS_BLOCKS * sizeof(double))) && ok(cudaMalloc(&n->loss, sizeof(double)));
  for (int l = 1; good && l <= n->L; ++l) good = ok(cudaMalloc(&n->act[l], (size_t)max_batch * sizes[l] * sizeof(float)));
  if (!good) {
    msgfem_net_destroy(n);
    return MSGFEM_ENOMEM;
  }
  *out = n;
  if (init_params) return msgfem_net_set_params(n, init_params);
  if (!ok(cudaMemsetAsync(n->p, 0, off * sizeof(float), n->st)) || !ok(cudaMemsetAsync(n->m, 0, off * sizeof(float), n->st)) ||
      !ok(cudaMemsetAsync(n->v, 0, off * sizeof(float), n->st)))
    return MSGFEM_ECUDA;
  return MSGFEM_OK;
}

long long msgfem_net_param_count(msgfem_net_h n) { return n ? n->np : 0; }

msgfem_status msgfem_net_get_params(msgfem_net_h n, float* host_out) {
  if (!n || !host_out) return MSGFEM_EINVAL;
  if (!ok(cudaMemcpyAsync(host_out, n->p, n->np * sizeof(float), cudaMemcpyDeviceToHost, n->st)) ||
      !ok(cudaStreamSynchronize(n->st)))
    return MSGFEM_ECUDA;
  return MSGFEM_OK;
}

msgfem_status msgfem_net_set_params(msgfem_net_h n, const float* host_in) {
  if (!n || !host_in) return MSGFEM_EINVAL;
  if (!ok(cudaMemcpyAsync(n->p, host_in, n->np * sizeof(float), cudaMemcpyHostToDevice, n->st)) ||
      !ok(cudaMemsetAsync(n->m, 0, n->np * sizeof(float), n->st)) ||
      !ok(cudaMemsetAsync(n->v, 0, n->np * sizeof(float), n->st)) || !ok(cudaStreamSynchronize(n->st)))
    return MSGFEM_ECUDA;
  n->t = 0;
  return MSGFEM_OK;
}

msgfem_status msgfem_net_forward(msgfem_net_h n, const float* X, int batch, float* Y) {
  if (!n || !X || !Y || batch < 1 || batch > n->bmax) return MSGFEM_EINVAL;
  forward(n, X, batch, Y);
  return ok(cudaGetLastError()) ? MSGFEM_OK : MSGFEM_ECUDA;
}

msgfem_status msgfem_net_gradient(msgfem_net_h n, const float* X, const float* T, int batch, float* grad_out,
                                  double* loss_out) {
  if (!n || !X || !T || batch < 1 || batch > n->bmax) return MSGFEM_EINVAL;
  gradient(n, X, T, batch);
  if (!ok(cudaGetLastError())) return MSGFEM_ECUDA;
  if (grad_out && !ok(cudaMemcpyAsync(grad_out, n->g, n->np * sizeof(float), cudaMemcpyDeviceToHost, n->st)))
    return MSGFEM_ECUDA;
  if (loss_out && !ok(cudaMemcpyAsync(loss_out, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->st)))
    return MSGFEM_ECUDA;
  if ((grad_out || loss_out) && !ok(cudaStreamSynchronize(n->st))) return MSGFEM_ECUDA;
  return MSGFEM_OK;
}

msgfem_status msgfem_net_adam_step(msgfem_net_h n, const float* X, const float* T, int batch, float lr, float beta1,
                                   float beta2, float eps, double* loss_out) {
  if (!n || !X || !T || batch < 1 || batch > n->bmax) return MSGFEM_EINVAL;
  if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f)) return MSGFEM_EINVAL;
  gradient(n, X, T, batch);
  n->t += 1;
  double p1 = 1.0, p2 = 1.0;
  for (int i = 0; i < n->t; ++i) { p1 *= beta1; p2 *= beta2; }
  const float c1 = (float)(1.0 / (1.0 - p1)), c2 = (float)(1.0 / (1.0 - p2));
  k_adam<<<304, 256, 0, n->st>>>(n->p, n->g, n->m, n->v, n->np, lr, beta1, beta2, eps, c1, c2);
  ++g_launch_count;
  if (!ok(cudaGetLastError())) return MSGFEM_ECUDA;
  if (loss_out) {
    if (!ok(cudaMemcpyAsync(loss_out, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->st)) ||
        !ok(cudaStreamSynchronize(n->st)))
      return MSGFEM_ECUDA;
  }
  return MSGFEM_OK;
}

void msgfem_net_destroy(msgfem_net_h n) {
  if (!n) return;
  for (float* q : {n->p, n->g, n->m, n->v, n->d1, n->d2}) if (q) cudaFree(q);
  for (size_t l = 1; l < n->act.size(); ++l) if (n->act[l]) cudaFree(n->act[l]);
  if (n->part) cudaFree(n->part);
  if (n->loss) cudaFree(n->loss);
  delete n;
}

}  // extern "C"
