// Energy-error evaluation that allocates no memory (msgfem_energy_error_noalloc).
//
// The partial sums live in a file-scope __device__ array of fixed size instead
// of memory owned by the handle, so a caller that cannot allocate device memory
// at the point of the call can still evaluate ||u_ref - u||_a / ||u_ref||_a for
// its own device vectors.  Every GPU that loads the library holds this array
// until the process exits.
#include "internal.h"

#define NOALLOC_EPT 4                 // elements per thread
#define NOALLOC_THREADS 256
#define NOALLOC_MAX_BLOCKS 4096       // -> at most 4,194,304 elements per call

// [2 b], [2 b + 1]: per-block sums of d^T K_e d and ref^T K_e ref; the last
// slot holds the result of the most recent call.  64 KiB + 8 bytes.
static __device__ __align__(256) double g_noalloc_scratch[2 * NOALLOC_MAX_BLOCKS + 1];

namespace {

// Each thread sums NOALLOC_EPT consecutive elements; each block writes its own
// two slots, so no slot has to be cleared between calls.
__global__ void __launch_bounds__(NOALLOC_THREADS)
k_energy_blocks(const double* __restrict__ Ke, int layered, const int* __restrict__ etype,
                const double* __restrict__ ref, const double* __restrict__ u, int NX, int NY, int NZ,
                const int* __restrict__ user_of_node, double* __restrict__ scratch) {
  __shared__ double red[2][NOALLOC_THREADS];
  double e0 = 0.0, e1 = 0.0;
  const int nel = NX * NY * NZ;
  const int first = (blockIdx.x * NOALLOC_THREADS + threadIdx.x) * NOALLOC_EPT;
  for (int el = first; el < min(first + NOALLOC_EPT, nel); ++el) {
    const int ke = el % NZ, ij = el / NZ, je = ij % NY, ie = ij / NY;
    double d[24], r[24];
    for (int a = 0; a < 8; ++a) {
      int node = ((ie + (a & 1)) * (NY + 1) + je + ((a >> 1) & 1)) * (NZ + 1) + ke + (a >> 2);
      if (user_of_node) node = user_of_node[node];   // hexahedron list: vectors in the list's node order
      for (int c = 0; c < 3; ++c) {
        r[3 * a + c] = ref[3 * node + c];
        d[3 * a + c] = r[3 * a + c] - u[3 * node + c];
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
  for (int st = NOALLOC_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      red[0][threadIdx.x] += red[0][threadIdx.x + st];
      red[1][threadIdx.x] += red[1][threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scratch[2 * blockIdx.x] = red[0][0];
    scratch[2 * blockIdx.x + 1] = red[1][0];
  }
}

// Fixed-order reduction of the block sums; writes the ratio to the result
// slot and, when given, to a device output.
__global__ void k_energy_final(double* __restrict__ scratch, int nblocks, double* __restrict__ out_dev) {
  __shared__ double red[2][256];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += 256) {
    a += scratch[2 * i];
    b += scratch[2 * i + 1];
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      red[0][threadIdx.x] += red[0][threadIdx.x + st];
      red[1][threadIdx.x] += red[1][threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double num = red[0][0], den = red[1][0];
    const double e = den > 0.0 ? sqrt(fmax(num, 0.0) / den) : 0.0;
    scratch[2 * NOALLOC_MAX_BLOCKS] = e;
    if (out_dev) *out_dev = e;
  }
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// Device address of the array on the handle's device, looked up once by
// msgfem_setup with that device current: host code may not pass the symbol
// itself to a kernel (in host code it names a host-side stand-in).  Taking the
// address also loads this file's module, so a later call loads nothing.
msgfem_status noalloc_prepare(msgfem* h) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaGetSymbolAddress", __FILE__, __LINE__);
  h->noalloc_scratch = static_cast<double*>(p);
  return MSGFEM_OK;
}

extern "C" msgfem_status msgfem_energy_error_noalloc(msgfem_h h, const double* u, const double* u_ref,
                                                     double* energy_err_out) {
  if (!h || !u || !u_ref || !energy_err_out) return MSGFEM_EINVAL;
  if (h->stage < 2) {
    h->err = "msgfem_energy_error_noalloc needs the element stiffness of msgfem_local_spaces";
    return MSGFEM_ESTATE;
  }
  const long long nel = (long long)h->NX * h->NY * h->NZ;
  const long long per_block = (long long)NOALLOC_THREADS * NOALLOC_EPT;
  const long long nblocks = (nel + per_block - 1) / per_block;
  if (nblocks > NOALLOC_MAX_BLOCKS) {
    h->err = "msgfem_energy_error_noalloc: mesh has " + std::to_string(nel) + " elements, more than the " +
             std::to_string((long long)NOALLOC_MAX_BLOCKS * per_block) + " its fixed scratch array supports";
    return MSGFEM_EINVAL;
  }
  if (!on_device(u) || !on_device(u_ref)) {
    h->err = "msgfem_energy_error_noalloc: u and u_ref must be device pointers";
    return MSGFEM_EINVAL;
  }
  // kernels go to the current device: it must be the handle's, whose copy of
  // the array msgfem_setup resolved
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaGetDevice", __FILE__, __LINE__);
  if (dev != h->device || h->noalloc_scratch == nullptr) {
    h->err = "msgfem_energy_error_noalloc: call with the handle's device (" + std::to_string(h->device) +
             ") current, not device " + std::to_string(dev);
    return MSGFEM_EINVAL;
  }
  double* scratch = h->noalloc_scratch;
  const bool dev_out = on_device(energy_err_out);
  if (!dev_out) {
    // a host result needs a copy and a wait on the stream, which a stream capture cannot hold
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(h->stream, &cs);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamIsCapturing", __FILE__, __LINE__);
    if (cs != cudaStreamCaptureStatusNone) {
      h->err = "msgfem_energy_error_noalloc: the stream is being captured; pass a device pointer as energy_err_out";
      return MSGFEM_ESTATE;
    }
  }
  k_energy_blocks<<<(unsigned)nblocks, NOALLOC_THREADS, 0, h->stream>>>(h->d_Ke, h->layered,
                                                                       h->typed ? h->d_etype : nullptr, u_ref, u,
                                                                       h->NX, h->NY, h->NZ, h->d_user_of_node,
                                                                       scratch);
  k_energy_final<<<1, 256, 0, h->stream>>>(scratch, (int)nblocks, dev_out ? energy_err_out : nullptr);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "energy kernels", __FILE__, __LINE__);
  if (!dev_out) {
    e = cudaMemcpyAsync(energy_err_out, scratch + 2 * NOALLOC_MAX_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost,
                        h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync", __FILE__, __LINE__);
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize", __FILE__, __LINE__);
  }
  return MSGFEM_OK;
}
