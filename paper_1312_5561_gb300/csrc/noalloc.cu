// Allocation-free dot products.
//
// fsi_dots_static computes the same deterministic FP64 dot products as the
// Krylov reduction of the solver (304 CTA partial sums, then a fixed-order
// sum of the partials), but its partial sums live in a file-scope
// __device__ array instead of memory allocated by a handle.  It exists for
// callers that may not allocate device memory at all: a coupling driver or
// host application that owns every device allocation (for example a fluid
// code that hands the solid library fixed buffers and forbids allocation in
// its time loop), or code with a no-allocation policy after start-up because
// cudaMalloc / cudaFree synchronise the device and stall the other streams.
#include <cuda_runtime.h>

#include "fsi_solid.h"

namespace {

// Partial sums per vector: the solver's reductions split every dot product
// into 2 x 152 CTA partials (two per SM of a GB300), and so does this call,
// so its sums are bit-identical to the solver's.
constexpr int kBlocks = 2 * 152;
constexpr int kMaxVectors = FSI_DOTS_STATIC_MAX_VECTORS;
constexpr int kThreads = 256;

// Scratch: one partial sum per CTA and vector (kMaxVectors * kBlocks * 8 B = 76 KiB).
// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) double g_dots_scratch[kMaxVectors * kBlocks];

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double s[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < kThreads / 32) ? s[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;
}

__global__ void dots_partial_kernel(const double* __restrict__ V, long long ldv, const double* __restrict__ y,
                                    long long n, double* __restrict__ partial) {
  const int i = blockIdx.y;
  const double* x = V + (size_t)i * ldv;
  double acc = 0.0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    acc += x[k] * y[k];
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[(size_t)i * kBlocks + blockIdx.x] = acc;
}

__global__ void dots_final_kernel(const double* __restrict__ partial, double* __restrict__ out) {
  const int i = blockIdx.x;
  double acc = 0.0;
  for (int k = threadIdx.x; k < kBlocks; k += blockDim.x) acc += partial[(size_t)i * kBlocks + k];
  acc = block_sum(acc);
  if (threadIdx.x == 0) out[i] = acc;
}

// Device address of the scratch array in the current device's current
// context.  The address belongs to a context, not to a device (it changes
// after cudaDeviceReset, for instance), so it is looked up on every call; the
// lookup allocates nothing.
cudaError_t scratch_address(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_dots_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

}  // namespace

extern "C" fsi_status fsi_dots_static(const double* V, int64_t ldv, int32_t k, const double* y, int64_t n,
                                      double* out, void* stream) {
  if (!V || !y || !out || n < 0 || k <= 0 || k > kMaxVectors || (k > 1 && ldv < n)) return FSI_ERR_ARG;
  double* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return FSI_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dim3 grid(kBlocks, k);
  dots_partial_kernel<<<grid, kThreads, 0, s>>>(V, ldv, y, n, scratch);
  dots_final_kernel<<<k, kThreads, 0, s>>>(scratch, out);
  if (cudaGetLastError() != cudaSuccess) return FSI_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return FSI_ERR_CUDA;
  return FSI_OK;
}
