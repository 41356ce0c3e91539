// Per-node MLP of the learned Newton initial guess: forward, backward and Adam
// in hand-written kernels.  Layers l = 0..L-1: Z_l = A_l W_l^T + b_l,
// A_(l+1) = tanh(Z_l) for hidden layers, the last layer is affine.  Loss
// L = 1/(2N) sum_n sum_o w_o (Y_no - T_no)^2.  Training is FP32 (weights,
// activations, gradients); inference can run in BF16 on the tensor cores
// (mma.sync m16n8k16, FP32 accumulation).  All reductions run in a fixed
// order (no atomics), so training is bit-reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "fsi_solid.h"
#include "internal.h"

namespace fsi {
namespace {

constexpr int TS = 64;   // output tile (rows and columns)
constexpr int TK = 16;   // reduction tile

inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

// C[m][n] = sum_k A[m][k] * B[n][k] (+ bias[n]); optional tanh.  A [M][K], B [N][K] row-major.
// 256 threads, each computes a 4x4 sub-tile of the 64x64 output tile.
template <bool TANH, bool BIAS>
__global__ void __launch_bounds__(256) gemm_nt_kernel(int M, int N, int K, const float* __restrict__ A,
                                                      const float* __restrict__ B, const float* __restrict__ bias,
                                                      float* __restrict__ C) {
  __shared__ float As[TK][TS + 4];
  __shared__ float Bs[TK][TS + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * TS, n0 = blockIdx.x * TS;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int q = threadIdx.x; q < TS * TK; q += 256) {
      const int r = q / TK, kk = q % TK;
      const int gm = m0 + r, gn = n0 + r, gk = k0 + kk;
      As[kk][r] = (gm < M && gk < K) ? A[(size_t)gm * K + gk] : 0.f;
      Bs[kk][r] = (gn < N && gk < K) ? B[(size_t)gn * K + gk] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[kk][ty * 4 + i];
        b[i] = Bs[kk][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
      if (gm < M && gn < N) {
        float v = acc[i][j] + (BIAS ? bias[gn] : 0.f);
        C[(size_t)gm * N + gn] = TANH ? tanhf(v) : v;
      }
    }
}

// C[m][n] = sum_k A[k][m] * B[k][n]  (A [K][M], B [K][N]): weight gradients dW = dZ^T A_in.
__global__ void __launch_bounds__(256) gemm_tn_kernel(int M, int N, int K, const float* __restrict__ A,
                                                      const float* __restrict__ B, float* __restrict__ C) {
  __shared__ float As[TK][TS + 4];
  __shared__ float Bs[TK][TS + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * TS, n0 = blockIdx.x * TS;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int q = threadIdx.x; q < TS * TK; q += 256) {
      const int kk = q / TS, r = q % TS;
      const int gk = k0 + kk;
      As[kk][r] = (gk < K && m0 + r < M) ? A[(size_t)gk * M + m0 + r] : 0.f;
      Bs[kk][r] = (gk < K && n0 + r < N) ? B[(size_t)gk * N + n0 + r] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[kk][ty * 4 + i];
        b[i] = Bs[kk][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
      if (gm < M && gn < N) C[(size_t)gm * N + gn] = acc[i][j];
    }
}

// C[m][n] = sum_k A[m][k] * B[k][n] * (GATE ? (1 - G[m][n]^2) : 1)   (A [M][K], B [K][N]):
// back-propagation through a layer, dA_in = dZ W, then through tanh.
template <bool GATE>
__global__ void __launch_bounds__(256) gemm_nn_kernel(int M, int N, int K, const float* __restrict__ A,
                                                      const float* __restrict__ B, const float* __restrict__ G,
                                                      float* __restrict__ C) {
  __shared__ float As[TK][TS + 4];
  __shared__ float Bs[TK][TS + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * TS, n0 = blockIdx.x * TS;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int q = threadIdx.x; q < TS * TK; q += 256) {
      const int r = q / TK, kk = q % TK;
      const int gm = m0 + r, gk = k0 + kk;
      As[kk][r] = (gm < M && gk < K) ? A[(size_t)gm * K + gk] : 0.f;
      const int kb = q / TS, c = q % TS;
      const int gkb = k0 + kb, gn = n0 + c;
      Bs[kb][c] = (gkb < K && gn < N) ? B[(size_t)gkb * N + gn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[kk][ty * 4 + i];
        b[i] = Bs[kk][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
      if (gm < M && gn < N) {
        float v = acc[i][j];
        if (GATE) {
          const float g = G[(size_t)gm * N + gn];
          v *= 1.f - g * g;
        }
        C[(size_t)gm * N + gn] = v;
      }
    }
}

// dY = w_o (Y - T) / N and the per-row loss contributions
__global__ void loss_grad_kernel(int n, int O, const float* __restrict__ Y, const float* __restrict__ T,
                                 const float* __restrict__ w, float* __restrict__ dY, float* __restrict__ row_loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float l = 0.f;
  for (int o = 0; o < O; ++o) {
    const float wo = w ? w[o] : 1.f;
    const float d = Y[(size_t)i * O + o] - T[(size_t)i * O + o];
    dY[(size_t)i * O + o] = wo * d / (float)n;
    l += 0.5f * wo * d * d;
  }
  row_loss[i] = l;
}

// column sums of a [n][N] matrix (bias gradients, loss), fixed order: one thread per column
__global__ void colsum_kernel(int n, int N, const float* __restrict__ X, float scale, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  double acc = 0.0;
  for (int i = 0; i < n; ++i) acc += (double)X[(size_t)i * N + c];
  out[c] = (float)(acc * scale);
}

__global__ void adam_kernel(long n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float c1, float c2, float eps) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void to_bf16_kernel(long n, const float* __restrict__ x, __nv_bfloat16* __restrict__ y) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

// BF16 tensor-core layer: C = A W^T + b (optional tanh), A [M][K] bf16, W [N][K] bf16,
// K a multiple of 16.  One warp per 16 x 8 output tile; mma.sync m16n8k16 with FP32
// accumulation.  Output written as FP32 and, for hidden layers, as BF16 input of the next layer.
template <bool TANH>
__global__ void mma_layer_kernel(int M, int N, int K, const __nv_bfloat16* __restrict__ A,
                                 const __nv_bfloat16* __restrict__ W, const float* __restrict__ bias,
                                 float* __restrict__ Cf, __nv_bfloat16* __restrict__ Cb) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int tiles_n = (N + 7) / 8;
  const int tm = warp / tiles_n, tn = warp % tiles_n;
  if (tm * 16 >= M) return;
  const int g = lane >> 2, t = lane & 3;
  float c[4] = {0.f, 0.f, 0.f, 0.f};
  const int r0 = tm * 16 + g, r1 = r0 + 8;
  const int ncol = tn * 8 + g;
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t a[4], b[2];
    auto ldA = [&](int r, int k) -> uint32_t {
      __nv_bfloat162 v;
      v.x = (r < M) ? A[(size_t)r * K + k] : __float2bfloat16(0.f);
      v.y = (r < M) ? A[(size_t)r * K + k + 1] : __float2bfloat16(0.f);
      return *reinterpret_cast<uint32_t*>(&v);
    };
    auto ldB = [&](int n, int k) -> uint32_t {
      __nv_bfloat162 v;
      v.x = (n < N) ? W[(size_t)n * K + k] : __float2bfloat16(0.f);
      v.y = (n < N) ? W[(size_t)n * K + k + 1] : __float2bfloat16(0.f);
      return *reinterpret_cast<uint32_t*>(&v);
    };
    a[0] = ldA(r0, k0 + 2 * t);
    a[1] = ldA(r1, k0 + 2 * t);
    a[2] = ldA(r0, k0 + 2 * t + 8);
    a[3] = ldA(r1, k0 + 2 * t + 8);
    b[0] = ldB(ncol, k0 + 2 * t);
    b[1] = ldB(ncol, k0 + 2 * t + 8);
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
  const int cc = tn * 8 + 2 * t;
  const int rows[2] = {r0, r1};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int r = rows[h], col = cc + q;
      if (r < M && col < N) {
        float v = c[2 * h + q] + bias[col];
        if (TANH) v = tanhf(v);
        if (Cf) Cf[(size_t)r * N + col] = v;
        if (Cb) Cb[(size_t)r * N + col] = __float2bfloat16(v);
      }
    }
  }
}

}  // namespace

struct Mlp {
  std::vector<int> sizes;
  std::vector<size_t> w_off, b_off;
  size_t n_params = 0;
  float* p = nullptr;   // parameters
  float* g = nullptr;   // gradients
  float* m = nullptr;   // Adam moments
  float* v = nullptr;
  __nv_bfloat16* pb = nullptr;   // BF16 copy of the weights
  int t = 0;
  int cap = 0;          // samples the activation buffers hold
  std::vector<float*> act;   // act[l]: [cap][sizes[l]] (act[0] unused: the input)
  float* dz = nullptr;
  float* dz2 = nullptr;
  float* rowloss = nullptr;
  float* lossdev = nullptr;
  __nv_bfloat16* xb = nullptr;
  __nv_bfloat16* hb = nullptr;
  __nv_bfloat16* hb2 = nullptr;
  std::string err;
};

namespace {

template <typename T>
void release(T*& q) {
  if (q) cudaFree(q);
  q = nullptr;
}

// Grows the per-sample buffers to n samples.  The old buffers are released
// and the capacity cleared first, so a failed allocation (CudaError) leaves
// the handle with no buffers rather than with freed ones; the next call
// allocates again.
void mlp_reserve(Mlp& M, int n) {
  if (n <= M.cap) return;
  M.cap = 0;
  for (float*& a : M.act) release(a);
  release(M.dz);
  release(M.dz2);
  release(M.rowloss);
  release(M.xb);
  release(M.hb);
  release(M.hb2);
  int wmax = 0;
  for (int s : M.sizes) wmax = std::max(wmax, s);
  M.act.assign(M.sizes.size(), nullptr);
  for (size_t l = 1; l < M.sizes.size(); ++l)
    FSI_CUDA_TRY(cudaMalloc(&M.act[l], sizeof(float) * (size_t)n * M.sizes[l]));
  FSI_CUDA_TRY(cudaMalloc(&M.dz, sizeof(float) * (size_t)n * wmax));
  FSI_CUDA_TRY(cudaMalloc(&M.dz2, sizeof(float) * (size_t)n * wmax));
  FSI_CUDA_TRY(cudaMalloc(&M.rowloss, sizeof(float) * (size_t)n));
  FSI_CUDA_TRY(cudaMalloc(&M.xb, sizeof(__nv_bfloat16) * (size_t)n * wmax));
  FSI_CUDA_TRY(cudaMalloc(&M.hb, sizeof(__nv_bfloat16) * (size_t)n * wmax));
  FSI_CUDA_TRY(cudaMalloc(&M.hb2, sizeof(__nv_bfloat16) * (size_t)n * wmax));
  M.cap = n;
}

void forward_f32(Mlp& M, const float* X, int n, cudaStream_t s) {
  const int L = (int)M.sizes.size() - 1;
  const float* in = X;
  for (int l = 0; l < L; ++l) {
    const int K = M.sizes[l], N = M.sizes[l + 1];
    dim3 grid(cdiv(N, TS), cdiv(n, TS));
    if (l < L - 1)
      FSI_LAUNCH(KC_OTHER, s, gemm_nt_kernel<true, true><<<grid, 256, 0, s>>>(n, N, K, in, M.p + M.w_off[l],
                                                                               M.p + M.b_off[l], M.act[l + 1]));
    else
      FSI_LAUNCH(KC_OTHER, s, gemm_nt_kernel<false, true><<<grid, 256, 0, s>>>(n, N, K, in, M.p + M.w_off[l],
                                                                                M.p + M.b_off[l], M.act[l + 1]));
    in = M.act[l + 1];
  }
}

float backward(Mlp& M, const float* X, const float* T, const float* w, int n, cudaStream_t s) {
  const int L = (int)M.sizes.size() - 1;
  const int O = M.sizes[L];
  FSI_LAUNCH(KC_OTHER, s, loss_grad_kernel<<<cdiv(n, 256), 256, 0, s>>>(n, O, M.act[L], T, w, M.dz, M.rowloss));
  FSI_LAUNCH(KC_OTHER, s, colsum_kernel<<<1, 32, 0, s>>>(n, 1, M.rowloss, 1.f / (float)n, M.lossdev));
  float* d = M.dz;
  float* d2 = M.dz2;
  for (int l = L - 1; l >= 0; --l) {
    const int K = M.sizes[l], N = M.sizes[l + 1];
    const float* ain = (l == 0) ? X : M.act[l];
    // dW_l = d^T a_in  [N][K], db_l = colsum(d)
    dim3 gw(cdiv(K, TS), cdiv(N, TS));
    FSI_LAUNCH(KC_OTHER, s, gemm_tn_kernel<<<gw, 256, 0, s>>>(N, K, n, d, ain, M.g + M.w_off[l]));
    FSI_LAUNCH(KC_OTHER, s, colsum_kernel<<<cdiv(N, 128), 128, 0, s>>>(n, N, d, 1.f, M.g + M.b_off[l]));
    if (l > 0) {
      dim3 gd(cdiv(K, TS), cdiv(n, TS));
      FSI_LAUNCH(KC_OTHER, s, gemm_nn_kernel<true><<<gd, 256, 0, s>>>(n, K, N, d, M.p + M.w_off[l], M.act[l], d2));
      std::swap(d, d2);
    }
  }
  float loss = 0.f;
  FSI_CUDA_TRY(cudaMemcpyAsync(&loss, M.lossdev, sizeof(float), cudaMemcpyDeviceToHost, s));
  FSI_CUDA_TRY(cudaStreamSynchronize(s));
  return loss;
}

}  // namespace
}  // namespace fsi

using fsi::Mlp;

extern "C" {

fsi_status fsi_mlp_create(int32_t n_layers, const int32_t* sizes, uint64_t seed, fsi_mlp_t* out) {
  if (!out || !sizes || n_layers < 1 || n_layers > 16) return FSI_ERR_ARG;
  *out = nullptr;
  for (int l = 0; l <= n_layers; ++l)
    if (sizes[l] <= 0 || sizes[l] > 4096) return FSI_ERR_ARG;
  Mlp* M = new Mlp();
  M->sizes.assign(sizes, sizes + n_layers + 1);
  size_t off = 0;
  for (int l = 0; l < n_layers; ++l) {
    M->w_off.push_back(off);
    off += (size_t)sizes[l] * sizes[l + 1];
    M->b_off.push_back(off);
    off += (size_t)sizes[l + 1];
  }
  M->n_params = off;
  // U(-a, a), a = sqrt(6 / (fan_in + fan_out)), biases zero; splitmix64 stream
  std::vector<float> h(off, 0.f);
  uint64_t st = seed;
  auto next = [&]() {
    st += 0x9E3779B97F4A7C15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  for (int l = 0; l < n_layers; ++l) {
    const double a = std::sqrt(6.0 / (sizes[l] + sizes[l + 1]));
    for (size_t q = 0; q < (size_t)sizes[l] * sizes[l + 1]; ++q) h[M->w_off[l] + q] = (float)((2.0 * next() - 1.0) * a);
  }
  if (cudaMalloc(&M->p, sizeof(float) * off) != cudaSuccess || cudaMalloc(&M->g, sizeof(float) * off) != cudaSuccess ||
      cudaMalloc(&M->m, sizeof(float) * off) != cudaSuccess || cudaMalloc(&M->v, sizeof(float) * off) != cudaSuccess ||
      cudaMalloc(&M->pb, sizeof(__nv_bfloat16) * off) != cudaSuccess ||
      cudaMalloc(&M->lossdev, sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    fsi_mlp_destroy(reinterpret_cast<fsi_mlp_t>(M));   // frees what was allocated
    return FSI_ERR_OOM;
  }
  if (cudaMemcpy(M->p, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(M->m, 0, sizeof(float) * off) != cudaSuccess || cudaMemset(M->v, 0, sizeof(float) * off) != cudaSuccess ||
      cudaMemset(M->g, 0, sizeof(float) * off) != cudaSuccess) {
    cudaGetLastError();
    fsi_mlp_destroy(reinterpret_cast<fsi_mlp_t>(M));
    return FSI_ERR_CUDA;
  }
  *out = reinterpret_cast<fsi_mlp_t>(M);
  return FSI_OK;
}

fsi_status fsi_mlp_destroy(fsi_mlp_t h) {
  Mlp* M = reinterpret_cast<Mlp*>(h);
  if (!M) return FSI_OK;
  cudaDeviceSynchronize();
  for (float* a : M->act) if (a) cudaFree(a);
  for (void* q : {(void*)M->p, (void*)M->g, (void*)M->m, (void*)M->v, (void*)M->pb, (void*)M->dz, (void*)M->dz2,
                  (void*)M->rowloss, (void*)M->lossdev, (void*)M->xb, (void*)M->hb, (void*)M->hb2})
    if (q) cudaFree(q);
  delete M;
  return FSI_OK;
}

int64_t fsi_mlp_num_params(fsi_mlp_t h) {
  Mlp* M = reinterpret_cast<Mlp*>(h);
  return M ? (int64_t)M->n_params : -1;
}

fsi_status fsi_mlp_params(fsi_mlp_t h, float* host, int32_t set) {
  Mlp* M = reinterpret_cast<Mlp*>(h);
  if (!M || !host) return FSI_ERR_ARG;
  cudaError_t e = set ? cudaMemcpy(M->p, host, sizeof(float) * M->n_params, cudaMemcpyHostToDevice)
                      : cudaMemcpy(host, M->p, sizeof(float) * M->n_params, cudaMemcpyDeviceToHost);
  if (set) M->t = 0;
  return e == cudaSuccess ? FSI_OK : FSI_ERR_CUDA;
}

fsi_status fsi_mlp_forward(fsi_mlp_t h, const float* X, int32_t n, float* Y, int32_t bf16, void* stream) {
  Mlp* M = reinterpret_cast<Mlp*>(h);
  if (!M || !X || !Y || n <= 0) return FSI_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    fsi::mlp_reserve(*M, n);
    const int L = (int)M->sizes.size() - 1;
    if (!bf16) {
      fsi::forward_f32(*M, X, n, s);
      FSI_CUDA_TRY(cudaMemcpyAsync(Y, M->act[L], sizeof(float) * (size_t)n * M->sizes[L], cudaMemcpyDeviceToDevice, s));
    } else {
      for (int l = 0; l < L; ++l)
        if (M->sizes[l] % 16) return FSI_ERR_ARG;   // BF16 path needs layer inputs in multiples of 16
      FSI_LAUNCH(fsi::KC_OTHER, s, fsi::to_bf16_kernel<<<512, 256, 0, s>>>((long)M->n_params, M->p, M->pb));
      FSI_LAUNCH(fsi::KC_OTHER, s, fsi::to_bf16_kernel<<<512, 256, 0, s>>>((long)n * M->sizes[0], X, M->xb));
      const __nv_bfloat16* in = M->xb;
      for (int l = 0; l < L; ++l) {
        const int K = M->sizes[l], N = M->sizes[l + 1];
        const long warps = (long)((n + 15) / 16) * ((N + 7) / 8);
        __nv_bfloat16* outb = (l % 2 == 0) ? M->hb : M->hb2;
        if (l < L - 1)
          FSI_LAUNCH(fsi::KC_OTHER, s, fsi::mma_layer_kernel<true><<<fsi::cdiv(warps * 32, 128), 128, 0, s>>>(
              n, N, K, in, M->pb + M->w_off[l], M->p + M->b_off[l], nullptr, outb));
        else
          FSI_LAUNCH(fsi::KC_OTHER, s, fsi::mma_layer_kernel<false><<<fsi::cdiv(warps * 32, 128), 128, 0, s>>>(
              n, N, K, in, M->pb + M->w_off[l], M->p + M->b_off[l], Y, nullptr));
        in = outb;
      }
    }
    FSI_CUDA_TRY(cudaGetLastError());
    FSI_CUDA_TRY(cudaStreamSynchronize(s));
  } catch (const fsi::CudaError& e) {
    M->err = e.msg;
    return FSI_ERR_CUDA;
  } catch (const std::bad_alloc&) {
    M->err = "host allocation failed";
    return FSI_ERR_OOM;
  } catch (const std::exception& e) {
    M->err = e.what();
    return FSI_ERR_ARG;
  }
  return FSI_OK;
}

fsi_status fsi_mlp_train_step(fsi_mlp_t h, const float* X, const float* T, int32_t n, const float* w_out, float lr,
                              int32_t apply, float* loss_out, float* grad_host, void* stream) {
  Mlp* M = reinterpret_cast<Mlp*>(h);
  if (!M || !X || !T || n <= 0) return FSI_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    fsi::mlp_reserve(*M, n);
    fsi::forward_f32(*M, X, n, s);
    const float loss = fsi::backward(*M, X, T, w_out, n, s);
    if (loss_out) *loss_out = loss;
    if (grad_host)
      FSI_CUDA_TRY(cudaMemcpy(grad_host, M->g, sizeof(float) * M->n_params, cudaMemcpyDeviceToHost));
    if (apply) {
      M->t += 1;
      const float b1 = 0.9f, b2 = 0.999f;
      const float c1 = 1.f - std::pow(b1, (float)M->t), c2 = 1.f - std::pow(b2, (float)M->t);
      FSI_LAUNCH(fsi::KC_OTHER, s, fsi::adam_kernel<<<512, 256, 0, s>>>((long)M->n_params, M->p, M->g, M->m, M->v,
                                                                         lr, b1, b2, c1, c2, 1e-8f));
    }
    FSI_CUDA_TRY(cudaGetLastError());
    FSI_CUDA_TRY(cudaStreamSynchronize(s));
  } catch (const fsi::CudaError& e) {
    M->err = e.msg;
    return FSI_ERR_CUDA;
  } catch (const std::bad_alloc&) {
    M->err = "host allocation failed";
    return FSI_ERR_OOM;
  } catch (const std::exception& e) {
    M->err = e.what();
    return FSI_ERR_ARG;
  }
  return FSI_OK;
}

}  // extern "C"
