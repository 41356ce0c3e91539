// Sparse and dense linear algebra of the linear solve: 4x4 block-CSR SpMV and
// residuals, damped block-Jacobi smoothing, aggregation transfers, Galerkin
// coarse operators, the block-diagonal dense coarse solve and the FP64
// vector kernels of the Krylov method (deterministic reductions).
#include <cuda_bf16.h>

#include <cmath>
#include <type_traits>
#include <utility>

#include "internal.h"

namespace fsi {

namespace {

inline int blocks_for(long n, int t) { return (int)((n + t - 1) / t); }

template <typename T>
struct Vec4;
template <>
struct Vec4<double> {
  __device__ __forceinline__ static void load(const double* p, double v[4]) {
    double2 a = reinterpret_cast<const double2*>(p)[0];
    double2 b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  __device__ __forceinline__ static void store(double* p, const double v[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
};
template <>
struct Vec4<float> {
  __device__ __forceinline__ static void load(const float* p, float v[4]) {
    float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
  __device__ __forceinline__ static void store(float* p, const float v[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};

template <int R>
struct Lanes {
  static constexpr int v = R <= 4 ? 4 : 8;
};

// Block-row kernel for R x C blocks: a group of Lanes<R> threads owns one
// block row; thread r accumulates row r of every block of that row.
//   MODE 0: y = A x     MODE 1: y = b - A x     MODE 3: y += A x
//   MODE 2: y = x + omega D^-1 (b - A x)   (one damped block-Jacobi sweep, R == C)
template <typename TV, typename TX, typename TA, int R, int C, int MODE>
__global__ void bsr_kernel(int n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                           const TV* __restrict__ vals, const TX* __restrict__ x, const TX* __restrict__ b,
                           const TV* __restrict__ dinv, TA omega, TX* __restrict__ y) {
  constexpr int LN = Lanes<R>::v;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = t / LN, r = t % LN;
  const bool active = row < n && r < R;
  TA acc = 0;
  if (active) {
    const int k0 = row_ptr[row], k1 = row_ptr[row + 1];
    int k = k0;
    if constexpr (C == 4) {
      // four blocks per step: all index, value and vector loads are issued
      // before the products, so each warp keeps four blocks in flight
      for (; k + 4 <= k1; k += 4) {
        int j[4];
        TV v[4][4];
        TX xx[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) j[u] = col_idx[k + u];
#pragma unroll
        for (int u = 0; u < 4; ++u) Vec4<TV>::load(vals + (size_t)(k + u) * (R * C) + r * C, v[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) Vec4<TX>::load(x + (size_t)j[u] * C, xx[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u)
          acc += (TA)v[u][0] * (TA)xx[u][0] + (TA)v[u][1] * (TA)xx[u][1] + (TA)v[u][2] * (TA)xx[u][2] +
                 (TA)v[u][3] * (TA)xx[u][3];
      }
    }
    for (; k < k1; ++k) {
      const int j = col_idx[k];
      const TV* a = vals + (size_t)k * (R * C) + r * C;
      const TX* xv = x + (size_t)j * C;
      if constexpr (C == 4) {
        TV v[4];
        TX xx[4];
        Vec4<TV>::load(a, v);
        Vec4<TX>::load(xv, xx);
        acc += (TA)v[0] * (TA)xx[0] + (TA)v[1] * (TA)xx[1] + (TA)v[2] * (TA)xx[2] + (TA)v[3] * (TA)xx[3];
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) acc += (TA)a[c] * (TA)xv[c];
      }
    }
  }
  const size_t o = (size_t)row * R + r;
  if constexpr (MODE == 0) {
    if (active) y[o] = (TX)acc;
  } else if constexpr (MODE == 1) {
    if (active) y[o] = (TX)((TA)b[o] - acc);
  } else if constexpr (MODE == 3) {
    if (active) y[o] = (TX)((TA)y[o] + acc);
  } else {
    static_assert(R == C, "Jacobi sweep needs square blocks");
    const TA res = active ? (TA)b[o] - acc : (TA)0;
    const unsigned base = (threadIdx.x & 31) & ~(unsigned)(LN - 1);
    TA rr[R];
#pragma unroll
    for (int c = 0; c < R; ++c) rr[c] = __shfl_sync(0xffffffffu, res, base + c);
    if (active) {
      const TV* d = dinv + (size_t)row * (R * R) + r * R;
      TA corr = 0;
#pragma unroll
      for (int c = 0; c < R; ++c) corr += (TA)d[c] * rr[c];
      y[o] = (TX)((TA)x[o] + omega * corr);
    }
  }
}

// Block-row kernel for 7-row blocks (coarse levels, restriction): one warp
// per block row.  Lane (j, r) = (lane / 7, lane % 7), j < 4: slot j takes
// every fourth block of the row and row r of each; the four slot sums are
// then added in a fixed order ((s0 + s2) + (s1 + s3)).  Long coarse rows
// (~50 blocks) thereby keep 28 lanes busy instead of 7.  Modes as above.
// (Staging each group of four blocks through shared memory with aligned
// vector loads, software-pipelined one group ahead, measured 5 % slower on
// the 3.1M-element tube, and 40 % slower with BF16 values; a warp that
// streams the row's values with coalesced scalar loads and keeps one running
// sum per lane position lost to the CTA-per-row kernel in the autotuner on
// every coarse level of that tube.)
template <typename TV, typename TX, typename TA, int C, int MODE, typename TD = TV>
__global__ void bsr7_kernel(int n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                            const TV* __restrict__ vals, const TX* __restrict__ x, const TX* __restrict__ b,
                            const TD* __restrict__ dinv, TA omega, TX* __restrict__ y) {
  constexpr int R = 7;
  const int row = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int j = lane / R, r = lane % R;
  TA acc = 0;
  if (row < n && lane < 4 * R) {
    const int k1 = row_ptr[row + 1];
    int k = row_ptr[row] + j;
    if constexpr (C == R) {
      // two blocks per slot and step: both blocks' loads are issued before the products
      // (four blocks per slot, or prefetching the next pair in the Galerkin products,
      // measured no faster)
      for (; k + 4 < k1; k += 8) {
        const TV* a0 = vals + (size_t)k * (R * C) + r * C;
        const TV* a1 = vals + (size_t)(k + 4) * (R * C) + r * C;
        const TX* x0 = x + (size_t)col_idx[k] * C;
        const TX* x1 = x + (size_t)col_idx[k + 4] * C;
        TA v0[C], v1[C], y0[C], y1[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
          v0[c] = (TA)a0[c];
          v1[c] = (TA)a1[c];
          y0[c] = (TA)x0[c];
          y1[c] = (TA)x1[c];
        }
#pragma unroll
        for (int c = 0; c < C; ++c) acc += v0[c] * y0[c];
#pragma unroll
        for (int c = 0; c < C; ++c) acc += v1[c] * y1[c];
      }
    }
    for (; k < k1; k += 4) {
      const TV* a = vals + (size_t)k * (R * C) + r * C;
      const TX* xv = x + (size_t)col_idx[k] * C;
      if constexpr (C == 4) {
        TV v[4];
        TX xx[4];
        Vec4<TV>::load(a, v);
        Vec4<TX>::load(xv, xx);
        acc += (TA)v[0] * (TA)xx[0] + (TA)v[1] * (TA)xx[1] + (TA)v[2] * (TA)xx[2] + (TA)v[3] * (TA)xx[3];
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) acc += (TA)a[c] * (TA)xv[c];
      }
    }
  }
  acc += __shfl_down_sync(0xffffffffu, acc, 2 * R);
  acc += __shfl_down_sync(0xffffffffu, acc, R);
  const bool out = row < n && lane < R;
  const size_t o = (size_t)row * R + lane;
  if constexpr (MODE == 0) {
    if (out) y[o] = (TX)acc;
  } else if constexpr (MODE == 1) {
    if (out) y[o] = (TX)((TA)b[o] - acc);
  } else if constexpr (MODE == 3) {
    if (out) y[o] = (TX)((TA)y[o] + acc);
  } else {
    static_assert(C == R, "Jacobi sweep needs square blocks");
    const TA res = out ? (TA)b[o] - acc : (TA)0;
    TA rr[R];
#pragma unroll
    for (int c = 0; c < R; ++c) rr[c] = __shfl_sync(0xffffffffu, res, c);
    if (out) {
      const TD* d = dinv + (size_t)row * (R * R) + lane * R;
      TA corr = 0;
#pragma unroll
      for (int c = 0; c < R; ++c) corr += (TA)d[c] * rr[c];
      y[o] = (TX)((TA)x[o] + omega * corr);
    }
  }
}

// ---- FP64-accurate operator with FP32 values, without the FP64 pipe.
// x (FP64) is first split into a pair of floats xh + xl (|xl| <= ulp(xh)/2).
// Each product a * xh is formed exactly as p + e (p = a*xh, e = fma(a, xh, -p)),
// a * xl is added as a plain FP32 product, and the row sum is carried as an
// unevaluated pair of floats (Knuth's two-sum; Dekker/Knuth double-float
// arithmetic), giving ~46-bit accuracy for ~10 FP32 operations per product.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_add(DF s, float p) {
  const float t = s.hi + p;
  const float bp = t - s.hi;
  const float err = (s.hi - (t - bp)) + (p - bp);   // two-sum error of s.hi + p
  const float lo = s.lo + err;
  const float hi = t + lo;
  return DF{hi, lo - (hi - t)};
}

__global__ void split_df_kernel(const double* __restrict__ x, float2* __restrict__ xs, long n) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    const double v = x[t];
    const float h = (float)v;
    xs[t] = make_float2(h, (float)(v - (double)h));
  }
}

// MODE 0: y = A x, MODE 1: y = b - A x; A: FP32 4x4 blocks, x given as float pairs.
template <int MODE>
__global__ void bsr_df_kernel(int n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                              const float* __restrict__ vals, const float2* __restrict__ xs,
                              const double* __restrict__ b, double* __restrict__ y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = t >> 2, r = t & 3;
  if (row >= n) return;
  DF s{0.f, 0.f};
  float small = 0.f;
  const int k1 = row_ptr[row + 1];
  for (int k = row_ptr[row]; k < k1; ++k) {
    const int j = col_idx[k];
    const float4 a = *reinterpret_cast<const float4*>(vals + 16 * (size_t)k + 4 * r);
    const float4 x01 = *reinterpret_cast<const float4*>(xs + 4 * (size_t)j);
    const float4 x23 = *reinterpret_cast<const float4*>(xs + 4 * (size_t)j + 2);
    const float av[4] = {a.x, a.y, a.z, a.w};
    const float xh[4] = {x01.x, x01.z, x23.x, x23.z};
    const float xl[4] = {x01.y, x01.w, x23.y, x23.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float p = av[c] * xh[c];
      const float e = fmaf(av[c], xh[c], -p);
      s = df_add(s, p);
      small = fmaf(av[c], xl[c], small + e);
    }
  }
  const double acc = (double)s.hi + ((double)s.lo + (double)small);
  const size_t o = 4 * (size_t)row + r;
  if (MODE == 0)
    y[o] = acc;
  else
    y[o] = b[o] - acc;
}

// Small coarse levels have few but long block rows (~50-110 blocks): one CTA
// of 32 slots x 7 rows per block row, slot partial sums added in slot order.
template <typename TV, typename TX, typename TA, int C, int MODE, typename TD = TV>
__global__ void __launch_bounds__(224) bsr7_cta_kernel(int n, const int32_t* __restrict__ row_ptr,
                                                       const int32_t* __restrict__ col_idx,
                                                       const TV* __restrict__ vals, const TX* __restrict__ x,
                                                       const TX* __restrict__ b, const TD* __restrict__ dinv,
                                                       TA omega, TX* __restrict__ y) {
  constexpr int R = 7, SLOTS = 32;
  __shared__ TA part[SLOTS][R];
  __shared__ TA rowsum[R];
  const int row = blockIdx.x;
  const int t = threadIdx.x, j = t / R, r = t % R;
  TA acc = 0;
  const int k1 = row_ptr[row + 1];
  for (int k = row_ptr[row] + j; k < k1; k += SLOTS) {
    const TV* a = vals + (size_t)k * (R * C) + r * C;
    const TX* xv = x + (size_t)col_idx[k] * C;
#pragma unroll
    for (int c = 0; c < C; ++c) acc += (TA)a[c] * (TA)xv[c];
  }
  part[j][r] = acc;
  __syncthreads();
  if (t < R) {
    TA s = 0;
    for (int q = 0; q < SLOTS; ++q) s += part[q][t];
    rowsum[t] = s;
  }
  __syncthreads();
  if (t >= R) return;
  const size_t o = (size_t)row * R + t;
  if constexpr (MODE == 0) {
    y[o] = (TX)rowsum[t];
  } else if constexpr (MODE == 1) {
    y[o] = (TX)((TA)b[o] - rowsum[t]);
  } else if constexpr (MODE == 3) {
    y[o] = (TX)((TA)y[o] + rowsum[t]);
  } else {
    static_assert(C == R, "Jacobi sweep needs square blocks");
    const TD* d = dinv + (size_t)row * (R * R) + t * R;
    TA corr = 0;
#pragma unroll
    for (int c = 0; c < R; ++c) corr += (TA)d[c] * ((TA)b[(size_t)row * R + c] - rowsum[c]);
    y[o] = (TX)((TA)x[o] + omega * corr);
  }
}

// x = omega D^-1 b (first Jacobi sweep from a zero guess), B x B blocks
template <typename T, int B>
__global__ void jacobi_zero_kernel(int n, const T* __restrict__ dinv, const T* __restrict__ b, T omega,
                                   T* __restrict__ x) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = t / B, r = t % B;
  if (row >= n) return;
  const T* d = dinv + (size_t)row * (B * B) + r * B;
  const T* bv = b + (size_t)row * B;
  T acc = 0;
#pragma unroll
  for (int c = 0; c < B; ++c) acc += d[c] * bv[c];
  x[(size_t)row * B + r] = omega * acc;
}

// ---- minimal-residual block Jacobi (coarse levels).  One sweep:
// z = D^-1 r, w = A z, a = (r.w)/(w.w), x += a z, r -= a w.  The step length
// minimises ||r - a w||_2 over a, so a sweep never raises the residual, even
// where D^-1 A has eigenvalues with which a fixed damping diverges.  The two
// dot products are summed in FP64 over a fixed partition (one partial per
// CTA, then the partials in index order): deterministic.
constexpr int kMrThreads = 256;

__device__ __forceinline__ double mr_block_sum(double v) {
  __shared__ double sh[kMrThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < kMrThreads / 32) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;
}

// part[blk] = sum r.w, part[gridDim.x + blk] = sum w.w over this CTA's grid-stride entries
template <typename T>
__global__ void __launch_bounds__(kMrThreads) mr_dots_kernel(long m, const T* __restrict__ r,
                                                             const T* __restrict__ w, double* __restrict__ part) {
  double rw = 0.0, ww = 0.0;
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (long)gridDim.x * blockDim.x) {
    const double wk = (double)w[k];
    rw += (double)r[k] * wk;
    ww += wk * wk;
  }
  rw = mr_block_sum(rw);
  ww = mr_block_sum(ww);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = rw;
    part[gridDim.x + blockIdx.x] = ww;
  }
}

// a = (r.w)/(w.w) from the CTA partials (every CTA sums them in the same
// order), then x += a z, r -= a w and z = D^-1 r for the next sweep (one
// thread per block row)
template <typename T, int B>
__global__ void __launch_bounds__(kMrThreads) mr_update_kernel(int n, int nblk, const double* __restrict__ part,
                                                               const T* __restrict__ dinv, T* __restrict__ x,
                                                               T* __restrict__ r, const T* __restrict__ w,
                                                               T* __restrict__ z) {
  __shared__ double s_alpha;
  double rw = 0.0, ww = 0.0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) {
    rw += part[k];
    ww += part[nblk + k];
  }
  rw = mr_block_sum(rw);
  ww = mr_block_sum(ww);
  if (threadIdx.x == 0) s_alpha = (ww > 0.0 && isfinite(rw / ww)) ? rw / ww : 0.0;
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T a = (T)s_alpha;
  T rr[B];
  const size_t o = (size_t)i * B;
#pragma unroll
  for (int c = 0; c < B; ++c) {
    x[o + c] += a * z[o + c];
    rr[c] = r[o + c] - a * w[o + c];
    r[o + c] = rr[c];
  }
  const T* d = dinv + (size_t)i * (B * B);
#pragma unroll
  for (int q = 0; q < B; ++q) {
    T acc = 0;
#pragma unroll
    for (int c = 0; c < B; ++c) acc += d[q * B + c] * rr[c];
    z[o + q] = acc;
  }
}

// number of displacement-like unknowns in a B-block (3 of 4, 6 of 7)
template <int B>
struct NU {
  static constexpr int v = (B == 4) ? 3 : 6;
};

// Inverse of each B x B diagonal block (Gauss-Jordan, partial pivoting, FP64);
// FILTER drops the displacement-pressure couplings first.
template <typename T, int B, bool FILTER = false>
__global__ void block_inverse_kernel(int n, const int32_t* __restrict__ diag_idx, const T* __restrict__ vals,
                                     T* __restrict__ dinv, int* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a[B][2 * B];
  const T* v = vals + (size_t)(B * B) * diag_idx[i];
  for (int r = 0; r < B; ++r)
    for (int c = 0; c < B; ++c) {
      a[r][c] = (FILTER && ((r < NU<B>::v) != (c < NU<B>::v))) ? 0.0 : (double)v[B * r + c];
      a[r][B + c] = (r == c) ? 1.0 : 0.0;
    }
  bool ok = true;
  for (int k = 0; k < B; ++k) {
    int p = k;
    double best = fabs(a[k][k]);
    for (int r = k + 1; r < B; ++r)
      if (fabs(a[r][k]) > best) { best = fabs(a[r][k]); p = r; }
    if (!(best > 0.0)) { ok = false; break; }
    if (p != k)
      for (int c = 0; c < 2 * B; ++c) { double t = a[k][c]; a[k][c] = a[p][c]; a[p][c] = t; }
    const double ip = 1.0 / a[k][k];
    for (int c = 0; c < 2 * B; ++c) a[k][c] *= ip;
    for (int r = 0; r < B; ++r) {
      if (r == k) continue;
      const double f = a[r][k];
      for (int c = 0; c < 2 * B; ++c) a[r][c] -= f * a[k][c];
    }
  }
  T* o = dinv + (size_t)(B * B) * i;
  for (int r = 0; r < B; ++r)
    for (int c = 0; c < B; ++c) o[B * r + c] = ok ? (T)a[r][B + c] : T(0);
  if (!ok && err) atomicOr(err, 4);
}

constexpr int NS = 7;

// W[q] = sum over the plan of A_k P_t(col(k))   (B x B times B x 7); FILTER
// skips the displacement-pressure couplings of A.
template <typename T, int B, bool FILTER>
__global__ void galerkin_w_kernel(int p_nb, const int32_t* __restrict__ w_ptr, const int32_t* __restrict__ w_k,
                                  const int32_t* __restrict__ a_ci, const T* __restrict__ a_v,
                                  const T* __restrict__ ptent, T* __restrict__ w_v) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int q = (int)(t / (B * NS)), e = (int)(t % (B * NS));
  if (q >= p_nb) return;
  const int r = e / NS, c = e % NS;
  T acc = 0;
  for (int s = w_ptr[q]; s < w_ptr[q + 1]; ++s) {
    const int k = w_k[s];
    const T* a = a_v + (size_t)k * (B * B) + r * B;
    const T* p = ptent + (size_t)a_ci[k] * (B * NS) + c;
#pragma unroll
    for (int m = 0; m < B; ++m)
      if (!FILTER || ((r < NU<B>::v) == (m < NU<B>::v))) acc += a[m] * p[m * NS];
  }
  w_v[(size_t)q * (B * NS) + e] = acc;
}

// P[q] = free (.) ([col(q) == agg(i)] P_t(i) - omega D_i^-1 W[q])
template <typename T, int B>
__global__ void galerkin_p_kernel(int p_nb, const int32_t* __restrict__ p_brow, const int32_t* __restrict__ p_ci,
                                  const int32_t* __restrict__ agg, const uint8_t* __restrict__ freem,
                                  const T* __restrict__ dinv, const T* __restrict__ ptent, const T* __restrict__ w_v,
                                  T omega, T* __restrict__ p_v) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int q = (int)(t / (B * NS)), e = (int)(t % (B * NS));
  if (q >= p_nb) return;
  const int r = e / NS, c = e % NS;
  const int i = p_brow[q];
  T v = 0;
  if (freem[(size_t)i * B + r]) {
    const T* d = dinv + (size_t)i * (B * B) + r * B;
    const T* w = w_v + (size_t)q * (B * NS) + c;
    T acc = 0;
#pragma unroll
    for (int m = 0; m < B; ++m) acc += d[m] * w[m * NS];
    v = -omega * acc;
    if (p_ci[q] == agg[i]) v += ptent[(size_t)i * (B * NS) + e];
  }
  p_v[(size_t)q * (B * NS) + e] = v;
}

// PT[t] = P[pt_src[t]]^T  (7 x B blocks)
template <typename T, int B>
__global__ void galerkin_pt_kernel(int p_nb, const int32_t* __restrict__ pt_src, const T* __restrict__ p_v,
                                   T* __restrict__ pt_v) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int u = (int)(t / (B * NS)), e = (int)(t % (B * NS));
  if (u >= p_nb) return;
  const int r = e / B, c = e % B;   // PT block entry (r, c) = P entry (c, r)
  pt_v[(size_t)u * (B * NS) + e] = p_v[(size_t)pt_src[u] * (B * NS) + c * NS + r];
}

// One thread per output block (all B x 7 entries in registers): every pair's
// two blocks are read once per output block instead of once per entry.
template <typename T, int B>
__global__ void __launch_bounds__(128) galerkin_ap_block_kernel(int ap_nb, const int32_t* __restrict__ ap_ptr,
                                                                const int32_t* __restrict__ pairs,
                                                                const T* __restrict__ a_v, const T* __restrict__ p_v,
                                                                T* __restrict__ ap_v) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= ap_nb) return;
  T acc[B][NS];
#pragma unroll
  for (int r = 0; r < B; ++r)
#pragma unroll
    for (int c = 0; c < NS; ++c) acc[r][c] = 0;
  for (int s = ap_ptr[o]; s < ap_ptr[o + 1]; ++s) {
    const T* a = a_v + (size_t)pairs[2 * s] * (B * B);
    const T* p = p_v + (size_t)pairs[2 * s + 1] * (B * NS);
    T pv[B][NS];
#pragma unroll
    for (int m = 0; m < B; ++m)
#pragma unroll
      for (int c = 0; c < NS; ++c) pv[m][c] = p[m * NS + c];
#pragma unroll
    for (int r = 0; r < B; ++r)
#pragma unroll
      for (int m = 0; m < B; ++m) {
        const T ar = a[r * B + m];
#pragma unroll
        for (int c = 0; c < NS; ++c) acc[r][c] += ar * pv[m][c];
      }
  }
  T* out = ap_v + (size_t)o * (B * NS);
#pragma unroll
  for (int r = 0; r < B; ++r)
#pragma unroll
    for (int c = 0; c < NS; ++c) out[r * NS + c] = acc[r][c];
}

// AP[r] = sum over the plan of A_k P_q   (B x B times B x 7)
template <typename T, int B>
__global__ void galerkin_ap_kernel(int ap_nb, const int32_t* __restrict__ ap_ptr, const int32_t* __restrict__ pairs,
                                   const T* __restrict__ a_v, const T* __restrict__ p_v, T* __restrict__ ap_v) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int o = (int)(t / (B * NS)), e = (int)(t % (B * NS));
  if (o >= ap_nb) return;
  const int r = e / NS, c = e % NS;
  T acc = 0;
  for (int s = ap_ptr[o]; s < ap_ptr[o + 1]; ++s) {
    const T* a = a_v + (size_t)pairs[2 * s] * (B * B) + r * B;
    const T* p = p_v + (size_t)pairs[2 * s + 1] * (B * NS) + c;
#pragma unroll
    for (int m = 0; m < B; ++m) acc += a[m] * p[m * NS];
  }
  ap_v[(size_t)o * (B * NS) + e] = acc;
}

// Ac[o] = sum over the plan of P_q^T AP_r   (7 x B times B x 7)
template <typename T, int B>
__global__ void galerkin_ac_kernel(int ac_nb, const int32_t* __restrict__ ac_ptr, const int32_t* __restrict__ pairs,
                                   const T* __restrict__ p_v, const T* __restrict__ ap_v, T* __restrict__ c_v) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int o = (int)(t / (NS * NS)), e = (int)(t % (NS * NS));
  if (o >= ac_nb) return;
  const int r = e / NS, c = e % NS;
  T acc = 0;
  for (int s = ac_ptr[o]; s < ac_ptr[o + 1]; ++s) {
    const T* p = p_v + (size_t)pairs[2 * s] * (B * NS) + r;
    const T* ap = ap_v + (size_t)pairs[2 * s + 1] * (B * NS) + c;
#pragma unroll
    for (int m = 0; m < B; ++m) acc += p[m * NS] * ap[m * NS];
  }
  c_v[(size_t)o * (NS * NS) + e] = acc;
}

// ---- Galerkin pair products on the tensor cores (FP32 levels).
// out[o] = sum over the plan of op(X[qa]) Y[qb], with X blocks RX x CX
// (row-major; op = identity, or the transpose when TRANS), Y blocks KY x NY,
// out blocks MO x NY, MO, K, NY <= 8.  One warp owns one output block and
// runs through its pairs in plan order; each pair is one m16n8k8 product
// with the block padded into rows 0..7 of the 16 x 8 A operand.  FP32
// accuracy comes from the split x = hi + lo into two TF32 numbers (hi = x
// rounded to TF32, lo = x - hi rounded again) and three products
// hi*hi + hi*lo + lo*hi (the dropped lo*lo term is below FP32 rounding).
// Per pair a lane loads four operand values, against 14 scattered loads per
// output entry in the one-thread-per-entry form.
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  uint32_t h, l;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  const float r = x - __uint_as_float(h);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(r));
  hi = h;
  lo = l;
}

__device__ __forceinline__ void mma_tf32_16x8x8(float c[4], uint32_t a0, uint32_t a2, uint32_t b0, uint32_t b1) {
  const uint32_t z = 0u;   // rows 8..15 of the A operand are padding
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(z), "r"(a2), "r"(z), "r"(b0), "r"(b1));
}

template <int RX, int CX, int KY, int NY, bool TRANS>
__global__ void __launch_bounds__(128) pair_mma_kernel(int n_out, const int32_t* __restrict__ ptr,
                                                       const int32_t* __restrict__ pairs,
                                                       const float* __restrict__ xv, const float* __restrict__ yv,
                                                       float* __restrict__ out) {
  constexpr int MO = TRANS ? CX : RX;
  constexpr int K = TRANS ? RX : CX;
  static_assert(K == KY && MO <= 8 && K <= 8 && NY <= 8, "block shapes of a pair product");
  const int o = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (o >= n_out) return;   // warp-uniform
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // fragment positions (PTX m16n8k8 .tf32): A a0 = (g, t), a2 = (g, t + 4);
  // B b0 = (k = t, n = g), b1 = (k = t + 4, n = g); C c0 = (g, 2t), c1 = (g, 2t + 1)
  const bool a0_in = g < MO && t < K, a2_in = g < MO && t + 4 < K;
  const bool b0_in = t < K && g < NY, b1_in = t + 4 < K && g < NY;
  const int xa0 = TRANS ? t * CX + g : g * CX + t;
  const int xa2 = TRANS ? (t + 4) * CX + g : g * CX + t + 4;
  const int yb0 = t * NY + g, yb1 = (t + 4) * NY + g;
  float c[4] = {0.f, 0.f, 0.f, 0.f};
  const int s1 = ptr[o + 1];
  for (int s = ptr[o]; s < s1; ++s) {
    const int qa = pairs[2 * s], qb = pairs[2 * s + 1];
    const float* X = xv + (size_t)qa * (RX * CX);
    const float* Y = yv + (size_t)qb * (KY * NY);
    const float fa0 = a0_in ? X[xa0] : 0.f, fa2 = a2_in ? X[xa2] : 0.f;
    const float fb0 = b0_in ? Y[yb0] : 0.f, fb1 = b1_in ? Y[yb1] : 0.f;
    uint32_t a0h, a0l, a2h, a2l, b0h, b0l, b1h, b1l;
    tf32_split(fa0, a0h, a0l);
    tf32_split(fa2, a2h, a2l);
    tf32_split(fb0, b0h, b0l);
    tf32_split(fb1, b1h, b1l);
    mma_tf32_16x8x8(c, a0l, a2l, b0h, b1h);
    mma_tf32_16x8x8(c, a0h, a2h, b0l, b1l);
    mma_tf32_16x8x8(c, a0h, a2h, b0h, b1h);
  }
  float* po = out + (size_t)o * (MO * NY);
  if (g < MO) {
    if (2 * t < NY) po[g * NY + 2 * t] = c[0];
    if (2 * t + 1 < NY) po[g * NY + 2 * t + 1] = c[1];
  }
}

template <typename T>
__global__ void identity_fix_kernel(int n_fix, const int32_t* __restrict__ blk, const int32_t* __restrict__ dof,
                                    T* __restrict__ vals) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_fix) return;
  vals[(size_t)blk[t] * (NS * NS) + dof[t] * (NS + 1)] = T(1);
}

// In-place Gauss-Jordan inversion (partial pivoting) of the dense operator of
// each coarse component; one CTA per component, FP64 working storage.
template <typename T>
__global__ void coarse_factor_kernel(int bs, const int32_t* __restrict__ comp_ptr, const int64_t* __restrict__ inv_off,
                                     const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                                     const T* __restrict__ vals, double* __restrict__ work, T* __restrict__ inv,
                                     int* __restrict__ err) {
  const int comp = blockIdx.x;
  const int n0 = comp_ptr[comp], n1 = comp_ptr[comp + 1];
  const int nd = bs * (n1 - n0);
  double* A = work + inv_off[comp];
  __shared__ int piv_row;
  __shared__ double s_best[32];
  __shared__ int s_idx[32];
  extern __shared__ int s_perm[];
  for (long k = threadIdx.x; k < (long)nd * nd; k += blockDim.x) A[k] = 0.0;
  __syncthreads();
  for (int i = n0 + threadIdx.x; i < n1; i += blockDim.x) {
    for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      const int j = col_idx[k];
      if (j < n0 || j >= n1) continue;
      for (int r = 0; r < bs; ++r)
        for (int c = 0; c < bs; ++c)
          A[(size_t)(bs * (i - n0) + r) * nd + bs * (j - n0) + c] = (double)vals[(size_t)(bs * bs) * k + bs * r + c];
    }
  }
  __syncthreads();
  bool singular = false;
  for (int k = 0; k < nd; ++k) {
    // pivot search in column k, rows k..nd-1
    double best = -1.0;
    int bi = k;
    for (int r = k + threadIdx.x; r < nd; r += blockDim.x) {
      double v = fabs(A[(size_t)r * nd + k]);
      if (v > best) { best = v; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_down_sync(0xffffffffu, best, o);
      int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if ((threadIdx.x & 31) == 0) { s_best[threadIdx.x >> 5] = best; s_idx[threadIdx.x >> 5] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = -1.0;
      int idx = k;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
        if (s_best[w] > b || (s_best[w] == b && s_idx[w] < idx)) { b = s_best[w]; idx = s_idx[w]; }
      piv_row = (b > 0.0) ? idx : -1;
      s_perm[k] = idx;
    }
    __syncthreads();
    const int p = piv_row;
    if (p < 0) { singular = true; break; }
    if (p != k)
      for (int c = threadIdx.x; c < nd; c += blockDim.x) {
        double t = A[(size_t)k * nd + c];
        A[(size_t)k * nd + c] = A[(size_t)p * nd + c];
        A[(size_t)p * nd + c] = t;
      }
    __syncthreads();
    const double ip = 1.0 / A[(size_t)k * nd + k];
    __syncthreads();
    for (int c = threadIdx.x; c < nd; c += blockDim.x) {
      double v = (c == k) ? 1.0 : A[(size_t)k * nd + c];
      A[(size_t)k * nd + c] = v * ip;
    }
    __syncthreads();
    for (long q = threadIdx.x; q < (long)nd * nd; q += blockDim.x) {
      const int r = (int)(q / nd), c = (int)(q % nd);
      if (r == k) continue;
      const double f = A[(size_t)r * nd + k];
      if (c == k) continue;
      A[(size_t)r * nd + c] -= f * A[(size_t)k * nd + c];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nd; r += blockDim.x) {
      if (r == k) continue;
      A[(size_t)r * nd + k] = -A[(size_t)r * nd + k] * A[(size_t)k * nd + k];
    }
    __syncthreads();
  }
  if (singular) {
    if (threadIdx.x == 0) atomicOr(err, 8);
    return;
  }
  // undo the row interchanges as column interchanges, in reverse order
  for (int k = nd - 1; k >= 0; --k) {
    const int p = s_perm[k];
    if (p != k)
      for (int r = threadIdx.x; r < nd; r += blockDim.x) {
        double t = A[(size_t)r * nd + k];
        A[(size_t)r * nd + k] = A[(size_t)r * nd + p];
        A[(size_t)r * nd + p] = t;
      }
    __syncthreads();
  }
  T* o = inv + inv_off[comp];
  for (long q = threadIdx.x; q < (long)nd * nd; q += blockDim.x) o[q] = (T)A[q];
}

// x_comp = Inv_comp b_comp
template <typename T>
__global__ void coarse_apply_kernel(int bs, const int32_t* __restrict__ comp_ptr, const int64_t* __restrict__ inv_off,
                                    const T* __restrict__ inv, const T* __restrict__ b, T* __restrict__ x) {
  const int comp = blockIdx.x;
  const int n0 = comp_ptr[comp], n1 = comp_ptr[comp + 1];
  const int nd = bs * (n1 - n0);
  const T* A = inv + inv_off[comp];
  const T* bb = b + (size_t)bs * n0;
  for (int r = threadIdx.x; r < nd; r += blockDim.x) {
    T acc = 0;
    for (int c = 0; c < nd; ++c) acc += A[(size_t)r * nd + c] * bb[c];
    x[(size_t)bs * n0 + r] = acc;
  }
}

// ---------------------------------------------------------------- FP64 vector kernels
constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double s[kRedThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < kRedThreads / 32) ? s[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;
}

// partial[i * nblk + blk] = sum over this block's chunk of V_i . y   (V_i = V + i ldv)
__global__ void multidot_kernel(const double* __restrict__ V, long ldv, const double* __restrict__ y, long n,
                                double* __restrict__ partial) {
  const int i = blockIdx.y;
  const double* x = V + (size_t)i * ldv;
  double acc = 0.0;
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
    acc += x[k] * y[k];
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[(size_t)i * gridDim.x + blockIdx.x] = acc;
}

__global__ void reduce_partials_kernel(const double* __restrict__ partial, int nblk, double* __restrict__ out) {
  const int i = blockIdx.x;
  double acc = 0.0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) acc += partial[(size_t)i * nblk + k];
  acc = block_sum(acc);
  if (threadIdx.x == 0) out[i] = acc;
}

// w += sign * sum_i coef[i] V_i   (V row-major [k][n]); coef in device memory
__global__ void multi_axpy_kernel(const double* __restrict__ coef, const double* __restrict__ V, int k, long n,
                                  double sign, double* __restrict__ w) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < k; ++i) acc += coef[i] * V[(size_t)i * n + t];
    w[t] += sign * acc;
  }
}

__global__ void axpy_kernel(double a, const double* __restrict__ x, double* __restrict__ y, long n) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
    y[t] += a * x[t];
}

__global__ void scale_copy_kernel(double a, const double* __restrict__ x, double* __restrict__ y, long n) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
    y[t] = a * x[t];
}

__global__ void to_float_kernel(const double* __restrict__ x, float* __restrict__ y, long n) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
    y[t] = (float)x[t];
}

__global__ void to_double_kernel(const float* __restrict__ x, double* __restrict__ y, long n) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
    y[t] = (double)x[t];
}

__global__ void mask_vector_kernel(const uint8_t* __restrict__ cmask, double* __restrict__ x, long n) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
    if (cmask[t]) x[t] = 0.0;
}

// out[s] = sum of squares over the unknowns of segment s (nodes seg_ptr[s]..seg_ptr[s+1])
__global__ void segment_sumsq_kernel(const int32_t* __restrict__ seg_ptr, const double* __restrict__ x,
                                     double* __restrict__ out) {
  const int sg = blockIdx.x;
  const long d0 = 4L * seg_ptr[sg], d1 = 4L * seg_ptr[sg + 1];
  double acc = 0.0;
  for (long t = d0 + threadIdx.x; t < d1; t += blockDim.x) acc += x[t] * x[t];
  acc = block_sum(acc);
  if (threadIdx.x == 0) out[sg] = acc;
}

// Segmented reductions of the per-segment Krylov method: out[i n_seg + s] =
// V_i . y over the unknowns of segment s (one CTA per (segment, vector), fixed
// order: deterministic).
__global__ void seg_multidot_kernel(const int32_t* __restrict__ seg_ptr, int n_seg, const double* __restrict__ V,
                                    long ldv, const double* __restrict__ y, double* __restrict__ out) {
  const int sg = blockIdx.x, i = blockIdx.y;
  const long d0 = 4L * seg_ptr[sg], d1 = 4L * seg_ptr[sg + 1];
  const double* v = V + (size_t)i * ldv;
  double acc = 0.0;
  for (long t = d0 + threadIdx.x; t < d1; t += blockDim.x) acc += v[t] * y[t];
  acc = block_sum(acc);
  if (threadIdx.x == 0) out[(size_t)i * n_seg + sg] = acc;
}

// w += sign * sum_i coef[i n_seg + seg(t)] V_i[t]
__global__ void seg_multi_axpy_kernel(const int32_t* __restrict__ seg_node, int n_seg,
                                      const double* __restrict__ coef, const double* __restrict__ V, int k, long n,
                                      double sign, double* __restrict__ w) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    const int sg = seg_node[t >> 2];
    double acc = 0.0;
    for (int i = 0; i < k; ++i) acc += coef[(size_t)i * n_seg + sg] * V[(size_t)i * n + t];
    w[t] += sign * acc;
  }
}

// mode 0: a[s] = 1/sqrt(sumsq) (1 if zero), b[s] = sqrt(sumsq); x *= a[seg]  (normalise)
__global__ void segment_normalise_kernel(int n_seg, double* __restrict__ a, double* __restrict__ b) {
  const int sg = blockIdx.x * blockDim.x + threadIdx.x;
  if (sg >= n_seg) return;
  const double s = sqrt(a[sg]);
  b[sg] = s > 0.0 ? s : 1.0;
  a[sg] = s > 0.0 ? 1.0 / s : 1.0;
}

__global__ void segment_scale_kernel(const int32_t* __restrict__ seg_node, const double* __restrict__ scale,
                                     double* __restrict__ x, long n) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
    x[t] *= scale[seg_node[t >> 2]];
}

inline int grid_stride_blocks(long n) {
  long b = (n + 255) / 256;
  return (int)(b < 152 * 8 ? (b > 0 ? b : 1) : 152 * 8);
}

}  // namespace

// ---------------------------------------------------------------- launchers
// shape: the launch shape chosen by the autotuner for the level (0: default).
// 7-row blocks: 1 = one CTA per block row (bsr7_cta_kernel), 2 = one warp per
// block row (bsr7_kernel), 0 = CTA per row below 4096 rows; 4-row blocks: the
// CTA size (64, 128 or 256; 0 = 128).
template <typename TV, typename TX, typename TA, int R, int C, int MODE, typename TD = TV>
static void bsr_launch(int n, const int32_t* rp, const int32_t* ci, const void* vals, const TX* x, const TX* b,
                       const void* dinv, TA omega, TX* y, cudaStream_t s, int cls, int shape = 0) {
  if constexpr (R == 7) {
    if (n == 0) return;
    if (shape == 1 || (shape == 0 && n < 4096))
      FSI_LAUNCH(cls, s, bsr7_cta_kernel<TV, TX, TA, C, MODE, TD><<<n, 224, 0, s>>>(
          n, rp, ci, (const TV*)vals, x, b, (const TD*)dinv, omega, y));
    else
      FSI_LAUNCH(cls, s, bsr7_kernel<TV, TX, TA, C, MODE, TD><<<blocks_for((long)n * 32, 128), 128, 0, s>>>(
          n, rp, ci, (const TV*)vals, x, b, (const TD*)dinv, omega, y));
    return;
  }
  constexpr int LN = Lanes<R>::v;
  const long threads = (long)n * LN;
  if (threads == 0) return;
  const int cta = (shape == 64 || shape == 256) ? shape : 128;
  FSI_LAUNCH(cls, s, bsr_kernel<TV, TX, TA, R, C, MODE><<<blocks_for(threads, cta), cta, 0, s>>>(
      n, rp, ci, (const TV*)vals, x, b, (const TV*)dinv, omega, y));
}

template <typename T>
void launch_spmv(const Level& L, const T* x, T* y, cudaStream_t s) {
  if (L.bs == 4)
    bsr_launch<T, T, T, 4, 4, 0>(L.n, L.row_ptr, L.col_idx, L.vals, x, nullptr, nullptr, T(0), y, s, fsi::KC_BSR0,
                                 L.shape);
  else
    bsr_launch<T, T, T, 7, 7, 0>(L.n, L.row_ptr, L.col_idx, L.vals, x, nullptr, nullptr, T(0), y, s,
                                 fsi::KC_COARSE_BSR, L.shape);
  FSI_CUDA_TRY(cudaGetLastError());
}
template void launch_spmv<double>(const Level&, const double*, double*, cudaStream_t);
template void launch_spmv<float>(const Level&, const float*, float*, cudaStream_t);

void split_df(const double* x, float2* xs, long n, cudaStream_t s) {
  FSI_LAUNCH(fsi::KC_VECTOR, s, split_df_kernel<<<grid_stride_blocks(n), 256, 0, s>>>(x, xs, n));
}

// FP32 values, FP64 vectors: double-float accumulation (xs is scratch of 4 n float2)
void launch_spmv_df(const Level& L, const void* vals, const double* x, float2* xs, const double* b, double* y,
                    cudaStream_t s) {
  split_df(x, xs, 4L * L.n, s);
  if (b)
    FSI_LAUNCH(fsi::KC_BSR0, s, bsr_df_kernel<1><<<blocks_for(4L * L.n, 128), 128, 0, s>>>(
        L.n, L.row_ptr, L.col_idx, (const float*)vals, xs, b, y));
  else
    FSI_LAUNCH(fsi::KC_BSR0, s, bsr_df_kernel<0><<<blocks_for(4L * L.n, 128), 128, 0, s>>>(
        L.n, L.row_ptr, L.col_idx, (const float*)vals, xs, nullptr, y));
  FSI_CUDA_TRY(cudaGetLastError());
}

void launch_spmv_f64acc(const Level& L, const void* vals, const double* x, double* y, bool fp32vals, cudaStream_t s) {
  if (fp32vals)
    bsr_launch<float, double, double, 4, 4, 0>(L.n, L.row_ptr, L.col_idx, vals, x, nullptr, nullptr, 0.0, y, s, fsi::KC_BSR0);
  else
    bsr_launch<double, double, double, 4, 4, 0>(L.n, L.row_ptr, L.col_idx, vals, x, nullptr, nullptr, 0.0, y, s, fsi::KC_BSR0);
  FSI_CUDA_TRY(cudaGetLastError());
}

void launch_residual_f64(const Level& L, const void* vals, const double* b, const double* x, double* r,
                         bool fp32vals, cudaStream_t s) {
  if (fp32vals)
    bsr_launch<float, double, double, 4, 4, 1>(L.n, L.row_ptr, L.col_idx, vals, x, b, nullptr, 0.0, r, s, fsi::KC_BSR0);
  else
    bsr_launch<double, double, double, 4, 4, 1>(L.n, L.row_ptr, L.col_idx, vals, x, b, nullptr, 0.0, r, s, fsi::KC_BSR0);
  FSI_CUDA_TRY(cudaGetLastError());
}

// ---- block lower-triangular preconditioner P_L (Sec. 5.4.2, Eq. lpre)
// A from K: one thread per block entry.  Entries coupling u and p are dropped;
// the pressure row of a diagonal block becomes (0 0 0 1), of any other block 0.
template <typename T>
__global__ void split_a_kernel(int nb, const int32_t* __restrict__ brow, const int32_t* __restrict__ col,
                               const T* __restrict__ k, T* __restrict__ a) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= 16L * nb) return;
  const int blk = (int)(q >> 4), i = (int)(q >> 2) & 3, j = (int)q & 3;
  T v = k[q];
  if ((i == 3) != (j == 3)) v = T(0);
  if (i == 3 && j == 3) v = brow[blk] == col[blk] ? T(1) : T(0);
  a[q] = v;
}

void launch_split_a(const Level& L, const void* k_vals, bool fp32, cudaStream_t s) {
  const int nbk = blocks_for(16L * L.nb, 256);
  if (fp32)
    FSI_LAUNCH(fsi::KC_OTHER, s, split_a_kernel<float><<<nbk, 256, 0, s>>>(L.nb, L.block_row, L.col_idx,
                                                                           (const float*)k_vals, (float*)L.vals));
  else
    FSI_LAUNCH(fsi::KC_OTHER, s, split_a_kernel<double><<<nbk, 256, 0, s>>>(L.nb, L.block_row, L.col_idx,
                                                                            (const double*)k_vals, (double*)L.vals));
  FSI_CUDA_TRY(cudaGetLastError());
}

template <typename T>
__global__ void pl_stage_kernel(long n4, const double* __restrict__ r, T* __restrict__ b) {
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += (long)gridDim.x * blockDim.x)
    b[q] = (q & 3) == 3 ? T(0) : T(r[q]);
}

template <typename T>
__global__ void pl_unstage_kernel(long n4, const T* __restrict__ x, double* __restrict__ z) {
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += (long)gridDim.x * blockDim.x)
    z[q] = (q & 3) == 3 ? 0.0 : (double)x[q];
}

__global__ void pl_pressure_kernel(long nn, const double* __restrict__ y, const double* __restrict__ r,
                                   const double* __restrict__ sinv, double* __restrict__ z) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x)
    z[4 * i + 3] = (y[4 * i + 3] - r[4 * i + 3]) * sinv[i];
}

void pl_stage(const double* r, void* b, bool fp32, long n_nodes, cudaStream_t s) {
  const long n4 = 4 * n_nodes;
  if (fp32)
    FSI_LAUNCH(fsi::KC_VECTOR, s, pl_stage_kernel<float><<<grid_stride_blocks(n4), 256, 0, s>>>(n4, r, (float*)b));
  else
    FSI_LAUNCH(fsi::KC_VECTOR, s, pl_stage_kernel<double><<<grid_stride_blocks(n4), 256, 0, s>>>(n4, r, (double*)b));
}

void pl_unstage(const void* x, double* z, bool fp32, long n_nodes, cudaStream_t s) {
  const long n4 = 4 * n_nodes;
  if (fp32)
    FSI_LAUNCH(fsi::KC_VECTOR, s, pl_unstage_kernel<float><<<grid_stride_blocks(n4), 256, 0, s>>>(n4, (const float*)x, z));
  else
    FSI_LAUNCH(fsi::KC_VECTOR, s, pl_unstage_kernel<double><<<grid_stride_blocks(n4), 256, 0, s>>>(n4, (const double*)x, z));
}

void pl_pressure(const double* y, const double* r, const double* sinv, double* z, long n_nodes, cudaStream_t s) {
  FSI_LAUNCH(fsi::KC_VECTOR, s, pl_pressure_kernel<<<grid_stride_blocks(n_nodes), 256, 0, s>>>(n_nodes, y, r, sinv, z));
}

template <typename T>
static void block_inverse_t(Level& L, int* err, cudaStream_t s) {
  if (L.bs == 4)
    FSI_LAUNCH(fsi::KC_BLOCKINV, s, block_inverse_kernel<T, 4><<<blocks_for(L.n, 128), 128, 0, s>>>(L.n, L.diag_idx, (const T*)L.vals, (T*)L.dinv,
                                                                    err));
  else
    FSI_LAUNCH(fsi::KC_BLOCKINV, s, block_inverse_kernel<T, 7><<<blocks_for(L.n, 64), 64, 0, s>>>(L.n, L.diag_idx, (const T*)L.vals, (T*)L.dinv,
                                                                  err));
}

void launch_block_inverse(Level& L, bool fp32, int* err, cudaStream_t s) {
  if (fp32)
    block_inverse_t<float>(L, err, s);
  else
    block_inverse_t<double>(L, err, s);
  FSI_CUDA_TRY(cudaGetLastError());
}

template <typename T, int B>
static void galerkin_t(Level& L, Level& C, bool filter, cudaStream_t s) {
  const long pe = (long)L.p_nb * B * NS;
  const T* dsm = (const T*)L.dinv;
  if (filter) {
    FSI_LAUNCH(fsi::KC_GALERKIN, s, block_inverse_kernel<T, B, true><<<blocks_for(L.n, 64), 64, 0, s>>>(
        L.n, L.diag_idx, (const T*)L.vals, (T*)L.dinv_f, nullptr));
    dsm = (const T*)L.dinv_f;
    FSI_LAUNCH(fsi::KC_GALERKIN, s, galerkin_w_kernel<T, B, true><<<blocks_for(pe, 256), 256, 0, s>>>(
        L.p_nb, L.w_ptr, L.w_k, L.col_idx, (const T*)L.vals, (const T*)L.ptent, (T*)L.w_v));
  } else {
    FSI_LAUNCH(fsi::KC_GALERKIN, s, galerkin_w_kernel<T, B, false><<<blocks_for(pe, 256), 256, 0, s>>>(
        L.p_nb, L.w_ptr, L.w_k, L.col_idx, (const T*)L.vals, (const T*)L.ptent, (T*)L.w_v));
  }
  FSI_LAUNCH(fsi::KC_GALERKIN, s, galerkin_p_kernel<T, B><<<blocks_for(pe, 256), 256, 0, s>>>(L.p_nb, L.p_brow, L.p_ci, L.agg, L.freem,
                                                              dsm, (const T*)L.ptent, (const T*)L.w_v,
                                                              (T)L.omega_p, (T*)L.p_v));
  FSI_LAUNCH(fsi::KC_GALERKIN, s, galerkin_pt_kernel<T, B><<<blocks_for(pe, 256), 256, 0, s>>>(L.p_nb, L.pt_src, (const T*)L.p_v, (T*)L.pt_v));
  // A P: one thread per output block on the 4x4 level (16 x 28 register
  // tile, each A block read once per output block), one thread per output
  // entry on the 7x7 levels (per-entry threads of one output block share its
  // pair blocks through L1).  P^T (A P): one thread
  // per entry everywhere.  Both choices measured faster on the 393k-tet tube
  // (a warp-staged variant, 32 output blocks per warp with their pair blocks
  // copied through shared memory, measured 3x slower on the 3.1M-tet tube).
  // FP32 levels: both products on the tensor cores (pair_mma_kernel, one warp per
  // output block, 3xTF32 for FP32 accuracy)
  if constexpr (std::is_same<T, float>::value) {
    FSI_LAUNCH(fsi::KC_GALERKIN, s, pair_mma_kernel<B, B, B, NS, false><<<blocks_for(32L * L.ap_nb, 128), 128, 0, s>>>(
        L.ap_nb, L.ap_ptr, L.ap_pairs, (const float*)L.vals, (const float*)L.p_v, (float*)L.ap_v));
    FSI_LAUNCH(fsi::KC_GALERKIN, s, pair_mma_kernel<B, NS, B, NS, true><<<blocks_for(32L * C.nb, 128), 128, 0, s>>>(
        C.nb, L.ac_ptr, L.ac_pairs, (const float*)L.p_v, (const float*)L.ap_v, (float*)C.vals));
  } else {
  if constexpr (B == 4)
    FSI_LAUNCH(fsi::KC_GALERKIN, s, galerkin_ap_block_kernel<T, B><<<blocks_for(L.ap_nb, 128), 128, 0, s>>>(
        L.ap_nb, L.ap_ptr, L.ap_pairs, (const T*)L.vals, (const T*)L.p_v, (T*)L.ap_v));
  else
    FSI_LAUNCH(fsi::KC_GALERKIN, s, galerkin_ap_kernel<T, B><<<blocks_for((long)L.ap_nb * B * NS, 256), 256, 0, s>>>(
        L.ap_nb, L.ap_ptr, L.ap_pairs, (const T*)L.vals, (const T*)L.p_v, (T*)L.ap_v));
  FSI_LAUNCH(fsi::KC_GALERKIN, s, galerkin_ac_kernel<T, B><<<blocks_for((long)C.nb * NS * NS, 256), 256, 0, s>>>(
      C.nb, L.ac_ptr, L.ac_pairs, (const T*)L.p_v, (const T*)L.ap_v, (T*)C.vals));
  }
  if (L.n_fix > 0)
    FSI_LAUNCH(fsi::KC_GALERKIN, s, identity_fix_kernel<T><<<blocks_for(L.n_fix, 128), 128, 0, s>>>(L.n_fix, L.fix_blk, L.fix_dof, (T*)C.vals));
}

void launch_galerkin(Level& L, Level& C, bool fp32, bool filter, cudaStream_t s) {
  if (fp32) {
    if (L.bs == 4) galerkin_t<float, 4>(L, C, filter, s); else galerkin_t<float, 7>(L, C, filter, s);
  } else {
    if (L.bs == 4) galerkin_t<double, 4>(L, C, filter, s); else galerkin_t<double, 7>(L, C, filter, s);
  }
  FSI_CUDA_TRY(cudaGetLastError());
}

__global__ void values_to_bf16_kernel(long m, const float* __restrict__ x, __nv_bfloat16* __restrict__ y) {
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (long)gridDim.x * blockDim.x)
    y[q] = __float2bfloat16_rn(x[q]);
}

void launch_values_to_bf16(const Level& L, cudaStream_t s) {
  const long m = (long)L.nb * L.bs * L.bs;
  FSI_LAUNCH(fsi::KC_GALERKIN, s, values_to_bf16_kernel<<<grid_stride_blocks(m), 256, 0, s>>>(
      m, (const float*)L.vals, (__nv_bfloat16*)L.vals_lp));
  FSI_CUDA_TRY(cudaGetLastError());
}

void launch_coarse_factor(Handle& h, bool fp32, cudaStream_t s) {
  const Level& L = h.levels.back();
  const Coarse& C = h.coarse;
  size_t shm = sizeof(int) * (size_t)C.max_dofs;
  if (fp32)
    FSI_LAUNCH(fsi::KC_COARSE, s, coarse_factor_kernel<float><<<C.n_comp, 256, shm, s>>>(L.bs, C.comp_ptr, C.inv_off, L.row_ptr, L.col_idx,
                                                           (const float*)L.vals, C.work, (float*)C.inv, h.d_err));
  else
    FSI_LAUNCH(fsi::KC_COARSE, s, coarse_factor_kernel<double><<<C.n_comp, 256, shm, s>>>(L.bs, C.comp_ptr, C.inv_off, L.row_ptr, L.col_idx,
                                                            (const double*)L.vals, C.work, (double*)C.inv, h.d_err));
  FSI_CUDA_TRY(cudaGetLastError());
}

template <typename T, int B>
static void smooth_b(const Level& L, T omega, int sweeps, bool zero_start, cudaStream_t s) {
  T* x = (T*)L.x;
  T* x2 = (T*)L.x2;
  const T* b = (const T*)L.b;
  int k = 0;
  if (zero_start) {
    if (sweeps > 0) {
      FSI_LAUNCH((B == 4 ? fsi::KC_BSR0 : fsi::KC_COARSE_BSR), s, jacobi_zero_kernel<T, B><<<blocks_for((long)L.n * B, 128), 128, 0, s>>>(L.n, (const T*)L.dinv, b, omega, x));
      k = 1;
    } else {
      FSI_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(T) * B * (size_t)L.n, s));
    }
  }
  for (; k < sweeps; ++k) {
    if constexpr (B == 7 && std::is_same<T, float>::value) {
      if (L.vals_lp) {
        bsr_launch<__nv_bfloat16, float, float, 7, 7, 2, float>(L.n, L.row_ptr, L.col_idx, L.vals_lp, x, b, L.dinv,
                                                                 omega, x2, s, fsi::KC_COARSE_BSR, L.shape);
        std::swap(x, x2);
        continue;
      }
    }
    bsr_launch<T, T, T, B, B, 2>(L.n, L.row_ptr, L.col_idx, L.vals, x, b, L.dinv, omega, x2, s,
                                 (B == 4 ? fsi::KC_JACOBI0 : fsi::KC_COARSE_BSR), L.shape);
    std::swap(x, x2);
  }
  // the result must live in L.x
  if (x != (T*)L.x) FSI_CUDA_TRY(cudaMemcpyAsync(L.x, x, sizeof(T) * B * (size_t)L.n, cudaMemcpyDeviceToDevice, s));
}

template <typename T>
static void smooth(const Level& L, T omega, int sweeps, bool zero_start, cudaStream_t s) {
  if (L.bs == 4)
    smooth_b<T, 4>(L, omega, sweeps, zero_start, s);
  else
    smooth_b<T, 7>(L, omega, sweeps, zero_start, s);
}

// nu minimal-residual block-Jacobi sweeps on a 7x7 level.  zero_start: x = 0,
// r = b; otherwise r = b - A x is formed first.  On return x = L.x and
// r = L.r = b - A x (the restriction reads it directly).
template <typename T>
static void smooth_mr(const Level& L, int sweeps, bool zero_start, cudaStream_t s) {
  constexpr int B = 7;
  T* x = (T*)L.x;
  T* r = (T*)L.r;
  T* z = (T*)L.x2;
  T* w = (T*)L.w;
  const T* b = (const T*)L.b;
  const long m = (long)L.n * B;
  if (zero_start) {
    FSI_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(T) * m, s));
    FSI_CUDA_TRY(cudaMemcpyAsync(r, b, sizeof(T) * m, cudaMemcpyDeviceToDevice, s));
  } else {
    bool done = false;
    if constexpr (std::is_same<T, float>::value) {
      if (L.vals_lp) {
        bsr_launch<__nv_bfloat16, float, float, 7, 7, 1, float>(L.n, L.row_ptr, L.col_idx, L.vals_lp, (const float*)x,
                                                                 (const float*)b, nullptr, 0.0f, (float*)r, s,
                                                                 fsi::KC_COARSE_BSR, L.shape);
        done = true;
      }
    }
    if (!done)
      bsr_launch<T, T, T, 7, 7, 1>(L.n, L.row_ptr, L.col_idx, L.vals, (const T*)x, b, nullptr, T(0), r, s,
                                   fsi::KC_COARSE_BSR, L.shape);
  }
  if (sweeps <= 0) return;
  FSI_LAUNCH(fsi::KC_COARSE_BSR, s, jacobi_zero_kernel<T, B><<<blocks_for(m, 128), 128, 0, s>>>(
      L.n, (const T*)L.dinv, r, T(1), z));
  for (int k = 0; k < sweeps; ++k) {
    bool done = false;
    if constexpr (std::is_same<T, float>::value) {
      if (L.vals_lp) {
        bsr_launch<__nv_bfloat16, float, float, 7, 7, 0, float>(L.n, L.row_ptr, L.col_idx, L.vals_lp, (const float*)z,
                                                                 nullptr, nullptr, 0.0f, (float*)w, s, L.kc_spmv,
                                                                 L.shape);
        done = true;
      }
    }
    if (!done)
      bsr_launch<T, T, T, 7, 7, 0>(L.n, L.row_ptr, L.col_idx, L.vals, (const T*)z, nullptr, nullptr, T(0), w, s,
                                   L.kc_spmv, L.shape);
    FSI_LAUNCH(fsi::KC_COARSE_BSR, s, mr_dots_kernel<T><<<kMrBlocks, kMrThreads, 0, s>>>(m, r, w, L.mr));
    FSI_LAUNCH(fsi::KC_COARSE_BSR, s, mr_update_kernel<T, B><<<blocks_for(L.n, kMrThreads), kMrThreads, 0, s>>>(
        L.n, kMrBlocks, L.mr, (const T*)L.dinv, x, r, w, z));
  }
}

// One V-cycle on levels[level..]: approximately solves K_l x_l = b_l from x_l = 0.
template <typename T>
void vcycle(Handle& h, int level, cudaStream_t s) {
  Level& L = h.levels[level];
  const int nl = (int)h.levels.size();
  const T omega = (T)h.opts.omega;
  if (level == nl - 1) {
    const Coarse& C = h.coarse;
    FSI_LAUNCH(fsi::KC_COARSE, s, coarse_apply_kernel<T><<<C.n_comp, 256, 0, s>>>(L.bs, C.comp_ptr, C.inv_off, (const T*)C.inv, (const T*)L.b,
                                                    (T*)L.x));
    FSI_CUDA_TRY(cudaGetLastError());
    return;
  }
  Level& Lc = h.levels[level + 1];
  const int nu_pre = level == 0 ? h.opts.nu_pre : h.opts.nu_coarse;
  const int nu_post = level == 0 ? h.opts.nu_post : h.opts.nu_coarse;
  const bool vanka = level == 0 && h.opts.smoother == FSI_SMOOTHER_VANKA;
  const bool mr = L.bs == 7 && L.mr != nullptr;
  if (vanka)
    vanka_smooth<T>(h, nu_pre, true, s);
  else if (mr)
    smooth_mr<T>(L, nu_pre, true, s);   // leaves r = b - A x in L.r
  else
    smooth<T>(L, omega, nu_pre, true, s);
  if (mr) {
    bsr_launch<T, T, T, 7, 7, 0>(Lc.n, L.pt_rp, L.pt_ci, L.pt_v, (const T*)L.r, nullptr, nullptr, T(0), (T*)Lc.b, s,
                                 fsi::KC_TRANSFER);
  } else if (L.bs == 4) {
    bsr_launch<T, T, T, 4, 4, 1>(L.n, L.row_ptr, L.col_idx, L.vals, (const T*)L.x, (const T*)L.b, nullptr, T(0),
                                 (T*)L.r, s, fsi::KC_BSR0, L.shape);
    bsr_launch<T, T, T, 7, 4, 0>(Lc.n, L.pt_rp, L.pt_ci, L.pt_v, (const T*)L.r, nullptr, nullptr, T(0), (T*)Lc.b, s, fsi::KC_TRANSFER);
  } else {
    bool done = false;
    if constexpr (std::is_same<T, float>::value) {
      if (L.vals_lp) {
        bsr_launch<__nv_bfloat16, float, float, 7, 7, 1, float>(L.n, L.row_ptr, L.col_idx, L.vals_lp,
                                                                 (const float*)L.x, (const float*)L.b, nullptr,
                                                                 0.0f, (float*)L.r, s, fsi::KC_COARSE_BSR, L.shape);
        done = true;
      }
    }
    if (!done)
      bsr_launch<T, T, T, 7, 7, 1>(L.n, L.row_ptr, L.col_idx, L.vals, (const T*)L.x, (const T*)L.b, nullptr, T(0),
                                   (T*)L.r, s, fsi::KC_COARSE_BSR, L.shape);
    bsr_launch<T, T, T, 7, 7, 0>(Lc.n, L.pt_rp, L.pt_ci, L.pt_v, (const T*)L.r, nullptr, nullptr, T(0), (T*)Lc.b, s, fsi::KC_TRANSFER);
  }
  vcycle<T>(h, level + 1, s);
  if (L.bs == 4)
    bsr_launch<T, T, T, 4, 7, 3>(L.n, L.p_rp, L.p_ci, L.p_v, (const T*)Lc.x, nullptr, nullptr, T(0), (T*)L.x, s, fsi::KC_TRANSFER);
  else
    bsr_launch<T, T, T, 7, 7, 3>(L.n, L.p_rp, L.p_ci, L.p_v, (const T*)Lc.x, nullptr, nullptr, T(0), (T*)L.x, s, fsi::KC_TRANSFER);
  if (vanka)
    vanka_smooth<T>(h, nu_post, false, s);
  else if (mr)
    smooth_mr<T>(L, nu_post, false, s);
  else
    smooth<T>(L, omega, nu_post, false, s);
  FSI_CUDA_TRY(cudaGetLastError());
}
template void vcycle<double>(Handle&, int, cudaStream_t);
template void vcycle<float>(Handle&, int, cudaStream_t);

// ---- autotuner of the block-row launch shapes (create time, once per handle).
// For every level that is smoothed, the damped block-Jacobi sweep of its own
// operator (the kernel that dominates the V-cycle) is timed with CUDA events
// on the handle's stream, three repetitions after one warm-up, for each
// candidate shape; the fastest is kept in Level::shape.  Candidates: CTA
// sizes 64, 128, 256 for the 4x4 level; CTA-per-row and warp-per-row kernels
// for the 7x7 levels.  The vectors are zeroed first (the timing does not
// depend on the values).
template <typename T>
static float time_sweep(Level& L, int shape, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  const T omega = T(0.7);
  auto run = [&]() {
    if (L.bs == 4)
      bsr_launch<T, T, T, 4, 4, 2>(L.n, L.row_ptr, L.col_idx, L.vals, (const T*)L.x, (const T*)L.b, L.dinv, omega,
                                   (T*)L.x2, s, fsi::KC_OTHER, shape);
    else
      bsr_launch<T, T, T, 7, 7, 2>(L.n, L.row_ptr, L.col_idx, L.vals, (const T*)L.x, (const T*)L.b, L.dinv, omega,
                                   (T*)L.x2, s, fsi::KC_OTHER, shape);
  };
  run();
  FSI_CUDA_TRY(cudaEventRecord(e0, s));
  for (int r = 0; r < 3; ++r) run();
  FSI_CUDA_TRY(cudaEventRecord(e1, s));
  FSI_CUDA_TRY(cudaEventSynchronize(e1));
  float ms = 0.f;
  FSI_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
  return ms;
}

template <typename T>
static void autotune_t(Handle& h, cudaStream_t s) {
  cudaEvent_t e0, e1;
  FSI_CUDA_TRY(cudaEventCreate(&e0));
  FSI_CUDA_TRY(cudaEventCreate(&e1));
  const int nl = (int)h.levels.size();
  for (int l = 0; l + 1 < nl; ++l) {
    Level& L = h.levels[l];
    const size_t bytes = sizeof(T) * L.bs * (size_t)L.n;
    FSI_CUDA_TRY(cudaMemsetAsync(L.x, 0, bytes, s));
    FSI_CUDA_TRY(cudaMemsetAsync(L.b, 0, bytes, s));
    const int c4[3] = {64, 128, 256}, c7[2] = {1, 2};
    const int* cand = L.bs == 4 ? c4 : c7;
    const int nc = L.bs == 4 ? 3 : 2;
    float best = 1e30f;
    int pick = 0;
    for (int q = 0; q < nc; ++q) {
      const float ms = time_sweep<T>(L, cand[q], s, e0, e1);
      if (ms < best) {
        best = ms;
        pick = cand[q];
      }
    }
    L.shape = pick;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

void autotune_levels(Handle& h, cudaStream_t s) {
  if (h.precision == FSI_PREC_FP32_IR)
    autotune_t<float>(h, s);
  else
    autotune_t<double>(h, s);
  FSI_CUDA_TRY(cudaGetLastError());
}

void dots(Handle& h, const double* V, long ldv, int k, const double* y, long n, double* out_dev, cudaStream_t s) {
  dim3 grid(h.red_blocks, k);
  FSI_LAUNCH(fsi::KC_VECTOR, s, multidot_kernel<<<grid, kRedThreads, 0, s>>>(V, ldv, y, n, h.d_partial));
  FSI_LAUNCH(fsi::KC_VECTOR, s, reduce_partials_kernel<<<k, kRedThreads, 0, s>>>(h.d_partial, h.red_blocks, out_dev));
  FSI_CUDA_TRY(cudaGetLastError());
}

void multi_axpy(const double* coef_dev, const double* V, int k, long n, double* w, double sign, cudaStream_t s) {
  FSI_LAUNCH(fsi::KC_VECTOR, s, multi_axpy_kernel<<<grid_stride_blocks(n), 256, 0, s>>>(coef_dev, V, k, n, sign, w));
  FSI_CUDA_TRY(cudaGetLastError());
}

void axpy(double a, const double* x, double* y, long n, cudaStream_t s) {
  FSI_LAUNCH(fsi::KC_VECTOR, s, axpy_kernel<<<grid_stride_blocks(n), 256, 0, s>>>(a, x, y, n));
  FSI_CUDA_TRY(cudaGetLastError());
}

void scale_copy(double a, const double* x, double* y, long n, cudaStream_t s) {
  FSI_LAUNCH(fsi::KC_VECTOR, s, scale_copy_kernel<<<grid_stride_blocks(n), 256, 0, s>>>(a, x, y, n));
  FSI_CUDA_TRY(cudaGetLastError());
}

void to_float(const double* x, float* y, long n, cudaStream_t s) {
  FSI_LAUNCH(fsi::KC_VECTOR, s, to_float_kernel<<<grid_stride_blocks(n), 256, 0, s>>>(x, y, n));
  FSI_CUDA_TRY(cudaGetLastError());
}

void to_double(const float* x, double* y, long n, cudaStream_t s) {
  FSI_LAUNCH(fsi::KC_VECTOR, s, to_double_kernel<<<grid_stride_blocks(n), 256, 0, s>>>(x, y, n));
  FSI_CUDA_TRY(cudaGetLastError());
}

void segment_sumsq(const int32_t* seg_ptr, int n_seg, const double* x, double* out, cudaStream_t s) {
  FSI_LAUNCH(fsi::KC_VECTOR, s, segment_sumsq_kernel<<<n_seg, kRedThreads, 0, s>>>(seg_ptr, x, out));
  FSI_CUDA_TRY(cudaGetLastError());
}

void seg_dots(const int32_t* seg_ptr, int n_seg, const double* V, long ldv, int k, const double* y, double* out_dev,
              cudaStream_t s) {
  dim3 grid(n_seg, k);
  FSI_LAUNCH(fsi::KC_VECTOR, s, seg_multidot_kernel<<<grid, kRedThreads, 0, s>>>(seg_ptr, n_seg, V, ldv, y, out_dev));
  FSI_CUDA_TRY(cudaGetLastError());
}

void seg_multi_axpy(const int32_t* seg_node, int n_seg, const double* coef_dev, const double* V, int k, long n,
                    double* w, double sign, cudaStream_t s) {
  FSI_LAUNCH(fsi::KC_VECTOR, s, seg_multi_axpy_kernel<<<grid_stride_blocks(n), 256, 0, s>>>(seg_node, n_seg, coef_dev, V,
                                                                                             k, n, sign, w));
  FSI_CUDA_TRY(cudaGetLastError());
}

void segment_normalise(int n_seg, double* a, double* b, cudaStream_t s) {
  FSI_LAUNCH(fsi::KC_VECTOR, s, segment_normalise_kernel<<<blocks_for(n_seg, 128), 128, 0, s>>>(n_seg, a, b));
  FSI_CUDA_TRY(cudaGetLastError());
}

void segment_scale(const int32_t* seg_node, const double* scale, double* x, long n, cudaStream_t s) {
  FSI_LAUNCH(fsi::KC_VECTOR, s, segment_scale_kernel<<<grid_stride_blocks(n), 256, 0, s>>>(seg_node, scale, x, n));
  FSI_CUDA_TRY(cudaGetLastError());
}

void mask_vector(const uint8_t* cmask, double* x, long n, cudaStream_t s) {
  FSI_LAUNCH(fsi::KC_VECTOR, s, mask_vector_kernel<<<grid_stride_blocks(n), 256, 0, s>>>(cmask, x, n));
  FSI_CUDA_TRY(cudaGetLastError());
}

}  // namespace fsi
