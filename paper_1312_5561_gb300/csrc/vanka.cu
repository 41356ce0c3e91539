// Multiplicative Vanka smoother of the finest AMG level (Sec. 5.5.2, Eq. locsys
// and vankasmooth).
//
// Patch P_i: the pressure unknown p_i and the displacement unknowns of every
// node that B2 couples to it, i.e. the nodes of block row i of K (node i and
// its mesh neighbours; 15 nodes, 46 unknowns at an interior Kuhn node).  Local
// unknown order: (u_x, u_y, u_z) of the row's nodes in column order, then p_i.
//
// Per Newton step (vanka_factor): each CTA forms K^i, the restriction of K to
// the patch, in shared memory and inverts it by Gauss-Jordan elimination with
// partial pivoting; the inverse is stored densely per patch.
//
// Per sweep: the patches are visited colour by colour.  Colours come from a
// greedy distance-2 colouring of the nodes, so two patches of one colour share
// no unknown.  Within a colour every patch first computes its local residual
// from the current iterate and its correction (vanka_solve), then all of them
// add omega times the correction (vanka_update): Gauss-Seidel across colours,
// simultaneous within a colour, deterministic.
#include <algorithm>

#include "internal.h"

namespace fsi {
namespace {

constexpr int kVkThreads = 128;

__device__ __forceinline__ void vk_row(int l, int deg, int i, int r0, const int32_t* __restrict__ ci, int& g,
                                       int& comp) {
  if (l < 3 * deg) {
    g = ci[r0 + l / 3];
    comp = l % 3;
  } else {
    g = i;
    comp = 3;
  }
}

template <typename T>
__device__ __forceinline__ T vk_abs(T v) {
  return v < T(0) ? -v : v;
}

// K^i -> (K^i)^-1, one CTA per patch; shared memory: augmented [m][2m] matrix
template <typename T>
__global__ void __launch_bounds__(kVkThreads) vanka_factor_kernel(
    int n, const int32_t* __restrict__ order, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
    const int32_t* __restrict__ diag, const T* __restrict__ vals, int m_max, T* __restrict__ inv,
    int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char vk_smem[];
  T* M = reinterpret_cast<T*>(vk_smem);
  T* fac = M + (size_t)m_max * (2 * m_max + 1);
  __shared__ int piv;
  const int k = blockIdx.x;
  if (k >= n) return;
  const int i = order[k];
  const int r0 = rp[i], deg = rp[i + 1] - r0;
  const int m = 3 * deg + 1;
  const int ld = 2 * m_max + 1;
  for (int q = threadIdx.x; q < m * ld; q += blockDim.x) {
    const int r = q / ld, c = q % ld;
    M[q] = (c == m + r) ? T(1) : T(0);
  }
  __syncthreads();
  for (int ab = threadIdx.x; ab < deg * deg; ab += blockDim.x) {
    const int a = ab / deg, b = ab % deg;
    const int ga = ci[r0 + a], gb = ci[r0 + b];
    int q = -1;
    for (int t = rp[ga]; t < rp[ga + 1]; ++t)
      if (ci[t] == gb) {
        q = t;
        break;
      }
    if (q < 0) continue;
    const T* B = vals + 16L * q;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) M[(3 * a + r) * ld + 3 * b + c] = B[4 * r + c];
    if (gb == i)
      for (int r = 0; r < 3; ++r) M[(3 * a + r) * ld + 3 * deg] = B[4 * r + 3];   // K(u_a, p_i)
  }
  for (int b = threadIdx.x; b < deg; b += blockDim.x) {
    const T* B = vals + 16L * (r0 + b);                                          // block (i, b)
    for (int c = 0; c < 3; ++c) M[3 * deg * ld + 3 * b + c] = B[12 + c];         // K(p_i, u_b)
  }
  if (threadIdx.x == 0) M[3 * deg * ld + 3 * deg] = vals[16L * diag[i] + 15];
  __syncthreads();
  const int w = 2 * m;
  for (int c = 0; c < m; ++c) {
    if (threadIdx.x == 0) {
      int p = c;
      T best = vk_abs(M[c * ld + c]);
      for (int r = c + 1; r < m; ++r) {
        const T v = vk_abs(M[r * ld + c]);
        if (v > best) {
          best = v;
          p = r;
        }
      }
      piv = best > T(0) ? p : -1;
      if (piv < 0) atomicOr(err, 16);
    }
    __syncthreads();
    const int p = piv;
    if (p < 0) return;   // singular patch: reported through err, inverse left unwritten
    if (p != c)
      for (int j = threadIdx.x; j < w; j += blockDim.x) {
        const T t = M[c * ld + j];
        M[c * ld + j] = M[p * ld + j];
        M[p * ld + j] = t;
      }
    __syncthreads();
    const T d = T(1) / M[c * ld + c];
    for (int r = threadIdx.x; r < m; r += blockDim.x) fac[r] = M[r * ld + c];
    __syncthreads();
    for (int j = threadIdx.x; j < w; j += blockDim.x) M[c * ld + j] *= d;
    __syncthreads();
    for (int q = threadIdx.x; q < m * w; q += blockDim.x) {
      const int r = q / w, j = q % w;
      if (r != c) M[r * ld + j] -= fac[r] * M[c * ld + j];
    }
    __syncthreads();
  }
  T* out = inv + (size_t)k * m_max * m_max;
  for (int q = threadIdx.x; q < m * m; q += blockDim.x) {
    const int r = q / m, c = q % m;
    out[r * m_max + c] = M[r * ld + m + c];
  }
}

// z_k = (K^k)^-1 (b - K x) restricted to patch k, for the patches k0..k1-1 of one colour
template <typename T>
__global__ void __launch_bounds__(kVkThreads) vanka_solve_kernel(
    int k0, int k1, const int32_t* __restrict__ order, const int32_t* __restrict__ rp,
    const int32_t* __restrict__ ci, const T* __restrict__ vals, const T* __restrict__ x, const T* __restrict__ b,
    const T* __restrict__ inv, int m_max, T* __restrict__ z) {
  __shared__ T r[kVankaMaxM];
  const int k = k0 + blockIdx.x;
  if (k >= k1) return;
  const int i = order[k];
  const int r0 = rp[i], deg = rp[i + 1] - r0;
  const int m = 3 * deg + 1;
  for (int l = threadIdx.x; l < m; l += blockDim.x) {
    int g, comp;
    vk_row(l, deg, i, r0, ci, g, comp);
    T acc = b[4L * g + comp];
    for (int q = rp[g]; q < rp[g + 1]; ++q) {
      const T* B = vals + 16L * q + 4 * comp;
      const T* xc = x + 4L * ci[q];
      acc -= B[0] * xc[0] + B[1] * xc[1] + B[2] * xc[2] + B[3] * xc[3];
    }
    r[l] = acc;
  }
  __syncthreads();
  const T* I = inv + (size_t)k * m_max * m_max;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int l = warp; l < m; l += nw) {
    T s = T(0);
    for (int j = lane; j < m; j += 32) s += I[l * m_max + j] * r[j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) z[(size_t)k * m_max + l] = s;
  }
}

template <typename T>
__global__ void __launch_bounds__(kVkThreads) vanka_update_kernel(
    int k0, int k1, const int32_t* __restrict__ order, const int32_t* __restrict__ rp,
    const int32_t* __restrict__ ci, const T* __restrict__ z, int m_max, T omega, T* __restrict__ x) {
  const int k = k0 + blockIdx.x;
  if (k >= k1) return;
  const int i = order[k];
  const int r0 = rp[i], deg = rp[i + 1] - r0;
  const int m = 3 * deg + 1;
  for (int l = threadIdx.x; l < m; l += blockDim.x) {
    int g, comp;
    vk_row(l, deg, i, r0, ci, g, comp);
    x[4L * g + comp] += omega * z[(size_t)k * m_max + l];
  }
}

template <typename T>
size_t vk_factor_smem(int m_max) {
  return sizeof(T) * ((size_t)m_max * (2 * m_max + 1) + m_max);
}

}  // namespace

// Greedy distance-2 colouring of the nodes (node order): node i takes the
// smallest colour not used by any node j whose block row shares a column with
// row i.  Returns the colour-major order and the colour ranges.
void vanka_colouring(const HostPattern& pat, int n, std::vector<int32_t>& order, std::vector<int32_t>& cptr,
                     int* max_deg) {
  std::vector<int32_t> col(n, -1), mark;
  int md = 0, ncol = 0;
  for (int i = 0; i < n; ++i) {
    md = std::max(md, pat.row_ptr[i + 1] - pat.row_ptr[i]);
    for (int q = pat.row_ptr[i]; q < pat.row_ptr[i + 1]; ++q) {
      const int kk = pat.col_idx[q];
      for (int t = pat.row_ptr[kk]; t < pat.row_ptr[kk + 1]; ++t) {
        const int j = pat.col_idx[t];
        if (col[j] >= 0) mark[col[j]] = i;
      }
    }
    int c = 0;
    while (c < (int)mark.size() && mark[c] == i) ++c;
    if (c == (int)mark.size()) mark.push_back(-1);
    col[i] = c;
    ncol = std::max(ncol, c + 1);
  }
  cptr.assign(ncol + 1, 0);
  for (int i = 0; i < n; ++i) cptr[col[i] + 1]++;
  for (int c = 0; c < ncol; ++c) cptr[c + 1] += cptr[c];
  std::vector<int32_t> fill(cptr.begin(), cptr.end() - 1);
  order.assign(n, 0);
  for (int i = 0; i < n; ++i) order[fill[col[i]]++] = i;
  *max_deg = md;
}

void launch_vanka_factor(Handle& h, bool fp32, cudaStream_t s) {
  const Level& L = h.levels[0];
  if (fp32) {
    const size_t shm = vk_factor_smem<float>(h.vk_m);
    FSI_CUDA_TRY(cudaFuncSetAttribute(vanka_factor_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)shm));
    FSI_LAUNCH(fsi::KC_BLOCKINV, s, vanka_factor_kernel<float><<<L.n, kVkThreads, shm, s>>>(
        L.n, h.d_vk_order, L.row_ptr, L.col_idx, L.diag_idx, (const float*)L.vals, h.vk_m, (float*)h.d_vk_inv,
        h.d_err));
  } else {
    const size_t shm = vk_factor_smem<double>(h.vk_m);
    FSI_CUDA_TRY(cudaFuncSetAttribute(vanka_factor_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)shm));
    FSI_LAUNCH(fsi::KC_BLOCKINV, s, vanka_factor_kernel<double><<<L.n, kVkThreads, shm, s>>>(
        L.n, h.d_vk_order, L.row_ptr, L.col_idx, L.diag_idx, (const double*)L.vals, h.vk_m, (double*)h.d_vk_inv,
        h.d_err));
  }
  FSI_CUDA_TRY(cudaGetLastError());
}

template <typename T>
void vanka_smooth(Handle& h, int sweeps, bool zero_start, cudaStream_t s) {
  const Level& L = h.levels[0];
  T* x = (T*)L.x;
  if (zero_start) FSI_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(T) * 4 * (size_t)L.n, s));
  const T omega = (T)h.opts.vanka_omega;
  for (int sw = 0; sw < sweeps; ++sw)
    for (int c = 0; c < h.vk_ncol; ++c) {
      const int k0 = h.vk_cptr[c], k1 = h.vk_cptr[c + 1];
      if (k1 <= k0) continue;
      FSI_LAUNCH(fsi::KC_JACOBI0, s, vanka_solve_kernel<T><<<k1 - k0, kVkThreads, 0, s>>>(
          k0, k1, h.d_vk_order, L.row_ptr, L.col_idx, (const T*)L.vals, x, (const T*)L.b, (const T*)h.d_vk_inv,
          h.vk_m, (T*)h.d_vk_z));
      FSI_LAUNCH(fsi::KC_JACOBI0, s, vanka_update_kernel<T><<<k1 - k0, kVkThreads, 0, s>>>(
          k0, k1, h.d_vk_order, L.row_ptr, L.col_idx, (const T*)h.d_vk_z, h.vk_m, omega, x));
    }
  FSI_CUDA_TRY(cudaGetLastError());
}

template void vanka_smooth<float>(Handle&, int, bool, cudaStream_t);
template void vanka_smooth<double>(Handle&, int, bool, cudaStream_t);

}  // namespace fsi
