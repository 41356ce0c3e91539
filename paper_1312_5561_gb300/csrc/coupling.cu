// Interface kernels of the Dirichlet-Neumann coupling loop (Sec. 5.1, 5.2):
// the surrogate fluid map, the restriction of the solid state to Gamma^0, the
// interface residual and the Aitken-relaxed update (Eq. acceit).  All are
// grid-stride loops over the n_Gamma interface nodes (a few thousand to a few
// tens of thousands): launch-bound, each one pass over O(n_Gamma) doubles.
#include <algorithm>

#include "internal.h"

namespace fsi {
namespace {

inline int gs_blocks(long n) {
  long b = (n + 255) / 256;
  return (int)std::min<long>(std::max<long>(b, 1), 4L * 152);
}

// node_p[idx_j] = p0 - c w_j . (d_j - d_ref(idx_j)); other entries untouched (zero)
__global__ void dn_fluid_kernel(int ng, const int32_t* __restrict__ idx, const double* __restrict__ w,
                                const double* __restrict__ d, const double* __restrict__ dref, double p0, double c,
                                double* __restrict__ node_p) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ng; j += gridDim.x * blockDim.x) {
    const int i = idx[j];
    double s = 0.0;
    for (int q = 0; q < 3; ++q) {
      const double dd = d[3 * j + q] - (dref ? dref[4L * i + q] : 0.0);
      s = fma(w[3 * j + q], dd, s);
    }
    node_p[i] = p0 - c * s;
  }
}

// out = the displacement of state on Gamma^0; with d != nullptr also r = out - d
__global__ void dn_restrict_kernel(int ng, const int32_t* __restrict__ idx, const double* __restrict__ state,
                                   double* __restrict__ out, const double* __restrict__ d, double* __restrict__ r) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ng; j += gridDim.x * blockDim.x) {
    const int i = idx[j];
    for (int q = 0; q < 3; ++q) {
      const double v = state[4L * i + q];
      out[3 * j + q] = v;
      if (r) r[3 * j + q] = v - d[3 * j + q];
    }
  }
}

// d = omega d~ + (1 - omega) d;  also dr = r - r_prev, r_prev = r for the next cycle
__global__ void dn_relax_kernel(long m, double omega, const double* __restrict__ dt, double* __restrict__ d) {
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (long)gridDim.x * blockDim.x)
    d[q] = omega * dt[q] + (1.0 - omega) * d[q];
}

__global__ void dn_diff_kernel(long m, const double* __restrict__ r, const double* __restrict__ r_prev,
                               double* __restrict__ dr) {
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (long)gridDim.x * blockDim.x)
    dr[q] = r[q] - r_prev[q];
}

}  // namespace

void dn_fluid(int ng, const int32_t* idx, const double* w, const double* d, const double* dref, double p0, double c,
              double* node_p, cudaStream_t s) {
  FSI_LAUNCH(fsi::KC_VECTOR, s, dn_fluid_kernel<<<gs_blocks(ng), 256, 0, s>>>(ng, idx, w, d, dref, p0, c, node_p));
  FSI_CUDA_TRY(cudaGetLastError());
}

void dn_restrict(int ng, const int32_t* idx, const double* state, double* out, const double* d, double* r,
                 cudaStream_t s) {
  FSI_LAUNCH(fsi::KC_VECTOR, s, dn_restrict_kernel<<<gs_blocks(ng), 256, 0, s>>>(ng, idx, state, out, d, r));
  FSI_CUDA_TRY(cudaGetLastError());
}

void dn_relax(long m, double omega, const double* dt, double* d, cudaStream_t s) {
  FSI_LAUNCH(fsi::KC_VECTOR, s, dn_relax_kernel<<<gs_blocks(m), 256, 0, s>>>(m, omega, dt, d));
  FSI_CUDA_TRY(cudaGetLastError());
}

void dn_diff(long m, const double* r, const double* r_prev, double* dr, cudaStream_t s) {
  FSI_LAUNCH(fsi::KC_VECTOR, s, dn_diff_kernel<<<gs_blocks(m), 256, 0, s>>>(m, r, r_prev, dr));
  FSI_CUDA_TRY(cudaGetLastError());
}

}  // namespace fsi
