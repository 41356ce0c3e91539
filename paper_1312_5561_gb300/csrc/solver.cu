// Handle set-up, AMG hierarchy, Krylov methods, Newton's method and the C ABI.
//
// Newton's method follows Sec. 4.4: at each iterate the residual R(v_k) of the
// stabilised weak form (Eq. stabweakelas) and the consistent tangent K_k
// (Eq. globsys) are assembled, K_k dv = -R(v_k) is solved by a Krylov method
// to a relative reduction eps_1, and v_(k+1) = v_k + dv.  The stop test is
// the relative residual ||R(v_k)|| <= eps_2 ||R(v_0)||; with adaptive_tol the
// inner reduction follows eps_(1,k) = eps_(2,k-1)^2 (Sec. 4.4, end).
//
// The Krylov method is FGMRES(m) with classical Gram-Schmidt applied twice
// (or BiCGStab), right-preconditioned by one V-cycle of a smoothed-aggregation
// AMG on the 4x4 block system (damped block-Jacobi or Vanka smoothing,
// Galerkin coarse operators, a dense block-diagonal solve on the coarsest
// level), or by the block-triangular P_L of Sec. 5.4.2.  Vectors,
// orthogonalisation and the outer residual are FP64; in FSI_PREC_FP32_IR the
// tangent and the V-cycle are FP32 while the Newton residual stays FP64, so
// each Newton step acts as one step of iterative refinement.  The
// Dirichlet-Neumann coupling loop of Sec. 5.1-5.2 (dn_impl) runs Newton solves
// under a surrogate fluid load.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <exception>
#include <new>
#include <numeric>

#include "amg_setup.h"
#include "internal.h"

namespace fsi {

thread_local Profiler* g_prof = nullptr;
std::atomic<long long> g_launches{0};
// While this thread captures a V-cycle into a graph, its launches are recorded,
// not run: they are counted here and added to g_launches per graph launch.
static thread_local long long* t_captured = nullptr;

void launch_begin(int cls, cudaStream_t s) {
  if (t_captured)
    ++*t_captured;
  else
    g_launches.fetch_add(1, std::memory_order_relaxed);
  Profiler* p = g_prof;
  if (!p || !p->on) return;
  if (p->pool.size() < 2 * (p->used + 1)) {
    for (int q = 0; q < 2; ++q) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      p->pool.push_back(e);
    }
    p->cls.push_back(cls);
  }
  p->cls[p->used] = cls;
  cudaEventRecord(p->pool[2 * p->used], s);
}

void launch_end(cudaStream_t s) {
  Profiler* p = g_prof;
  if (!p || !p->on || p->pool.size() < 2 * (p->used + 1)) return;
  cudaEventRecord(p->pool[2 * p->used + 1], s);
  ++p->used;
}

// Sets the handle's profiler as the current one for the duration of a call.
struct ProfScope {
  explicit ProfScope(Profiler* p) { g_prof = p; }
  ~ProfScope() { g_prof = nullptr; }
};

namespace {

// layout of the small device/pinned scratch used by the Krylov methods
constexpr int kMaxRestart = 128;
constexpr int kDotH2 = kMaxRestart + 8;        // second Gram-Schmidt pass
constexpr int kDotW = 2 * (kMaxRestart + 8);   // ||w||^2
constexpr int kDotY = kDotW + 8;               // least-squares coefficients
constexpr int kDotNorm = kDotY + kMaxRestart + 8;
constexpr int kDotSize = kDotNorm + 8;

struct OomError {
  std::string msg;
};

template <typename T>
T* dalloc(size_t count) {
  if (count == 0) count = 1;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, sizeof(T) * count);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw OomError{std::string("cudaMalloc of ") + std::to_string(sizeof(T) * count) + " bytes: " +
                   cudaGetErrorString(e)};
  }
  return (T*)p;
}

template <typename T>
T* upload(const T* host, size_t count, cudaStream_t s) {
  T* d = dalloc<T>(count);
  if (count) FSI_CUDA_TRY(cudaMemcpyAsync(d, host, sizeof(T) * count, cudaMemcpyHostToDevice, s));
  return d;
}

template <typename T>
T* upload(const std::vector<T>& v, cudaStream_t s) {
  return upload(v.data(), v.size(), s);
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

int check_err(Handle& h, cudaStream_t s) {
  int e = 0;
  FSI_CUDA_TRY(cudaMemcpyAsync(&e, h.d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  FSI_CUDA_TRY(cudaStreamSynchronize(s));
  if (e) FSI_CUDA_TRY(cudaMemsetAsync(h.d_err, 0, sizeof(int), s));
  return e;
}

// sqrt(x^T M x) with the P1 mass matrices (Sec. 4.4, Eq. newstop)
double mass_norm_host(Handle& h, const double* x, cudaStream_t s) {
  launch_mass_norm2(h, x, h.d_dots + kDotNorm + 4, s);
  double v = 0.0;
  FSI_CUDA_TRY(cudaMemcpyAsync(&v, h.d_dots + kDotNorm + 4, sizeof(double), cudaMemcpyDeviceToHost, s));
  FSI_CUDA_TRY(cudaStreamSynchronize(s));
  return std::sqrt(std::max(v, 0.0));
}

double norm2_host(Handle& h, const double* x, long n, cudaStream_t s) {
  dots(h, x, 0, 1, x, n, h.d_dots + kDotNorm, s);
  double v = 0.0;
  FSI_CUDA_TRY(cudaMemcpyAsync(&v, h.d_dots + kDotNorm, sizeof(double), cudaMemcpyDeviceToHost, s));
  FSI_CUDA_TRY(cudaStreamSynchronize(s));
  return std::sqrt(v);
}

void alloc_level_vectors(Level& L, bool f32) {
  const size_t ts = f32 ? 4 : 8;
  L.x = dalloc<char>(ts * L.bs * (size_t)L.n);
  L.x2 = dalloc<char>(ts * L.bs * (size_t)L.n);
  L.b = dalloc<char>(ts * L.bs * (size_t)L.n);
  L.r = dalloc<char>(ts * L.bs * (size_t)L.n);
}

void upload_pattern(Level& L, cudaStream_t s) {
  const HostPattern& P = L.hpat;
  L.n = (int)P.row_ptr.size() - 1;
  L.nb = (int)P.col_idx.size();
  std::vector<int32_t> diag(L.n), brow(L.nb);
  for (int i = 0; i < L.n; ++i) {
    diag[i] = find_block(P, i, i);
    for (int k = P.row_ptr[i]; k < P.row_ptr[i + 1]; ++k) brow[k] = i;
  }
  L.row_ptr = upload(P.row_ptr, s);
  L.col_idx = upload(P.col_idx, s);
  L.diag_idx = upload(diag, s);
  L.block_row = upload(brow, s);
}

// values as T on the device
void* upload_values(const std::vector<double>& v, bool f32, cudaStream_t s) {
  if (!f32) return upload(v, s);
  std::vector<float> f(v.begin(), v.end());
  float* d = upload(f, s);
  FSI_CUDA_TRY(cudaStreamSynchronize(s));   // the host staging vector dies here
  return d;
}

// Smoothed-aggregation hierarchy from the reference tangent (zero state).
void build_hierarchy(Handle& h, const std::vector<uint8_t>& free0, const std::vector<int32_t>& comp0,
                     const double* X, cudaStream_t s) {
  const bool f32 = h.precision == FSI_PREC_FP32_IR;
  Level& L0 = h.levels[0];
  // reference tangent, FP64, Dirichlet rows/columns applied
  double* zero = dalloc<double>(4 * (size_t)h.n_nodes);
  double* kref = dalloc<double>(16 * (size_t)L0.nb);
  FSI_CUDA_TRY(cudaMemsetAsync(zero, 0, sizeof(double) * 4 * h.n_nodes, s));
  launch_assemble(h, zero, nullptr, nullptr, true, s, kref, 0);
  HostBsr A0;
  A0.n = A0.nc = L0.n;
  A0.br = A0.bc = 4;
  A0.rp = L0.hpat.row_ptr;
  A0.ci = L0.hpat.col_idx;
  A0.v.resize(16 * (size_t)L0.nb);
  FSI_CUDA_TRY(cudaMemcpyAsync(A0.v.data(), kref, sizeof(double) * A0.v.size(), cudaMemcpyDeviceToHost, s));
  FSI_CUDA_TRY(cudaStreamSynchronize(s));
  cudaFree(zero);
  cudaFree(kref);
  if (check_err(h, s) & 1) throw ArgError("reference configuration has an inverted element");
  if (h.opts.precond == FSI_PRECOND_BLOCK_LT) {
    // P_L: the hierarchy is built for the displacement block A alone (same
    // transformation as launch_split_a)
    for (int i = 0; i < A0.n; ++i)
      for (int q = A0.rp[i]; q < A0.rp[i + 1]; ++q)
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) {
            double& v = A0.v[16 * (size_t)q + 4 * a + b];
            if ((a == 3) != (b == 3)) v = 0.0;
            if (a == 3 && b == 3) v = A0.ci[q] == i ? 1.0 : 0.0;
          }
  }

  std::vector<HostLevel> hl;
  HostCoarse hc;
  h.filter_p = h.opts.inertia_coef > 0.0;
  build_sa_hierarchy(A0, free0, X, comp0, std::max(1, h.opts.coarse_max_nodes), std::max(1, h.opts.max_levels),
                     8, h.filter_p, hl, hc, h.opts.aggregation == FSI_AGG_GROW, h.opts.exact_candidates != 0,
                     h.opts.power_steps);
  const int nl = (int)hl.size();
  const size_t ts = f32 ? 4 : 8;
  for (int l = 1; l < nl; ++l) {
    Level C;
    const HostBsr& A = hl[l].A;
    C.bs = A.br;
    C.hpat.row_ptr = A.rp;
    C.hpat.col_idx = A.ci;
    upload_pattern(C, s);
    C.vals = upload_values(A.v, f32, s);
    C.dinv = upload_values(hl[l].Dinv, f32, s);
    if (f32 && h.opts.coarse_bf16 && l + 1 < nl) {   // the coarsest level is solved, not smoothed
      C.vals_lp = dalloc<char>(2 * (size_t)C.nb * C.bs * C.bs);
      launch_values_to_bf16(C, s);
    }
    alloc_level_vectors(C, f32);
    C.kc_spmv = l == 1 ? KC_LEVEL1_SPMV : KC_COARSE_BSR;
    if (h.opts.coarse_smoother == FSI_COARSE_MR && l + 1 < nl) {   // the coarsest level is solved, not smoothed
      C.w = dalloc<char>(ts * C.bs * (size_t)C.n);
      C.mr = dalloc<double>(2 * kMrBlocks + 8);
    }
    h.levels.push_back(std::move(C));
  }
  for (int l = 0; l + 1 < nl; ++l) {
    Level& L = h.levels[l];
    const HostLevel& H = hl[l];
    const int bs = L.bs;
    L.p_nb = H.P.nb();
    L.p_rp = upload(H.P.rp, s);
    L.p_ci = upload(H.P.ci, s);
    L.p_v = upload_values(H.P.v, f32, s);
    std::vector<int32_t> brow(L.p_nb);
    for (int i = 0; i < H.P.n; ++i)
      for (int q = H.P.rp[i]; q < H.P.rp[i + 1]; ++q) brow[q] = i;
    L.p_brow = upload(brow, s);
    L.pt_nb = H.PT.nb();
    L.pt_rp = upload(H.PT.rp, s);
    L.pt_ci = upload(H.PT.ci, s);
    L.pt_v = upload_values(H.PT.v, f32, s);
    L.pt_src = upload(H.pt_src, s);
    L.agg = upload(H.agg, s);
    L.ptent = upload_values(H.Pt, f32, s);
    L.freem = upload(H.free, s);
    L.omega_p = H.omega_p;
    L.w_ptr = upload(H.w_ptr, s);
    L.w_k = upload(H.w_k, s);
    L.w_v = dalloc<char>(ts * (size_t)L.p_nb * bs * 7);
    if (h.filter_p) L.dinv_f = dalloc<char>(ts * (size_t)L.n * bs * bs);
    L.ap_nb = H.AP.nb();
    L.ap_ptr = upload(H.ap_ptr, s);
    L.ap_pairs = upload(H.ap_pairs, s);
    L.ap_v = dalloc<char>(ts * (size_t)L.ap_nb * bs * 7);
    L.ac_ptr = upload(H.ac_ptr, s);
    L.ac_pairs = upload(H.ac_pairs, s);
    L.n_fix = (int)H.fix_blk.size();
    L.fix_blk = upload(H.fix_blk, s);
    L.fix_dof = upload(H.fix_dof, s);
    FSI_CUDA_TRY(cudaStreamSynchronize(s));
  }
  Coarse& C = h.coarse;
  C.n_comp = (int)hc.comp_ptr.size() - 1;
  C.max_dofs = hc.max_dofs;
  C.comp_ptr = upload(hc.comp_ptr, s);
  C.inv_off = upload(hc.inv_off, s);
  C.inv = dalloc<char>(ts * (size_t)hc.inv_size);
  C.work = dalloc<double>((size_t)hc.inv_size);
  FSI_CUDA_TRY(cudaStreamSynchronize(s));
}

// Per Newton step, from the current tangent: block-Jacobi inverses, smoothed
// prolongators and Galerkin operators of every level, and the dense inverse
// of the coarsest operator.
// With amg_lag = L > 0 the coarse levels (smoothed P, Galerkin operators,
// coarsest factorisation) are recomputed only on every (L+1)-th call; the
// finest level always uses the current K and its current block inverses.
void amg_numeric(Handle& h, cudaStream_t s) {
  const bool f32 = h.precision == FSI_PREC_FP32_IR;
  const int nl = (int)h.levels.size();
  if (h.opts.precond == FSI_PRECOND_BLOCK_LT) launch_split_a(h.levels[0], h.k_vals, f32, s);
  launch_block_inverse(h.levels[0], f32, h.d_err, s);
  if (h.opts.smoother == FSI_SMOOTHER_VANKA) launch_vanka_factor(h, f32, s);
  const bool refresh = h.opts.amg_lag <= 0 || (h.amg_calls % (h.opts.amg_lag + 1)) == 0;
  ++h.amg_calls;
  if (!refresh) return;
  for (int l = 0; l + 1 < nl; ++l) {
    if (l > 0) launch_block_inverse(h.levels[l], f32, h.d_err, s);
    launch_galerkin(h.levels[l], h.levels[l + 1], f32, h.filter_p, s);
    if (h.levels[l + 1].vals_lp) launch_values_to_bf16(h.levels[l + 1], s);
  }
  launch_coarse_factor(h, f32, s);
}

// The V-cycle reads and writes only level buffers whose addresses are fixed
// for the life of the handle, so it can be captured once into a CUDA graph and
// replayed on any stream (use_graphs).  Kernel event timing is suspended while
// capturing, so a replayed V-cycle is not split by kernel class.
void run_vcycle(Handle& h, cudaStream_t s) {
  const bool f32 = h.precision == FSI_PREC_FP32_IR;
  // while kernel timing is recording, launch eagerly so that every kernel is timed
  if (!h.opts.use_graphs || (g_prof && g_prof->on)) {
    if (f32) vcycle<float>(h, 0, s); else vcycle<double>(h, 0, s);
    return;
  }
  if (!h.vc_exec) {
    FSI_CUDA_TRY(cudaStreamSynchronize(h.stream));
    Profiler* saved = g_prof;
    g_prof = nullptr;
    long long captured = 0;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h.stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      t_captured = &captured;
      try {
        if (f32) vcycle<float>(h, 0, h.stream); else vcycle<double>(h, 0, h.stream);
      } catch (...) {
        // a failure while capturing: end the capture so that the handle's
        // stream stays usable, and restore the accounting, then report it
        t_captured = nullptr;
        if (cudaStreamEndCapture(h.stream, &graph) == cudaSuccess && graph) cudaGraphDestroy(graph);
        g_prof = saved;
        throw;
      }
      t_captured = nullptr;
      e = cudaStreamEndCapture(h.stream, &graph);
    }
    g_prof = saved;
    if (e != cudaSuccess && graph) cudaGraphDestroy(graph);
    FSI_CUDA_TRY(e);
    h.vc_kernels = captured;
    e = cudaGraphInstantiate(&h.vc_exec, graph, 0);
    cudaGraphDestroy(graph);
    FSI_CUDA_TRY(e);
  }
  FSI_CUDA_TRY(cudaGraphLaunch(h.vc_exec, s));
  g_launches.fetch_add(h.vc_kernels, std::memory_order_relaxed);
}

void apply_operator(Handle& h, const double* x, double* y, cudaStream_t s);

// z = P_L^-1 v (Eq. lpre): z_u = one V-cycle on A applied to v_u, then
// z_p = S~^-1 (B2 z_u - v_p); B2 z_u is the pressure part of K (z_u, 0)
static void precondition_pl(Handle& h, const double* v, double* z, cudaStream_t s) {
  Level& L0 = h.levels[0];
  const bool f32 = h.precision == FSI_PREC_FP32_IR;
  pl_stage(v, L0.b, f32, L0.n, s);
  run_vcycle(h, s);
  pl_unstage(L0.x, z, f32, L0.n, s);
  apply_operator(h, z, h.d_pl_y, s);
  pl_pressure(h.d_pl_y, v, h.d_sinv, z, L0.n, s);
}

// z = M^-1 v (one V-cycle, or P_L)
void precondition(Handle& h, const double* v, double* z, cudaStream_t s) {
  if (h.opts.precond == FSI_PRECOND_BLOCK_LT) {
    precondition_pl(h, v, z, s);
    return;
  }
  Level& L0 = h.levels[0];
  const long n = 4L * L0.n;
  if (h.precision == FSI_PREC_FP32_IR) {
    to_float(v, (float*)L0.b, n, s);
    run_vcycle(h, s);
    to_double((const float*)L0.x, z, n, s);
  } else {
    FSI_CUDA_TRY(cudaMemcpyAsync(L0.b, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    run_vcycle(h, s);
    FSI_CUDA_TRY(cudaMemcpyAsync(z, L0.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
}

// y = K x (FP64 vectors).  With FP32 values the sum is carried in
// double-float arithmetic; with FP64 values in FP64.
void apply_operator(Handle& h, const double* x, double* y, cudaStream_t s) {
  if (h.precision == FSI_PREC_FP32_IR)
    launch_spmv_df(h.levels[0], h.k_vals, x, h.d_xdf, nullptr, y, s);
  else
    launch_spmv_f64acc(h.levels[0], h.k_vals, x, y, false, s);
}

void operator_residual(Handle& h, const double* b, const double* x, double* r, cudaStream_t s) {
  if (h.precision == FSI_PREC_FP32_IR)
    launch_spmv_df(h.levels[0], h.k_vals, x, h.d_xdf, b, r, s);
  else
    launch_residual_f64(h.levels[0], h.k_vals, b, x, r, false, s);
}

// FGMRES(m), right preconditioned.  Returns iterations; *rel = ||b - A x|| / ||b||.
// Orthogonalisation: classical Gram-Schmidt applied twice (one pass alone lost
// enough orthogonality here to multiply the iteration count by 2.5).  The new
// direction is formed in place in V_(j+1), so each reduction also returns
// ||w||^2 and the norm after the second pass follows from Pythagoras.
int fgmres(Handle& h, const double* b, double* x, double rtol, int maxit, double* rel, cudaStream_t s) {
  const long n = 4L * h.n_nodes;
  const int m = h.m;
  double* V = h.d_V;
  double* Z = h.d_Z;
  double* r = h.d_r;
  operator_residual(h, b, x, r, s);
  const double bnorm = norm2_host(h, b, n, s);
  double beta = norm2_host(h, r, n, s);
  if (bnorm == 0.0) {
    FSI_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    *rel = 0.0;
    return 0;
  }
  const double target = rtol * bnorm;
  int total = 0;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  while (beta > target && total < maxit) {
    scale_copy(1.0 / beta, r, V, n, s);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jj = 0;
    for (int j = 0; j < m; ++j) {
      double* vj = V + (size_t)j * n;
      double* zj = Z + (size_t)j * n;
      double* w = V + (size_t)(j + 1) * n;
      precondition(h, vj, zj, s);
      apply_operator(h, zj, w, s);
      // pass 1: h1 = V^T w (w is vector j+1); the update reads h1 from device
      // memory, so the host waits only once, after pass 2
      dots(h, V, n, j + 2, w, n, h.d_dots, s);
      multi_axpy(h.d_dots, V, j + 1, n, w, -1.0, s);
      // pass 2: h2 = V^T w and ||w||^2 of the once-orthogonalised w
      dots(h, V, n, j + 2, w, n, h.d_dots + kDotH2, s);
      FSI_CUDA_TRY(cudaMemcpyAsync(h.h_dots, h.d_dots, sizeof(double) * (kDotH2 + j + 2), cudaMemcpyDeviceToHost,
                                   s));
      FSI_CUDA_TRY(cudaStreamSynchronize(s));
      double proj2 = 0.0;
      for (int i = 0; i <= j; ++i) {
        H[(size_t)i * m + j] = h.h_dots[i] + h.h_dots[kDotH2 + i];
        proj2 += h.h_dots[kDotH2 + i] * h.h_dots[kDotH2 + i];
      }
      multi_axpy(h.d_dots + kDotH2, V, j + 1, n, w, -1.0, s);
      const double hn2 = h.h_dots[kDotH2 + j + 1] - proj2;
      const double hn = std::sqrt(std::max(hn2, 0.0));
      H[(size_t)(j + 1) * m + j] = hn;
      if (hn > 0.0) scale_copy(1.0 / hn, w, w, n, s);
      // Givens rotations
      for (int i = 0; i < j; ++i) {
        double a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      {
        double a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
        double d = std::hypot(a, bb);
        cs[j] = d > 0 ? a / d : 1.0;
        sn[j] = d > 0 ? bb / d : 0.0;
        H[(size_t)j * m + j] = d;
        H[(size_t)(j + 1) * m + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
      }
      ++total;
      jj = j + 1;
      if (std::fabs(g[j + 1]) <= target || total >= maxit || hn == 0.0) break;
    }
    for (int i = jj - 1; i >= 0; --i) {
      double acc = g[i];
      for (int k = i + 1; k < jj; ++k) acc -= H[(size_t)i * m + k] * y[k];
      y[i] = acc / H[(size_t)i * m + i];
    }
    FSI_CUDA_TRY(cudaMemcpyAsync(h.d_dots + kDotY, y.data(), sizeof(double) * jj, cudaMemcpyHostToDevice, s));
    multi_axpy(h.d_dots + kDotY, Z, jj, n, x, 1.0, s);
    operator_residual(h, b, x, r, s);
    beta = norm2_host(h, r, n, s);
  }
  *rel = beta / bnorm;
  return total;
}

// FGMRES(m) with one Arnoldi process per segment of a batched mesh.  The
// system is block diagonal by segment, so every inner product, norm,
// Hessenberg column, Givens rotation and least-squares solve is taken per
// segment: each segment converges at its own rate to rtol relative to its own
// right-hand side, and a segment that has converged stops contributing (its
// basis vectors and coefficients are zero from then on).  The preconditioner
// (one V-cycle over the union hierarchy) acts on the union of the segments'
// basis vectors; flexible GMRES asks nothing more of it.  Returns the
// iterations of the slowest segment; *rel = the largest segment's
// ||b_s - A x_s|| / ||b_s||.
int fgmres_seg(Handle& h, const double* b, double* x, double rtol, int maxit, double* rel, cudaStream_t s) {
  const long n = 4L * h.n_nodes;
  const int m = h.m, ns = h.n_seg;
  double* V = h.d_V;
  double* Z = h.d_Z;
  double* r = h.d_r;
  auto seg_norms = [&](const double* v, std::vector<double>& out) {
    segment_sumsq(h.d_seg_ptr, ns, v, h.d_seg_a, s);
    FSI_CUDA_TRY(cudaMemcpyAsync(h.h_seg, h.d_seg_a, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
    FSI_CUDA_TRY(cudaStreamSynchronize(s));
    out.resize(ns);
    for (int q = 0; q < ns; ++q) out[q] = std::sqrt(h.h_seg[q]);
  };
  auto set_scale = [&](const std::vector<double>& sc) {
    for (int q = 0; q < ns; ++q) h.h_seg[q] = sc[q];
    FSI_CUDA_TRY(cudaMemcpyAsync(h.d_seg_a, h.h_seg, sizeof(double) * ns, cudaMemcpyHostToDevice, s));
  };
  std::vector<double> bn, beta;
  seg_norms(b, bn);
  operator_residual(h, b, x, r, s);
  seg_norms(r, beta);
  std::vector<char> done(ns), live(ns);
  auto converged = [&](int q) { return bn[q] == 0.0 || beta[q] <= rtol * bn[q]; };
  for (int q = 0; q < ns; ++q) done[q] = converged(q);
  const size_t hs = (size_t)(m + 1) * m;
  std::vector<double> H(hs * ns), cs((size_t)m * ns), sn((size_t)m * ns), g((size_t)(m + 1) * ns), y(m),
      sc(ns);
  std::vector<int> jj(ns);
  double* d_h1 = h.d_sdots;
  double* d_h2 = h.d_sdots + (size_t)(m + 2) * ns;
  int total = 0;
  auto any_open = [&](const std::vector<char>& f, bool want) {
    for (int q = 0; q < ns; ++q)
      if ((bool)f[q] == want) return true;
    return false;
  };
  while (any_open(done, false) && total < maxit) {
    for (int q = 0; q < ns; ++q) {
      live[q] = !done[q];
      sc[q] = live[q] ? 1.0 / beta[q] : 0.0;
      jj[q] = 0;
      std::fill(g.begin() + (size_t)q * (m + 1), g.begin() + (size_t)(q + 1) * (m + 1), 0.0);
      g[(size_t)q * (m + 1)] = live[q] ? beta[q] : 0.0;
    }
    FSI_CUDA_TRY(cudaMemcpyAsync(V, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    set_scale(sc);
    segment_scale(h.d_seg_node, h.d_seg_a, V, n, s);
    int jmax = 0;
    for (int j = 0; j < m; ++j) {
      double* vj = V + (size_t)j * n;
      double* zj = Z + (size_t)j * n;
      double* w = V + (size_t)(j + 1) * n;
      precondition(h, vj, zj, s);
      apply_operator(h, zj, w, s);
      seg_dots(h.d_seg_ptr, ns, V, n, j + 2, w, d_h1, s);
      seg_multi_axpy(h.d_seg_node, ns, d_h1, V, j + 1, n, w, -1.0, s);
      seg_dots(h.d_seg_ptr, ns, V, n, j + 2, w, d_h2, s);
      FSI_CUDA_TRY(cudaMemcpyAsync(h.h_sdots, h.d_sdots, sizeof(double) * (size_t)2 * (m + 2) * ns,
                                   cudaMemcpyDeviceToHost, s));
      FSI_CUDA_TRY(cudaStreamSynchronize(s));
      seg_multi_axpy(h.d_seg_node, ns, d_h2, V, j + 1, n, w, -1.0, s);
      const double* h1 = h.h_sdots;
      const double* h2 = h.h_sdots + (size_t)(m + 2) * ns;
      for (int q = 0; q < ns; ++q) {
        sc[q] = 0.0;
        if (!live[q]) continue;
        double* Hq = &H[hs * q];
        double* csq = &cs[(size_t)m * q];
        double* snq = &sn[(size_t)m * q];
        double* gq = &g[(size_t)(m + 1) * q];
        double proj2 = 0.0;
        for (int i = 0; i <= j; ++i) {
          Hq[(size_t)i * m + j] = h1[(size_t)i * ns + q] + h2[(size_t)i * ns + q];
          proj2 += h2[(size_t)i * ns + q] * h2[(size_t)i * ns + q];
        }
        const double hn = std::sqrt(std::max(h2[(size_t)(j + 1) * ns + q] - proj2, 0.0));
        Hq[(size_t)(j + 1) * m + j] = hn;
        sc[q] = hn > 0.0 ? 1.0 / hn : 0.0;
        for (int i = 0; i < j; ++i) {
          const double a = Hq[(size_t)i * m + j], bb = Hq[(size_t)(i + 1) * m + j];
          Hq[(size_t)i * m + j] = csq[i] * a + snq[i] * bb;
          Hq[(size_t)(i + 1) * m + j] = -snq[i] * a + csq[i] * bb;
        }
        const double a = Hq[(size_t)j * m + j], bb = Hq[(size_t)(j + 1) * m + j];
        const double d = std::hypot(a, bb);
        csq[j] = d > 0 ? a / d : 1.0;
        snq[j] = d > 0 ? bb / d : 0.0;
        Hq[(size_t)j * m + j] = d;
        Hq[(size_t)(j + 1) * m + j] = 0.0;
        gq[j + 1] = -snq[j] * gq[j];
        gq[j] = csq[j] * gq[j];
        jj[q] = j + 1;
        if (std::fabs(gq[j + 1]) <= rtol * bn[q] || hn == 0.0) {
          live[q] = 0;   // converged in this cycle: no further basis vectors
          sc[q] = 0.0;
        }
      }
      set_scale(sc);
      segment_scale(h.d_seg_node, h.d_seg_a, w, n, s);
      ++total;
      jmax = j + 1;
      if (!any_open(live, true) || total >= maxit) break;
    }
    // per-segment least squares: y_q = R_q^-1 g_q over its first jj[q] columns
    std::fill(h.h_scoef, h.h_scoef + (size_t)(m + 1) * ns, 0.0);
    for (int q = 0; q < ns; ++q) {
      const double* Hq = &H[hs * q];
      const double* gq = &g[(size_t)(m + 1) * q];
      const int k = jj[q];
      for (int i = k - 1; i >= 0; --i) {
        double acc = gq[i];
        for (int c = i + 1; c < k; ++c) acc -= Hq[(size_t)i * m + c] * y[c];
        y[i] = acc / Hq[(size_t)i * m + i];
      }
      for (int i = 0; i < k; ++i) h.h_scoef[(size_t)i * ns + q] = y[i];
    }
    FSI_CUDA_TRY(cudaMemcpyAsync(h.d_scoef, h.h_scoef, sizeof(double) * (size_t)jmax * ns, cudaMemcpyHostToDevice,
                                 s));
    if (jmax > 0) seg_multi_axpy(h.d_seg_node, ns, h.d_scoef, Z, jmax, n, x, 1.0, s);
    operator_residual(h, b, x, r, s);
    seg_norms(r, beta);
    for (int q = 0; q < ns; ++q) done[q] = converged(q);
  }
  double worst = 0.0;
  for (int q = 0; q < ns; ++q)
    if (bn[q] > 0.0) worst = std::max(worst, beta[q] / bn[q]);
  *rel = worst;
  return total;
}

// BiCGStab (van der Vorst), right-preconditioned by the same V-cycle: the
// paper's Krylov method for the solid (Sec. 5.4.2), here with the coupled AMG
// preconditioner.  Short recurrences: no restart length, two preconditioner
// and two operator applications per iteration.  Returns iterations.
int bicgstab(Handle& h, const double* b, double* x, double rtol, int maxit, double* rel, cudaStream_t s) {
  const long n = 4L * h.n_nodes;
  double* r = h.d_r;
  double* r0 = h.d_V;                       // shadow residual
  double* p = h.d_V + (size_t)n;
  double* v = h.d_V + 2 * (size_t)n;
  double* phat = h.d_Z;
  double* shat = h.d_Z + (size_t)n;
  double* t = h.d_w;
  operator_residual(h, b, x, r, s);
  const double bnorm = norm2_host(h, b, n, s);
  if (bnorm == 0.0) {
    FSI_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    *rel = 0.0;
    return 0;
  }
  const double target = rtol * bnorm;
  double rn = norm2_host(h, r, n, s);
  FSI_CUDA_TRY(cudaMemcpyAsync(r0, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  FSI_CUDA_TRY(cudaMemsetAsync(p, 0, sizeof(double) * n, s));
  FSI_CUDA_TRY(cudaMemsetAsync(v, 0, sizeof(double) * n, s));
  double rho = 1.0, alpha = 1.0, omega = 1.0;
  int it = 0;
  auto dot = [&](const double* a, const double* bb) {
    dots(h, a, 0, 1, bb, n, h.d_dots + kDotNorm + 1, s);
    double v_ = 0.0;
    FSI_CUDA_TRY(cudaMemcpyAsync(&v_, h.d_dots + kDotNorm + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    FSI_CUDA_TRY(cudaStreamSynchronize(s));
    return v_;
  };
  while (rn > target && it < maxit) {
    const double rho1 = dot(r0, r);
    if (rho1 == 0.0) break;
    const double beta = (rho1 / rho) * (alpha / omega);
    // p = r + beta (p - omega v)
    axpy(-omega, v, p, n, s);
    scale_copy(beta, p, p, n, s);
    axpy(1.0, r, p, n, s);
    precondition(h, p, phat, s);
    apply_operator(h, phat, v, s);
    alpha = rho1 / dot(r0, v);
    axpy(-alpha, v, r, n, s);                 // r becomes s
    axpy(alpha, phat, x, n, s);
    ++it;
    rn = norm2_host(h, r, n, s);
    if (rn <= target) break;
    precondition(h, r, shat, s);
    apply_operator(h, shat, t, s);
    const double tt = dot(t, t);
    omega = tt > 0.0 ? dot(t, r) / tt : 0.0;
    axpy(omega, shat, x, n, s);
    axpy(-omega, t, r, n, s);
    rn = norm2_host(h, r, n, s);
    rho = rho1;
    if (omega == 0.0) break;
  }
  operator_residual(h, b, x, r, s);           // true residual
  *rel = norm2_host(h, r, n, s) / bnorm;
  return it;
}

void set_error(Handle* h, const std::string& msg) {
  if (h) h->last_error = msg;
}

int linear_solve(Handle& h, const double* b, double* x, double rtol, double* rel, cudaStream_t s) {
  if (h.opts.krylov == FSI_KRYLOV_BICGSTAB) return bicgstab(h, b, x, rtol, h.opts.max_krylov, rel, s);
  if (h.n_seg > 1 && h.opts.segment_krylov) return fgmres_seg(h, b, x, rtol, h.opts.max_krylov, rel, s);
  return fgmres(h, b, x, rtol, h.opts.max_krylov, rel, s);
}

}  // namespace

// ------------------------------------------------------------------ create / destroy
static void destroy_impl(Handle* hp);

static Handle* create_impl(const fsi_mesh_desc* mesh, int n_mat, const fsi_material* mats,
                           const fsi_solver_opts* opts) {
  if (!mesh || !mats || n_mat <= 0) throw ArgError("mesh and material table are required");
  if (mesh->n_nodes <= 0 || mesh->n_elems <= 0 || !mesh->X || !mesh->tets || !mesh->mat_id)
    throw ArgError("mesh needs n_nodes > 0, n_elems > 0, X, tets and mat_id");
  if (mesh->n_faces > 0 && !mesh->neu_faces) throw ArgError("n_faces > 0 but neu_faces is NULL");
  const int nn = mesh->n_nodes, ne = mesh->n_elems;
  bool need_fibre = false;
  for (int e = 0; e < ne; ++e) {
    if (mesh->mat_id[e] < 0 || mesh->mat_id[e] >= n_mat) throw ArgError("mat_id out of range at element " + std::to_string(e));
    for (int a = 0; a < 4; ++a) {
      int v = mesh->tets[4 * e + a];
      if (v < 0 || v >= nn) throw ArgError("vertex index out of range at element " + std::to_string(e));
    }
    if (mats[mesh->mat_id[e]].model == FSI_MODEL_ARTERY) need_fibre = true;
  }
  for (int m = 0; m < n_mat; ++m) {
    const fsi_material& M = mats[m];
    if (M.model != FSI_MODEL_MOONEY_RIVLIN && M.model != FSI_MODEL_ARTERY) throw ArgError("unknown material model");
    if (!(M.kappa > 0) || !(M.c10 >= 0) || (M.model == FSI_MODEL_ARTERY && !(M.k2 > 0)))
      throw ArgError("material parameters out of range");
  }
  if (need_fibre && !mesh->fibre) throw ArgError("artery material needs fibre directions");
  for (int f = 0; f < mesh->n_faces; ++f)
    for (int a = 0; a < 3; ++a) {
      int v = mesh->neu_faces[3 * f + a];
      if (v < 0 || v >= nn) throw ArgError("face vertex out of range");
    }
  if (mesh->seg_node) {
    // segments are independent meshes: contiguous node ranges, every element inside one
    const int32_t* sg = mesh->seg_node;
    if (mesh->n_segments < 1) throw ArgError("seg_node given but n_segments < 1");
    for (int i = 0; i < nn; ++i) {
      if (sg[i] < 0 || sg[i] >= mesh->n_segments) throw ArgError("seg_node out of range at node " + std::to_string(i));
      if (i > 0 && sg[i] < sg[i - 1]) throw ArgError("seg_node must be non-decreasing (segments contiguous)");
    }
    for (int e = 0; e < ne; ++e)
      for (int a = 1; a < 4; ++a)
        if (sg[mesh->tets[4 * e + a]] != sg[mesh->tets[4 * e]])
          throw ArgError("element " + std::to_string(e) + " joins two segments");
  }

  Handle* hp = new Handle();
  // a create that fails part-way releases what it has allocated
  struct Guard {
    Handle* p;
    ~Guard() { if (p) destroy_impl(p); }
  } guard{hp};
  Handle& h = *hp;
  fsi_solid_default_opts(&h.opts);
  if (opts) h.opts = *opts;
  if (h.opts.precond != FSI_PRECOND_AMG && h.opts.precond != FSI_PRECOND_BLOCK_LT)
    throw ArgError("unknown preconditioner");
  if (h.opts.smoother != FSI_SMOOTHER_JACOBI && h.opts.smoother != FSI_SMOOTHER_VANKA)
    throw ArgError("unknown smoother");
  if (h.opts.aggregation != FSI_AGG_RING && h.opts.aggregation != FSI_AGG_GROW)
    throw ArgError("unknown aggregation");
  if (h.opts.coarse_smoother != FSI_COARSE_JACOBI && h.opts.coarse_smoother != FSI_COARSE_MR)
    throw ArgError("unknown coarse smoother");
  if (h.opts.power_steps < 1 || h.opts.power_steps > 10000) throw ArgError("power_steps must lie in [1, 10000]");
  // BiCGStab needs a fixed (linear) preconditioner
  if (h.opts.krylov == FSI_KRYLOV_BICGSTAB) h.opts.coarse_smoother = FSI_COARSE_JACOBI;
  h.opts.restart = std::min(std::max(h.opts.restart, 1), kMaxRestart);
  if (h.opts.krylov == FSI_KRYLOV_BICGSTAB) h.opts.restart = std::max(h.opts.restart, 2);   // BiCGStab work vectors
  h.m = h.opts.restart;
  h.precision = h.opts.precision == FSI_PREC_FP32_IR ? FSI_PREC_FP32_IR : FSI_PREC_FP64;
  const bool f32 = h.precision == FSI_PREC_FP32_IR;
  h.n_nodes = nn;
  h.n_elems = ne;
  h.n_faces = mesh->n_faces;
  h.n_mat = n_mat;
  cudaStream_t s = nullptr;
  FSI_CUDA_TRY(cudaStreamCreateWithFlags(&h.stream, cudaStreamNonBlocking));
  s = h.stream;

  // colouring and colour-major element order (stable in element index)
  h.n_colours = colour_elements(nn, ne, mesh->tets, h.colour_host);
  h.colour_ptr.assign(h.n_colours + 1, 0);
  for (int e = 0; e < ne; ++e) h.colour_ptr[h.colour_host[e] + 1]++;
  for (int c = 0; c < h.n_colours; ++c) h.colour_ptr[c + 1] += h.colour_ptr[c];
  h.elem_perm_host.resize(ne);
  {
    std::vector<int32_t> fill(h.colour_ptr.begin(), h.colour_ptr.end() - 1);
    for (int e = 0; e < ne; ++e) h.elem_perm_host[fill[h.colour_host[e]]++] = e;
  }
  // level-0 pattern and element -> block map
  h.levels.resize(1);
  Level& L0 = h.levels[0];
  element_pattern(nn, ne, mesh->tets, L0.hpat);
  std::vector<int32_t> conn(4 * (size_t)ne), slot(16 * (size_t)ne), matp(ne);
  std::vector<double> fib(6 * (size_t)ne, 0.0);
  for (int k = 0; k < ne; ++k) {
    const int e = h.elem_perm_host[k];
    for (int a = 0; a < 4; ++a) conn[4 * k + a] = mesh->tets[4 * e + a];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) slot[16 * k + 4 * a + b] = find_block(L0.hpat, conn[4 * k + a], conn[4 * k + b]);
    matp[k] = mesh->mat_id[e];
    if (mesh->fibre)
      for (int q = 0; q < 6; ++q) fib[6 * k + q] = mesh->fibre[6 * (size_t)e + q];
  }
  std::vector<double> mt(8 * (size_t)n_mat);
  for (int m = 0; m < n_mat; ++m) {
    const fsi_material& M = mats[m];
    double mul = M.model == FSI_MODEL_ARTERY ? 2.0 * (M.c10 + M.k1 / (2.0 * M.k2)) : 2.0 * (M.c10 + M.c01);
    double row[8] = {(double)M.model, M.c10, M.c01, M.k1, M.k2, M.kappa, M.rho, mul};
    for (int q = 0; q < 8; ++q) mt[8 * m + q] = row[q];
  }
  std::vector<uint8_t> dmask(4 * (size_t)nn, 0);
  if (mesh->dir_mask)
    for (size_t k = 0; k < dmask.size(); ++k) dmask[k] = mesh->dir_mask[k] ? 1 : 0;
  std::vector<uint8_t> free0(dmask.size());
  for (size_t k = 0; k < dmask.size(); ++k) free0[k] = dmask[k] ? 0 : 1;
  // node -> face incidence for the deterministic load gather
  std::vector<int32_t> nfp(nn + 1, 0), nfi(3 * (size_t)std::max(mesh->n_faces, 0));
  for (int f = 0; f < mesh->n_faces; ++f)
    for (int a = 0; a < 3; ++a) nfp[mesh->neu_faces[3 * f + a] + 1]++;
  for (int i = 0; i < nn; ++i) nfp[i + 1] += nfp[i];
  {
    std::vector<int32_t> fill(nfp.begin(), nfp.end() - 1);
    for (int f = 0; f < mesh->n_faces; ++f)
      for (int a = 0; a < 3; ++a) nfi[fill[mesh->neu_faces[3 * f + a]]++] = 3 * f + a;
  }
  std::vector<int32_t> comp(nn, 0);
  if (mesh->seg_node)
    for (int i = 0; i < nn; ++i) comp[i] = mesh->seg_node[i];
  h.n_seg = nn ? comp[nn - 1] + 1 : 1;
  h.seg_ptr_host.assign(h.n_seg + 1, 0);
  for (int i = 0; i < nn; ++i) h.seg_ptr_host[comp[i] + 1]++;
  for (int q = 0; q < h.n_seg; ++q) h.seg_ptr_host[q + 1] += h.seg_ptr_host[q];

  h.d_conn = upload(conn, s);
  h.d_slot = upload(slot, s);
  h.d_mat = upload(matp, s);
  h.d_fibre = upload(fib, s);
  h.d_mats = upload(mt, s);
  h.d_X = upload(mesh->X, 3 * (size_t)nn, s);
  h.d_dir_mask = upload(dmask, s);
  h.d_faces = upload(mesh->neu_faces ? mesh->neu_faces : (const int32_t*)nullptr,
                     mesh->neu_faces ? 3 * (size_t)mesh->n_faces : 0, s);
  h.d_nf_ptr = upload(nfp, s);
  h.d_nf_idx = upload(nfi, s);
  h.d_seg_node = upload(comp, s);
  h.d_seg_ptr = upload(h.seg_ptr_host, s);
  h.d_seg_a = dalloc<double>(h.n_seg);
  h.d_seg_b = dalloc<double>(h.n_seg);
  FSI_CUDA_TRY(cudaMallocHost((void**)&h.h_seg, sizeof(double) * h.n_seg));
  h.d_err = dalloc<int>(1);
  FSI_CUDA_TRY(cudaMemsetAsync(h.d_err, 0, sizeof(int), s));
  h.d_geo = dalloc<double>(16 * (size_t)ne);
  launch_geometry(h, s);
  if (check_err(h, s) & 1) throw ArgError("an element has non-positive reference volume");

  // gather plans (deterministic assembly without colours): contributions of
  // each block / node in element order
  {
    std::vector<int32_t> bptr(L0.hpat.col_idx.size() + 1, 0), bsrc(16 * (size_t)ne);
    for (size_t q = 0; q < slot.size(); ++q) bptr[slot[q] + 1]++;
    for (size_t b = 0; b + 1 < bptr.size(); ++b) bptr[b + 1] += bptr[b];
    std::vector<int32_t> fill(bptr.begin(), bptr.end() - 1);
    for (size_t q = 0; q < slot.size(); ++q) bsrc[fill[slot[q]]++] = (int32_t)q;
    std::vector<int32_t> nptr(nn + 1, 0), nsrc(4 * (size_t)ne);
    for (size_t q = 0; q < conn.size(); ++q) nptr[conn[q] + 1]++;
    for (int i = 0; i < nn; ++i) nptr[i + 1] += nptr[i];
    std::vector<int32_t> fn(nptr.begin(), nptr.end() - 1);
    for (size_t q = 0; q < conn.size(); ++q) nsrc[fn[conn[q]]++] = (int32_t)q;
    h.d_gb_ptr = upload(bptr, s);
    h.d_gb_src = upload(bsrc, s);
    h.d_gn_ptr = upload(nptr, s);
    h.d_gn_src = upload(nsrc, s);
    h.d_ebuf = dalloc<char>((size_t)ne * 256 * 8);   // FP64 size: the reference tangent is FP64
    h.d_rbuf = dalloc<double>((size_t)ne * 16);
    FSI_CUDA_TRY(cudaStreamSynchronize(s));
  }
  upload_pattern(L0, s);
  L0.bs = 4;
  L0.cmask = h.d_dir_mask;
  L0.vals = dalloc<char>((f32 ? 4 : 8) * 16 * (size_t)L0.nb);
  h.k_vals = L0.vals;
  if (h.opts.precond == FSI_PRECOND_BLOCK_LT) {
    h.k_vals = dalloc<char>((f32 ? 4 : 8) * 16 * (size_t)L0.nb);
    // S~ = (1/theta + 1/kappa) diag(M_p), M_aa = V/10 per incident tetrahedron
    const double theta = h.opts.schur_theta > 0.0 ? h.opts.schur_theta : mats[0].c10;
    if (!(theta > 0.0)) throw ArgError("schur_theta must be positive (or c10 of material 0)");
    std::vector<double> sd(nn, 0.0);
    for (int e = 0; e < ne; ++e) {
      const int32_t* t = mesh->tets + 4 * (size_t)e;
      const double* x0 = mesh->X + 3 * (size_t)t[0];
      double d[3][3];
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) d[a][c] = mesh->X[3 * (size_t)t[a + 1] + c] - x0[c];
      const double vol = std::fabs(d[0][0] * (d[1][1] * d[2][2] - d[1][2] * d[2][1]) -
                                   d[0][1] * (d[1][0] * d[2][2] - d[1][2] * d[2][0]) +
                                   d[0][2] * (d[1][0] * d[2][1] - d[1][1] * d[2][0])) / 6.0;
      const double w = (1.0 / theta + 1.0 / mats[mesh->mat_id[e]].kappa) * vol / 10.0;
      for (int a = 0; a < 4; ++a) sd[t[a]] += w;
    }
    std::vector<double> sinv(nn);
    for (int i = 0; i < nn; ++i) sinv[i] = dmask[4 * (size_t)i + 3] ? -1.0 : (sd[i] > 0.0 ? 1.0 / sd[i] : 0.0);
    h.d_sinv = upload(sinv, s);
    h.d_pl_y = dalloc<double>(4 * (size_t)nn);
    FSI_CUDA_TRY(cudaStreamSynchronize(s));
  }
  L0.dinv = dalloc<char>((f32 ? 4 : 8) * 16 * (size_t)L0.n);
  alloc_level_vectors(L0, f32);
  if (h.opts.smoother == FSI_SMOOTHER_VANKA) {
    std::vector<int32_t> order;
    int max_deg = 0;
    vanka_colouring(L0.hpat, nn, order, h.vk_cptr, &max_deg);
    h.vk_ncol = (int)h.vk_cptr.size() - 1;
    h.vk_m = 3 * max_deg + 1;
    if (h.vk_m > kVankaMaxM) throw ArgError("a Vanka patch would exceed 64 unknowns (node with > 20 neighbours)");
    h.d_vk_order = upload(order, s);
    const size_t ts = f32 ? 4 : 8;
    h.d_vk_inv = dalloc<char>(ts * (size_t)nn * h.vk_m * h.vk_m);
    h.d_vk_z = dalloc<char>(ts * (size_t)nn * h.vk_m);
    FSI_CUDA_TRY(cudaStreamSynchronize(s));
  }
  build_hierarchy(h, free0, comp, mesh->X, s);

  const size_t ndof = 4 * (size_t)nn;
  h.d_V = dalloc<double>((size_t)(h.m + 1) * ndof);
  h.d_Z = dalloc<double>((size_t)h.m * ndof);
  h.d_w = dalloc<double>(ndof);
  h.d_r = dalloc<double>(ndof);
  h.d_t = dalloc<double>(ndof);
  h.d_t2 = dalloc<double>(ndof);
  h.d_t3 = dalloc<double>(ndof);
  h.d_res = dalloc<double>(ndof);
  h.d_xdf = dalloc<float2>(ndof);
  h.d_state_tmp = dalloc<double>(ndof);
  h.d_fext = dalloc<double>(3 * (size_t)nn);
  FSI_CUDA_TRY(cudaMemsetAsync(h.d_fext, 0, sizeof(double) * 3 * nn, s));
  if (mesh->n_faces > 0) {
    // coupling interface: vertices of the loaded faces, with the unit direction
    // of the P1 load of a unit pressure (-sum over faces of the doubled area normal)
    std::vector<double> f(3 * (size_t)nn, 0.0);
    std::vector<uint8_t> on(nn, 0);
    for (int q = 0; q < mesh->n_faces; ++q) {
      const int32_t* v = mesh->neu_faces + 3 * (size_t)q;
      double e1[3], e2[3];
      for (int c = 0; c < 3; ++c) {
        e1[c] = mesh->X[3 * (size_t)v[1] + c] - mesh->X[3 * (size_t)v[0] + c];
        e2[c] = mesh->X[3 * (size_t)v[2] + c] - mesh->X[3 * (size_t)v[0] + c];
      }
      const double nv[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                            e1[0] * e2[1] - e1[1] * e2[0]};
      for (int a = 0; a < 3; ++a) {
        on[v[a]] = 1;
        for (int c = 0; c < 3; ++c) f[3 * (size_t)v[a] + c] -= nv[c];
      }
    }
    std::vector<int32_t> gi;
    std::vector<double> gw;
    for (int i = 0; i < nn; ++i) {
      if (!on[i]) continue;
      const double* fi = &f[3 * (size_t)i];
      const double len = std::sqrt(fi[0] * fi[0] + fi[1] * fi[1] + fi[2] * fi[2]);
      gi.push_back(i);
      for (int c = 0; c < 3; ++c) gw.push_back(len > 0.0 ? fi[c] / len : 0.0);
    }
    h.n_gam = (int)gi.size();
    h.d_gam_idx = upload(gi, s);
    h.d_gam_w = upload(gw, s);
    h.d_dn = dalloc<double>(15 * (size_t)h.n_gam);
    h.d_dn_p = dalloc<double>(nn);
    FSI_CUDA_TRY(cudaStreamSynchronize(s));
  }
  if (h.n_seg > 1) {
    const size_t ns = (size_t)h.n_seg, mm = (size_t)h.m;
    h.d_sdots = dalloc<double>(2 * (mm + 2) * ns);
    h.d_scoef = dalloc<double>((mm + 1) * ns);
    FSI_CUDA_TRY(cudaMallocHost((void**)&h.h_sdots, sizeof(double) * 2 * (mm + 2) * ns));
    FSI_CUDA_TRY(cudaMallocHost((void**)&h.h_scoef, sizeof(double) * (mm + 1) * ns));
  }
  h.red_blocks = 2 * 152;
  h.d_partial = dalloc<double>((size_t)h.red_blocks * (kMaxRestart + 1));
  h.d_dots = dalloc<double>(kDotSize);
  FSI_CUDA_TRY(cudaMallocHost((void**)&h.h_dots, sizeof(double) * kDotSize));
  FSI_CUDA_TRY(cudaStreamSynchronize(s));
  if (h.opts.autotune) {
    autotune_elements(h, s);
    autotune_levels(h, s);
    if (check_err(h, s)) throw ArgError("reference configuration failed in the autotuning pass");
  }
  guard.p = nullptr;
  return hp;
}

static void destroy_impl(Handle* hp) {
  if (!hp) return;
  Handle& h = *hp;
  if (h.stream) cudaStreamSynchronize(h.stream);
  for (size_t l = 0; l < h.levels.size(); ++l) {
    Level& L = h.levels[l];
    dfree(L.vals_lp);
    for (void* p : {(void*)L.row_ptr, (void*)L.col_idx, (void*)L.diag_idx, (void*)L.block_row, L.vals, L.dinv,
                    (void*)L.p_rp, (void*)L.p_ci, L.p_v, (void*)L.pt_rp, (void*)L.pt_ci, L.pt_v, L.x, L.x2, L.b,
                    L.r, (void*)L.agg, L.ptent, (void*)L.freem, (void*)L.p_brow, (void*)L.w_ptr, (void*)L.w_k,
                    L.w_v, L.dinv_f, (void*)L.pt_src, (void*)L.ap_ptr, (void*)L.ap_pairs, L.ap_v, (void*)L.ac_ptr,
                    (void*)L.ac_pairs, (void*)L.fix_blk, (void*)L.fix_dof, L.w, (void*)L.mr})
      dfree(p);
  }
  if (h.k_vals && !h.levels.empty() && h.k_vals != h.levels[0].vals) dfree(h.k_vals);
  dfree(h.d_sinv);
  dfree(h.d_pl_y);
  dfree(h.d_gam_idx);
  dfree(h.d_gam_w);
  dfree(h.d_dn);
  dfree(h.d_dn_p);
  dfree(h.d_vk_order);
  dfree(h.d_vk_inv);
  dfree(h.d_vk_z);
  for (void* p : {(void*)h.coarse.comp_ptr, (void*)h.coarse.inv_off, h.coarse.inv, (void*)h.coarse.work,
                  (void*)h.d_conn, (void*)h.d_geo, (void*)h.d_fibre, (void*)h.d_mat, (void*)h.d_slot,
                  (void*)h.d_mats, (void*)h.d_X, (void*)h.d_dir_mask, (void*)h.d_faces, (void*)h.d_nf_ptr,
                  (void*)h.d_nf_idx, (void*)h.d_seg_node, h.d_ebuf, (void*)h.d_rbuf, (void*)h.d_gb_ptr,
                  (void*)h.d_gb_src, (void*)h.d_gn_ptr, (void*)h.d_gn_src, (void*)h.d_err, (void*)h.d_V, (void*)h.d_Z,
                  (void*)h.d_w, (void*)h.d_r, (void*)h.d_t, (void*)h.d_t2, (void*)h.d_t3, (void*)h.d_partial,
                  (void*)h.d_dots, (void*)h.d_xdf, (void*)h.d_xs, (void*)h.d_ys, (void*)h.d_fext, (void*)h.d_state_tmp,
                  (void*)h.d_res})
    dfree(p);
  if (h.vc_exec) cudaGraphExecDestroy(h.vc_exec);
  if (h.h_dots) cudaFreeHost(h.h_dots);
  if (h.h_sdots) cudaFreeHost(h.h_sdots);
  if (h.h_scoef) cudaFreeHost(h.h_scoef);
  dfree(h.d_sdots);
  dfree(h.d_scoef);
  if (h.h_seg) cudaFreeHost(h.h_seg);
  dfree(h.d_seg_ptr);
  dfree(h.d_seg_a);
  dfree(h.d_seg_b);
  for (cudaEvent_t e : h.prof.pool) cudaEventDestroy(e);
  if (h.stream) cudaStreamDestroy(h.stream);
  delete hp;
}

// ------------------------------------------------------------------ Newton
static int assemble_checked(Handle& h, const double* state, const double* hist, double* res, bool tangent,
                            cudaStream_t s) {
  launch_assemble(h, state, hist, res, tangent, s);
  int e = check_err(h, s);
  if (e & 1) return FSI_ERR_INVERTED;
  return FSI_OK;
}

static int newton_iterate(Handle& h, double* state, const fsi_load* load, double rn, double eps1, fsi_info* info,
                          cudaStream_t s) {
  const long n = 4L * h.n_nodes;
  const double* hist = load ? load->hist : nullptr;
  int st = assemble_checked(h, state, hist, nullptr, true, s);
  if (st) return st;
  amg_numeric(h, s);
  int e = check_err(h, s);
  if (e & 8) throw CudaError("singular coarsest-level operator");
  scale_copy(-1.0, h.d_res, h.d_t, n, s);
  FSI_CUDA_TRY(cudaMemsetAsync(h.d_t2, 0, sizeof(double) * n, s));
  // independent segments: solve with every segment's right-hand side scaled to
  // unit norm (exact, the system is block diagonal), so that each segment is
  // reduced by eps1 relative to its own residual
  const bool segs = h.n_seg > 1;
  if (segs) {
    segment_sumsq(h.d_seg_ptr, h.n_seg, h.d_t, h.d_seg_a, s);
    segment_normalise(h.n_seg, h.d_seg_a, h.d_seg_b, s);
    segment_scale(h.d_seg_node, h.d_seg_a, h.d_t, n, s);
  }
  double rel = 0.0;
  int its = linear_solve(h, h.d_t, h.d_t2, eps1, &rel, s);
  if (segs) segment_scale(h.d_seg_node, h.d_seg_b, h.d_t2, n, s);
  axpy(1.0, h.d_t2, state, n, s);
  if (info) {
    info->krylov_its_total += its;
    info->krylov_its_last = its;
    info->lin_res = rel;
    info->inc_norm = norm2_host(h, h.d_t2, n, s);
    info->inc_mnorm = mass_norm_host(h, h.d_t2, s);
  }
  (void)rn;
  if (rel > h.opts.krylov_rtol * 1e3 && its >= h.opts.max_krylov) return FSI_ERR_NOT_CONVERGED;
  return FSI_OK;
}

// per-segment residual norms (host copy)
static void segment_norms(Handle& h, const double* x, std::vector<double>& out, cudaStream_t s) {
  segment_sumsq(h.d_seg_ptr, h.n_seg, x, h.d_seg_a, s);
  FSI_CUDA_TRY(cudaMemcpyAsync(h.h_seg, h.d_seg_a, sizeof(double) * h.n_seg, cudaMemcpyDeviceToHost, s));
  FSI_CUDA_TRY(cudaStreamSynchronize(s));
  out.resize(h.n_seg);
  for (int q = 0; q < h.n_seg; ++q) out[q] = std::sqrt(h.h_seg[q]);
}

// Newton's method for one load (time) step.  The stop is relative to the
// initial residual norm, or to r_ref when r_ref > 0 (single-segment meshes).
static int solve_impl(Handle& h, double* state, const fsi_load* load, const double* guess, fsi_info* info,
                      cudaStream_t s, double r_ref = 0.0) {
  const long n = 4L * h.n_nodes;
  fsi_info loc{};
  if (!info) info = &loc;
  *info = fsi_info{};
  info->n_levels = (int)h.levels.size();
  if (load && load->dir_values) launch_set_dirichlet_values(h, state, load->dir_values, s);
  launch_external_force(h, load, s);
  const double* hist = load ? load->hist : nullptr;
  int st = assemble_checked(h, state, hist, h.d_res, false, s);
  if (st) return st;
  const double r0 = norm2_host(h, h.d_res, n, s);
  double rn = r0;
  info->res0 = r0;
  if (!std::isfinite(r0)) return FSI_ERR_INVERTED;   // a non-finite state or load
  if (guess) {
    FSI_CUDA_TRY(cudaMemcpyAsync(h.d_state_tmp, state, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    FSI_CUDA_TRY(cudaMemcpyAsync(h.d_t3, guess, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    mask_vector(h.d_dir_mask, h.d_t3, n, s);
    axpy(1.0, h.d_t3, h.d_state_tmp, n, s);
    int st2 = assemble_checked(h, h.d_state_tmp, hist, h.d_t, false, s);
    double rg = st2 ? INFINITY : norm2_host(h, h.d_t, n, s);
    if (rg <= r0) {   // false for a non-finite guess: the zero increment is kept
      FSI_CUDA_TRY(cudaMemcpyAsync(state, h.d_state_tmp, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      FSI_CUDA_TRY(cudaMemcpyAsync(h.d_res, h.d_t, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      rn = rg;
      info->guess_accepted = 1;
    }
  }
  double eps_prev = 1.0;
  std::vector<double> seg0, segk;
  if (h.n_seg > 1) segment_norms(h, h.d_res, seg0, s);
  auto converged = [&]() {
    if (h.n_seg == 1) {
      const double ref = r_ref > 0.0 ? r_ref : r0;
      return ref == 0.0 || rn <= h.opts.newton_rtol * ref;
    }
    segment_norms(h, h.d_res, segk, s);
    for (int q = 0; q < h.n_seg; ++q)
      if (segk[q] > h.opts.newton_rtol * seg0[q]) return false;
    return true;
  };
  int k = 0;
  for (;; ++k) {
    if (converged()) break;
    if (k >= h.opts.max_newton) {
      info->newton_its = k;
      info->res = rn;
      return FSI_ERR_NOT_CONVERGED;
    }
    double eps1 = h.opts.krylov_rtol;
    if (h.opts.adaptive_tol) eps1 = std::max(h.opts.krylov_rtol, std::min(0.1, eps_prev * eps_prev));
    st = newton_iterate(h, state, load, rn, eps1, info, s);
    if (st) {
      info->newton_its = k + 1;
      return st;
    }
    st = assemble_checked(h, state, hist, h.d_res, false, s);
    // safeguard (the paper's Newton has none): if the full step inverts an
    // element, halve it, up to six times; dv is still in d_t2
    for (int half = 1; st == FSI_ERR_INVERTED && half <= 6; ++half) {
      axpy(-std::ldexp(1.0, -half), h.d_t2, state, n, s);
      st = assemble_checked(h, state, hist, h.d_res, false, s);
    }
    if (st) {
      info->newton_its = k + 1;
      return st;
    }
    double rnew = norm2_host(h, h.d_res, n, s);
    if (!std::isfinite(rnew)) {
      info->newton_its = k + 1;
      return FSI_ERR_INVERTED;
    }
    eps_prev = rnew / std::max(rn, 1e-300);
    rn = rnew;
  }
  info->newton_its = k;
  info->res = rn;
  return FSI_OK;
}

// Dirichlet-Neumann iteration with Aitken relaxation (Sec. 5.1, 5.2).
static int dn_impl(Handle& h, double* state, const fsi_load* load, const fsi_dn_opts& o, fsi_dn_info* info,
                   cudaStream_t s) {
  const int ng = h.n_gam;
  const long m = 3L * ng;
  double* d = h.d_dn;
  double* dt = h.d_dn + m;
  double* r = h.d_dn + 2 * m;
  double* r_prev = h.d_dn + 3 * m;   // r_prev and dr adjacent: one dots() call gives both products
  double* dr = h.d_dn + 4 * m;
  fsi_load ld{};
  if (load) ld = *load;
  ld.pressure = 1.0;
  ld.node_pressure = h.d_dn_p;
  ld.face_pressure = nullptr;
  if (ld.dir_values) {
    launch_set_dirichlet_values(h, state, ld.dir_values, s);
    ld.dir_values = nullptr;
  }
  FSI_CUDA_TRY(cudaMemsetAsync(h.d_dn_p, 0, sizeof(double) * h.n_nodes, s));
  dn_restrict(ng, h.d_gam_idx, state, d, nullptr, nullptr, s);     // d_0
  double omega = o.omega0, r_ref = 0.0;
  bool have_prev = false;
  const double scale = 1.0 / std::sqrt((double)ng);
  for (int k = 1; k <= o.max_cycles; ++k) {
    dn_fluid(ng, h.d_gam_idx, h.d_gam_w, d, o.d_ref, o.p0, o.added_mass, h.d_dn_p, s);
    fsi_info ni{};
    int st = solve_impl(h, state, &ld, nullptr, &ni, s, r_ref);
    info->newton_its_total += ni.newton_its;
    info->krylov_its_total += ni.krylov_its_total;
    info->cycles = k;
    if (st) return st;
    if (k == 1) r_ref = ni.res0;
    dn_restrict(ng, h.d_gam_idx, state, dt, d, r, s);                 // d~_k, r_k
    const double res = norm2_host(h, r, m, s) * scale;
    if (k == 1) info->res_first = res;
    info->res_last = res;
    if (res < o.tol) {
      info->converged = 1;
      return FSI_OK;
    }
    if (o.aitken && have_prev) {
      dn_diff(m, r, r_prev, dr, s);
      dots(h, r_prev, m, 2, dr, m, h.d_dots + kDotNorm + 1, s);    // r_prev . dr, dr . dr
      double pr[2];
      FSI_CUDA_TRY(cudaMemcpyAsync(pr, h.d_dots + kDotNorm + 1, sizeof(pr), cudaMemcpyDeviceToHost, s));
      FSI_CUDA_TRY(cudaStreamSynchronize(s));
      if (pr[1] > 0.0) omega = -omega * pr[0] / pr[1];
    }
    info->omega_last = omega;
    dn_relax(m, omega, dt, d, s);
    FSI_CUDA_TRY(cudaMemcpyAsync(r_prev, r, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    have_prev = true;
  }
  return FSI_ERR_NOT_CONVERGED;
}

}  // namespace fsi

// ------------------------------------------------------------------ C ABI
using fsi::Handle;

struct fsi_solid_s {
  Handle h;
};

#define FSI_GUARD_BEGIN try {
#define FSI_GUARD_END(hptr)                                  \
  }                                                          \
  catch (const fsi::ArgError& e) {                           \
    fsi::set_error(hptr, e.msg);                             \
    return FSI_ERR_ARG;                                      \
  }                                                          \
  catch (const fsi::CudaError& e) {                          \
    fsi::set_error(hptr, e.msg);                             \
    return FSI_ERR_CUDA;                                     \
  }                                                          \
  catch (const fsi::OomError& e) {                           \
    fsi::set_error(hptr, e.msg);                             \
    return FSI_ERR_OOM;                                      \
  }                                                          \
  catch (const std::bad_alloc&) {                            \
    fsi::set_error(hptr, "host allocation failed");          \
    return FSI_ERR_OOM;                                      \
  }                                                          \
  catch (const std::exception& e) {                          \
    fsi::set_error(hptr, e.what());                          \
    return FSI_ERR_ARG;                                      \
  }

static inline Handle* H(fsi_solid_t h) { return reinterpret_cast<Handle*>(h); }
#define FSI_PROF(h) fsi::ProfScope fsi_prof_scope_(&(h)->prof)
static inline cudaStream_t S(Handle* h, void* stream) { return stream ? (cudaStream_t)stream : h->stream; }

static thread_local std::string g_create_error;

extern "C" {

void fsi_solid_default_opts(fsi_solver_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = FSI_PREC_FP64;
  o->krylov = FSI_KRYLOV_FGMRES;
  o->restart = 100;
  o->max_krylov = 300;
  o->max_newton = 25;
  o->smoother = FSI_SMOOTHER_JACOBI;
  o->nu_pre = 4;
  o->nu_post = 4;
  o->nu_coarse = 2;
  o->coarse_smoother = FSI_COARSE_MR;
  o->autotune = 1;
  o->segment_krylov = 1;
  o->exact_candidates = 0;
  o->power_steps = 20;
  o->coarse_max_nodes = 16;
  o->max_levels = 12;
  o->use_pspg = 1;
  o->adaptive_tol = 0;
  o->use_graphs = 1;
  o->amg_lag = 0;
  o->omega = 0.7;
  o->newton_rtol = 1e-8;
  o->krylov_rtol = 1e-8;
  o->fibre_factor = 2.0;
  o->inertia_coef = 0.0;
  o->assembly = 0;
  o->precond = FSI_PRECOND_AMG;
  o->schur_theta = 0.0;
  o->vanka_omega = 0.86;
}

fsi_status fsi_solid_create(const fsi_mesh_desc* mesh, int32_t n_mat, const fsi_material* mats,
                            const fsi_solver_opts* opts, fsi_solid_t* out) {
  if (!out) return FSI_ERR_ARG;
  *out = nullptr;
  Handle* hp = nullptr;
  try {
    hp = fsi::create_impl(mesh, n_mat, mats, opts);
    *out = reinterpret_cast<fsi_solid_t>(hp);
    return FSI_OK;
  } catch (const fsi::ArgError& e) {
    g_create_error = e.msg;
    return FSI_ERR_ARG;
  } catch (const fsi::CudaError& e) {
    g_create_error = e.msg;
    return FSI_ERR_CUDA;
  } catch (const fsi::OomError& e) {
    g_create_error = e.msg;
    return FSI_ERR_OOM;
  } catch (const std::bad_alloc&) {
    g_create_error = "host allocation failed";
    return FSI_ERR_OOM;
  } catch (const std::exception& e) {
    g_create_error = e.what();
    return FSI_ERR_ARG;
  }
}

fsi_status fsi_solid_destroy(fsi_solid_t h) {
  fsi::destroy_impl(H(h));
  return FSI_OK;
}

fsi_status fsi_solid_residual_tangent(fsi_solid_t hh, const double* state, const fsi_load* load, double* residual,
                                      int32_t want_tangent, void* stream) {
  Handle* h = H(hh);
  if (!h || !state) return FSI_ERR_ARG;
  FSI_GUARD_BEGIN
  FSI_PROF(h);
  cudaStream_t s = S(h, stream);
  fsi::launch_external_force(*h, load, s);
  int st = fsi::assemble_checked(*h, state, load ? load->hist : nullptr, residual, want_tangent != 0, s);
  if (st) {
    fsi::set_error(h, "inverted or non-finite element");
    return (fsi_status)st;
  }
  return FSI_OK;
  FSI_GUARD_END(h)
}

fsi_status fsi_solid_get_bsr(fsi_solid_t hh, const int32_t** row_ptr, const int32_t** col_idx, const void** vals,
                             int32_t* dtype, int32_t* n_blocks) {
  Handle* h = H(hh);
  if (!h) return FSI_ERR_ARG;
  const fsi::Level& L = h->levels[0];
  if (row_ptr) *row_ptr = L.row_ptr;
  if (col_idx) *col_idx = L.col_idx;
  if (vals) *vals = h->k_vals;
  if (dtype) *dtype = h->precision == FSI_PREC_FP32_IR ? 1 : 0;
  if (n_blocks) *n_blocks = L.nb;
  return FSI_OK;
}

fsi_status fsi_solid_spmv(fsi_solid_t hh, const double* x, double* y, void* stream) {
  Handle* h = H(hh);
  if (!h || !x || !y) return FSI_ERR_ARG;
  FSI_GUARD_BEGIN
  FSI_PROF(h);
  cudaStream_t s = S(h, stream);
  fsi::apply_operator(*h, x, y, s);
  FSI_CUDA_TRY(cudaStreamSynchronize(s));
  return FSI_OK;
  FSI_GUARD_END(h)
}

fsi_status fsi_solid_linear_solve(fsi_solid_t hh, const double* b, double* x, fsi_info* info, void* stream) {
  Handle* h = H(hh);
  if (!h || !b || !x) return FSI_ERR_ARG;
  FSI_GUARD_BEGIN
  FSI_PROF(h);
  cudaStream_t s = S(h, stream);
  fsi::amg_numeric(*h, s);
  if (fsi::check_err(*h, s) & 8) throw fsi::CudaError("singular coarsest-level operator");
  double rel = 0.0;
  int its = fsi::linear_solve(*h, b, x, h->opts.krylov_rtol, &rel, s);
  FSI_CUDA_TRY(cudaStreamSynchronize(s));
  if (info) {
    *info = fsi_info{};
    info->krylov_its_total = its;
    info->krylov_its_last = its;
    info->lin_res = rel;
    info->n_levels = (int)h->levels.size();
  }
  if (rel > h->opts.krylov_rtol) {
    fsi::set_error(h, "Krylov iteration cap reached");
    if (info) info->status = FSI_ERR_NOT_CONVERGED;
    return FSI_ERR_NOT_CONVERGED;
  }
  return FSI_OK;
  FSI_GUARD_END(h)
}

fsi_status fsi_solid_newton_step(fsi_solid_t hh, double* state, const fsi_load* load, fsi_info* info, void* stream) {
  Handle* h = H(hh);
  if (!h || !state) return FSI_ERR_ARG;
  FSI_GUARD_BEGIN
  FSI_PROF(h);
  cudaStream_t s = S(h, stream);
  fsi_info loc{};
  if (!info) info = &loc;
  *info = fsi_info{};
  info->n_levels = (int)h->levels.size();
  const long n = 4L * h->n_nodes;
  fsi::launch_external_force(*h, load, s);
  int st = fsi::assemble_checked(*h, state, load ? load->hist : nullptr, h->d_res, false, s);
  if (st) return (fsi_status)st;
  info->res0 = fsi::norm2_host(*h, h->d_res, n, s);
  if (!std::isfinite(info->res0)) {
    fsi::set_error(h, "non-finite residual");
    info->status = FSI_ERR_INVERTED;
    return FSI_ERR_INVERTED;
  }
  st = fsi::newton_iterate(*h, state, load, info->res0, h->opts.krylov_rtol, info, s);
  info->newton_its = 1;
  info->status = st;
  FSI_CUDA_TRY(cudaStreamSynchronize(s));
  return (fsi_status)st;
  FSI_GUARD_END(h)
}

fsi_status fsi_solid_solve(fsi_solid_t hh, double* state, const fsi_load* load, const double* guess, fsi_info* info,
                           void* stream) {
  Handle* h = H(hh);
  if (!h || !state) return FSI_ERR_ARG;
  FSI_GUARD_BEGIN
  FSI_PROF(h);
  cudaStream_t s = S(h, stream);
  int st = fsi::solve_impl(*h, state, load, guess, info, s);
  FSI_CUDA_TRY(cudaStreamSynchronize(s));
  if (info) info->status = st;
  if (st) fsi::set_error(h, st == FSI_ERR_INVERTED ? "inverted or non-finite element" : "Newton did not converge");
  return (fsi_status)st;
  FSI_GUARD_END(h)
}

void fsi_dn_default_opts(fsi_dn_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->omega0 = 0.5;
  o->tol = 1e-8;
  o->max_cycles = 50;
  o->aitken = 1;
}

fsi_status fsi_solid_dn_solve(fsi_solid_t hh, double* state, const fsi_load* load, const fsi_dn_opts* o,
                              fsi_dn_info* info, void* stream) {
  Handle* h = H(hh);
  if (!h || !state || !o) return FSI_ERR_ARG;
  FSI_GUARD_BEGIN
  FSI_PROF(h);
  fsi_dn_info loc{};
  if (!info) info = &loc;
  *info = fsi_dn_info{};
  info->n_interface = h->n_gam;
  if (h->n_gam == 0) throw fsi::ArgError("no loaded faces: the coupling interface is empty");
  if (!(o->omega0 > 0.0 && o->omega0 <= 1.0)) throw fsi::ArgError("omega0 must lie in (0, 1]");
  if (!(o->added_mass >= 0.0)) throw fsi::ArgError("added_mass must be >= 0");
  if (o->max_cycles < 1) throw fsi::ArgError("max_cycles must be >= 1");
  cudaStream_t s = S(h, stream);
  int st = fsi::dn_impl(*h, state, load, *o, info, s);
  FSI_CUDA_TRY(cudaStreamSynchronize(s));
  if (st) fsi::set_error(h, st == FSI_ERR_INVERTED ? "inverted or non-finite element"
                                                     : "DN iteration or Newton did not converge");
  return (fsi_status)st;
  FSI_GUARD_END(h)
}

fsi_status fsi_solid_newmark_advance(fsi_solid_t hh, const double* state, double* disp, double* vel, double* acc,
                                     double* hist, double beta, double gamma, double dt, void* stream) {
  Handle* h = H(hh);
  if (!h || !state || !disp || !vel || !acc || !hist || !(beta > 0) || !(dt > 0)) return FSI_ERR_ARG;
  FSI_GUARD_BEGIN
  FSI_PROF(h);
  cudaStream_t s = S(h, stream);
  fsi::launch_newmark(*h, state, disp, vel, acc, hist, beta, gamma, dt, s);
  FSI_CUDA_TRY(cudaStreamSynchronize(s));
  return FSI_OK;
  FSI_GUARD_END(h)
}

fsi_status fsi_solid_get_colouring(fsi_solid_t hh, int32_t* colour_out, int32_t* n_colours) {
  Handle* h = H(hh);
  if (!h) return FSI_ERR_ARG;
  if (colour_out) std::memcpy(colour_out, h->colour_host.data(), sizeof(int32_t) * h->n_elems);
  if (n_colours) *n_colours = h->n_colours;
  return FSI_OK;
}

fsi_status fsi_solid_get_tuning(fsi_solid_t hh, int32_t* out, int32_t capacity, int32_t* n_out) {
  Handle* h = H(hh);
  if (!h || (capacity > 0 && !out)) return FSI_ERR_ARG;
  std::vector<int32_t> v;
  v.push_back(h->elem_threads);
  for (size_t l = 0; l + 1 < h->levels.size(); ++l) v.push_back(h->levels[l].shape);
  if (n_out) *n_out = (int32_t)v.size();
  for (int q = 0; q < capacity && q < (int)v.size(); ++q) out[q] = v[q];
  return FSI_OK;
}

fsi_status fsi_solid_get_levels(fsi_solid_t hh, int32_t* nodes_out, int32_t* blocks_out, int32_t capacity,
                                int32_t* n_levels) {
  Handle* h = H(hh);
  if (!h) return FSI_ERR_ARG;
  int nl = (int)h->levels.size();
  if (n_levels) *n_levels = nl;
  for (int l = 0; l < nl && l < capacity; ++l) {
    if (nodes_out) nodes_out[l] = h->levels[l].n;
    if (blocks_out) blocks_out[l] = h->levels[l].nb;
  }
  return FSI_OK;
}

int64_t fsi_solid_launch_count(void) { return (int64_t)fsi::g_launches.load(std::memory_order_relaxed); }

fsi_status fsi_solid_kernel_timing(fsi_solid_t hh, int32_t enable, double* ms_out, int64_t* launches_out) {
  Handle* h = H(hh);
  if (!h) return FSI_ERR_ARG;
  fsi::Profiler& p = h->prof;
  for (int c = 0; c < FSI_KC_COUNT; ++c) {
    if (ms_out) ms_out[c] = 0.0;
    if (launches_out) launches_out[c] = 0;
  }
  for (size_t q = 0; q < p.used; ++q) {
    float ms = 0.0f;
    if (cudaEventSynchronize(p.pool[2 * q + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&ms, p.pool[2 * q], p.pool[2 * q + 1]) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    const int c = p.cls[q];
    if (ms_out) ms_out[c] += ms;
    if (launches_out) launches_out[c] += 1;
  }
  p.used = 0;
  p.on = enable != 0;
  return FSI_OK;
}

const char* fsi_solid_last_error(fsi_solid_t hh) {
  Handle* h = H(hh);
  if (!h) return g_create_error.c_str();
  return h->last_error.c_str();
}

}  // extern "C"
