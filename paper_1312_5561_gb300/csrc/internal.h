// Internal declarations shared by the translation units of libfsi_solid.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "fsi_solid.h"

// ------------------------------------------------------------------ launch accounting
// Every kernel launch of the library goes through FSI_LAUNCH, which counts it
// and, while a handle's kernel timing is switched on, brackets it with a pair
// of CUDA events recorded on the launching stream.
namespace fsi {
enum KernelClass {
  KC_TANGENT = 0,     // element residual + tangent + colour-ordered scatter
  KC_RESIDUAL,        // element residual only
  KC_JACOBI0,         // damped block-Jacobi sweep (x + w D^-1 (b - A x)) on the finest level
  KC_BSR0,            // other finest-level block-row kernels (SpMV, residual)
  KC_COARSE_BSR,      // block-row kernels on coarser levels (smoothing, residuals)
  KC_TRANSFER,        // restriction / prolongation
  KC_GALERKIN,        // numeric set-up: smoothed P, P^T, A P, P^T A P
  KC_BLOCKINV,        // block-diagonal inverses
  KC_COARSE,          // dense coarsest-level factorisation and solve
  KC_VECTOR,          // Krylov vector kernels and reductions
  KC_OTHER,
  KC_LEVEL1_SPMV,     // w = A z on level 1 inside the minimal-residual sweeps
  KC_COUNT
};
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<int> cls;      // class of pair p (events 2p, 2p+1)
  size_t used = 0;
};
extern thread_local Profiler* g_prof;
extern std::atomic<long long> g_launches;   // kernels launched by this process
void launch_begin(int cls, cudaStream_t s);
void launch_end(cudaStream_t s);
}  // namespace fsi

#define FSI_LAUNCH(cls, s, ...)      \
  do {                               \
    fsi::launch_begin((cls), (s));   \
    __VA_ARGS__;                     \
    fsi::launch_end((s));            \
  } while (0)


namespace fsi {

// ------------------------------------------------------------------ host setup
struct HostPattern {
  std::vector<int32_t> row_ptr;   // [n+1]
  std::vector<int32_t> col_idx;   // [nb], sorted within a row
};

// Greedy first-fit colouring of elements in element order: an element takes
// the smallest colour not used by an earlier element sharing a vertex.
int colour_elements(int n_nodes, int n_elems, const int32_t* tets, std::vector<int32_t>& colour);

// Node adjacency through shared elements (every node is its own neighbour).
void element_pattern(int n_nodes, int n_elems, const int32_t* tets, HostPattern& pat);

// Find block (i, j) in a pattern; -1 if absent.
int32_t find_block(const HostPattern& pat, int32_t i, int32_t j);

// ------------------------------------------------------------------ device level
// One level of the AMG hierarchy.  Level 0 holds the assembled tangent (4x4
// blocks); coarser levels hold Galerkin operators with 7x7 blocks.  P maps
// the next coarser level to this one (blocks bs x 7), PT is its transpose.
struct Level {
  int n = 0;                 // block rows
  int nb = 0;                // stored blocks
  int bs = 4;                // block size of this level
  int32_t* row_ptr = nullptr;
  int32_t* col_idx = nullptr;
  int32_t* diag_idx = nullptr;
  int32_t* block_row = nullptr;
  void* vals = nullptr;      // T [nb][bs*bs]
  void* dinv = nullptr;      // T [n][bs*bs] inverses of the diagonal blocks
  void* vals_lp = nullptr;   // BF16 copy of vals read by the V-cycle (coarse levels, FP32 mode, coarse_bf16)
  uint8_t* cmask = nullptr;  // level 0: [n][4] 1 = constrained component
  // prolongation from level+1 (rows: this level's nodes) and restriction (its transpose)
  int p_nb = 0, pt_nb = 0;
  int32_t* p_rp = nullptr;
  int32_t* p_ci = nullptr;
  void* p_v = nullptr;       // T [p_nb][bs*7]
  int32_t* pt_rp = nullptr;
  int32_t* pt_ci = nullptr;
  void* pt_v = nullptr;      // T [pt_nb][7*bs]
  // numeric set-up of the next level (fixed plans, values recomputed per Newton step)
  int32_t* agg = nullptr;        // [n] aggregate of each node
  void* ptent = nullptr;         // T [n][bs*7] tentative prolongator rows
  uint8_t* freem = nullptr;      // [n*bs] 1 = free unknown
  double omega_p = 0.0;
  void* dinv_f = nullptr;        // T [n][bs*bs] filtered block inverses (prolongator smoothing)
  int32_t* p_brow = nullptr;     // [p_nb] block row of each P block
  int32_t* w_ptr = nullptr;      // [p_nb+1]
  int32_t* w_k = nullptr;        // A blocks summed into each W = A P_t block
  void* w_v = nullptr;           // T [p_nb][bs*7]
  int32_t* pt_src = nullptr;     // [p_nb] P block transposed into PT block t
  int ap_nb = 0;
  int32_t* ap_ptr = nullptr;     // [ap_nb+1]
  int32_t* ap_pairs = nullptr;   // (A block, P block) pairs
  void* ap_v = nullptr;          // T [ap_nb][bs*7]
  int32_t* ac_ptr = nullptr;     // [nb of next level + 1]
  int32_t* ac_pairs = nullptr;   // (P block, AP block) pairs
  int n_fix = 0;
  int32_t* fix_blk = nullptr;    // identity rows of the next level
  int32_t* fix_dof = nullptr;
  // V-cycle vectors (T)
  void* x = nullptr;
  void* x2 = nullptr;
  void* b = nullptr;
  void* r = nullptr;
  void* w = nullptr;         // minimal-residual smoothing: A z (coarse levels)
  int shape = 0;             // launch shape of this level's block-row kernels (autotuner; 0 = default)
  int kc_spmv = 4;           // launch class of w = A z in the minimal-residual sweeps (KC_COARSE_BSR or KC_LEVEL1_SPMV)
  double* mr = nullptr;      // minimal-residual smoothing: 2 x kMrBlocks dot partials
  HostPattern hpat;          // level 0 pattern (host copy)
};

struct Coarse {              // block-diagonal dense inverse of the coarsest level
  int n_comp = 0;
  int max_dofs = 0;
  int32_t* comp_ptr = nullptr;   // [n_comp+1] node ranges (components are contiguous)
  int64_t* inv_off = nullptr;    // [n_comp] offsets into inv (in entries)
  void* inv = nullptr;           // T dense inverses, row-major per component
  double* work = nullptr;        // FP64 factorisation workspace (same layout as inv)
};

struct Handle {
  // sizes
  int n_nodes = 0, n_elems = 0, n_faces = 0, n_mat = 0, n_colours = 0, n_seg = 1;
  fsi_solver_opts opts{};
  std::string last_error;
  int precision = 0;   // 0 fp64, 1 fp32

  // element data, colour-major order
  std::vector<int32_t> colour_host;     // [n_elems] original order
  std::vector<int32_t> colour_ptr;      // [n_colours+1] ranges in colour-major order
  std::vector<int32_t> elem_perm_host;  // colour-major position -> original element
  int32_t* d_conn = nullptr;     // [n_elems][4]
  double* d_geo = nullptr;       // [n_elems][16]: g (12), V, tauV, 0, 0
  double* d_fibre = nullptr;     // [n_elems][6]
  int32_t* d_mat = nullptr;      // [n_elems]
  int32_t* d_slot = nullptr;     // [n_elems][16] block index of (a, b)
  double* d_mats = nullptr;      // [n_mat][8]: model, c10, c01, k1, k2, kappa, rho, mu_l
  double* d_X = nullptr;         // [n_nodes][3]
  uint8_t* d_dir_mask = nullptr; // [n_nodes][4]
  int32_t* d_faces = nullptr;    // [n_faces][3]
  int32_t* d_nf_ptr = nullptr;   // [n_nodes+1] node -> (face, local vertex) incidence
  int32_t* d_nf_idx = nullptr;   // [3 n_faces]: 3 * face + local vertex
  int32_t* d_seg_node = nullptr; // [n_nodes]
  std::vector<int32_t> seg_ptr_host;  // [n_seg+1] node ranges of the segments
  int32_t* d_seg_ptr = nullptr;
  double* d_seg_a = nullptr;     // [n_seg] per-segment scratch
  double* d_seg_b = nullptr;
  double* h_seg = nullptr;       // pinned [n_seg]
  // per-segment FGMRES (segment_krylov): [2 (m+2)][n_seg] dot products and
  // [m+1][n_seg] coefficients, device and pinned host copies
  double* d_sdots = nullptr;
  double* h_sdots = nullptr;
  double* d_scoef = nullptr;
  double* h_scoef = nullptr;
  int* d_err = nullptr;          // device error word (bit 0 inverted, bit 1 bounds)
  // gather-based assembly: element buffers and fixed gather plans
  void* d_ebuf = nullptr;        // T [n_elems][16][16] element tangent blocks
  double* d_rbuf = nullptr;      // [n_elems][16] element residuals
  int32_t* d_gb_ptr = nullptr;   // [n_b+1] contributions of each BSR block
  int32_t* d_gb_src = nullptr;   // [16 n_elems] element block index 16 e + (4a + b)
  int32_t* d_gn_ptr = nullptr;   // [n_nodes+1] contributions of each node
  int32_t* d_gn_src = nullptr;   // [4 n_elems] element node index 4 e + a

  // AMG hierarchy (level 0 = assembled matrix)
  std::vector<Level> levels;
  Coarse coarse;

  // Krylov workspace (FP64)
  int m = 30;
  double* d_V = nullptr;     // [(m+1)][ndof]
  double* d_Z = nullptr;     // [m][ndof]
  double* d_w = nullptr;     // [ndof]
  double* d_r = nullptr;     // [ndof]
  double* d_t = nullptr;     // [ndof] scratch
  double* d_t2 = nullptr;    // [ndof] scratch
  double* d_t3 = nullptr;    // [ndof] scratch
  double* d_partial = nullptr;   // reduction partials [n_red_blocks * 72]
  double* d_dots = nullptr;      // [72]
  double* h_dots = nullptr;      // pinned host [72]
  float2* d_xdf = nullptr;       // [ndof] double-float split of an FP64 vector (FP32 mode)
  float* d_xs = nullptr;         // FP32 vector scratch for the mixed precision preconditioner
  float* d_ys = nullptr;
  double* d_fext = nullptr;      // [n_nodes][3]
  double* d_state_tmp = nullptr; // [ndof]
  double* d_res = nullptr;       // [ndof]
  int red_blocks = 0;
  // the assembled tangent K.  With the AMG preconditioner on K it is level 0's
  // value array; with the block-triangular P_L level 0 holds the displacement
  // block A (u-p couplings removed, identity pressure rows) and K lives here
  void* k_vals = nullptr;
  double* d_sinv = nullptr;      // [n_nodes] 1 / S~_ii of Eq. lpreschur (-1 on constrained p)
  double* d_pl_y = nullptr;      // [ndof] K x_u scratch of P_L
  // Dirichlet-Neumann coupling: interface Gamma^0 = vertices of the loaded faces
  int n_gam = 0;
  int32_t* d_gam_idx = nullptr;  // [n_gam] node ids (ascending)
  double* d_gam_w = nullptr;     // [n_gam][3] unit direction of the load of a unit pressure
  double* d_dn = nullptr;        // 5 x [3 n_gam]: d, d~, r, r_prev, dr (r_prev, dr adjacent)
  double* d_dn_p = nullptr;      // [n_nodes] nodal fluid pressure (zero off Gamma^0)
  // Vanka smoother of the finest level (smoother == FSI_SMOOTHER_VANKA)
  int vk_ncol = 0;
  std::vector<int32_t> vk_cptr;  // colour ranges into d_vk_order
  int32_t* d_vk_order = nullptr; // [n_nodes] patch centres, colour-major
  int vk_m = 0;                  // max local unknowns (3 x max row length + 1)
  void* d_vk_inv = nullptr;      // T [n_nodes][vk_m][vk_m] inverses of the local matrices
  void* d_vk_z = nullptr;        // T [n_nodes][vk_m] local corrections

  int elem_threads = 128;              // CTA size of the element kernels (autotuner)
  cudaStream_t stream = nullptr;
  cudaGraphExec_t vc_exec = nullptr;   // captured V-cycle (use_graphs)
  long long vc_kernels = 0;            // kernels in the captured V-cycle
  long long amg_calls = 0;             // numeric set-ups requested (amg_lag bookkeeping)
  bool filter_p = false;               // prolongator smoothing without u-p couplings (inertia)
  struct Profiler* prof_ptr() { return &prof; }
  Profiler prof;
};

// ------------------------------------------------------------------ kernels (launchers)
// element.cu
void launch_geometry(Handle& h, cudaStream_t s);
void launch_external_force(Handle& h, const fsi_load* load, cudaStream_t s);
// Residual (if residual != nullptr) and tangent (if want_tangent) at `state`;
// the tangent goes to level 0 (or to vals_target, FP32 if target_fp32 == 1).
void launch_assemble(Handle& h, const double* state, const double* hist, double* residual,
                     bool want_tangent, cudaStream_t s, void* vals_target = nullptr, int target_fp32 = -1);
void launch_assemble_gather(Handle& h, const double* state, const double* hist, double* residual,
                            bool want_tangent, cudaStream_t s, void* vals_target, int target_fp32);
void launch_assemble_colour(Handle& h, const double* state, const double* hist, double* residual,
                            bool want_tangent, cudaStream_t s, void* vals_target, int target_fp32);
void launch_set_dirichlet_values(Handle& h, double* state, const double* values, cudaStream_t s);
// out_dev[0] = x^T M x, M = diag[M_1, M_2] the P1 mass matrices (x: [n_nodes][4]; deterministic)
void launch_mass_norm2(Handle& h, const double* x, double* out_dev, cudaStream_t s);
void launch_newmark(Handle& h, const double* state, double* disp, double* vel, double* acc, double* hist,
                    double beta, double gamma, double dt, cudaStream_t s);

// linalg.cu
template <typename T>
void launch_spmv(const Level& L, const T* x, T* y, cudaStream_t s);
// the three operator products take the value array explicitly (level 0's
// pattern with the values of K, which differ from L.vals under P_L)
void launch_spmv_f64acc(const Level& L, const void* vals, const double* x, double* y, bool fp32vals, cudaStream_t s);
// FP32 values with FP64 vectors in double-float arithmetic; y = A x (b == nullptr) or y = b - A x
void launch_spmv_df(const Level& L, const void* vals, const double* x, float2* xs, const double* b, double* y,
                    cudaStream_t s);
void launch_residual_f64(const Level& L, const void* vals, const double* b, const double* x, double* r,
                         bool fp32vals, cudaStream_t s);
// P_L: level-0 values of A from K (u-p couplings dropped, pressure rows identity)
void launch_split_a(const Level& L, const void* k_vals, bool fp32, cudaStream_t s);
// P_L stages: b = (r_u, 0) in T; z = (x_u, 0) in FP64; z_p = (y_p - r_p) sinv
void pl_stage(const double* r, void* b, bool fp32, long n_nodes, cudaStream_t s);
void pl_unstage(const void* x, double* z, bool fp32, long n_nodes, cudaStream_t s);
void pl_pressure(const double* y, const double* r, const double* sinv, double* z, long n_nodes, cudaStream_t s);
void launch_block_inverse(Level& L, bool fp32, int* err, cudaStream_t s);
// numeric set-up of level+1 from level (smoothed P, P^T, A P, P^T A P)
void launch_galerkin(Level& L, Level& C, bool fp32, bool filter, cudaStream_t s);
void launch_coarse_factor(Handle& h, bool fp32, cudaStream_t s);
// times the launch shapes of every smoothed level's block-row kernels and keeps the fastest
void autotune_levels(Handle& h, cudaStream_t s);
// times the CTA size of the element tangent kernel and keeps the fastest (h.elem_threads)
void autotune_elements(Handle& h, cudaStream_t s);
// L.vals_lp = bf16(L.vals) (FP32 values, 7x7 blocks)
void launch_values_to_bf16(const Level& L, cudaStream_t s);
template <typename T>
void vcycle(Handle& h, int level, cudaStream_t s);
// CTAs of the deterministic dot partials of the minimal-residual smoother
constexpr int kMrBlocks = 2 * 152;
// FP64 vector helpers; reductions are deterministic (fixed two-pass order)
// out_dev[i] = V_i . y for V_i = V + i ldv, i < k
void dots(Handle& h, const double* V, long ldv, int k, const double* y, long n, double* out_dev,
          cudaStream_t s);
void multi_axpy(const double* coef_dev, const double* V, int k, long n, double* w, double sign,
                cudaStream_t s);
void axpy(double a, const double* x, double* y, long n, cudaStream_t s);
void scale_copy(double a, const double* x, double* y, long n, cudaStream_t s);
void to_float(const double* x, float* y, long n, cudaStream_t s);
void to_double(const float* x, double* y, long n, cudaStream_t s);
void mask_vector(const uint8_t* cmask, double* x, long n, cudaStream_t s);
// Vanka smoother (vanka.cu)
constexpr int kVankaMaxM = 64;   // local unknowns per patch (3 x 21 nodes + 1)
void vanka_colouring(const HostPattern& pat, int n, std::vector<int32_t>& order, std::vector<int32_t>& cptr,
                     int* max_deg);
void launch_vanka_factor(Handle& h, bool fp32, cudaStream_t s);
template <typename T>
void vanka_smooth(Handle& h, int sweeps, bool zero_start, cudaStream_t s);
// Dirichlet-Neumann coupling (coupling.cu)
void dn_fluid(int ng, const int32_t* idx, const double* w, const double* d, const double* dref, double p0, double c,
              double* node_p, cudaStream_t s);
void dn_restrict(int ng, const int32_t* idx, const double* state, double* out, const double* d, double* r,
                 cudaStream_t s);
void dn_relax(long m, double omega, const double* dt, double* d, cudaStream_t s);
void dn_diff(long m, const double* r, const double* r_prev, double* dr, cudaStream_t s);
// independent segments (batched meshes)
void segment_sumsq(const int32_t* seg_ptr, int n_seg, const double* x, double* out, cudaStream_t s);
void segment_normalise(int n_seg, double* a, double* b, cudaStream_t s);
void segment_scale(const int32_t* seg_node, const double* scale, double* x, long n, cudaStream_t s);
// out_dev[i n_seg + s] = V_i . y over segment s (deterministic)
void seg_dots(const int32_t* seg_ptr, int n_seg, const double* V, long ldv, int k, const double* y, double* out_dev,
              cudaStream_t s);
// w += sign * sum_i coef_dev[i n_seg + seg(t)] V_i[t]
void seg_multi_axpy(const int32_t* seg_node, int n_seg, const double* coef_dev, const double* V, int k, long n,
                    double* w, double sign, cudaStream_t s);

}  // namespace fsi

#define FSI_CUDA_TRY(expr)                                                         \
  do {                                                                             \
    cudaError_t _e = (expr);                                                       \
    if (_e != cudaSuccess) {                                                       \
      throw fsi::CudaError(std::string(#expr) + ": " + cudaGetErrorString(_e));     \
    }                                                                              \
  } while (0)

namespace fsi {
struct CudaError {
  std::string msg;
  explicit CudaError(std::string m) : msg(std::move(m)) {}
};
struct ArgError {
  std::string msg;
  explicit ArgError(std::string m) : msg(std::move(m)) {}
};
}  // namespace fsi
