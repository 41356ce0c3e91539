// Element kernels of the residual-stabilised P1/P1 u-p solid.
//
// One thread owns one tetrahedron.  It gathers the element's nodal state and
// geometry, forms the kinematics and the isochoric stress in registers
// (Sec. 2.3: F, J, C, I1, I2, I3; Eq. mmrpkt / arpkt for S'), and then adds
// the 16 residual entries (Sec. 4.2.3 + Eq. stelas) and, when asked, the
// 16 4x4 blocks of the consistent tangent (Eq. globsys) into the global
// arrays.  Elements are processed colour by colour: no two elements of one
// colour share a vertex, so the read-modify-write scatter needs no atomics
// and its summation order is fixed (bit-identical results run to run).
//
// Tangent, written in spatial vectors so that no 81-entry elasticity tensor
// is formed.  With gb_a = F^-T g_a, f_a = F g_a, b = F F^T and
// dS'/dC = sum_XY m_XY X (x) Y + gamma C^-1 (.) C^-1 + eta II over the basis
// {I, C, C^-1, A1, A2}:
//   A_ab = V (g_a.S' g_b) I + 2V sum_XY m_XY (F X g_a)(x)(F Y g_b)
//        + V gamma [gb_b (x) gb_a + (gb_a.gb_b) I] + V eta [f_b (x) f_a + (g_a.g_b) b]
//        - V pbar J [gb_a (x) gb_b - gb_b (x) gb_a] + rho c0 M_ab I
//   B1^T_ab = -(V/4) J gb_a,   -C_ab = -M_ab/kappa - tau V J gb_a.gb_b
//   B2_ab = -(V/4) J gb_b + tau V [-(rho c0/4) gb_a - (w.gb_b) gb_a
//           - J (q.gb_a) gb_b + J (q.gb_b) gb_a + J (gb_a.gb_b) q]
// with q = F^-T grad p and w = rho hbar - rho c0 ubar.
#include <cmath>

#include "internal.h"

namespace fsi {

namespace {

constexpr int kThreads = 128;

template <typename T>
__device__ __forceinline__ T dot3(const T* a, const T* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// symmetric 3x3 stored as (00, 11, 22, 01, 02, 12)
template <typename T>
__device__ __forceinline__ void sym_mul_vec(const T* S, const T* v, T* o) {
  o[0] = S[0] * v[0] + S[3] * v[1] + S[4] * v[2];
  o[1] = S[3] * v[0] + S[1] * v[1] + S[5] * v[2];
  o[2] = S[4] * v[0] + S[5] * v[1] + S[2] * v[2];
}

__global__ void geometry_kernel(int ne, const double* __restrict__ X, const int32_t* __restrict__ conn,
                                const int32_t* __restrict__ mat, const double* __restrict__ mats,
                                int use_pspg, double* __restrict__ geo, int* __restrict__ err) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  double x[4][3];
  for (int a = 0; a < 4; ++a) {
    int n = conn[4 * e + a];
    for (int i = 0; i < 3; ++i) x[a][i] = X[3 * n + i];
  }
  double d1[3], d2[3], d3[3];
  for (int i = 0; i < 3; ++i) {
    d1[i] = x[1][i] - x[0][i];
    d2[i] = x[2][i] - x[0][i];
    d3[i] = x[3][i] - x[0][i];
  }
  // grad N_1..3 = (d2 x d3, d3 x d1, d1 x d2) / det, det = d1 . (d2 x d3)
  double c1[3] = {d2[1] * d3[2] - d2[2] * d3[1], d2[2] * d3[0] - d2[0] * d3[2], d2[0] * d3[1] - d2[1] * d3[0]};
  double c2[3] = {d3[1] * d1[2] - d3[2] * d1[1], d3[2] * d1[0] - d3[0] * d1[2], d3[0] * d1[1] - d3[1] * d1[0]};
  double c3[3] = {d1[1] * d2[2] - d1[2] * d2[1], d1[2] * d2[0] - d1[0] * d2[2], d1[0] * d2[1] - d1[1] * d2[0]};
  double det = dot3(d1, c1);
  if (!(det > 0.0)) atomicOr(err, 1);
  double* o = geo + 16 * (size_t)e;
  for (int i = 0; i < 3; ++i) {
    double g1 = c1[i] / det, g2 = c2[i] / det, g3 = c3[i] / det;
    o[3 + i] = g1;
    o[6 + i] = g2;
    o[9 + i] = g3;
    o[i] = -(g1 + g2 + g3);
  }
  double V = det / 6.0;
  double h2 = 0.0;
  for (int a = 0; a < 4; ++a)
    for (int b = a + 1; b < 4; ++b) {
      double dx = x[a][0] - x[b][0], dy = x[a][1] - x[b][1], dz = x[a][2] - x[b][2];
      h2 = fmax(h2, dx * dx + dy * dy + dz * dz);
    }
  const double* mp = mats + 8 * mat[e];
  double mul = mp[7];
  o[12] = V;
  o[13] = use_pspg ? h2 / (4.0 * mul) * V : 0.0;
  o[14] = sqrt(h2);
  o[15] = 0.0;
}

struct ElemIn {
  double u[4][3], p[4], g[4][3], hs[4][3];
  double V, tauV;
};

// Residual and (optionally) tangent of one element.  Writes R[a][c] and, when
// TANGENT, hands each 4x4 block (a, b) to emit(4 a + b, K) as soon as it is formed.
template <typename TC, bool TANGENT, typename Emit>
__device__ __forceinline__ bool element_eval(const ElemIn& in, const double* __restrict__ mp,
                                             const double* __restrict__ fibd, double inertia_d,
                                             double fibre_factor_d, TC R[4][4], Emit& emit) {
  const TC V = (TC)in.V, tauV = (TC)in.tauV;
  const int model = (int)mp[0];
  const TC c10 = (TC)mp[1], c01 = (TC)mp[2], k1 = (TC)mp[3], k2 = (TC)mp[4], kappa = (TC)mp[5], rho = (TC)mp[6];
  const TC inertia = (TC)inertia_d, fibre_factor = (TC)fibre_factor_d;
  TC fib[6];
  for (int q = 0; q < 6; ++q) fib[q] = (TC)fibd[q];
  TC ug[4][3], pg[4], gg_[4][3], hsg[4][3];
  for (int a = 0; a < 4; ++a) {
    pg[a] = (TC)in.p[a];
    for (int i = 0; i < 3; ++i) {
      ug[a][i] = (TC)in.u[a][i];
      gg_[a][i] = (TC)in.g[a][i];
      hsg[a][i] = (TC)in.hs[a][i];
    }
  }

  // ---- kinematics (Sec. 2.3).  The volumetric terms J - 1, log J and J^{-2/3}
  // are always formed in FP64 (they decide the pressure coupling at large kappa).
  double Hd[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      Hd[i][j] = in.u[0][i] * in.g[0][j] + in.u[1][i] * in.g[1][j] + in.u[2][i] * in.g[2][j] +
                 in.u[3][i] * in.g[3][j];
  const double trH = Hd[0][0] + Hd[1][1] + Hd[2][2];
  double trHH = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) trHH += Hd[i][j] * Hd[j][i];
  const double detH = Hd[0][0] * (Hd[1][1] * Hd[2][2] - Hd[1][2] * Hd[2][1]) -
                      Hd[0][1] * (Hd[1][0] * Hd[2][2] - Hd[1][2] * Hd[2][0]) +
                      Hd[0][2] * (Hd[1][0] * Hd[2][1] - Hd[1][1] * Hd[2][0]);
  const double Jm1d = trH + 0.5 * (trH * trH - trHH) + detH;   // det(I + H) - 1, no cancellation
  const double Jd = 1.0 + Jm1d;
  if (!(Jd > 0.0) || !isfinite(Jd)) return false;
  TC H[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) H[i][j] = (TC)Hd[i][j];
  const TC Jm1 = (TC)Jm1d;
  const TC J = (TC)Jd;
  TC F[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) F[i][j] = H[i][j] + (i == j ? TC(1.0) : TC(0.0));
  TC Fi[3][3];   // F^-1 = adj(F) / J
  {
    const TC iJ = TC(1.0) / J;
    Fi[0][0] = (F[1][1] * F[2][2] - F[1][2] * F[2][1]) * iJ;
    Fi[0][1] = (F[0][2] * F[2][1] - F[0][1] * F[2][2]) * iJ;
    Fi[0][2] = (F[0][1] * F[1][2] - F[0][2] * F[1][1]) * iJ;
    Fi[1][0] = (F[1][2] * F[2][0] - F[1][0] * F[2][2]) * iJ;
    Fi[1][1] = (F[0][0] * F[2][2] - F[0][2] * F[2][0]) * iJ;
    Fi[1][2] = (F[0][2] * F[1][0] - F[0][0] * F[1][2]) * iJ;
    Fi[2][0] = (F[1][0] * F[2][1] - F[1][1] * F[2][0]) * iJ;
    Fi[2][1] = (F[0][1] * F[2][0] - F[0][0] * F[2][1]) * iJ;
    Fi[2][2] = (F[0][0] * F[1][1] - F[0][1] * F[1][0]) * iJ;
  }
  // E = (H + H^T + H^T H) / 2, C = I + 2E; symmetric storage (00,11,22,01,02,12)
  const int si[6] = {0, 1, 2, 0, 0, 1}, sj[6] = {0, 1, 2, 1, 2, 2};
  TC E[6], C[6], Ci[6], B[6];
  for (int k = 0; k < 6; ++k) {
    int i = si[k], j = sj[k];
    TC hth = H[0][i] * H[0][j] + H[1][i] * H[1][j] + H[2][i] * H[2][j];
    E[k] = TC(0.5) * (H[i][j] + H[j][i] + hth);
    C[k] = TC(2.0) * E[k] + (i == j ? TC(1.0) : TC(0.0));
    Ci[k] = Fi[i][0] * Fi[j][0] + Fi[i][1] * Fi[j][1] + Fi[i][2] * Fi[j][2];   // F^-1 F^-T
    B[k] = F[i][0] * F[j][0] + F[i][1] * F[j][1] + F[i][2] * F[j][2];         // F F^T
  }
  const TC I1 = C[0] + C[1] + C[2];
  const TC CC = C[0] * C[0] + C[1] * C[1] + C[2] * C[2] + TC(2.0) * (C[3] * C[3] + C[4] * C[4] + C[5] * C[5]);
  const TC I2 = TC(0.5) * (I1 * I1 - CC);
  const double lj = log1p(Jm1d);
  const double J23d = exp(-(2.0 / 3.0) * lj);
  const TC J23 = (TC)J23d;                 // I3^{-1/3}
  const TC J43 = J23 * J23;                // I3^{-2/3}

  // ---- isochoric stress S' and dS'/dC coefficients
  TC S[6];
  for (int k = 0; k < 6; ++k) {
    TC d = (si[k] == sj[k]) ? TC(1.0) : TC(0.0);
    S[k] = c10 * J23 * (d - (I1 / TC(3.0)) * Ci[k]) + c01 * J43 * (I1 * d - C[k] - (TC(2.0) / TC(3.0)) * I2 * Ci[k]);
  }
  // m over basis 0:I 1:C 2:Ci 3:A1 4:A2 (symmetric), gamma (Ci.Ci), eta (II)
  TC m[5][5];
  for (int x = 0; x < 5; ++x)
    for (int y = 0; y < 5; ++y) m[x][y] = TC(0.0);
  TC gam = TC(0.0), eta = TC(0.0);
  if (TANGENT) {
    m[0][2] += -c10 * J23 / TC(3.0);
    m[2][2] += c10 * J23 * I1 / TC(9.0);
    gam += c10 * J23 * I1 / TC(3.0);
    m[0][2] += -(TC(2.0) / TC(3.0)) * c01 * J43 * I1;
    m[1][2] += (TC(2.0) / TC(3.0)) * c01 * J43;
    m[2][2] += (TC(4.0) / TC(9.0)) * c01 * J43 * I2;
    m[0][0] += c01 * J43;
    eta += -c01 * J43;
    gam += (TC(2.0) / TC(3.0)) * c01 * J43 * I2;
  }
  TC af[2][3] = {{0, 0, 0}, {0, 0, 0}};
  if (model == FSI_MODEL_ARTERY) {
    const double J23m1 = expm1(-(2.0 / 3.0) * lj);
    for (int f = 0; f < 2; ++f) {
      const TC* a = fib + 3 * f;
      TC Ca[3], Ea[3];
      sym_mul_vec(C, a, Ca);
      sym_mul_vec(E, a, Ea);
      const TC I4 = dot3(a, Ca);
      const TC Jim1 = (TC)(J23m1 + J23d * 2.0 * (double)dot3(a, Ea));   // J_i - 1 (Eq. arinv46), FP64
      if (!(Jim1 > TC(0.0))) continue;                             // fibres act in extension only
      for (int i = 0; i < 3; ++i) af[f][i] = a[i];
      const TC ex = exp(k2 * Jim1 * Jim1);
      const TC beta = fibre_factor * k1 * ex * Jim1;
      for (int k = 0; k < 6; ++k) S[k] += beta * J23 * (a[si[k]] * a[sj[k]] - (I4 / TC(3.0)) * Ci[k]);
      if (TANGENT) {
        const TC alpha = fibre_factor * k1 * ex * (TC(1.0) + TC(2.0) * k2 * Jim1 * Jim1);
        const int X = 3 + f;
        m[X][X] += alpha * J43;
        m[X][2] += -alpha * J43 * I4 / TC(3.0) - beta * J23 / TC(3.0);
        m[2][2] += alpha * J43 * I4 * I4 / TC(9.0) + beta * J23 * I4 / TC(9.0);
        gam += beta * J23 * I4 / TC(3.0);
      }
    }
  }

  // ---- per-node vectors
  const TC pbar = TC(0.25) * (pg[0] + pg[1] + pg[2] + pg[3]);
  TC gp[3], ubar[3], hbar[3];
  for (int i = 0; i < 3; ++i) {
    gp[i] = pg[0] * gg_[0][i] + pg[1] * gg_[1][i] + pg[2] * gg_[2][i] + pg[3] * gg_[3][i];
    ubar[i] = TC(0.25) * (ug[0][i] + ug[1][i] + ug[2][i] + ug[3][i]);
    hbar[i] = TC(0.25) * (hsg[0][i] + hsg[1][i] + hsg[2][i] + hsg[3][i]);
  }
  TC q[3], w[3];
  for (int i = 0; i < 3; ++i) {
    q[i] = Fi[0][i] * gp[0] + Fi[1][i] * gp[1] + Fi[2][i] * gp[2];   // F^-T grad p
    w[i] = rho * hbar[i] - rho * inertia * ubar[i];
  }
  TC gb[4][3];   // F^-T g_a
  for (int a = 0; a < 4; ++a)
    for (int i = 0; i < 3; ++i)
      gb[a][i] = Fi[0][i] * gg_[a][0] + Fi[1][i] * gg_[a][1] + Fi[2][i] * gg_[a][2];
  TC FS[3][3];   // F S' (S' symmetric)
  for (int i = 0; i < 3; ++i) {
    for (int k = 0; k < 3; ++k) {
      TC s0 = (k == 0) ? S[0] : (k == 1 ? S[3] : S[4]);
      TC s1 = (k == 0) ? S[3] : (k == 1 ? S[1] : S[5]);
      TC s2 = (k == 0) ? S[4] : (k == 1 ? S[5] : S[2]);
      FS[i][k] = F[i][0] * s0 + F[i][1] * s1 + F[i][2] * s2;
    }
  }

  // ---- residual (always FP64): R^1_a rows 0..2, R^2_a row 3
  TC usum[3], hsum[3], psum = pg[0] + pg[1] + pg[2] + pg[3];
  for (int i = 0; i < 3; ++i) {
    usum[i] = ug[0][i] + ug[1][i] + ug[2][i] + ug[3][i];
    hsum[i] = hsg[0][i] + hsg[1][i] + hsg[2][i] + hsg[3][i];
  }
  const TC V20 = V / TC(20.0);
  for (int a = 0; a < 4; ++a) {
    for (int i = 0; i < 3; ++i) {
      TC fsg = FS[i][0] * gg_[a][0] + FS[i][1] * gg_[a][1] + FS[i][2] * gg_[a][2];
      R[a][i] = V * (fsg - pbar * J * gb[a][i]) + rho * inertia * V20 * (ug[a][i] + usum[i]) -
                rho * V20 * (hsg[a][i] + hsum[i]);
    }
    TC wq = (w[0] - J * q[0]) * gb[a][0] + (w[1] - J * q[1]) * gb[a][1] + (w[2] - J * q[2]) * gb[a][2];
    R[a][3] = -V * Jm1 * TC(0.25) - V20 * (pg[a] + psum) / kappa + tauV * wq;
  }
  if (!TANGENT) return true;

  // ---- tangent blocks
  TC fv[4][3];   // F g_a
  for (int a = 0; a < 4; ++a)
    for (int i = 0; i < 3; ++i) fv[a][i] = F[i][0] * gg_[a][0] + F[i][1] * gg_[a][1] + F[i][2] * gg_[a][2];
  TC Fa[2][3];   // F a_i
  for (int f = 0; f < 2; ++f)
    for (int i = 0; i < 3; ++i) Fa[f][i] = F[i][0] * af[f][0] + F[i][1] * af[f][1] + F[i][2] * af[f][2];
  // pressure geometric term folded into the C^-1 (x) C^-1 coefficient and the swap term
  m[2][2] += -TC(0.5) * pbar * J;
  // symmetric completion
  for (int x = 0; x < 5; ++x)
    for (int y = x + 1; y < 5; ++y) {
      TC s = m[x][y] + m[y][x];
      m[x][y] = s;
      m[y][x] = s;
    }
  // w_X(b) = F X g_b, z_X(b) = sum_Y m_XY w_Y(b)
  TC z[4][5][3];
  TC wv[4][5][3];
  for (int b = 0; b < 4; ++b) {
    TC Bf[3];
    sym_mul_vec(B, fv[b], Bf);
    for (int i = 0; i < 3; ++i) {
      wv[b][0][i] = fv[b][i];
      wv[b][1][i] = Bf[i];
      wv[b][2][i] = gb[b][i];
      wv[b][3][i] = Fa[0][i] * dot3(af[0], gg_[b]);
      wv[b][4][i] = Fa[1][i] * dot3(af[1], gg_[b]);
    }
    for (int x = 0; x < 5; ++x)
      for (int i = 0; i < 3; ++i) {
        TC acc = TC(0.0);
        for (int y = 0; y < 5; ++y) acc += m[x][y] * wv[b][y][i];
        z[b][x][i] = TC(2.0) * V * acc;
      }
  }
  TC Sg[4][3];
  for (int b = 0; b < 4; ++b) sym_mul_vec(S, gg_[b], Sg[b]);
  TC qg[4], wg[4];
  for (int a = 0; a < 4; ++a) {
    qg[a] = dot3(q, gb[a]);
    wg[a] = dot3(w, gb[a]);
  }
  const TC Vswap = V * (gam + pbar * J);
  const TC Vgam = V * gam, Veta = V * eta;
  const TC c_in = rho * inertia;
  for (int a = 0; a < 4; ++a) {
    for (int b = 0; b < 4; ++b) {
      const TC Mab = V20 * (a == b ? TC(2.0) : TC(1.0));
      const TC gg = dot3(gg_[a], gg_[b]);
      const TC gbgb = dot3(gb[a], gb[b]);
      const TC diag = V * dot3(gg_[a], Sg[b]) + Vgam * gbgb + c_in * Mab;
      TC K[4][4];
      for (int i = 0; i < 3; ++i) {
        for (int k = 0; k < 3; ++k) {
          TC v = TC(0.0);
          for (int x = 0; x < 5; ++x) v += wv[a][x][i] * z[b][x][k];
          v += Vswap * gb[b][i] * gb[a][k] + Veta * fv[b][i] * fv[a][k];
          int sk = (i == k) ? i : (i + k == 1 ? 3 : (i + k == 2 ? 4 : 5));
          v += Veta * gg * B[sk];
          if (i == k) v += diag;
          K[i][k] = v;
        }
        K[i][3] = -TC(0.25) * V * J * gb[a][i];
      }
      const TC ca = tauV * (-TC(0.25) * c_in - wg[b] + J * qg[b]);
      const TC cb = -TC(0.25) * V * J - tauV * J * qg[a];
      const TC cq = tauV * J * gbgb;
      for (int k = 0; k < 3; ++k) K[3][k] = cb * gb[b][k] + ca * gb[a][k] + cq * q[k];
      K[3][3] = -Mab / kappa - tauV * J * gbgb;
      emit(4 * a + b, K);
    }
  }
  return true;
}

template <typename T>
struct BsrEmit {
  T* vals;
  const int32_t* slot;
  template <typename TC>
  __device__ __forceinline__ void operator()(int ab, const TC (&K)[4][4]) const {
    T* v = vals + 16 * (size_t)slot[ab];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) v[4 * r + c] += (T)K[r][c];
  }
};

// T: storage type of the tangent; TC: arithmetic type of the element math
// (the volumetric J terms are FP64 in both cases).
template <typename T, typename TC, bool TANGENT>
__global__ void __launch_bounds__(kThreads) assemble_kernel(
    int e0, int e1, const int32_t* __restrict__ conn, const double* __restrict__ geo,
    const double* __restrict__ fibre, const int32_t* __restrict__ mat, const double* __restrict__ mats,
    const double* __restrict__ state, const double* __restrict__ hist, double inertia, double fibre_factor,
    const int32_t* __restrict__ slot, T* __restrict__ vals, double* __restrict__ res, int* __restrict__ err) {
  const int e = e0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= e1) return;
  ElemIn in;
  int nid[4];
  const double* ge = geo + 16 * (size_t)e;
  for (int a = 0; a < 4; ++a) {
    nid[a] = conn[4 * e + a];
    const double* s = state + 4 * (size_t)nid[a];
    for (int i = 0; i < 3; ++i) {
      in.u[a][i] = s[i];
      in.g[a][i] = ge[3 * a + i];
      in.hs[a][i] = hist ? hist[3 * (size_t)nid[a] + i] : 0.0;
    }
    in.p[a] = s[3];
  }
  in.V = ge[12];
  in.tauV = ge[13];
  const double* mp = mats + 8 * mat[e];
  const double* fib = fibre + 6 * (size_t)e;
  TC R[4][4];
  BsrEmit<T> emit{vals, slot + 16 * (size_t)e};
  if (!element_eval<TC, TANGENT>(in, mp, fib, inertia, fibre_factor, R, emit)) {
    atomicOr(err, 1);
    return;
  }
  if (res) {
    for (int a = 0; a < 4; ++a) {
      double* r = res + 4 * (size_t)nid[a];
      for (int c = 0; c < 4; ++c) r[c] += (double)R[a][c];
    }
  }
}

// Gather-based assembly.  Every element writes its 16 residual entries and
// 16 tangent blocks to a per-element buffer in one launch; the global
// residual and BSR values are then formed by gathering, for each node and
// each block, its contributions in a fixed order (deterministic without
// colours or atomics, and every launch fills the GPU).
template <typename T>
struct BufEmit {
  T* out;   // [16][16] of this element
  template <typename TC>
  __device__ __forceinline__ void operator()(int ab, const TC (&K)[4][4]) const {
    T* v = out + 16 * ab;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) v[4 * r + c] = (T)K[r][c];
  }
};

template <typename T, typename TC, bool TANGENT>
__global__ void __launch_bounds__(kThreads) element_buffer_kernel(
    int ne, const int32_t* __restrict__ conn, const double* __restrict__ geo, const double* __restrict__ fibre,
    const int32_t* __restrict__ mat, const double* __restrict__ mats, const double* __restrict__ state,
    const double* __restrict__ hist, double inertia, double fibre_factor, T* __restrict__ ek,
    double* __restrict__ er, int* __restrict__ err) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  ElemIn in;
  const double* ge = geo + 16 * (size_t)e;
  for (int a = 0; a < 4; ++a) {
    const int nid = conn[4 * e + a];
    const double* s = state + 4 * (size_t)nid;
    for (int i = 0; i < 3; ++i) {
      in.u[a][i] = s[i];
      in.g[a][i] = ge[3 * a + i];
      in.hs[a][i] = hist ? hist[3 * (size_t)nid + i] : 0.0;
    }
    in.p[a] = s[3];
  }
  in.V = ge[12];
  in.tauV = ge[13];
  TC R[4][4];
  BufEmit<T> emit{ek + 256 * (size_t)e};
  if (!element_eval<TC, TANGENT>(in, mats + 8 * mat[e], fibre + 6 * (size_t)e, inertia, fibre_factor, R, emit)) {
    atomicOr(err, 1);
    if (er)
      for (int q = 0; q < 16; ++q) er[16 * (size_t)e + q] = 0.0;
    if (TANGENT)
      for (int q = 0; q < 256; ++q) ek[256 * (size_t)e + q] = T(0);
    return;
  }
  if (er)
    for (int a = 0; a < 4; ++a)
      for (int c = 0; c < 4; ++c) er[16 * (size_t)e + 4 * a + c] = (double)R[a][c];
}

// vals[b][q] = sum over the contributions of block b (fixed order), with the
// Dirichlet rows/columns replaced by identity rows and zero columns.
template <typename T>
__global__ void gather_tangent_kernel(int nb, const int32_t* __restrict__ bptr, const int32_t* __restrict__ bsrc,
                                      const T* __restrict__ ek, const int32_t* __restrict__ block_row,
                                      const int32_t* __restrict__ col_idx, const uint8_t* __restrict__ mask,
                                      T* __restrict__ vals) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = (int)(t >> 4), q = (int)(t & 15);
  if (b >= nb) return;
  const int i = block_row[b], j = col_idx[b];
  const int r = q >> 2, c = q & 3;
  T v;
  if (mask[4 * i + r] || mask[4 * j + c]) {
    v = (i == j && r == c && mask[4 * i + r]) ? T(1) : T(0);
  } else {
    float accf = 0.f;
    double accd = 0.0;
    for (int k = bptr[b]; k < bptr[b + 1]; ++k) {
      const T x = ek[16 * (size_t)bsrc[k] + q];
      if (sizeof(T) == 4) accf += (float)x; else accd += (double)x;
    }
    v = (sizeof(T) == 4) ? (T)accf : (T)accd;
  }
  vals[16 * (size_t)b + q] = v;
}

// res[i][c] = sum over the element contributions of node i - f_ext, masked
__global__ void gather_residual_kernel(int n, const int32_t* __restrict__ nptr, const int32_t* __restrict__ nsrc,
                                       const double* __restrict__ er, const double* __restrict__ fext,
                                       const uint8_t* __restrict__ mask, double* __restrict__ res) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4 * n) return;
  const int i = t >> 2, c = t & 3;
  double acc = (c < 3 && fext) ? -fext[3 * (size_t)i + c] : 0.0;
  for (int k = nptr[i]; k < nptr[i + 1]; ++k) acc += er[4 * (size_t)nsrc[k] + c];
  res[t] = mask[t] ? 0.0 : acc;
}

// R = -f_ext on displacement rows, 0 on pressure rows
__global__ void init_residual_kernel(int n, const double* __restrict__ fext, double* __restrict__ res) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int c = 0; c < 3; ++c) res[4 * i + c] = fext ? -fext[3 * i + c] : 0.0;
  res[4 * i + 3] = 0.0;
}

__global__ void mask_residual_kernel(int n, const uint8_t* __restrict__ mask, double* __restrict__ res) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 4 * n) return;
  if (mask[k]) res[k] = 0.0;
}

// Dead pressure on boundary triangles, gathered per node in a fixed order:
// f_a = -((x1-x0) x (x2-x0)) * sum_b P_b (1 + delta_ab) / 24.
__global__ void external_force_kernel(int n, const int32_t* __restrict__ nf_ptr, const int32_t* __restrict__ nf_idx,
                                      const int32_t* __restrict__ faces, const double* __restrict__ X, double pressure,
                                      const double* __restrict__ node_p, const double* __restrict__ face_p,
                                      double* __restrict__ fext) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double f[3] = {0, 0, 0};
  for (int k = nf_ptr[i]; k < nf_ptr[i + 1]; ++k) {
    int code = nf_idx[k];
    int fc = code / 3, a = code % 3;
    int v0 = faces[3 * fc], v1 = faces[3 * fc + 1], v2 = faces[3 * fc + 2];
    double e1[3], e2[3];
    for (int c = 0; c < 3; ++c) {
      e1[c] = X[3 * v1 + c] - X[3 * v0 + c];
      e2[c] = X[3 * v2 + c] - X[3 * v0 + c];
    }
    double nrm[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double P[3];
    int vv[3] = {v0, v1, v2};
    for (int b = 0; b < 3; ++b) {
      double pb = pressure;
      if (node_p) pb *= node_p[vv[b]];
      else if (face_p) pb *= face_p[fc];
      P[b] = pb;
    }
    double wa = (P[0] + P[1] + P[2] + P[a]) / 24.0;
    for (int c = 0; c < 3; ++c) f[c] -= nrm[c] * wa;
  }
  for (int c = 0; c < 3; ++c) fext[3 * i + c] = f[c];
}

template <typename T>
__global__ void dirichlet_matrix_kernel(int nb, const int32_t* __restrict__ block_row, const int32_t* __restrict__ col_idx,
                                        const uint8_t* __restrict__ mask, T* __restrict__ vals) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nb) return;
  int i = block_row[k], j = col_idx[k];
  uint32_t mi = *reinterpret_cast<const uint32_t*>(mask + 4 * i);
  uint32_t mj = *reinterpret_cast<const uint32_t*>(mask + 4 * j);
  if (!mi && !mj) return;
  T* v = vals + 16 * (size_t)k;
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      bool cr = mask[4 * i + r] != 0, cc = mask[4 * j + c] != 0;
      if (cr || cc) v[4 * r + c] = (i == j && r == c && cr) ? T(1) : T(0);
    }
}

__global__ void set_dirichlet_kernel(int n, const uint8_t* __restrict__ mask, const double* __restrict__ values,
                                     double* __restrict__ state) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 4 * n) return;
  if (mask[k]) state[k] = values[k];
}

inline int blocks_for(long n, int t) { return (int)((n + t - 1) / t); }

__global__ void newmark_kernel(int n, const double* __restrict__ state, double* __restrict__ disp,
                               double* __restrict__ vel, double* __restrict__ acc, double* __restrict__ hist,
                               double beta, double gamma, double dt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * n) return;
  const int i = t / 3, c = t % 3;
  const double dn = state[4 * (size_t)i + c];
  const double a_new = (dn - disp[t]) / (beta * dt * dt) - vel[t] / (beta * dt) -
                       (1.0 - 2.0 * beta) / (2.0 * beta) * acc[t];
  const double v_new = vel[t] + dt * ((1.0 - gamma) * acc[t] + gamma * a_new);
  disp[t] = dn;
  vel[t] = v_new;
  acc[t] = a_new;
  hist[t] = dn / (beta * dt * dt) + v_new / (beta * dt) + (1.0 - 2.0 * beta) / (2.0 * beta) * a_new;
}

// ||x||_M^2 with M = diag[M_1, M_2], the P1 mass matrices of the displacement
// components and of the pressure (Sec. 4.4, Eq. newstop): element e adds
// sum_ab M_ab x_a . x_b = (V/20) (sum_a |x_a|^2 + |sum_a x_a|^2) over the
// 4 unknowns per node (M_ab = V (1 + delta_ab) / 20).  Each CTA sums a fixed
// grid-stride set of elements; a second pass adds the CTA partials in index
// order, so the result is deterministic.
constexpr int kNormThreads = 256;

__device__ __forceinline__ double cta_sum(double v) {
  __shared__ double w[kNormThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < kNormThreads / 32) ? w[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(kNormThreads) mass_norm_partial_kernel(int ne, const int32_t* __restrict__ conn,
                                                                       const double* __restrict__ geo,
                                                                       const double* __restrict__ x,
                                                                       double* __restrict__ partial) {
  double acc = 0.0;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (long)gridDim.x * blockDim.x) {
    const int4 c = *reinterpret_cast<const int4*>(conn + 4 * e);
    const int nd[4] = {c.x, c.y, c.z, c.w};
    double sq = 0.0, sum[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const double2 lo = *reinterpret_cast<const double2*>(x + 4 * (size_t)nd[a]);
      const double2 hi = *reinterpret_cast<const double2*>(x + 4 * (size_t)nd[a] + 2);
      sq += lo.x * lo.x + lo.y * lo.y + hi.x * hi.x + hi.y * hi.y;
      sum[0] += lo.x;
      sum[1] += lo.y;
      sum[2] += hi.x;
      sum[3] += hi.y;
    }
    const double V = geo[16 * e + 12];
    acc += V / 20.0 * (sq + sum[0] * sum[0] + sum[1] * sum[1] + sum[2] * sum[2] + sum[3] * sum[3]);
  }
  acc = cta_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kNormThreads) sum_partials_kernel(const double* __restrict__ partial, int nblk,
                                                                  double* __restrict__ out) {
  double acc = 0.0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) acc += partial[k];
  acc = cta_sum(acc);
  if (threadIdx.x == 0) *out = acc;
}

}  // namespace

void launch_newmark(Handle& h, const double* state, double* disp, double* vel, double* acc, double* hist,
                    double beta, double gamma, double dt, cudaStream_t s) {
  FSI_LAUNCH(fsi::KC_OTHER, s, newmark_kernel<<<blocks_for(3L * h.n_nodes, 256), 256, 0, s>>>(
      h.n_nodes, state, disp, vel, acc, hist, beta, gamma, dt));
  FSI_CUDA_TRY(cudaGetLastError());
}

void launch_geometry(Handle& h, cudaStream_t s) {
  if (h.n_elems == 0) return;
  FSI_LAUNCH(fsi::KC_OTHER, s, geometry_kernel<<<blocks_for(h.n_elems, 256), 256, 0, s>>>(h.n_elems, h.d_X, h.d_conn, h.d_mat, h.d_mats,
                                                              h.opts.use_pspg, h.d_geo, h.d_err));
  FSI_CUDA_TRY(cudaGetLastError());
}

void launch_external_force(Handle& h, const fsi_load* load, cudaStream_t s) {
  if (h.n_nodes == 0) return;
  double P = load ? load->pressure : 0.0;
  FSI_LAUNCH(fsi::KC_OTHER, s, external_force_kernel<<<blocks_for(h.n_nodes, 256), 256, 0, s>>>(
      h.n_nodes, h.d_nf_ptr, h.d_nf_idx, h.d_faces, h.d_X, P, load ? load->node_pressure : nullptr,
      load ? load->face_pressure : nullptr, h.d_fext));
  FSI_CUDA_TRY(cudaGetLastError());
}

void launch_assemble(Handle& h, const double* state, const double* hist, double* residual, bool want_tangent,
                     cudaStream_t s, void* vals_target, int target_fp32) {
  if (h.opts.assembly == 0 && h.d_ebuf) {
    launch_assemble_gather(h, state, hist, residual, want_tangent, s, vals_target, target_fp32);
    return;
  }
  launch_assemble_colour(h, state, hist, residual, want_tangent, s, vals_target, target_fp32);
}

void launch_assemble_gather(Handle& h, const double* state, const double* hist, double* residual, bool want_tangent,
                            cudaStream_t s, void* vals_target, int target_fp32) {
  Level& L0 = h.levels[0];
  void* vals = vals_target ? vals_target : h.k_vals;
  const bool f32 = vals_target ? (target_fp32 == 1) : (h.precision == FSI_PREC_FP32_IR);
  const int ne = h.n_elems;
  const int et = h.elem_threads;
  const int nbk = blocks_for(ne, et);
  double* er = residual ? h.d_rbuf : nullptr;
  if (want_tangent && f32) {
    FSI_LAUNCH(fsi::KC_TANGENT, s, element_buffer_kernel<float, float, true><<<nbk, et, 0, s>>>(
        ne, h.d_conn, h.d_geo, h.d_fibre, h.d_mat, h.d_mats, state, hist, h.opts.inertia_coef, h.opts.fibre_factor,
        (float*)h.d_ebuf, (double*)nullptr, h.d_err));
    if (er)
      FSI_LAUNCH(fsi::KC_RESIDUAL, s, element_buffer_kernel<double, double, false><<<nbk, et, 0, s>>>(
          ne, h.d_conn, h.d_geo, h.d_fibre, h.d_mat, h.d_mats, state, hist, h.opts.inertia_coef,
          h.opts.fibre_factor, (double*)nullptr, er, h.d_err));
  } else if (want_tangent) {
    FSI_LAUNCH(fsi::KC_TANGENT, s, element_buffer_kernel<double, double, true><<<nbk, et, 0, s>>>(
        ne, h.d_conn, h.d_geo, h.d_fibre, h.d_mat, h.d_mats, state, hist, h.opts.inertia_coef, h.opts.fibre_factor,
        (double*)h.d_ebuf, er, h.d_err));
  } else if (er) {
    FSI_LAUNCH(fsi::KC_RESIDUAL, s, element_buffer_kernel<double, double, false><<<nbk, et, 0, s>>>(
        ne, h.d_conn, h.d_geo, h.d_fibre, h.d_mat, h.d_mats, state, hist, h.opts.inertia_coef, h.opts.fibre_factor,
        (double*)nullptr, er, h.d_err));
  }
  if (want_tangent) {
    if (f32)
      FSI_LAUNCH(fsi::KC_TANGENT, s, gather_tangent_kernel<float><<<blocks_for(16L * L0.nb, 256), 256, 0, s>>>(
          L0.nb, h.d_gb_ptr, h.d_gb_src, (const float*)h.d_ebuf, L0.block_row, L0.col_idx, h.d_dir_mask,
          (float*)vals));
    else
      FSI_LAUNCH(fsi::KC_TANGENT, s, gather_tangent_kernel<double><<<blocks_for(16L * L0.nb, 256), 256, 0, s>>>(
          L0.nb, h.d_gb_ptr, h.d_gb_src, (const double*)h.d_ebuf, L0.block_row, L0.col_idx, h.d_dir_mask,
          (double*)vals));
  }
  if (residual)
    FSI_LAUNCH(fsi::KC_RESIDUAL, s, gather_residual_kernel<<<blocks_for(4L * h.n_nodes, 256), 256, 0, s>>>(
        h.n_nodes, h.d_gn_ptr, h.d_gn_src, er, h.d_fext, h.d_dir_mask, residual));
  FSI_CUDA_TRY(cudaGetLastError());
}

void launch_assemble_colour(Handle& h, const double* state, const double* hist, double* residual, bool want_tangent,
                            cudaStream_t s, void* vals_target, int target_fp32) {
  Level& L0 = h.levels[0];
  void* vals = vals_target ? vals_target : h.k_vals;
  const bool f32 = vals_target ? (target_fp32 == 1) : (h.precision == FSI_PREC_FP32_IR);
  if (residual)
    FSI_LAUNCH(fsi::KC_OTHER, s, init_residual_kernel<<<blocks_for(h.n_nodes, 256), 256, 0, s>>>(h.n_nodes, h.d_fext, residual));
  if (want_tangent) FSI_CUDA_TRY(cudaMemsetAsync(vals, 0, (size_t)L0.nb * 16 * (f32 ? 4 : 8), s));
  // FP32 tangents are formed by an FP32 kernel; the residual always comes from the FP64 kernel
  const bool split = want_tangent && f32;
  for (int c = 0; c < h.n_colours; ++c) {
    int e0 = h.colour_ptr[c], e1 = h.colour_ptr[c + 1];
    if (e1 <= e0) continue;
    int nbk = blocks_for(e1 - e0, kThreads);
    if (want_tangent && f32) {
      FSI_LAUNCH(fsi::KC_TANGENT, s, assemble_kernel<float, float, true><<<nbk, kThreads, 0, s>>>(
          e0, e1, h.d_conn, h.d_geo, h.d_fibre, h.d_mat, h.d_mats, state, hist, h.opts.inertia_coef,
          h.opts.fibre_factor, h.d_slot, (float*)vals, (double*)nullptr, h.d_err));
    } else if (want_tangent) {
      FSI_LAUNCH(fsi::KC_TANGENT, s, assemble_kernel<double, double, true><<<nbk, kThreads, 0, s>>>(
          e0, e1, h.d_conn, h.d_geo, h.d_fibre, h.d_mat, h.d_mats, state, hist, h.opts.inertia_coef,
          h.opts.fibre_factor, h.d_slot, (double*)vals, residual, h.d_err));
    }
    if ((!want_tangent || split) && residual) {
      FSI_LAUNCH(fsi::KC_RESIDUAL, s, assemble_kernel<double, double, false><<<nbk, kThreads, 0, s>>>(
          e0, e1, h.d_conn, h.d_geo, h.d_fibre, h.d_mat, h.d_mats, state, hist, h.opts.inertia_coef,
          h.opts.fibre_factor, h.d_slot, (double*)nullptr, residual, h.d_err));
    }
  }
  FSI_CUDA_TRY(cudaGetLastError());
  if (residual)
    FSI_LAUNCH(fsi::KC_OTHER, s, mask_residual_kernel<<<blocks_for(4L * h.n_nodes, 256), 256, 0, s>>>(h.n_nodes, h.d_dir_mask, residual));
  if (want_tangent) {
    if (f32)
      FSI_LAUNCH(fsi::KC_OTHER, s, dirichlet_matrix_kernel<float><<<blocks_for(L0.nb, 256), 256, 0, s>>>(L0.nb, L0.block_row, L0.col_idx,
                                                                            h.d_dir_mask, (float*)vals));
    else
      FSI_LAUNCH(fsi::KC_OTHER, s, dirichlet_matrix_kernel<double><<<blocks_for(L0.nb, 256), 256, 0, s>>>(L0.nb, L0.block_row, L0.col_idx,
                                                                             h.d_dir_mask, (double*)vals));
  }
  FSI_CUDA_TRY(cudaGetLastError());
}

void launch_mass_norm2(Handle& h, const double* x, double* out_dev, cudaStream_t s) {
  FSI_LAUNCH(fsi::KC_VECTOR, s, mass_norm_partial_kernel<<<h.red_blocks, kNormThreads, 0, s>>>(
      h.n_elems, h.d_conn, h.d_geo, x, h.d_partial));
  FSI_LAUNCH(fsi::KC_VECTOR, s, sum_partials_kernel<<<1, kNormThreads, 0, s>>>(h.d_partial, h.red_blocks, out_dev));
  FSI_CUDA_TRY(cudaGetLastError());
}

// CTA size of the element kernels: 64 or 128 threads (the tangent kernel holds
// ~220 registers per thread, so the CTA size decides how many CTAs fit on an
// SM); the tangent of the reference state is timed with each, three
// repetitions after one warm-up, and the faster is kept.
void autotune_elements(Handle& h, cudaStream_t s) {
  const bool f32 = h.precision == FSI_PREC_FP32_IR;
  double* zero = h.d_state_tmp;
  FSI_CUDA_TRY(cudaMemsetAsync(zero, 0, sizeof(double) * 4 * (size_t)h.n_nodes, s));
  cudaEvent_t e0, e1;
  FSI_CUDA_TRY(cudaEventCreate(&e0));
  FSI_CUDA_TRY(cudaEventCreate(&e1));
  const int ne = h.n_elems;
  float best = 1e30f;
  int pick = 128;
  for (int et : {64, 128}) {
    auto run = [&]() {
      if (f32)
        element_buffer_kernel<float, float, true><<<blocks_for(ne, et), et, 0, s>>>(
            ne, h.d_conn, h.d_geo, h.d_fibre, h.d_mat, h.d_mats, zero, nullptr, h.opts.inertia_coef,
            h.opts.fibre_factor, (float*)h.d_ebuf, (double*)nullptr, h.d_err);
      else
        element_buffer_kernel<double, double, true><<<blocks_for(ne, et), et, 0, s>>>(
            ne, h.d_conn, h.d_geo, h.d_fibre, h.d_mat, h.d_mats, zero, nullptr, h.opts.inertia_coef,
            h.opts.fibre_factor, (double*)h.d_ebuf, (double*)nullptr, h.d_err);
    };
    run();
    FSI_CUDA_TRY(cudaEventRecord(e0, s));
    for (int r = 0; r < 3; ++r) run();
    FSI_CUDA_TRY(cudaEventRecord(e1, s));
    FSI_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    FSI_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) {
      best = ms;
      pick = et;
    }
  }
  h.elem_threads = pick;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  FSI_CUDA_TRY(cudaGetLastError());
}

void launch_set_dirichlet_values(Handle& h, double* state, const double* values, cudaStream_t s) {
  FSI_LAUNCH(fsi::KC_OTHER, s, set_dirichlet_kernel<<<blocks_for(4L * h.n_nodes, 256), 256, 0, s>>>(h.n_nodes, h.d_dir_mask, values, state));
  FSI_CUDA_TRY(cudaGetLastError());
}

}  // namespace fsi
