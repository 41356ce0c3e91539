// Host set-up of the smoothed-aggregation AMG hierarchy (once per handle).
//
// The coarse spaces are built from the tangent at the reference state
// (zero displacement, zero pressure).  Level 0 is the assembled 4x4-block
// matrix; each coarser level has 7 unknowns per aggregate: the rigid-body
// modes of the displacement (3 translations, 3 rotations) and a constant
// pressure, orthonormalised per aggregate (QR).  The tentative prolongator is
// smoothed once by damped Jacobi, P = (I - w D^-1 A) P_t with
// w = 4 / (3 lambda), lambda a power-iteration estimate of lambda_max(D^-1 A)
// (power_steps steps; a few tens of steps fall short of lambda_max where the
// top eigenvalues cluster), and the coarse operators are the Galerkin
// products P^T A P.  What stays fixed per mesh is computed here: the
// aggregates, P_t, w, and the sparsity patterns of P, A P and P^T A P
// together with the index plans of those products (the value loops run on
// the host's cores with OpenMP, every row or block written by one thread, so
// the result does not depend on the thread count).  Every Newton step then
// recomputes on the device, with the current tangent, the smoothed P and the
// Galerkin operators of all levels (a numeric-only set-up); keeping the
// coarse operators of the reference state instead lets the Krylov iteration
// count grow without bound along a pressure ramp.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "amg_setup.h"

namespace fsi {

namespace {

constexpr int NS = 7;   // near-null-space size: 6 rigid-body modes + constant pressure

// Gauss-Jordan inverse of a dense b x b block with partial pivoting.
bool invert_block(const double* a_in, int b, double* out) {
  std::vector<double> a(2 * b * b);
  for (int r = 0; r < b; ++r)
    for (int c = 0; c < b; ++c) {
      a[r * 2 * b + c] = a_in[r * b + c];
      a[r * 2 * b + b + c] = (r == c) ? 1.0 : 0.0;
    }
  for (int k = 0; k < b; ++k) {
    int p = k;
    double best = std::fabs(a[k * 2 * b + k]);
    for (int r = k + 1; r < b; ++r)
      if (std::fabs(a[r * 2 * b + k]) > best) { best = std::fabs(a[r * 2 * b + k]); p = r; }
    if (!(best > 0.0)) return false;
    if (p != k)
      for (int c = 0; c < 2 * b; ++c) std::swap(a[k * 2 * b + c], a[p * 2 * b + c]);
    const double ip = 1.0 / a[k * 2 * b + k];
    for (int c = 0; c < 2 * b; ++c) a[k * 2 * b + c] *= ip;
    for (int r = 0; r < b; ++r) {
      if (r == k) continue;
      const double f = a[r * 2 * b + k];
      if (f == 0.0) continue;
      for (int c = 0; c < 2 * b; ++c) a[r * 2 * b + c] -= f * a[k * 2 * b + c];
    }
  }
  for (int r = 0; r < b; ++r)
    for (int c = 0; c < b; ++c) out[r * b + c] = a[r * 2 * b + b + c];
  return true;
}

// y (br x nc) += A (br x bk) * B (bk x nc)
inline void gemm_acc(const double* A, const double* B, double* Y, int br, int bk, int nc, double alpha = 1.0) {
  for (int r = 0; r < br; ++r)
    for (int k = 0; k < bk; ++k) {
      const double a = alpha * A[r * bk + k];
      if (a == 0.0) continue;
      for (int c = 0; c < nc; ++c) Y[r * nc + c] += a * B[k * nc + c];
    }
}

// Y (nc x nd) += A^T (A: bk x nc) * B (bk x nd)
inline void gemm_tn_acc(const double* A, const double* B, double* Y, int bk, int nc, int nd) {
  for (int k = 0; k < bk; ++k)
    for (int r = 0; r < nc; ++r) {
      const double a = A[k * nc + r];
      if (a == 0.0) continue;
      for (int c = 0; c < nd; ++c) Y[r * nd + c] += a * B[k * nd + c];
    }
}

// Capped aggregation on the block-norm strength graph:
//  1. nodes in index order: a free node with at least one free neighbour is a
//     root; it takes up to cap-1 free neighbours, strongest ||A_ij||_F first
//     (ties: lower index);
//  2. each remaining node joins the aggregate of its strongest aggregated
//     neighbour (decided against the state after step 1);
//  3. the rest become singletons.
// Aggregates are renumbered component-major (stable).
// grow = false: a root takes its cap-1 strongest free neighbours (1-ring);
// grow = true:  the aggregate grows one node at a time by the strongest
//               connection from any member to a free node, so that on thin,
//               stretched elements it becomes a line across the wall.
int aggregate_capped(const HostBsr& A, const std::vector<int32_t>& comp, int cap, bool grow,
                     std::vector<int32_t>& agg) {
  const int n = A.n;
  const int bb = A.br * A.bc;
  std::vector<double> w(A.nb());
  for (int k = 0; k < A.nb(); ++k) {
    double s = 0.0;
    for (int q = 0; q < bb; ++q) s += A.v[(size_t)k * bb + q] * A.v[(size_t)k * bb + q];
    w[k] = std::sqrt(s);
  }
  agg.assign(n, -1);
  int na = 0;
  std::vector<std::pair<double, int>> cand;
  std::vector<int> members;
  for (int i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    cand.clear();
    for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      int j = A.ci[k];
      if (j != i && agg[j] < 0) cand.push_back({-w[k], j});
    }
    if (cand.empty()) continue;
    if (grow) {
      // grow by the strongest connection from any member to a free node
      agg[i] = na;
      members.assign(1, i);
      while ((int)members.size() < cap) {
        double best = -1.0;
        int bj = -1;
        for (int m : members)
          for (int k = A.rp[m]; k < A.rp[m + 1]; ++k) {
            const int j = A.ci[k];
            if (j == m || agg[j] >= 0) continue;
            if (w[k] > best || (w[k] == best && j < bj)) { best = w[k]; bj = j; }
          }
        if (bj < 0) break;
        agg[bj] = na;
        members.push_back(bj);
      }
      ++na;
      continue;
    }
    std::sort(cand.begin(), cand.end());
    agg[i] = na;
    for (int q = 0; q < (int)cand.size() && q < cap - 1; ++q) agg[cand[q].second] = na;
    ++na;
  }
  std::vector<int32_t> join(n, -1);
  for (int i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    double best = -1.0;
    for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      int j = A.ci[k];
      if (j != i && agg[j] >= 0 && w[k] > best) { best = w[k]; join[i] = agg[j]; }
    }
  }
  for (int i = 0; i < n; ++i)
    if (agg[i] < 0 && join[i] >= 0) agg[i] = join[i];
  for (int i = 0; i < n; ++i)
    if (agg[i] < 0) agg[i] = na++;
  std::vector<int32_t> acomp(na, 0);
  for (int i = 0; i < n; ++i) acomp[agg[i]] = comp[i];
  std::vector<int32_t> order(na);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return acomp[a] < acomp[b]; });
  std::vector<int32_t> newid(na);
  for (int k = 0; k < na; ++k) newid[order[k]] = k;
  for (int i = 0; i < n; ++i) agg[i] = newid[agg[i]];
  return na;
}

// Transpose of a block matrix (blocks transposed as well).
HostBsr transpose(const HostBsr& P) {
  HostBsr T;
  T.n = P.nc;
  T.nc = P.n;
  T.br = P.bc;
  T.bc = P.br;
  T.rp.assign(T.n + 1, 0);
  for (int k = 0; k < P.nb(); ++k) T.rp[P.ci[k] + 1]++;
  for (int I = 0; I < T.n; ++I) T.rp[I + 1] += T.rp[I];
  T.ci.resize(P.nb());
  const int bb = P.br * P.bc;
  T.v.resize((size_t)P.nb() * bb);
  std::vector<int32_t> fill(T.rp.begin(), T.rp.end() - 1);
  for (int i = 0; i < P.n; ++i)
    for (int k = P.rp[i]; k < P.rp[i + 1]; ++k) {
      const int I = P.ci[k];
      const int d = fill[I]++;
      T.ci[d] = i;
      for (int r = 0; r < P.br; ++r)
        for (int c = 0; c < P.bc; ++c) T.v[(size_t)d * bb + c * P.br + r] = P.v[(size_t)k * bb + r * P.bc + c];
    }
  return T;
}

// Pattern and pair plan of a sparse product built row by row: enum_row(i,
// emit) calls emit(column, x, y) for every pair (x, y) that contributes to
// output row i, in a fixed order.  The pairs are grouped by output column
// (ascending), each group keeping that order, so that a later sum over a
// group adds its products in the same order every time.  force_diag adds the
// diagonal column to every row, with no pairs if none reach it.  Rows are
// processed in contiguous chunks on the host's cores and the chunks are
// concatenated in row order: the result does not depend on the thread count.
template <typename EnumRow>
void pair_plan(int n_rows, bool force_diag, const EnumRow& enum_row, std::vector<int32_t>& rp,
               std::vector<int32_t>& ci, std::vector<int32_t>& ptr, std::vector<int32_t>& pairs) {
  struct Chunk {
    std::vector<int32_t> row_len, ci, grp_len, pairs;
  };
  constexpr int kRows = 512;
  const int n_chunks = (n_rows + kRows - 1) / kRows;
  std::vector<Chunk> chunks(n_chunks);
#pragma omp parallel for schedule(dynamic, 1)
  for (int c = 0; c < n_chunks; ++c) {
    Chunk& ch = chunks[c];
    struct Trip {
      int32_t col, x, y;
    };
    std::vector<Trip> trip;
    for (int i = c * kRows; i < std::min(n_rows, (c + 1) * kRows); ++i) {
      trip.clear();
      enum_row(i, [&](int32_t col, int32_t x, int32_t y) { trip.push_back({col, x, y}); });
      std::stable_sort(trip.begin(), trip.end(), [](const Trip& a, const Trip& b) { return a.col < b.col; });
      bool diag_open = force_diag;
      int len = 0;
      auto open_group = [&](int32_t col) {
        ch.ci.push_back(col);
        ch.grp_len.push_back(0);
        ++len;
      };
      for (size_t t = 0; t < trip.size(); ++t) {
        if (t == 0 || trip[t].col != trip[t - 1].col) {
          if (diag_open && trip[t].col >= i) {
            if (trip[t].col > i) open_group(i);
            diag_open = false;
          }
          open_group(trip[t].col);
        }
        ch.grp_len.back()++;
        ch.pairs.push_back(trip[t].x);
        ch.pairs.push_back(trip[t].y);
      }
      if (diag_open) open_group(i);
      ch.row_len.push_back(len);
    }
  }
  rp.assign(1, 0);
  ci.clear();
  ptr.assign(1, 0);
  pairs.clear();
  for (const Chunk& ch : chunks) {
    for (int l : ch.row_len) rp.push_back(rp.back() + l);
    ci.insert(ci.end(), ch.ci.begin(), ch.ci.end());
    for (int l : ch.grp_len) ptr.push_back(ptr.back() + l);
    pairs.insert(pairs.end(), ch.pairs.begin(), ch.pairs.end());
  }
}

double power_lambda(const HostBsr& A, const std::vector<double>& Dinv, const std::vector<uint8_t>& freem,
                    int steps) {
  const int b = A.br;
  const size_t N = (size_t)A.n * b;
  std::vector<double> v(N), y(N), t(b);
  uint64_t st = 0x9E3779B97F4A7C15ull;
  for (size_t k = 0; k < N; ++k) {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    v[k] = freem[k] ? ((double)(st >> 11) * (1.0 / 9007199254740992.0) - 0.5) : 0.0;
  }
  double lam = 1.0;
  for (int it = 0; it < steps; ++it) {
    double nv = 0.0;
    for (double x : v) nv += x * x;
    nv = std::sqrt(nv);
    if (nv == 0.0) return 1.0;
    for (double& x : v) x /= nv;
#pragma omp parallel for schedule(static) firstprivate(t)
    for (int i = 0; i < A.n; ++i) {
      std::fill(t.begin(), t.end(), 0.0);
      for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
        const int j = A.ci[k];
        for (int r = 0; r < b; ++r)
          for (int c = 0; c < b; ++c) t[r] += A.v[((size_t)k * b + r) * b + c] * v[(size_t)j * b + c];
      }
      for (int r = 0; r < b; ++r) {
        double s = 0.0;
        for (int c = 0; c < b; ++c) s += Dinv[((size_t)i * b + r) * b + c] * t[c];
        y[(size_t)i * b + r] = freem[(size_t)i * b + r] ? s : 0.0;
      }
    }
    double ny = 0.0;
    for (double x : y) ny += x * x;
    lam = std::sqrt(ny);
    v.swap(y);
  }
  return lam;
}

// Copy of A without the couplings between displacement-like unknowns (the
// first 3 of a 4-block, the first 6 of a 7-block) and pressure-like ones.
HostBsr filter_up(const HostBsr& A) {
  HostBsr F = A;
  const int b = A.br, nu = (b == 4) ? 3 : 6;
  for (int k = 0; k < F.nb(); ++k)
    for (int r = 0; r < b; ++r)
      for (int c = 0; c < b; ++c)
        if ((r < nu) != (c < nu)) F.v[((size_t)k * b + r) * b + c] = 0.0;
  return F;
}

void block_inverses(const HostBsr& A, std::vector<double>& Dinv) {
  const int b = A.br;
  Dinv.assign((size_t)A.n * b * b, 0.0);
  std::vector<double> blk(b * b);
  int bad = 0;   // 1: a row without a diagonal block, 2: a singular diagonal block
#pragma omp parallel for schedule(static) firstprivate(blk) reduction(| : bad)
  for (int i = 0; i < A.n; ++i) {
    int kd = -1;
    for (int k = A.rp[i]; k < A.rp[i + 1]; ++k)
      if (A.ci[k] == i) kd = k;
    if (kd < 0) {
      bad |= 1;
      continue;
    }
    for (int q = 0; q < b * b; ++q) blk[q] = A.v[(size_t)kd * b * b + q];
    if (!invert_block(blk.data(), b, &Dinv[(size_t)i * b * b])) bad |= 2;
  }
  if (bad & 1) throw ArgError("AMG level without a diagonal block");
  if (bad & 2) throw ArgError("singular diagonal block in AMG set-up");
}

}  // namespace

void build_sa_hierarchy(const HostBsr& A0, const std::vector<uint8_t>& free0, const double* X,
                        const std::vector<int32_t>& comp0, int coarse_max, int max_levels, int cap, bool filter,
                        std::vector<HostLevel>& levels, HostCoarse& coarse, bool grow, bool exact_candidates,
                        int power_steps) {
  levels.clear();
  levels.emplace_back();
  levels[0].A = A0;
  levels[0].free = free0;
  levels[0].comp = comp0;
  // level-0 near null space: per node a 4 x 7 block
  const int n0 = A0.n;
  int ncomp = comp0.empty() ? 1 : comp0.back() + 1;
  std::vector<double> ctr(3 * (size_t)ncomp, 0.0), cnt(ncomp, 0.0);
  for (int i = 0; i < n0; ++i) {
    for (int d = 0; d < 3; ++d) ctr[3 * comp0[i] + d] += X[3 * (size_t)i + d];
    cnt[comp0[i]] += 1.0;
  }
  for (int c = 0; c < ncomp; ++c)
    for (int d = 0; d < 3; ++d) ctr[3 * c + d] /= std::max(cnt[c], 1.0);
  std::vector<double> Bn((size_t)n0 * 4 * NS, 0.0);
  for (int i = 0; i < n0; ++i) {
    const double x = X[3 * (size_t)i] - ctr[3 * comp0[i]];
    const double y = X[3 * (size_t)i + 1] - ctr[3 * comp0[i] + 1];
    const double z = X[3 * (size_t)i + 2] - ctr[3 * comp0[i] + 2];
    double* B = &Bn[(size_t)i * 4 * NS];   // rows (ux, uy, uz, p), cols (tx, ty, tz, rx, ry, rz, p)
    B[0 * NS + 0] = 1.0;
    B[1 * NS + 1] = 1.0;
    B[2 * NS + 2] = 1.0;
    B[1 * NS + 3] = -z; B[2 * NS + 3] = y;     // e_x x r
    B[0 * NS + 4] = z;  B[2 * NS + 4] = -x;    // e_y x r
    B[0 * NS + 5] = -y; B[1 * NS + 5] = x;     // e_z x r
    B[3 * NS + 6] = 1.0;
  }
  for (int l = 0;; ++l) {
    HostLevel& L = levels[l];
    const HostBsr& A = L.A;
    const int n = A.n, b = A.br;
    block_inverses(A, L.Dinv);
    int max_run = 0, run = 0;
    for (int i = 0; i < n; ++i) {
      run = (i > 0 && L.comp[i] == L.comp[i - 1]) ? run + 1 : 1;
      max_run = std::max(max_run, run);
    }
    if (max_run <= coarse_max || l + 1 >= max_levels) break;
    std::vector<int32_t> agg;
    const int nc = aggregate_capped(A, L.comp, cap, grow, agg);
    if (nc >= n) break;
    // tentative prolongator (one b x 7 block per fine node) and coarse null space
    std::vector<std::vector<int32_t>> members(nc);
    for (int i = 0; i < n; ++i) members[agg[i]].push_back(i);
    HostBsr Pt;
    Pt.n = n;
    Pt.nc = nc;
    Pt.br = b;
    Pt.bc = NS;
    Pt.rp.resize(n + 1);
    Pt.ci.resize(n);
    Pt.v.assign((size_t)n * b * NS, 0.0);
    for (int i = 0; i <= n; ++i) Pt.rp[i] = i;
    for (int i = 0; i < n; ++i) Pt.ci[i] = agg[i];
    std::vector<double> Bc((size_t)nc * NS * NS, 0.0);
#pragma omp parallel for schedule(dynamic, 64)
    for (int I = 0; I < nc; ++I) {
      const auto& mem = members[I];
      const int rows = b * (int)mem.size();
      std::vector<double> Q((size_t)rows * NS, 0.0);
      for (int m = 0; m < (int)mem.size(); ++m)
        for (int d = 0; d < b; ++d)
          if (L.free[(size_t)mem[m] * b + d])
            for (int c = 0; c < NS; ++c) Q[(size_t)(m * b + d) * NS + c] = Bn[((size_t)mem[m] * b + d) * NS + c];
      double* R = &Bc[(size_t)I * NS * NS];
      // modified Gram-Schmidt with one re-orthogonalisation; dependent columns dropped
      for (int c = 0; c < NS; ++c) {
        double n_orig = 0.0;
        for (int r = 0; r < rows; ++r) n_orig += Q[(size_t)r * NS + c] * Q[(size_t)r * NS + c];
        n_orig = std::sqrt(n_orig);
        for (int pass = 0; pass < 2; ++pass)
          for (int k = 0; k < c; ++k) {
            double dot = 0.0;
            for (int r = 0; r < rows; ++r) dot += Q[(size_t)r * NS + k] * Q[(size_t)r * NS + c];
            R[k * NS + c] += dot;
            for (int r = 0; r < rows; ++r) Q[(size_t)r * NS + c] -= dot * Q[(size_t)r * NS + k];
          }
        double nn = 0.0;
        for (int r = 0; r < rows; ++r) nn += Q[(size_t)r * NS + c] * Q[(size_t)r * NS + c];
        nn = std::sqrt(nn);
        if (nn > 1e-10 * n_orig && nn > 0.0) {
          for (int r = 0; r < rows; ++r) Q[(size_t)r * NS + c] /= nn;
          R[c * NS + c] = nn;
        } else {
          // dependent column: no basis vector; with exact candidates its
          // projections on the earlier columns stay in R, so Q R = B still
          for (int r = 0; r < rows; ++r) Q[(size_t)r * NS + c] = 0.0;
          if (!exact_candidates)
            for (int k = 0; k < c; ++k) R[k * NS + c] = 0.0;
          R[c * NS + c] = 0.0;
        }
      }
      for (int m = 0; m < (int)mem.size(); ++m)
        for (int d = 0; d < b; ++d)
          for (int c = 0; c < NS; ++c) Pt.v[((size_t)mem[m] * b + d) * NS + c] = Q[(size_t)(m * b + d) * NS + c];
    }
    // P pattern = pattern of A P_t; W plan: the A blocks of row i whose column
    // lies in aggregate J feed P block (i, J)
    // prolongator smoothing operator: A itself, or (filter) A without the
    // displacement-pressure couplings
    HostBsr Af;
    std::vector<double> Dinv_f;
    if (filter) {
      Af = filter_up(A);
      block_inverses(Af, Dinv_f);
    }
    const HostBsr& As = filter ? Af : A;
    const std::vector<double>& Ds = filter ? Dinv_f : L.Dinv;
    const double lam = power_lambda(As, Ds, L.free, std::max(1, power_steps));
    const double wP = 4.0 / (3.0 * std::max(lam, 1e-300));
    const int pb = b * NS;
    HostBsr P;
    P.n = n;
    P.nc = nc;
    P.br = b;
    P.bc = NS;
    P.rp.assign(n + 1, 0);
    std::vector<int32_t> w_ptr{0}, w_k;
    {
      std::vector<int32_t> cols;
      for (int i = 0; i < n; ++i) {
        cols.clear();
        for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) cols.push_back(agg[A.ci[k]]);
        std::sort(cols.begin(), cols.end());
        cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
        for (int J : cols) {
          P.ci.push_back(J);
          for (int k = A.rp[i]; k < A.rp[i + 1]; ++k)
            if (agg[A.ci[k]] == J) w_k.push_back(k);
          w_ptr.push_back((int32_t)w_k.size());
        }
        P.rp[i + 1] = (int32_t)P.ci.size();
      }
    }
    P.v.assign((size_t)P.nb() * pb, 0.0);
    {
      std::vector<double> W(pb), tmp(pb);
#pragma omp parallel for schedule(dynamic, 256) firstprivate(W, tmp)
      for (int i = 0; i < n; ++i)
        for (int q = P.rp[i]; q < P.rp[i + 1]; ++q) {
          std::fill(W.begin(), W.end(), 0.0);
          for (int s = w_ptr[q]; s < w_ptr[q + 1]; ++s) {
            const int k = w_k[s];
            gemm_acc(&As.v[(size_t)k * b * b], &Pt.v[(size_t)A.ci[k] * pb], W.data(), b, b, NS);
          }
          std::fill(tmp.begin(), tmp.end(), 0.0);
          gemm_acc(&Ds[(size_t)i * b * b], W.data(), tmp.data(), b, b, NS, -wP);
          if (P.ci[q] == agg[i])
            for (int e = 0; e < pb; ++e) tmp[e] += Pt.v[(size_t)i * pb + e];
          for (int d = 0; d < b; ++d)
            for (int c = 0; c < NS; ++c)
              P.v[(size_t)q * pb + d * NS + c] = L.free[(size_t)i * b + d] ? tmp[d * NS + c] : 0.0;
        }
    }
    HostBsr PT = transpose(P);
    std::vector<int32_t> pt_src(P.nb());
    {
      std::vector<int32_t> fill(PT.rp.begin(), PT.rp.end() - 1);
      for (int i = 0; i < n; ++i)
        for (int q = P.rp[i]; q < P.rp[i + 1]; ++q) pt_src[fill[P.ci[q]]++] = q;
    }
    // AP = A P with its pair plan
    HostBsr AP;
    AP.n = n;
    AP.nc = nc;
    AP.br = b;
    AP.bc = NS;
    std::vector<int32_t> ap_ptr, ap_pairs;
    {
      pair_plan(n, false, [&](int i, auto&& emit) {
        for (int k = A.rp[i]; k < A.rp[i + 1]; ++k)
          for (int q = P.rp[A.ci[k]]; q < P.rp[A.ci[k] + 1]; ++q) emit(P.ci[q], k, q);
      }, AP.rp, AP.ci, ap_ptr, ap_pairs);
      AP.v.assign((size_t)AP.nb() * pb, 0.0);
#pragma omp parallel for schedule(dynamic, 1024)
      for (int r = 0; r < AP.nb(); ++r)
        for (int s = ap_ptr[r]; s < ap_ptr[r + 1]; ++s)
          gemm_acc(&A.v[(size_t)ap_pairs[2 * s] * b * b], &P.v[(size_t)ap_pairs[2 * s + 1] * pb],
                   &AP.v[(size_t)r * pb], b, b, NS);
    }
    // Ac = P^T (A P): coarse row I gathers the fine rows i of P column I
    HostBsr Ac;
    Ac.n = Ac.nc = nc;
    Ac.br = Ac.bc = NS;
    std::vector<int32_t> ac_ptr, ac_pairs;
    {
      pair_plan(nc, true, [&](int I, auto&& emit) {
        for (int t = PT.rp[I]; t < PT.rp[I + 1]; ++t) {
          const int i = PT.ci[t];
          for (int r = AP.rp[i]; r < AP.rp[i + 1]; ++r) emit(AP.ci[r], pt_src[t], r);
        }
      }, Ac.rp, Ac.ci, ac_ptr, ac_pairs);
      Ac.v.assign((size_t)Ac.nb() * NS * NS, 0.0);
#pragma omp parallel for schedule(dynamic, 1024)
      for (int B = 0; B < Ac.nb(); ++B)
        for (int s = ac_ptr[B]; s < ac_ptr[B + 1]; ++s)
          gemm_tn_acc(&P.v[(size_t)ac_pairs[2 * s] * pb], &AP.v[(size_t)ac_pairs[2 * s + 1] * pb],
                      &Ac.v[(size_t)B * NS * NS], b, NS, NS);
    }
    // coarse unknowns whose prolongator column is empty become identity rows
    HostLevel C;
    C.free.assign((size_t)nc * NS, 1);
    {
      std::vector<uint8_t> has(nc * NS, 0);
      for (int q = 0; q < P.nb(); ++q)
        for (int d = 0; d < b; ++d)
          for (int c = 0; c < NS; ++c)
            if (P.v[(size_t)q * pb + d * NS + c] != 0.0) has[(size_t)P.ci[q] * NS + c] = 1;
      for (int I = 0; I < nc; ++I) {
        int kd = -1;
        for (int k = Ac.rp[I]; k < Ac.rp[I + 1]; ++k)
          if (Ac.ci[k] == I) kd = k;
        for (int c = 0; c < NS; ++c)
          if (!has[(size_t)I * NS + c]) {
            Ac.v[((size_t)kd * NS + c) * NS + c] = 1.0;
            C.free[(size_t)I * NS + c] = 0;
            L.fix_blk.push_back(kd);
            L.fix_dof.push_back(c);
          }
      }
    }
    C.A = std::move(Ac);
    C.comp.assign(nc, 0);
    for (int i = 0; i < n; ++i) C.comp[agg[i]] = L.comp[i];
    L.agg = agg;
    L.Pt = std::move(Pt.v);
    L.omega_p = wP;
    L.P = std::move(P);
    L.PT = std::move(PT);
    L.pt_src = std::move(pt_src);
    L.w_ptr = std::move(w_ptr);
    L.w_k = std::move(w_k);
    L.AP = std::move(AP);
    L.ap_ptr = std::move(ap_ptr);
    L.ap_pairs = std::move(ap_pairs);
    L.ac_ptr = std::move(ac_ptr);
    L.ac_pairs = std::move(ac_pairs);
    Bn = std::move(Bc);
    levels.push_back(std::move(C));
  }
  // coarsest level: dense inverse per component
  HostLevel& Lc = levels.back();
  const int b = Lc.A.br;
  coarse.comp_ptr.assign(1, 0);
  for (int i = 1; i <= Lc.A.n; ++i)
    if (i == Lc.A.n || Lc.comp[i] != Lc.comp[i - 1]) coarse.comp_ptr.push_back(i);
  const int ncomp_c = (int)coarse.comp_ptr.size() - 1;
  coarse.inv_off.assign(ncomp_c, 0);
  int64_t tot = 0;
  coarse.max_dofs = 0;
  for (int c = 0; c < ncomp_c; ++c) {
    const int nd = b * (coarse.comp_ptr[c + 1] - coarse.comp_ptr[c]);
    coarse.inv_off[c] = tot;
    tot += (int64_t)nd * nd;
    coarse.max_dofs = std::max(coarse.max_dofs, nd);
  }
  // the dense inverses themselves are formed on the device every Newton step,
  // since the coarsest operator changes with K
  coarse.inv_size = tot;
}

}  // namespace fsi
