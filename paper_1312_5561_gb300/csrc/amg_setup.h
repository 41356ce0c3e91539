// Host data structures of the smoothed-aggregation AMG set-up.
#pragma once

#include <cstdint>
#include <vector>

#include "internal.h"

namespace fsi {

// Block-sparse matrix on the host: n block rows, nc block columns, blocks
// br x bc stored row-major; column indices sorted within each row.
struct HostBsr {
  int n = 0, nc = 0, br = 0, bc = 0;
  std::vector<int32_t> rp, ci;
  std::vector<double> v;
  int nb() const { return (int)ci.size(); }
};

struct HostLevel {
  HostBsr A;                    // level operator at the reference state (level 0: reference tangent)
  std::vector<uint8_t> free;    // [n * br] 1 = free unknown
  std::vector<double> Dinv;     // [n][br][br] inverses of the diagonal blocks
  std::vector<int32_t> comp;    // component (segment) of each node
  // transfer to the next coarser level (absent on the coarsest level)
  std::vector<int32_t> agg;     // aggregate of each node
  std::vector<double> Pt;       // [n][br][7] tentative prolongator rows (one block per node)
  double omega_p = 0.0;         // prolongator smoothing weight 4 / (3 lambda_max(D^-1 A))
  HostBsr P, PT;                // smoothed prolongator and its transpose (reference values)
  std::vector<int32_t> pt_src;  // PT block t holds the transpose of P block pt_src[t]
  std::vector<int32_t> w_ptr, w_k;          // W = A Pt: A blocks summed into each P block
  HostBsr AP;                               // A P pattern
  std::vector<int32_t> ap_ptr, ap_pairs;    // A P: (A block, P block) pairs per AP block
  std::vector<int32_t> ac_ptr, ac_pairs;    // P^T (A P): (P block, AP block) pairs per coarse block
  std::vector<int32_t> fix_blk, fix_dof;    // coarse unknowns with no fine support: identity rows
};

struct HostCoarse {
  std::vector<int32_t> comp_ptr;   // node ranges of the components of the coarsest level
  std::vector<int64_t> inv_off;    // offsets of the dense inverses
  int64_t inv_size = 0;            // entries of all dense inverses together
  int max_dofs = 0;
};

// Builds levels[0..] from the level-0 matrix A0 (4x4 blocks), its free mask,
// the node coordinates X [n][3] and components comp0 (non-decreasing).
// filter: smooth the prolongator with A minus its displacement-pressure
// couplings (needed when inertia dominates the displacement block: the PSPG
// inertia coupling then blows up the pressure rows of D^-1 A).
// grow: aggregates grow along the strongest connections (see aggregate_capped).
// exact_candidates: the coarse near-null space is the whole R factor of each
// aggregate's QR (P_t B_c = B on the free unknowns); otherwise a column that
// depends on the earlier ones within an aggregate is dropped with its
// projections.
// power_steps: steps of the power iteration that estimates lambda_max(D^-1 A)
// for the prolongator smoothing weight 4 / (3 lambda).
void build_sa_hierarchy(const HostBsr& A0, const std::vector<uint8_t>& free0, const double* X,
                        const std::vector<int32_t>& comp0, int coarse_max, int max_levels, int cap, bool filter,
                        std::vector<HostLevel>& levels, HostCoarse& coarse, bool grow = false,
                        bool exact_candidates = false, int power_steps = 20);

}  // namespace fsi
