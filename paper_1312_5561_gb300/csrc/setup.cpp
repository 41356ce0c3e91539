// Host-side set-up of the solver: element colouring, the 4x4 block-CSR
// pattern, and the aggregation hierarchy of the AMG preconditioner.  These
// are one-time graph algorithms per mesh; all numerical work runs on the GPU.
#include <algorithm>
#include <numeric>

#include "internal.h"

namespace fsi {

int colour_elements(int n_nodes, int n_elems, const int32_t* tets, std::vector<int32_t>& colour) {
  // used[node] = bit set of colours already used around that node (64-bit
  // words, grown on demand).
  std::vector<std::vector<uint64_t>> used(n_nodes);
  colour.assign(n_elems, 0);
  int n_colours = 0;
  std::vector<uint64_t> taken;
  for (int e = 0; e < n_elems; ++e) {
    taken.clear();
    for (int a = 0; a < 4; ++a) {
      const auto& u = used[tets[4 * e + a]];
      if (u.size() > taken.size()) taken.resize(u.size(), 0);
      for (size_t w = 0; w < u.size(); ++w) taken[w] |= u[w];
    }
    int c = 0;
    for (;; ++c) {
      size_t w = c >> 6;
      if (w >= taken.size() || !((taken[w] >> (c & 63)) & 1)) break;
    }
    colour[e] = c;
    n_colours = std::max(n_colours, c + 1);
    for (int a = 0; a < 4; ++a) {
      auto& u = used[tets[4 * e + a]];
      size_t w = c >> 6;
      if (u.size() <= w) u.resize(w + 1, 0);
      u[w] |= uint64_t(1) << (c & 63);
    }
  }
  return n_colours;
}

void element_pattern(int n_nodes, int n_elems, const int32_t* tets, HostPattern& pat) {
  std::vector<std::vector<int32_t>> nb(n_nodes);
  for (int i = 0; i < n_nodes; ++i) nb[i].push_back(i);
  for (int e = 0; e < n_elems; ++e)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        if (a != b) nb[tets[4 * e + a]].push_back(tets[4 * e + b]);
  pat.row_ptr.assign(n_nodes + 1, 0);
  pat.col_idx.clear();
  for (int i = 0; i < n_nodes; ++i) {
    auto& v = nb[i];
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    pat.col_idx.insert(pat.col_idx.end(), v.begin(), v.end());
    pat.row_ptr[i + 1] = (int32_t)pat.col_idx.size();
  }
}

int32_t find_block(const HostPattern& pat, int32_t i, int32_t j) {
  auto b = pat.col_idx.begin() + pat.row_ptr[i];
  auto e = pat.col_idx.begin() + pat.row_ptr[i + 1];
  auto it = std::lower_bound(b, e, j);
  if (it == e || *it != j) return -1;
  return (int32_t)(it - pat.col_idx.begin());
}

// Aggregation (unsmoothed, block-identity prolongation), deterministic:
//  1. nodes in index order: a node whose neighbours are all unaggregated
//     becomes a root; it and its neighbours form a new aggregate;
//  2. every node left over joins the neighbouring aggregate it has the most
//     links to (ties: the lowest aggregate id);
//  3. nodes with no aggregated neighbour form singleton aggregates.
// Aggregates are then renumbered component-major (stable), so that the nodes
// of one component are contiguous on every level.
int aggregate_nodes(const HostPattern& pat, const std::vector<int32_t>& comp, std::vector<int32_t>& agg) {
  const int n = (int)pat.row_ptr.size() - 1;
  agg.assign(n, -1);
  int n_agg = 0;
  for (int i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    bool free_all = true;
    for (int k = pat.row_ptr[i]; k < pat.row_ptr[i + 1]; ++k)
      if (agg[pat.col_idx[k]] >= 0) { free_all = false; break; }
    if (!free_all) continue;
    for (int k = pat.row_ptr[i]; k < pat.row_ptr[i + 1]; ++k) agg[pat.col_idx[k]] = n_agg;
    ++n_agg;
  }
  std::vector<int32_t> join(n, -1);
  std::vector<int32_t> cand, cnt;
  for (int i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    cand.clear();
    for (int k = pat.row_ptr[i]; k < pat.row_ptr[i + 1]; ++k) {
      int a = agg[pat.col_idx[k]];
      if (a >= 0) cand.push_back(a);
    }
    if (cand.empty()) continue;
    std::sort(cand.begin(), cand.end());
    int best = -1, best_c = 0;
    for (size_t s = 0; s < cand.size();) {
      size_t t = s;
      while (t < cand.size() && cand[t] == cand[s]) ++t;
      int c = (int)(t - s);
      if (c > best_c) { best_c = c; best = cand[s]; }
      s = t;
    }
    join[i] = best;   // decided against the phase-1 state: order independent
  }
  for (int i = 0; i < n; ++i)
    if (agg[i] < 0 && join[i] >= 0) agg[i] = join[i];
  for (int i = 0; i < n; ++i)
    if (agg[i] < 0) agg[i] = n_agg++;
  // component-major renumbering
  std::vector<int32_t> acomp(n_agg, -1);
  for (int i = 0; i < n; ++i) acomp[agg[i]] = comp[i];
  std::vector<int32_t> order(n_agg);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return acomp[a] < acomp[b]; });
  std::vector<int32_t> newid(n_agg);
  for (int k = 0; k < n_agg; ++k) newid[order[k]] = k;
  for (int i = 0; i < n; ++i) agg[i] = newid[agg[i]];
  return n_agg;
}

void coarse_pattern(const HostPattern& fine, const std::vector<int32_t>& agg, int n_coarse,
                    HostPattern& coarse) {
  const int n = (int)fine.row_ptr.size() - 1;
  std::vector<std::vector<int32_t>> nb(n_coarse);
  for (int i = 0; i < n; ++i)
    for (int k = fine.row_ptr[i]; k < fine.row_ptr[i + 1]; ++k) nb[agg[i]].push_back(agg[fine.col_idx[k]]);
  coarse.row_ptr.assign(n_coarse + 1, 0);
  coarse.col_idx.clear();
  for (int I = 0; I < n_coarse; ++I) {
    auto& v = nb[I];
    v.push_back(I);
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    coarse.col_idx.insert(coarse.col_idx.end(), v.begin(), v.end());
    coarse.row_ptr[I + 1] = (int32_t)coarse.col_idx.size();
  }
}

}  // namespace fsi
