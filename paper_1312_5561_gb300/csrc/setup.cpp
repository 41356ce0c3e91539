// Host-side set-up of the solver: element colouring and the 4x4 block-CSR
// pattern (the aggregation hierarchy is built in amg_setup.cpp).  These are
// one-time graph algorithms per mesh; all numerical work runs on the GPU.
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

}  // namespace fsi
