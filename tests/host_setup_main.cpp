// Test driver for the host mesh set-up (no GPU): element colouring, the
// node-block pattern and block lookup.
//
//   host_setup_main <dir>
//
// <dir>/dims.bin: int64 n_nodes, n_elems, n_queries; tets.bin int32[n_elems*4];
// queries.bin int32[n_queries*2] (i, j pairs).  Writes colour.bin
// int32[n_elems], rp.bin int32[n_nodes+1], ci.bin int32[nnz] and found.bin
// int32[n_queries] (block index or -1), and prints the number of colours.
#include <cstdio>
#include <fstream>
#include <stdexcept>
#include <string>
#include <vector>

#include "internal.h"

using namespace fsi;

template <typename T>
static std::vector<T> read_raw(const std::string& f, size_t n) {
  std::vector<T> v(n);
  std::ifstream in(f, std::ios::binary);
  in.read(reinterpret_cast<char*>(v.data()), (std::streamsize)(n * sizeof(T)));
  if (!in) throw std::runtime_error("short read: " + f);
  return v;
}

template <typename T>
static void write_raw(const std::string& f, const std::vector<T>& v) {
  std::ofstream out(f, std::ios::binary);
  out.write(reinterpret_cast<const char*>(v.data()), (std::streamsize)(v.size() * sizeof(T)));
}

int main(int argc, char** argv) {
  if (argc < 2) {
    std::fprintf(stderr, "usage: %s <dir>\n", argv[0]);
    return 2;
  }
  const std::string d = argv[1];
  try {
    const auto dims = read_raw<int64_t>(d + "/dims.bin", 3);
    const int nn = (int)dims[0], ne = (int)dims[1], nq = (int)dims[2];
    const auto tets = read_raw<int32_t>(d + "/tets.bin", (size_t)ne * 4);
    const auto q = read_raw<int32_t>(d + "/queries.bin", (size_t)nq * 2);
    std::vector<int32_t> colour;
    const int nc = colour_elements(nn, ne, tets.data(), colour);
    HostPattern pat;
    element_pattern(nn, ne, tets.data(), pat);
    std::vector<int32_t> found(nq);
    for (int k = 0; k < nq; ++k) found[k] = find_block(pat, q[2 * k], q[2 * k + 1]);
    write_raw(d + "/colour.bin", colour);
    write_raw(d + "/rp.bin", pat.row_ptr);
    write_raw(d + "/ci.bin", pat.col_idx);
    write_raw(d + "/found.bin", found);
    std::printf("%d\n", nc);
  } catch (const std::exception& e) {
    std::fprintf(stderr, "%s\n", e.what());
    return 1;
  }
  return 0;
}
