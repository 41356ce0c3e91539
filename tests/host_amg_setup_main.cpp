// Test driver for the host smoothed-aggregation set-up (no GPU): reads a 4x4
// block matrix, its free mask and the node coordinates from a directory, runs
// the set-up, and writes the arrays of levels 0 and 1 back as raw files
// together with an FNV-1a hash over every level array, so that a test can
// compare runs at different thread counts and check the products with scipy.
//
//   host_amg_setup_main <dir> <ring|grow> [exact] [filter] [steps=N]
//
// <dir>/dims.bin: int64 n, nb; rp.bin int32[n+1]; ci.bin int32[nb];
// v.bin double[nb*16]; free.bin uint8[n*4]; X.bin double[n*3].
#include <cstdio>
#include <fstream>
#include <stdexcept>
#include <string>
#include <vector>

#include "amg_setup.h"

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

template <typename T>
static uint64_t fnv(const std::vector<T>& v, uint64_t h) {
  const unsigned char* c = reinterpret_cast<const unsigned char*>(v.data());
  for (size_t i = 0; i < v.size() * sizeof(T); ++i) h = (h ^ c[i]) * 1099511628211ull;
  return h;
}

int main(int argc, char** argv) {
  if (argc < 3) {
    std::fprintf(stderr, "usage: %s <dir> <ring|grow>\n", argv[0]);
    return 2;
  }
  const std::string d = argv[1];
  const bool grow = std::string(argv[2]) == "grow";
  bool exact = false, filter = false;
  int steps = 20;
  for (int a = 3; a < argc; ++a) {
    const std::string f = argv[a];
    exact = exact || f == "exact";
    filter = filter || f == "filter";
    if (f.rfind("steps=", 0) == 0) steps = std::stoi(f.substr(6));
  }
  try {
    const auto dims = read_raw<int64_t>(d + "/dims.bin", 2);
    const int n = (int)dims[0], nb = (int)dims[1];
    HostBsr A;
    A.n = A.nc = n;
    A.br = A.bc = 4;
    A.rp = read_raw<int32_t>(d + "/rp.bin", (size_t)n + 1);
    A.ci = read_raw<int32_t>(d + "/ci.bin", (size_t)nb);
    A.v = read_raw<double>(d + "/v.bin", (size_t)nb * 16);
    const auto fr = read_raw<uint8_t>(d + "/free.bin", (size_t)n * 4);
    const auto X = read_raw<double>(d + "/X.bin", (size_t)n * 3);
    const std::vector<int32_t> comp(n, 0);
    std::vector<HostLevel> L;
    HostCoarse C;
    build_sa_hierarchy(A, fr, X.data(), comp, 16, 12, 8, filter, L, C, grow, exact, steps);
    uint64_t h = 1469598103934665603ull;
    for (const auto& l : L) {
      h = fnv(l.A.rp, h); h = fnv(l.A.ci, h); h = fnv(l.A.v, h); h = fnv(l.free, h); h = fnv(l.Dinv, h);
      h = fnv(l.agg, h); h = fnv(l.Pt, h); h = fnv(std::vector<double>{l.omega_p}, h);
      h = fnv(l.P.rp, h); h = fnv(l.P.ci, h); h = fnv(l.P.v, h); h = fnv(l.PT.v, h); h = fnv(l.pt_src, h);
      h = fnv(l.w_ptr, h); h = fnv(l.w_k, h); h = fnv(l.AP.ci, h); h = fnv(l.AP.v, h);
      h = fnv(l.ap_ptr, h); h = fnv(l.ap_pairs, h); h = fnv(l.ac_ptr, h); h = fnv(l.ac_pairs, h);
      h = fnv(l.fix_blk, h); h = fnv(l.fix_dof, h);
    }
    h = fnv(C.comp_ptr, h);
    h = fnv(C.inv_off, h);
    for (int k = 0; k < 3 && k < (int)L.size(); ++k) {
      const std::string p = d + "/l" + std::to_string(k) + "_";
      const HostLevel& l = L[k];
      write_raw(p + "A_rp.bin", l.A.rp);
      write_raw(p + "A_ci.bin", l.A.ci);
      write_raw(p + "A_v.bin", l.A.v);
      write_raw(p + "free.bin", l.free);
      write_raw(p + "Dinv.bin", l.Dinv);
      if (k + 1 < (int)L.size()) {
        write_raw(p + "agg.bin", l.agg);
        write_raw(p + "Pt.bin", l.Pt);
        write_raw(p + "P_rp.bin", l.P.rp);
        write_raw(p + "P_ci.bin", l.P.ci);
        write_raw(p + "P_v.bin", l.P.v);
        write_raw(p + "PT_rp.bin", l.PT.rp);
        write_raw(p + "PT_ci.bin", l.PT.ci);
        write_raw(p + "PT_v.bin", l.PT.v);
        write_raw(p + "pt_src.bin", l.pt_src);
        write_raw(p + "omega.bin", std::vector<double>{l.omega_p});
      }
    }
    std::printf("%zu %d %016llx\n", L.size(), L.size() > 1 ? L[1].A.n : 0, (unsigned long long)h);
  } catch (const ArgError& e) {
    std::fprintf(stderr, "%s\n", e.msg.c_str());
    return 1;
  } catch (const std::exception& e) {
    std::fprintf(stderr, "%s\n", e.what());
    return 1;
  }
  return 0;
}
