// Test harness: runs the library's host-side FEM builder (fem_host.h) on a grid read from
// binary files in the directory argv[1] and writes its arrays back there.
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "fem_host.h"

namespace {

std::string dir;

template <typename T>
std::vector<T> load(const char* name, size_t n) {
  std::vector<T> v(n);
  FILE* f = std::fopen((dir + "/" + name).c_str(), "rb");
  if (!f || std::fread(v.data(), sizeof(T), n, f) != n) std::exit(2);
  std::fclose(f);
  return v;
}

template <typename T>
void save(const char* name, const std::vector<T>& v) {
  FILE* f = std::fopen((dir + "/" + name).c_str(), "wb");
  if (!f) std::exit(3);
  std::fwrite(v.data(), sizeof(T), v.size(), f);
  std::fclose(f);
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 4) return 1;
  dir = argv[1];
  const int nn = std::atoi(argv[2]), ne = std::atoi(argv[3]);
  pdfx::FemHost m;
  if (!pdfx::build_fem_host(nn, ne, load<int32_t>("tri", 3 * ne), load<int8_t>("tag", 3 * ne),
                            load<double>("vx", 3 * ne), load<double>("vy", 3 * ne), load<double>("area2", ne), m))
    return 4;
  save("row", m.row); save("col", m.col); save("dpos", m.dpos); save("cptr", m.cptr); save("clist", m.clist);
  save("mval", m.mval); save("kval", m.kval); save("kdiag", m.kdiag); save("mlump", m.mlump);
  save("cls", m.cls); save("nrm", m.nrm); save("boff", m.boff); save("bnb", m.bnb); save("blen", m.blen);
  save("scal", std::vector<double>{m.area, m.cxi});
  return 0;
}
