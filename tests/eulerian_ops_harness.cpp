// Test harness: runs the coupled loop's per-node and per-element kernel arithmetic
// (eulerian_ops.h) in plain loops over a grid read from binary files in argv[1], in the
// order the kernels apply it, and writes the results back there.
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "eulerian_ops.h"
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

// Node-transferred gradients of nq quantities q[nq][nn] into g[nq][nn][2].
void node_gradients(const pdfx::FemHost& m, const std::vector<int32_t>& tri, const std::vector<int32_t>& off,
                    const std::vector<int32_t>& lst, int nn, int ne, int nq, const std::vector<double>& q,
                    std::vector<double>& g) {
  std::vector<double> eg(2 * static_cast<size_t>(ne));
  g.assign(2 * static_cast<size_t>(nq) * nn, 0.0);
  for (int j = 0; j < nq; ++j) {
    for (int e = 0; e < ne; ++e)
      pdfx::eops::elem_gradient(e, m.fe.data(), tri.data(), q.data() + static_cast<size_t>(j) * nn, &eg[2 * e],
                                &eg[2 * e + 1]);
    for (int n = 0; n < nn; ++n)
      pdfx::eops::node_mean(n, off.data(), lst.data(), eg.data(), &g[2 * (static_cast<size_t>(j) * nn + n)],
                            &g[2 * (static_cast<size_t>(j) * nn + n) + 1]);
  }
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 4) return 1;
  dir = argv[1];
  const int nn = std::atoi(argv[2]), ne = std::atoi(argv[3]);
  const auto tri = load<int32_t>("tri", 3 * ne);
  pdfx::FemHost m;
  if (!pdfx::build_fem_host(nn, ne, tri, load<int8_t>("tag", 3 * ne), load<double>("vx", 3 * ne),
                            load<double>("vy", 3 * ne), load<double>("area2", ne), m))
    return 4;
  const auto F = load<double>("fields", 32 * static_cast<size_t>(nn));
  const auto kc = load<double>("consts", 12);   // C1 C2 Cv gamma5 CL Ceta CT nu, dt Cp
  const pdfx::WpConst k{kc[0], kc[1], kc[2], kc[3], kc[4], kc[5], kc[6], kc[7], m.cxi};
  const double dt = kc[8], Cp = kc[9];
  // node -> elements, ascending element id
  std::vector<int32_t> off(static_cast<size_t>(nn) + 1, 0), lst(3 * static_cast<size_t>(ne));
  for (int e = 0; e < ne; ++e)
    for (int a = 0; a < 3; ++a) off[tri[3 * e + a] + 1]++;
  for (int n = 0; n < nn; ++n) off[n + 1] += off[n];
  {
    std::vector<int32_t> fill(off.begin(), off.end() - 1);
    for (int e = 0; e < ne; ++e)
      for (int a = 0; a < 3; ++a) lst[fill[tri[3 * e + a]]++] = e;
  }
  // Eqs. 12-18 and Eq. 59
  std::vector<double> rhs(9 * static_cast<size_t>(nn)), L(nn), x(9 * static_cast<size_t>(nn), 0.0);
  std::vector<uint8_t> fixed(9 * static_cast<size_t>(nn));
  std::vector<int32_t> bad(2, 0);
  for (int n = 0; n < nn; ++n) {
    const double* f = F.data() + 32 * static_cast<size_t>(n);
    if (!pdfx::eops::wp_rhs_node(f, k, rhs.data() + n, static_cast<size_t>(nn), &L[n])) bad[0]++;
    if (!pdfx::eops::wp_bc_node(f, k, m.cls[n], m.nrm[2 * n], m.nrm[2 * n + 1], fixed.data() + n, x.data() + n,
                                static_cast<size_t>(nn)))
      bad[1]++;
  }
  std::vector<double> aval(m.col.size());
  for (size_t i = 0; i < aval.size(); ++i)
    aval[i] = pdfx::eops::wp_entry(m.cptr[i], m.cptr[i + 1], m.clist.data(), m.fe.data(), tri.data(), L.data());
  // Eq. 33's source and Eq. 61's flux from ustar[nn][3] and P[nn], then the load
  const auto ustar = load<double>("ustar", 3 * static_cast<size_t>(nn));
  const auto P = load<double>("P", nn);
  std::vector<double> q6(6 * static_cast<size_t>(nn)), g6, q2(2 * static_cast<size_t>(nn)), g2;
  for (int n = 0; n < nn; ++n) {
    const double* f = F.data() + 32 * static_cast<size_t>(n);
    q6[n] = ustar[3 * n];
    q6[nn + n] = ustar[3 * n + 1];
    q6[2 * static_cast<size_t>(nn) + n] = P[n];
    q6[3 * static_cast<size_t>(nn) + n] = f[23];
    q6[4 * static_cast<size_t>(nn) + n] = f[24];
    q6[5 * static_cast<size_t>(nn) + n] = f[26];
  }
  node_gradients(m, tri, off, lst, nn, ne, 6, q6, g6);
  for (int n = 0; n < nn; ++n) {
    q2[n] = g6[2 * (2 * static_cast<size_t>(nn) + n)];
    q2[nn + n] = g6[2 * (2 * static_cast<size_t>(nn) + n) + 1];
  }
  node_gradients(m, tri, off, lst, nn, ne, 2, q2, g2);
  std::vector<double> src(nn), flux(nn), b(nn);
  const size_t N2 = 2 * static_cast<size_t>(nn);
  for (int n = 0; n < nn; ++n) {
    const double lapP = g2[2 * n] + g2[N2 + 2 * n + 1];
    pdfx::eops::pressure_node(&g6[2 * n], &g6[N2 + 2 * n], &g6[2 * N2 + 2 * n], &g6[3 * N2 + 2 * n],
                              &g6[4 * N2 + 2 * n], &g6[5 * N2 + 2 * n], lapP, F.data() + 32 * static_cast<size_t>(n),
                              m.cls[n], m.nrm[2 * n], m.nrm[2 * n + 1], k.nu, dt, Cp, &src[n], &flux[n]);
  }
  for (int n = 0; n < nn; ++n)
    b[n] = pdfx::eops::pressure_load_node(n, m.row.data(), m.col.data(), m.mval.data(), src.data(), flux.data(),
                                          m.boff.data(), m.bnb.data(), m.blen.data());
  save("rhs", rhs); save("L", L); save("x", x); save("fixed", fixed); save("bad", bad);
  save("row", m.row); save("col", m.col); save("aval", aval);
  save("src", src); save("flux", flux); save("b", b);
  return 0;
}
