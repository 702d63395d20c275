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

// Conjugate gradients over C systems [C][nn] with the library's per-node and per-component
// functions, in the order of its kernels: the reduced load's norm, the zero solution of a
// zero load, the initial residual, then iterations (A d, alpha, update, beta, direction)
// until every component meets its stopping rule.  Returns the largest iteration count, or
// -1 after max_iter.
int pcg(const pdfx::FemHost& m, const std::vector<double>& val, const std::vector<double>& diag, int C, int nn,
        const std::vector<uint8_t>* fixed, const std::vector<double>& b, std::vector<double>& x, double tol,
        int max_iter) {
  using namespace pdfx::eops;
  const size_t N = static_cast<size_t>(C) * nn;
  std::vector<double> r(N), z(N), d(N), q(N), sc(static_cast<size_t>(C) * kPcgScalars, 0.0);
  auto fr = [&](size_t o) { return !fixed || !(*fixed)[o]; };
  auto spmv = [&](const std::vector<double>& v) {
    for (int c = 0; c < C; ++c)
      for (int n = 0; n < nn; ++n)
        q[static_cast<size_t>(c) * nn + n] = csr_row(n, m.row.data(), m.col.data(), val.data(), v.data() + static_cast<size_t>(c) * nn);
  };
  auto pass = [&](int mode, int step) {
    for (int c = 0; c < C; ++c) {
      double s0 = 0.0, s1 = 0.0;
      double* s = &sc[static_cast<size_t>(c) * kPcgScalars];
      for (int n = 0; n < nn; ++n) {
        const size_t o = static_cast<size_t>(c) * nn + n;
        pcg_node(mode, fr(o), diag[n], s[S_ALPHA], &b[o], &x[o], &r[o], &z[o], &d[o], &q[o], &s0, &s1);
      }
      pcg_scalars(step, s0, s1, tol, s);
    }
  };
  for (size_t o = 0; o < N; ++o) d[o] = fr(o) ? 0.0 : x[o];
  spmv(d);
  pass(0, 0);
  for (size_t o = 0; o < N; ++o) pcg_trivial(fr(o), &sc[(o / nn) * kPcgScalars], &x[o]);
  spmv(x);
  pass(1, 1);
  int done = 0;
  for (;;) {
    bool any = false;
    for (int c = 0; c < C; ++c) any |= sc[static_cast<size_t>(c) * kPcgScalars + S_ACTIVE] != 0.0;
    if (!any) break;
    if (done >= max_iter) return -1;
    const int chunk = max_iter - done < 16 ? max_iter - done : 16;
    for (int j = 0; j < chunk; ++j) {
      spmv(d);
      pass(2, 2);
      pass(3, 3);
      for (size_t o = 0; o < N; ++o) pcg_direction(fr(o), &sc[(o / nn) * kPcgScalars], z[o], &d[o]);
    }
    done += chunk;
  }
  int most = 0;
  for (int c = 0; c < C; ++c) {
    const int it = static_cast<int>(sc[static_cast<size_t>(c) * kPcgScalars + S_ITERS]);
    most = it > most ? it : most;
  }
  return most;
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
  // Eq. 12 solved from the zero initial guess (Dirichlet values set above): the load M rhs
  std::vector<double> bw(9 * static_cast<size_t>(nn)), adiag(nn), wp = x;
  for (int c = 0; c < 9; ++c)
    for (int n = 0; n < nn; ++n)
      bw[static_cast<size_t>(c) * nn + n] = pdfx::eops::csr_row(n, m.row.data(), m.col.data(), m.mval.data(),
                                                                 rhs.data() + static_cast<size_t>(c) * nn);
  for (int n = 0; n < nn; ++n) adiag[n] = aval[m.dpos[n]];
  const double tol = kc[10];
  std::vector<int32_t> iters(2, 0);
  iters[0] = pcg(m, aval, adiag, 9, nn, &fixed, bw, wp, tol, 100000);
  // Eq. 33 from the zero initial guess: load with its nodal mean removed, zero integral
  std::vector<double> dP(nn, 0.0), bl = b;
  double mean = 0.0;
  for (int n = 0; n < nn; ++n) mean += bl[n];
  for (int n = 0; n < nn; ++n) bl[n] -= mean / nn;
  iters[1] = pcg(m, m.kval, m.kdiag, 1, nn, nullptr, bl, dP, tol, 100000);
  double num = 0.0;
  for (int n = 0; n < nn; ++n) num += m.mlump[n] * dP[n];
  for (int n = 0; n < nn; ++n) dP[n] -= num / m.area;
  save("wp", wp); save("dP", dP); save("iters", iters);
  save("rhs", rhs); save("L", L); save("x", x); save("fixed", fixed); save("bad", bad);
  save("row", m.row); save("col", m.col); save("aval", aval);
  save("src", src); save("flux", flux); save("b", b);
  return 0;
}
