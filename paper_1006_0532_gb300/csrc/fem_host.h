// Galerkin FEM data of a triangle grid for the coupled loop's solves (Sect. 3.2), built on
// the host in FP64 from the grid's connectivity, edge tags and element vertices (x taken as
// the image nearest to vertex A, so periodic seams need nothing else).  Plain C++: the
// library uploads the result.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <utility>
#include <vector>

namespace pdfx {

struct FemHost {
  std::vector<int32_t> row, col, dpos;   // CSR of the node graph, each row's diagonal position
  std::vector<int32_t> cptr, clist;      // each entry's element contributions: 9 e + 3 a + b
  std::vector<double> fe;                // [ne][7] dN/dx (3), dN/dy (3), area (Eq. 40)
  std::vector<double> mval, kval, kdiag; // consistent mass, laplacian stiffness, its diagonal
  std::vector<double> mlump;             // [nn] integral of each shapefunction
  std::vector<int8_t> cls;               // [nn] 0 interior, 1 no-slip, 2 free-slip
  std::vector<double> nrm;               // [nn][2] outward unit normal of no-slip nodes
  std::vector<int32_t> boff, bnb;        // no-slip edges at each node: the other node
  std::vector<double> blen;              //   and the edge's length
  double area = 0.0;                     // domain area
  double cxi = 1.0;                      // Eq. 17: 1 + 1.3 n_i n_i (2.3 with a no-slip wall)
};

// tri[ne][3], tag[ne][3] (edge opposite vertex k: 1 no-slip, 2 free-slip), vx, vy [ne][3],
// area2[ne] (twice the signed area, positive).  Returns false for a node of no element.
inline bool build_fem_host(int nn, int ne, const std::vector<int32_t>& tri, const std::vector<int8_t>& tag,
                           const std::vector<double>& vxs, const std::vector<double>& vys,
                           const std::vector<double>& area2, FemHost& m) {
  const size_t N = static_cast<size_t>(nn), E = static_cast<size_t>(ne);
  // element data: Eq. 40's derivatives in the element's frame, and the area
  m.fe.assign(7 * E, 0.0);
  m.mlump.assign(N, 0.0);
  m.area = 0.0;
  for (int e = 0; e < ne; ++e) {
    const double* vx = &vxs[3 * static_cast<size_t>(e)];
    const double* vy = &vys[3 * static_cast<size_t>(e)];
    const double xBA = vx[1] - vx[0], yBA = vy[1] - vy[0];
    const double xCA = vx[2] - vx[0], yCA = vy[2] - vy[0];
    const double a2 = area2[e], inv = 1.0 / a2;
    double* g = &m.fe[7 * static_cast<size_t>(e)];
    g[0] = (-yCA + yBA) * inv; g[1] = yCA * inv; g[2] = -yBA * inv;
    g[3] = (xCA - xBA) * inv;  g[4] = -xCA * inv; g[5] = xBA * inv;
    g[6] = 0.5 * a2;
    m.area += g[6];
    for (int a = 0; a < 3; ++a) m.mlump[tri[3 * e + a]] += g[6] / 3.0;
  }
  // CSR pattern of the node graph (each node with its neighbours and itself)
  std::vector<std::vector<int32_t>> adj(N);
  for (int e = 0; e < ne; ++e)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) adj[tri[3 * e + a]].push_back(tri[3 * e + b]);
  m.row.assign(N + 1, 0);
  m.col.clear();
  for (int n = 0; n < nn; ++n) {
    if (adj[n].empty()) return false;   // a node of no element has no equation
    std::sort(adj[n].begin(), adj[n].end());
    adj[n].erase(std::unique(adj[n].begin(), adj[n].end()), adj[n].end());
    m.row[n + 1] = m.row[n] + static_cast<int32_t>(adj[n].size());
  }
  const int nnz = m.row[nn];
  m.col.reserve(static_cast<size_t>(nnz));
  for (int n = 0; n < nn; ++n) m.col.insert(m.col.end(), adj[n].begin(), adj[n].end());
  auto entry = [&](int r, int cc) {
    return static_cast<int32_t>(std::lower_bound(m.col.begin() + m.row[r], m.col.begin() + m.row[r + 1], cc) -
                                m.col.begin());
  };
  m.dpos.assign(N, 0);
  for (int n = 0; n < nn; ++n) m.dpos[n] = entry(n, n);
  // contributions of each entry, ascending element
  m.cptr.assign(static_cast<size_t>(nnz) + 1, 0);
  m.clist.assign(9 * E, 0);
  std::vector<int32_t> epos(9 * E);
  for (int e = 0; e < ne; ++e)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const int32_t k = entry(tri[3 * e + a], tri[3 * e + b]);
        epos[9 * static_cast<size_t>(e) + 3 * a + b] = k;
        m.cptr[k + 1]++;
      }
  for (int k = 0; k < nnz; ++k) m.cptr[k + 1] += m.cptr[k];
  {
    std::vector<int32_t> fill(m.cptr.begin(), m.cptr.end() - 1);
    for (int e = 0; e < ne; ++e)
      for (int ab = 0; ab < 9; ++ab) m.clist[fill[epos[9 * static_cast<size_t>(e) + ab]]++] = 9 * e + ab;
  }
  // the fixed matrices: consistent mass and laplacian stiffness
  m.mval.assign(static_cast<size_t>(nnz), 0.0);
  m.kval.assign(static_cast<size_t>(nnz), 0.0);
  for (int k = 0; k < nnz; ++k)
    for (int j = m.cptr[k]; j < m.cptr[k + 1]; ++j) {
      const int e = m.clist[j] / 9, a = (m.clist[j] % 9) / 3, b = m.clist[j] % 3;
      const double* g = &m.fe[7 * static_cast<size_t>(e)];
      m.mval[k] += g[6] / 12.0 * (a == b ? 2.0 : 1.0);
      m.kval[k] += g[6] * (g[a] * g[b] + g[3 + a] * g[3 + b]);
    }
  m.kdiag.assign(N, 0.0);
  for (int n = 0; n < nn; ++n) m.kdiag[n] = m.kval[m.dpos[n]];
  // boundary classes, outward normals of no-slip nodes, no-slip edges at each node
  m.cls.assign(N, 0);
  m.nrm.assign(2 * N, 0.0);
  std::vector<std::vector<std::pair<int32_t, double>>> bed(N);
  bool wall = false;
  for (int e = 0; e < ne; ++e) {
    const double* vx = &vxs[3 * static_cast<size_t>(e)];
    const double* vy = &vys[3 * static_cast<size_t>(e)];
    for (int k = 0; k < 3; ++k) {
      const int t = tag[3 * static_cast<size_t>(e) + k];
      if (t != 1 && t != 2) continue;
      const int ia = (k + 1) % 3, ib = (k + 2) % 3;
      const int32_t na = tri[3 * e + ia], nb = tri[3 * e + ib];
      const double tx = vx[ib] - vx[ia], ty = vy[ib] - vy[ia];
      const double len = std::sqrt(tx * tx + ty * ty);
      double mx = -ty / len, my = tx / len;   // toward vertex k: into the domain
      if ((vx[k] - vx[ia]) * mx + (vy[k] - vy[ia]) * my < 0.0) { mx = -mx; my = -my; }
      for (const int32_t n : {na, nb}) {
        if (t == 1) {
          m.cls[n] = 1;
          m.nrm[2 * static_cast<size_t>(n)] -= mx;
          m.nrm[2 * static_cast<size_t>(n) + 1] -= my;
        } else if (m.cls[n] == 0) {
          m.cls[n] = 2;
        }
      }
      if (t == 1) {
        wall = true;
        bed[na].push_back({nb, len});
        bed[nb].push_back({na, len});
      }
    }
  }
  for (int n = 0; n < nn; ++n) {
    if (m.cls[n] != 1) continue;
    const double l = std::hypot(m.nrm[2 * static_cast<size_t>(n)], m.nrm[2 * static_cast<size_t>(n) + 1]);
    if (l > 0.0) { m.nrm[2 * static_cast<size_t>(n)] /= l; m.nrm[2 * static_cast<size_t>(n) + 1] /= l; }
  }
  m.boff.assign(N + 1, 0);
  m.bnb.clear();
  m.blen.clear();
  for (int n = 0; n < nn; ++n) {
    for (const auto& pr : bed[n]) { m.bnb.push_back(pr.first); m.blen.push_back(pr.second); }
    m.boff[n + 1] = static_cast<int32_t>(m.bnb.size());
  }
  m.cxi = 1.0 + 1.3 * (wall ? 1.0 : 0.0);   // Eq. 17 with n_i n_i of a unit normal
  return true;
}

}  // namespace pdfx
