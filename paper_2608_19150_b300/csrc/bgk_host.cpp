// Host-side set-up of the sweep solver: mesh connectivity and face normals, the
// Gauss-Legendre velocity grid, and the breaking of sweep-graph cycles.
//
// Compiled with -ffp-contract=off: the face normals and the signs of v_j . N decide the
// sweep graphs (Sec. 4.1), which must come out bit-identical on the host and the device.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "bgk_internal.h"
#include "bgk_tables.h"

namespace bgk {

namespace {

// Canonical normal of a face from its vertex ids sorted ascending (2D: edge (g0, g1);
// 3D: triangle (g0, g1, g2)).  2D: t = x1 - x0, N = (t_y, -t_x); 3D: N = (e1 x e2) / 2.
// One rounding per operation, no fused multiply-add.  |N| is the face measure.
void canonical_normal(const double* xyz, int dim, const int* g, double* N) {
  const double* p0 = xyz + (size_t)g[0] * dim;
  const double* p1 = xyz + (size_t)g[1] * dim;
  if (dim == 2) {
    double tx = p1[0] - p0[0];
    double ty = p1[1] - p0[1];
    N[0] = ty;
    N[1] = -tx;
    return;
  }
  const double* p2 = xyz + (size_t)g[2] * dim;
  double e1[3], e2[3];
  for (int i = 0; i < 3; ++i) {
    e1[i] = p1[i] - p0[i];
    e2[i] = p2[i] - p0[i];
  }
  double a = e1[1] * e2[2], b = e1[2] * e2[1];
  double c = e1[2] * e2[0], d = e1[0] * e2[2];
  double e = e1[0] * e2[1], f = e1[1] * e2[0];
  N[0] = (a - b) * 0.5;
  N[1] = (c - d) * 0.5;
  N[2] = (e - f) * 0.5;
}

struct FaceKey {
  int g[3];
  bool operator<(const FaceKey& o) const {
    return std::lexicographical_compare(g, g + 3, o.g, o.g + 3);
  }
};

// identity of a local node: a vertex id, or the sorted vertex pair of an edge midpoint
// (nvc: vertices per cell; every node of a Q1 quadrilateral is a vertex)
std::pair<int, int> node_id(const int* cv, int nvc, int a) {
  if (a < nvc) return {cv[a], -1};
  int k = a - 3, l = (k + 1) % 3;
  return {std::min(cv[k], cv[l]), std::max(cv[k], cv[l])};
}

}  // namespace

int finish_host_mesh(const int32_t* CV, int nv, HostMesh& hm);

// Q1 quadrilaterals (Sec. 3.1): four vertices per cell in order around it, nodes at the
// vertices, face i the edge from vertex i to vertex i+1.  Only parallelograms: their
// bilinear map is affine, so the local matrices are the reference tables combined with
// the face normals (ElemQ1Quad); a cell with x0 + x2 != x1 + x3 is rejected.
int build_host_mesh_quad(const bgk_mesh* m, HostMesh& hm) {
  if (m->dim != 2 || m->k_x != 1) return BGK_E_INVALID;
  if (m->n_cells <= 0 || m->n_vertices <= 0 || !m->xyz || !m->cell_vertices) return BGK_E_INVALID;
  if (m->n_cells > (int)kCellMask) return BGK_E_INVALID;
  const int d = 2, nv = 4;
  hm.dim = 2;
  hm.kx = 1;
  hm.quad = true;
  hm.nf = 4;
  hm.ndof = 4;
  hm.fd = 2;
  hm.ncell = m->n_cells;
  hm.nvert = m->n_vertices;
  hm.geo_stride = 10;  // N_0 .. N_3, 1/|K|, padding
  hm.geo.assign((size_t)hm.ncell * hm.geo_stride, 0.0);
  hm.nbr.assign((size_t)hm.ncell * 4, INT32_MIN);
  hm.nbr_face.assign((size_t)hm.ncell * 4, -1);
  hm.perm.assign(hm.ncell, 0);
  const double* X = m->xyz;
  const int32_t* CV = m->cell_vertices;
  std::map<FaceKey, std::pair<int, int>> open;
  double min_vol = INFINITY;
  for (int c = 0; c < hm.ncell; ++c) {
    const int* cv = CV + (size_t)c * nv;
    for (int a = 0; a < nv; ++a)
      if (cv[a] < 0 || cv[a] >= hm.nvert) return BGK_E_INVALID;
    const double* p[4];
    for (int a = 0; a < 4; ++a) p[a] = X + 2 * (size_t)cv[a];
    // parallelogram: x0 + x2 = x1 + x3 (relative to the longest edge)
    double hmax = 0.0;
    for (int a = 0; a < 4; ++a) {
      const double ex = p[(a + 1) % 4][0] - p[a][0], ey = p[(a + 1) % 4][1] - p[a][1];
      hmax = std::max(hmax, std::sqrt(ex * ex + ey * ey));
    }
    for (int al = 0; al < 2; ++al)
      if (!(std::fabs(p[0][al] + p[2][al] - p[1][al] - p[3][al]) <= 1e-12 * hmax)) return BGK_E_INVALID;
    const double vol = std::fabs((p[1][0] - p[0][0]) * (p[3][1] - p[0][1]) - (p[1][1] - p[0][1]) * (p[3][0] - p[0][0]));
    if (!(vol > 0.0) || !std::isfinite(vol)) return BGK_E_INVALID;
    min_vol = std::min(min_vol, vol);
    double* G = hm.geo.data() + (size_t)c * hm.geo_stride;
    G[hm.nf * d] = 1.0 / vol;
    for (int f = 0; f < 4; ++f) {
      int g[3] = {cv[f], cv[(f + 1) % 4], -1};
      std::sort(g, g + 2);
      double N[3] = {0, 0, 0};
      canonical_normal(X, d, g, N);
      // outward: a vertex off the face lies on the negative side
      const int off = cv[(f + 2) % 4];
      double sd = 0.0;
      for (int al = 0; al < d; ++al) sd += (X[(size_t)off * d + al] - X[(size_t)g[0] * d + al]) * N[al];
      if (sd == 0.0) return BGK_E_INVALID;
      const double sg = sd < 0.0 ? 1.0 : -1.0;
      for (int al = 0; al < d; ++al) G[f * d + al] = sg * N[al];
      FaceKey key{{g[0], g[1], -1}};
      auto it = open.find(key);
      if (it == open.end()) {
        open.emplace(key, std::make_pair(c, f));
      } else {
        int c2 = it->second.first, f2 = it->second.second;
        if (c2 == c) return BGK_E_INVALID;
        if (hm.nbr[(size_t)c2 * 4 + f2] != INT32_MIN) return BGK_E_INVALID;
        const double* G2 = hm.geo.data() + (size_t)c2 * hm.geo_stride + f2 * d;
        double dn = 0.0;
        for (int al = 0; al < d; ++al) dn += G[f * d + al] * G2[al];
        if (!(dn < 0.0)) return BGK_E_INVALID;
        hm.nbr[(size_t)c * 4 + f] = c2;
        hm.nbr_face[(size_t)c * 4 + f] = f2;
        hm.nbr[(size_t)c2 * 4 + f2] = c;
        hm.nbr_face[(size_t)c2 * 4 + f2] = f;
        open.erase(it);
      }
    }
  }
  hm.min_vol = min_vol;
  return finish_host_mesh(CV, nv, hm);
}

int build_host_mesh(const bgk_mesh* m, HostMesh& hm) {
  if (!m || (m->dim != 2 && m->dim != 3) || (m->k_x != 1 && m->k_x != 2) || (m->k_x == 2 && m->dim != 2))
    return BGK_E_INVALID;
  if (m->shape != 0 && m->shape != 1) return BGK_E_INVALID;
  if (m->shape == 1) return build_host_mesh_quad(m, hm);
  if (m->n_cells <= 0 || m->n_vertices <= 0 || !m->xyz || !m->cell_vertices) return BGK_E_INVALID;
  if (m->n_cells > (int)kCellMask) return BGK_E_INVALID;
  const int d = m->dim, nv = d + 1;
  hm.dim = d;
  hm.kx = m->k_x;
  hm.nf = d + 1;
  hm.ndof = (m->k_x == 1) ? d + 1 : 6;
  hm.fd = (m->k_x == 1) ? d : 3;
  hm.ncell = m->n_cells;
  hm.nvert = m->n_vertices;
  hm.geo_stride = d == 2 ? 8 : 16;
  hm.geo.assign((size_t)hm.ncell * hm.geo_stride, 0.0);
  hm.nbr.assign((size_t)hm.ncell * 4, INT32_MIN);
  hm.nbr_face.assign((size_t)hm.ncell * 4, -1);
  hm.perm.assign(hm.ncell, 0);
  const double* X = m->xyz;
  const int32_t* CV = m->cell_vertices;
  std::map<FaceKey, std::pair<int, int>> open;  // face -> (cell, face) seen once
  double min_vol = INFINITY;
  for (int c = 0; c < hm.ncell; ++c) {
    const int* cv = CV + (size_t)c * nv;
    for (int a = 0; a < nv; ++a)
      if (cv[a] < 0 || cv[a] >= hm.nvert) return BGK_E_INVALID;
    // volume from the vertex coordinates
    double vol;
    if (d == 2) {
      const double *a = X + 2 * (size_t)cv[0], *b = X + 2 * (size_t)cv[1], *cc = X + 2 * (size_t)cv[2];
      vol = 0.5 * std::fabs((b[0] - a[0]) * (cc[1] - a[1]) - (b[1] - a[1]) * (cc[0] - a[0]));
    } else {
      const double *a = X + 3 * (size_t)cv[0], *b = X + 3 * (size_t)cv[1], *cc = X + 3 * (size_t)cv[2],
                   *e = X + 3 * (size_t)cv[3];
      double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
      double v[3] = {cc[0] - a[0], cc[1] - a[1], cc[2] - a[2]};
      double w[3] = {e[0] - a[0], e[1] - a[1], e[2] - a[2]};
      vol = std::fabs(u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) +
                      u[2] * (v[0] * w[1] - v[1] * w[0])) / 6.0;
    }
    if (!(vol > 0.0) || !std::isfinite(vol)) return BGK_E_INVALID;
    min_vol = std::min(min_vol, vol);
    double* G = hm.geo.data() + (size_t)c * hm.geo_stride;
    G[hm.nf * d] = 1.0 / vol;
    for (int f = 0; f < hm.nf; ++f) {
      int g[3] = {-1, -1, -1}, k = 0;
      for (int a = 0; a < nv; ++a)
        if (a != f) g[k++] = cv[a];
      std::sort(g, g + d);
      double N[3] = {0, 0, 0};
      canonical_normal(X, d, g, N);
      // orient outward: the opposite vertex lies on the negative side
      double s = 0.0;
      for (int al = 0; al < d; ++al) s += (X[(size_t)cv[f] * d + al] - X[(size_t)g[0] * d + al]) * N[al];
      if (s == 0.0) return BGK_E_INVALID;
      double sg = s < 0.0 ? 1.0 : -1.0;
      for (int al = 0; al < d; ++al) G[f * d + al] = sg * N[al];
      FaceKey key{{g[0], g[1], d == 3 ? g[2] : -1}};
      auto it = open.find(key);
      if (it == open.end()) {
        open.emplace(key, std::make_pair(c, f));
      } else {
        int c2 = it->second.first, f2 = it->second.second;
        if (c2 == c) return BGK_E_INVALID;
        if (hm.nbr[(size_t)c2 * 4 + f2] != INT32_MIN) return BGK_E_INVALID;  // non-manifold
        // the two outward normals of a shared face are opposite unless the cells overlap
        const double* G2 = hm.geo.data() + (size_t)c2 * hm.geo_stride + f2 * d;
        double dn = 0.0;
        for (int al = 0; al < d; ++al) dn += G[f * d + al] * G2[al];
        if (!(dn < 0.0)) return BGK_E_INVALID;  // folded
        hm.nbr[(size_t)c * 4 + f] = c2;
        hm.nbr_face[(size_t)c * 4 + f] = f2;
        hm.nbr[(size_t)c2 * 4 + f2] = c;
        hm.nbr_face[(size_t)c2 * 4 + f2] = f;
        open.erase(it);
      }
    }
  }
  hm.min_vol = min_vol;
  return finish_host_mesh(CV, nv, hm);
}

// Boundary faces (numbered in (cell, face) order), their nodes and sides, and the node
// permutations across interior faces.
int finish_host_mesh(const int32_t* CV, int nv, HostMesh& hm) {
  const int d = hm.dim;
  int nb = 0;
  for (int c = 0; c < hm.ncell; ++c)
    for (int f = 0; f < hm.nf; ++f)
      if (hm.nbr[(size_t)c * 4 + f] == INT32_MIN) hm.nbr[(size_t)c * 4 + f] = -(++nb);
  hm.nbface = nb;
  hm.bnode.assign((size_t)nb * hm.fd, 0);
  hm.bside.assign((size_t)nb, -1);
  for (int c = 0; c < hm.ncell; ++c)
    for (int f = 0; f < hm.nf; ++f) {
      const int n2 = hm.nbr[(size_t)c * 4 + f];
      if (n2 >= 0) continue;
      const double* N = hm.geo.data() + (size_t)c * hm.geo_stride + f * d;
      double len = 0.0;
      for (int al = 0; al < d; ++al) len += N[al] * N[al];
      len = std::sqrt(len);
      for (int al = 0; al < d; ++al) {
        bool aligned = true;
        for (int be = 0; be < d; ++be)
          if (be != al && !(std::fabs(N[be]) <= 1e-10 * len)) aligned = false;
        if (aligned) hm.bside[(size_t)(-n2 - 1)] = (int8_t)(2 * al + (N[al] > 0.0 ? 1 : 0));
      }
    }
  for (int c = 0; c < hm.ncell; ++c) {
    const int* cv = CV + (size_t)c * nv;
    uint64_t pm = 0;
    for (int f = 0; f < hm.nf; ++f) {
      int n2 = hm.nbr[(size_t)c * 4 + f];
      for (int k = 0; k < hm.fd; ++k) {
        int a = hm.quad ? ElemQ1Quad::fn(f, k)
                        : hm.kx == 1 ? (d == 2 ? ElemP1Tri::fn(f, k) : ElemP1Tet::fn(f, k)) : ElemP2Tri::fn(f, k);
        if (n2 < 0) {
          hm.bnode[(size_t)(-n2 - 1) * hm.fd + k] = c * hm.ndof + a;
          continue;
        }
        auto id = node_id(cv, nv, a);
        const int* cv2 = CV + (size_t)n2 * nv;
        int match = -1;
        for (int b = 0; b < hm.ndof; ++b)
          if (node_id(cv2, nv, b) == id) { match = b; break; }
        if (match < 0) return BGK_E_INVALID;  // non-conforming
        pm |= (uint64_t)match << (16 * f + 4 * k);
      }
    }
    hm.perm[c] = pm;
  }
  return BGK_OK;
}

int build_vgrid(int dim, int N, int kv, double L, VGrid& g) {
  if ((dim != 2 && dim != 3) || kv < 1 || kv > kMaxKv || N < kv + 1 || N > kMaxN1D || N % (kv + 1) != 0 ||
      !(L > 0.0))
    return BGK_E_INVALID;
  std::memset(&g, 0, sizeof(g));
  g.dim = dim;
  g.N = N;
  g.kv = kv;
  g.np = kv + 1;
  g.ncl = N / g.np;
  g.nv = 1;
  for (int i = 0; i < dim; ++i) g.nv *= N;
  g.L = L;
  g.h = 2.0 * L / g.ncl;
  // Gauss-Legendre nodes by Newton's method on P_np (three-term recurrence)
  const int n = g.np;
  double xi[kMaxKv + 1], wi[kMaxKv + 1];
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double pn = n == 1 ? z : p1, pm = n == 1 ? 1.0 : p0;
      dp = n * (z * pn - pm) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    xi[n - 1 - i] = z;
    wi[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  for (int cl = 0; cl < g.ncl; ++cl)
    for (int k = 0; k < n; ++k) {
      double mid = -L + (cl + 0.5) * g.h;
      g.x[cl * n + k] = mid + 0.5 * g.h * xi[k];
      g.w[cl * n + k] = 0.5 * g.h * wi[k];
    }
  for (int m = 0; m < N; ++m) {
    g.wx[m] = g.w[m] * g.x[m];
    g.wxx[m] = g.w[m] * g.x[m] * g.x[m];
    const double src3[3] = {g.w[m], g.wx[m], g.wxx[m]};
    for (int k = 0; k < 3; ++k) {
      g.wh[k][m] = (float)src3[k];
      g.wl[k][m] = (float)(src3[k] - (double)g.wh[k][m]);
    }
  }
  // Lagrange basis on the reference cell: monomial coefficients by expansion
  for (int k = 0; k < n; ++k) {
    double c[kMaxKv + 2] = {1.0};
    int deg = 0;
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      double den = xi[k] - xi[i];
      for (int p = deg + 1; p >= 0; --p) c[p] = ((p > 0 ? c[p - 1] : 0.0) - xi[i] * c[p]) / den;
      ++deg;
    }
    for (int p = 0; p < n; ++p) g.lag[k][p] = c[p];
  }
  for (int cl = 0; cl <= g.ncl; ++cl) g.bnd_f[cl] = (float)(-L + cl * g.h);
  for (int cl = 0; cl < g.ncl; ++cl) g.mid_f[cl] = (float)(-L + (cl + 0.5) * g.h);
  for (int m = 0; m < N; ++m) g.iw_f[m] = (float)(1.0 / g.w[m]);
  for (int k = 0; k <= kMaxKv; ++k)
    for (int p = 0; p <= kMaxKv; ++p) g.lag_f[k][p] = (float)g.lag[k][p];
  g.hh_f = (float)(0.5 * g.h);
  return BGK_OK;
}

int host_face_sign(const HostMesh& hm, const VGrid& g, int j, int c, int f) {
  const double* N = hm.geo.data() + (size_t)c * hm.geo_stride + f * hm.dim;
  double v[3];
  int jj = j;
  for (int al = hm.dim - 1; al >= 0; --al) {
    v[al] = g.x[jj % g.N];
    jj /= g.N;
  }
  double s = v[0] * N[0];
  double t = v[1] * N[1];
  s = s + t;
  if (hm.dim == 3) {
    t = v[2] * N[2];
    s = s + t;
  }
  return s > 0.0 ? 1 : (s < 0.0 ? -1 : 0);
}

int host_break_cycles(const HostMesh& hm, const VGrid& g, int j, uint8_t* lag) {
  const int n = hm.ncell;
  // successors (downwind neighbours) in ascending id, with the face they enter through
  std::vector<int> off(n + 1, 0), succ, sface;
  succ.reserve((size_t)n * 2);
  sface.reserve((size_t)n * 2);
  for (int c = 0; c < n; ++c) {
    std::vector<std::pair<int, int>> s;
    for (int f = 0; f < hm.nf; ++f) {
      int nb = hm.nbr[(size_t)c * 4 + f];
      if (nb >= 0 && host_face_sign(hm, g, j, c, f) > 0) s.push_back({nb, hm.nbr_face[(size_t)c * 4 + f]});
    }
    std::sort(s.begin(), s.end());
    for (auto& p : s) {
      succ.push_back(p.first);
      sface.push_back(p.second);
    }
    off[c + 1] = (int)succ.size();
  }
  // Tarjan's SCC (iterative)
  std::vector<int> idx(n, -1), low(n, 0), comp(n, -1), stk, cs, it(n, 0);
  std::vector<char> on(n, 0);
  int counter = 0, ncomp = 0;
  for (int r = 0; r < n; ++r) {
    if (idx[r] >= 0) continue;
    cs.push_back(r);
    idx[r] = low[r] = counter++;
    stk.push_back(r);
    on[r] = 1;
    it[r] = off[r];
    while (!cs.empty()) {
      int v = cs.back();
      if (it[v] < off[v + 1]) {
        int w = succ[it[v]++];
        if (idx[w] < 0) {
          idx[w] = low[w] = counter++;
          stk.push_back(w);
          on[w] = 1;
          it[w] = off[w];
          cs.push_back(w);
        } else if (on[w]) {
          low[v] = std::min(low[v], idx[w]);
        }
      } else {
        if (low[v] == idx[v]) {
          int w;
          do {
            w = stk.back();
            stk.pop_back();
            on[w] = 0;
            comp[w] = ncomp;
          } while (w != v);
          ++ncomp;
        }
        cs.pop_back();
        if (!cs.empty()) low[cs.back()] = std::min(low[cs.back()], low[v]);
      }
    }
  }
  std::vector<int> csize(ncomp, 0);
  for (int c = 0; c < n; ++c) csize[comp[c]]++;
  // DFS inside each non-trivial component from its smallest id; back edges are lagged
  std::vector<char> state(n, 0);
  int nlag = 0;
  for (int r = 0; r < n; ++r) {
    if (csize[comp[r]] < 2 || state[r]) continue;
    std::vector<int> st{r};
    state[r] = 1;
    it[r] = off[r];
    while (!st.empty()) {
      int v = st.back();
      if (it[v] < off[v + 1]) {
        int e = it[v]++;
        int w = succ[e];
        if (comp[w] != comp[v]) continue;
        if (state[w] == 1) {
          lag[w] |= (uint8_t)(1u << sface[e]);
          ++nlag;
        } else if (state[w] == 0) {
          state[w] = 1;
          it[w] = off[w];
          st.push_back(w);
        }
      } else {
        state[v] = 2;
        st.pop_back();
      }
    }
  }
  return nlag;
}

}  // namespace bgk
