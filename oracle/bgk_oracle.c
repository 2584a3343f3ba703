/*
 * bgk_oracle.c -- plain, sequential FP64 CPU oracle of the sweep-based implicit BGK
 * solver (Hauck et al., "Sweep-based, implicit solutions of the multidimensional BGK
 * equation on unstructured grids").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or load this
 * file; only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code with the CUDA library.
 *
 * Every routine follows the paper's statement in its own order and notation:
 *   - velocity grid, nodal DG in v, Gauss-Legendre quadrature           (Sec. 3.2)
 *   - nodal DG in x on affine simplices, exact integration (Assumption 1, Table 1)
 *   - weak form with upwind flux, cell inflow / outflow boundaries         (Sec. 3.3)
 *   - conservative Maxwellian projection with the polynomial extension     (App. B)
 *   - moments U = (n, n u, 1/2 n |u|^2 + d/2 n theta)                      (Sec. 2)
 *   - DIRK stages in steady-state form, recursive stage derivative        (Sec. 3.5)
 *   - Picard iteration with lagged Maxwellian / boundary / cycle inflow    (Sec. 4)
 *   - sweep graph, DFS back-edge removal, generations (longest path)      (Sec. 4.1)
 *   - convergence criterion on the moments                                  (Sec. 4)
 *
 * Readings where the paper is silent or ambiguous (listed with reasons in the design
 * notes of the repository):
 *   R1  sign of v.n: computed from the face's canonical normal (see canon_normal) as the
 *       left-to-right sum of products without fused multiply-add; a zero sign means no
 *       flux through the face and no graph edge.
 *   R2  cycle breaking: Tarjan SCCs; inside each non-trivial SCC a DFS from its smallest
 *       cell id, visiting successors in ascending id, removes the back edges.
 *   R3  both inflow terms of the Picard equation carry the minus sign of Eq. (bgk-ss-
 *       inflow-outflow); the "+" on the non-lagged part is read as a typo.
 *   R4  the Maxwellian and all states are nodal in x (collocation at the DG nodes).
 *   R5  convergence: the m=1 denominator is max(|U^1|, |U^0|) so that a zero bulk
 *       velocity does not divide by zero.
 *   R6  BDF2: (3 f^{n+1} - 4 f^n + f^{n-1}) / (2 dt) = F(f^{n+1}), first step backward Euler.
 *   R7  DIRK3 uses the full-precision root of 6x^3 - 18x^2 + 9x - 1 (printed to 6 digits).
 *
 * Layouts (shared interface): f[j][cell][node]; nodal states [cell*ndof+node][d+2] as
 * (n, u_1..u_d, theta); moments U[cell*ndof+node][d+2] as (n, n u_1..n u_d, E).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define MAXD 3
#define MAXDOF 6
#define MAXF 4

enum { ORC_OK = 0, ORC_E_INVALID = 1, ORC_E_NOCONV = 4, ORC_E_NONPHYSICAL = 5 };
enum { INT_BE = 0, INT_DIRK2 = 1, INT_DIRK3 = 2, INT_BSTABLE2 = 3, INT_BDF2 = 4 };

typedef struct {
  int dim, kx, ndof, nface, fdof;
  int quad, nvc; /* Q1 quadrilaterals (2D); vertices per cell */
  int nvert, ncell, nnode;
  const double *xyz_in;
  double *xyz;
  int *cells;
  /* velocity grid */
  int n1d, kv, nv;
  double L;
  double *x1d, *w1d, *v, *w; /* v[nv][dim], w[nv] */
  /* per-cell exact matrices */
  double *vol;      /* |K| */
  double *M;        /* [cell][a][b] = int phi_a phi_b */
  double *G;        /* [cell][alpha][a][b] = int phi_b d_alpha phi_a */
  double *Fm;       /* [cell][face][a][b] = int_e phi_a phi_b (K-local indices) */
  double *ncan;     /* [cell][face][dim] canonical normal of the face (not oriented) */
  int *orient;      /* [cell][face] +1 if canonical normal points out of the cell */
  double *unit_n;   /* [cell][face][dim] unit outward normal */
  double *farea;    /* [cell][face] */
  int *nbr;         /* [cell][face] neighbour cell or -1 */
  int *nbr_face;    /* [cell][face] face index in the neighbour */
  int *nbr_node;    /* [cell][face][a] neighbour's local node matching node a (or -1) */
  int *face_nodes;  /* [face][fdof] local nodes on face (same for every cell) */
  /* sweep graphs */
  int *gen;         /* [nv][cell] */
  int *order;       /* [nv][cell] cells sorted by (gen, id) */
  unsigned char *lagged; /* [nv][cell][face]: inflow through this face is lagged */
  int *ngen;        /* [nv] */
  long n_lagged_total;
  /* physics */
  double nu, dt, tau;
  int integrator, lmax;
  int collision; /* 0: projected Maxwellian; 1: simplified Maxwellian N_h = n / |V|; 2: interpolated */
  /* wall boundary conditions (Sec. 4.2); NULL: inflow everywhere */
  int *wmirror;  /* [cell][face]: -1 inflow face, else the table row of mirror[] to use */
  int *mirror;   /* [1 + dim][nv]: row 0 = index of -v_j, row 1 + a = index of v_j with
                    component a negated (R_n v_j for n = +/-e_a) */
} orc_t;

/* ------------------------------------------------------------------ velocity grid */

/* Gauss-Legendre points and weights on [-1,1] (textbook closed forms). */
static int gauss_legendre(int npts, double *x, double *w) {
  if (npts == 2) {
    double a = 1.0 / sqrt(3.0);
    x[0] = -a; x[1] = a; w[0] = w[1] = 1.0;
  } else if (npts == 3) {
    double a = sqrt(3.0 / 5.0);
    x[0] = -a; x[1] = 0.0; x[2] = a;
    w[0] = w[2] = 5.0 / 9.0; w[1] = 8.0 / 9.0;
  } else if (npts == 4) {
    double r = 2.0 * sqrt(6.0 / 5.0);
    double a = sqrt((3.0 - r) / 7.0), b = sqrt((3.0 + r) / 7.0);
    double wa = (18.0 + sqrt(30.0)) / 36.0, wb = (18.0 - sqrt(30.0)) / 36.0;
    x[0] = -b; x[1] = -a; x[2] = a; x[3] = b;
    w[0] = wb; w[1] = wa; w[2] = wa; w[3] = wb;
  } else if (npts == 5) {
    double r = 2.0 * sqrt(10.0 / 7.0);
    double a = sqrt(5.0 - r) / 3.0, b = sqrt(5.0 + r) / 3.0;
    double s = 13.0 * sqrt(70.0);
    double wa = (322.0 + s) / 900.0, wb = (322.0 - s) / 900.0;
    x[0] = -b; x[1] = -a; x[2] = 0.0; x[3] = a; x[4] = b;
    w[0] = wb; w[1] = wa; w[2] = 128.0 / 225.0; w[3] = wa; w[4] = wb;
  } else {
    return ORC_E_INVALID;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------ barycentric algebra */
/* A polynomial in the d+1 barycentric coordinates is a list of terms c * prod l_i^e_i. */
typedef struct { double c; int e[4]; } term_t;
typedef struct { int n; term_t t[64]; } poly_t;

static void poly_basis(int dim, int kx, int a, poly_t *p) {
  memset(p, 0, sizeof(*p));
  if (kx == 1) {
    p->n = 1; p->t[0].c = 1.0; p->t[0].e[a] = 1;
    return;
  }
  /* P2 triangle: vertex a: 2 l_a^2 - l_a; edge node 3+k on edge (k, k+1 mod 3): 4 l_k l_{k+1} */
  (void)dim;
  if (a < 3) {
    p->n = 2;
    p->t[0].c = 2.0; p->t[0].e[a] = 2;
    p->t[1].c = -1.0; p->t[1].e[a] = 1;
  } else {
    int k = a - 3, l = (k + 1) % 3;
    p->n = 1; p->t[0].c = 4.0; p->t[0].e[k] = 1; p->t[0].e[l] += 1;
  }
}

static void poly_dlambda(const poly_t *p, int i, poly_t *out) {
  memset(out, 0, sizeof(*out));
  for (int k = 0; k < p->n; ++k) {
    if (p->t[k].e[i] == 0) continue;
    term_t t = p->t[k];
    t.c *= t.e[i];
    t.e[i] -= 1;
    out->t[out->n++] = t;
  }
}

static double factorial(int n) { double r = 1.0; for (int i = 2; i <= n; ++i) r *= i; return r; }

/* int over a k-simplex of measure meas of prod l_i^e_i (over the listed coordinates):
 * k! meas prod e_i! / (k + sum e)!  */
static double simplex_monomial(int k, double meas, const int *e, int nvar) {
  double num = factorial(k) * meas;
  int s = 0;
  for (int i = 0; i < nvar; ++i) { num *= factorial(e[i]); s += e[i]; }
  return num / factorial(k + s);
}

/* int_K p*q over the cell (d-simplex) */
static double integrate_prod_cell(int dim, double vol, const poly_t *p, const poly_t *q) {
  double s = 0.0;
  for (int a = 0; a < p->n; ++a)
    for (int b = 0; b < q->n; ++b) {
      int e[4];
      for (int i = 0; i < 4; ++i) e[i] = p->t[a].e[i] + q->t[b].e[i];
      s += p->t[a].c * q->t[b].c * simplex_monomial(dim, vol, e, dim + 1);
    }
  return s;
}

/* int_F p*q over the face opposite vertex f (where l_f = 0) */
static double integrate_prod_face(int dim, int f, double area, const poly_t *p, const poly_t *q) {
  double s = 0.0;
  for (int a = 0; a < p->n; ++a)
    for (int b = 0; b < q->n; ++b) {
      int e[4], ef[3], m = 0;
      for (int i = 0; i < 4; ++i) e[i] = p->t[a].e[i] + q->t[b].e[i];
      if (e[f] != 0) continue;
      for (int i = 0; i <= dim; ++i) if (i != f) ef[m++] = e[i];
      s += p->t[a].c * q->t[b].c * simplex_monomial(dim - 1, area, ef, dim);
    }
  return s;
}

/* ---------------------------------------------------------------- mesh geometry */

/* R1: canonical normal of the face with sorted global vertex ids g[0] < g[1] (< g[2]).
 * 2D: t = x_{g1} - x_{g0}, N = (t_y, -t_x), |N| = edge length.
 * 3D: N = ((x_{g1}-x_{g0}) x (x_{g2}-x_{g0})) / 2, |N| = face area.
 * Products and sums are evaluated one rounding at a time, left to right. */
static void canon_normal(const orc_t *o, const int *gsorted, double *N) {
  const double *p0 = o->xyz + (size_t)gsorted[0] * o->dim;
  const double *p1 = o->xyz + (size_t)gsorted[1] * o->dim;
  if (o->dim == 2) {
    double tx = p1[0] - p0[0], ty = p1[1] - p0[1];
    N[0] = ty; N[1] = -tx;
  } else {
    const double *p2 = o->xyz + (size_t)gsorted[2] * o->dim;
    double a[3], b[3];
    for (int i = 0; i < 3; ++i) { a[i] = p1[i] - p0[i]; b[i] = p2[i] - p0[i]; }
    double m0 = a[1] * b[2], m1 = a[2] * b[1];
    double m2 = a[2] * b[0], m3 = a[0] * b[2];
    double m4 = a[0] * b[1], m5 = a[1] * b[0];
    N[0] = (m0 - m1) * 0.5; N[1] = (m2 - m3) * 0.5; N[2] = (m4 - m5) * 0.5;
  }
}

static double vdotN(const double *v, const double *N, int dim) {
  double s = v[0] * N[0];
  double t = v[1] * N[1];
  s = s + t;
  if (dim == 3) { t = v[2] * N[2]; s = s + t; }
  return s;
}

typedef struct { int g[3]; int cell, face; } fkey_t;
static int fkey_cmp(const void *x, const void *y) {
  const fkey_t *a = x, *b = y;
  for (int i = 0; i < 3; ++i) if (a->g[i] != b->g[i]) return a->g[i] < b->g[i] ? -1 : 1;
  if (a->cell != b->cell) return a->cell < b->cell ? -1 : 1;
  return a->face - b->face;
}
static void sort_ints(int *v, int n) {
  for (int i = 1; i < n; ++i) { int x = v[i], j = i - 1; while (j >= 0 && v[j] > x) { v[j + 1] = v[j]; --j; } v[j + 1] = x; }
}

/* global identity of local node a of cell c: vertex id, or sorted pair for a midpoint */
static void node_identity(const orc_t *o, int c, int a, int *id2) {
  const int *cv = o->cells + (size_t)c * o->nvc;
  if (a < o->nvc) { id2[0] = cv[a]; id2[1] = -1; return; }
  int k = a - 3, l = (k + 1) % 3;
  int g0 = cv[k], g1 = cv[l];
  id2[0] = g0 < g1 ? g0 : g1; id2[1] = g0 < g1 ? g1 : g0;
}

/* Q1 quadrilateral (Sec. 3.1, the bilinear element): reference square [0,1]^2 with
 * phi_0 = (1-s)(1-t), phi_1 = s(1-t), phi_2 = s t, phi_3 = (1-s) t at the vertices in cell
 * order, the bilinear map x(s,t) = sum_a x_a phi_a(s,t) (any convex quadrilateral).
 * M = int phi_a phi_b, G_al = int phi_b d_al phi_a with grad phi = J^-T grad_ref phi,
 * integrated with 3x3 tensor Gauss-Legendre points: every integrand times |det J| is a
 * polynomial of degree <= 3 in each of s and t, integrated exactly.  Face f is the
 * straight edge from vertex f to vertex f+1 (mod 4); its mass matrix on the edge is
 * integrated the same way in the edge parameter. */
static void q1_phi(double s, double t, double *phi, double (*dphi)[2]) {
  phi[0] = (1 - s) * (1 - t); phi[1] = s * (1 - t); phi[2] = s * t; phi[3] = (1 - s) * t;
  dphi[0][0] = -(1 - t); dphi[0][1] = -(1 - s);
  dphi[1][0] = 1 - t;    dphi[1][1] = -s;
  dphi[2][0] = t;        dphi[2][1] = s;
  dphi[3][0] = -t;       dphi[3][1] = 1 - s;
}

static int quad_cell_geometry(orc_t *o, int c, fkey_t *keys) {
  const int nd = 4, nf = 4, d = 2;
  const int *cv = o->cells + (size_t)c * 4;
  double xg[3], wg[3];
  gauss_legendre(3, xg, wg);
  double *M = o->M + (size_t)c * nd * nd, *G = o->G + (size_t)c * d * nd * nd;
  memset(M, 0, sizeof(double) * nd * nd);
  memset(G, 0, sizeof(double) * d * nd * nd);
  double vol = 0.0;
  for (int qi = 0; qi < 3; ++qi)
    for (int qj = 0; qj < 3; ++qj) {
      double s = 0.5 * (xg[qi] + 1.0), t = 0.5 * (xg[qj] + 1.0), w = 0.25 * wg[qi] * wg[qj];
      double phi[4], dphi[4][2], J[2][2] = {{0, 0}, {0, 0}};
      q1_phi(s, t, phi, dphi);
      for (int a = 0; a < 4; ++a)
        for (int al = 0; al < 2; ++al)
          for (int r = 0; r < 2; ++r) J[al][r] += o->xyz[(size_t)cv[a] * 2 + al] * dphi[a][r];
      double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      if (!(det > 0.0) && !(det < 0.0)) return ORC_E_INVALID;
      double Ji[2][2] = {{J[1][1] / det, -J[0][1] / det}, {-J[1][0] / det, J[0][0] / det}};
      double adet = fabs(det);
      vol += w * adet;
      double gphi[4][2];
      for (int a = 0; a < 4; ++a)
        for (int al = 0; al < 2; ++al) gphi[a][al] = dphi[a][0] * Ji[0][al] + dphi[a][1] * Ji[1][al];
      for (int a = 0; a < nd; ++a)
        for (int b = 0; b < nd; ++b) {
          M[a * nd + b] += w * adet * phi[a] * phi[b];
          for (int al = 0; al < d; ++al) G[((size_t)al * nd + a) * nd + b] += w * adet * phi[b] * gphi[a][al];
        }
    }
  if (!(vol > 0.0)) return ORC_E_INVALID;
  o->vol[c] = vol;
  for (int f = 0; f < nf; ++f) {
    int g[2] = {cv[f], cv[(f + 1) % 4]};
    sort_ints(g, 2);
    double N[3] = {0, 0, 0};
    canon_normal(o, g, N);
    double area = sqrt(N[0] * N[0] + N[1] * N[1]);
    const double *xo = o->xyz + (size_t)cv[(f + 2) % 4] * 2, *x0 = o->xyz + (size_t)g[0] * 2;
    double sd = (xo[0] - x0[0]) * N[0] + (xo[1] - x0[1]) * N[1];
    int sg = sd < 0.0 ? 1 : -1;
    size_t cf = (size_t)c * nf + f;
    o->orient[cf] = sg;
    o->farea[cf] = area;
    for (int al = 0; al < d; ++al) {
      o->ncan[cf * d + al] = N[al];
      o->unit_n[cf * d + al] = sg * N[al] / area;
    }
    /* edge from vertex f to f+1: reference points (s, t)(e) along it, e in [0, 1] */
    static const double e0[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
    double *Fm = o->Fm + cf * nd * nd;
    memset(Fm, 0, sizeof(double) * nd * nd);
    for (int q = 0; q < 3; ++q) {
      double e = 0.5 * (xg[q] + 1.0), w = 0.5 * wg[q] * area;
      const double *pa = e0[f], *pb = e0[(f + 1) % 4];
      double phi[4], dphi[4][2];
      q1_phi(pa[0] + e * (pb[0] - pa[0]), pa[1] + e * (pb[1] - pa[1]), phi, dphi);
      for (int a = 0; a < nd; ++a)
        for (int b = 0; b < nd; ++b) Fm[a * nd + b] += w * phi[a] * phi[b];
    }
    fkey_t *k = &keys[cf];
    k->g[0] = g[0]; k->g[1] = g[1]; k->g[2] = -1;
    k->cell = c; k->face = f;
    o->nbr[cf] = -1; o->nbr_face[cf] = -1;
  }
  return ORC_OK;
}

static int build_geometry(orc_t *o) {
  int d = o->dim, nd = o->ndof, nf = o->nface;
  /* local nodes on face f: simplices, the face opposite vertex f; quadrilaterals, the
   * edge from vertex f to vertex f+1 */
  for (int f = 0; f < nf; ++f) {
    int m = 0;
    if (o->quad) {
      o->face_nodes[f * o->fdof] = f;
      o->face_nodes[f * o->fdof + 1] = (f + 1) % 4;
      continue;
    }
    for (int a = 0; a <= d; ++a) if (a != f) o->face_nodes[f * o->fdof + m++] = a;
    if (o->kx == 2) o->face_nodes[f * o->fdof + m++] = 3 + (f + 1) % 3;
  }
  fkey_t *keys = malloc(sizeof(fkey_t) * (size_t)o->ncell * nf);
  for (int c = 0; c < o->ncell; ++c) {
    if (o->quad) {
      if (quad_cell_geometry(o, c, keys) != ORC_OK) { free(keys); return ORC_E_INVALID; }
      continue;
    }
    const int *cv = o->cells + (size_t)c * (d + 1);
    const double *x0 = o->xyz + (size_t)cv[0] * d;
    /* affine map x = x0 + J xi, J columns x_i - x0 */
    double J[3][3] = {{0}}, Ji[3][3] = {{0}}, det;
    for (int i = 1; i <= d; ++i)
      for (int al = 0; al < d; ++al) J[al][i - 1] = o->xyz[(size_t)cv[i] * d + al] - x0[al];
    if (d == 2) {
      det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      Ji[0][0] = J[1][1] / det; Ji[0][1] = -J[0][1] / det;
      Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
    } else {
      det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
            J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
          int i1 = (k + 1) % 3, i2 = (k + 2) % 3, k1 = (i + 1) % 3, k2 = (i + 2) % 3;
          Ji[i][k] = (J[i1][k1] * J[i2][k2] - J[i1][k2] * J[i2][k1]) / det;
        }
    }
    if (!(fabs(det) > 0.0)) { free(keys); return ORC_E_INVALID; }
    double vol = fabs(det) / (d == 2 ? 2.0 : 6.0);
    o->vol[c] = vol;
    /* gradients of barycentric coordinates: grad l_i = row (i-1) of J^{-1}, l_0 = 1 - sum */
    double gl[4][3] = {{0}};
    for (int i = 1; i <= d; ++i)
      for (int al = 0; al < d; ++al) { gl[i][al] = Ji[i - 1][al]; gl[0][al] -= Ji[i - 1][al]; }
    poly_t phi[MAXDOF], dphi[MAXDOF][4];
    for (int a = 0; a < nd; ++a) {
      poly_basis(d, o->kx, a, &phi[a]);
      for (int i = 0; i <= d; ++i) poly_dlambda(&phi[a], i, &dphi[a][i]);
    }
    double *M = o->M + (size_t)c * nd * nd;
    double *G = o->G + (size_t)c * d * nd * nd;
    for (int a = 0; a < nd; ++a)
      for (int b = 0; b < nd; ++b) {
        M[a * nd + b] = integrate_prod_cell(d, vol, &phi[a], &phi[b]);
        /* int phi_b d_alpha phi_a = sum_i (d_alpha l_i) int phi_b dphi_a/dl_i */
        double t[4];
        for (int i = 0; i <= d; ++i) t[i] = integrate_prod_cell(d, vol, &phi[b], &dphi[a][i]);
        for (int al = 0; al < d; ++al) {
          double s = 0.0;
          for (int i = 0; i <= d; ++i) s += gl[i][al] * t[i];
          G[((size_t)al * nd + a) * nd + b] = s;
        }
      }
    /* faces */
    for (int f = 0; f < nf; ++f) {
      int g[3], m = 0;
      for (int a = 0; a <= d; ++a) if (a != f) g[m++] = cv[a];
      sort_ints(g, d);
      double N[3] = {0, 0, 0};
      canon_normal(o, g, N);
      double area = 0.0;
      for (int al = 0; al < d; ++al) area += N[al] * N[al];
      area = sqrt(area);
      /* orientation: outward if (x_opp - x_g0) . N < 0 */
      const double *xo = o->xyz + (size_t)cv[f] * d, *xg = o->xyz + (size_t)g[0] * d;
      double s = 0.0;
      for (int al = 0; al < d; ++al) s += (xo[al] - xg[al]) * N[al];
      int sg = s < 0.0 ? 1 : -1;
      size_t cf = (size_t)c * nf + f;
      o->orient[cf] = sg;
      o->farea[cf] = area;
      for (int al = 0; al < d; ++al) {
        o->ncan[cf * d + al] = N[al];
        o->unit_n[cf * d + al] = sg * N[al] / area;
      }
      double *Fm = o->Fm + cf * nd * nd;
      for (int a = 0; a < nd; ++a)
        for (int b = 0; b < nd; ++b) Fm[a * nd + b] = integrate_prod_face(d, f, area, &phi[a], &phi[b]);
      fkey_t *k = &keys[cf];
      k->g[0] = g[0]; k->g[1] = g[1]; k->g[2] = d == 3 ? g[2] : -1;
      k->cell = c; k->face = f;
      o->nbr[cf] = -1; o->nbr_face[cf] = -1;
    }
  }
  /* neighbours: identical sorted vertex triples */
  size_t nk = (size_t)o->ncell * nf;
  qsort(keys, nk, sizeof(fkey_t), fkey_cmp);
  for (size_t i = 0; i < nk;) {
    size_t j = i + 1;
    while (j < nk && keys[j].g[0] == keys[i].g[0] && keys[j].g[1] == keys[i].g[1] && keys[j].g[2] == keys[i].g[2]) ++j;
    if (j - i > 2) { free(keys); return ORC_E_INVALID; } /* non-manifold */
    if (j - i == 2) {
      size_t a = (size_t)keys[i].cell * nf + keys[i].face, b = (size_t)keys[i + 1].cell * nf + keys[i + 1].face;
      /* the two cells must lie on opposite sides of the shared face (else they overlap) */
      if (o->orient[a] == o->orient[b]) { free(keys); return ORC_E_INVALID; }
      o->nbr[a] = keys[i + 1].cell; o->nbr_face[a] = keys[i + 1].face;
      o->nbr[b] = keys[i].cell; o->nbr_face[b] = keys[i].face;
    }
    i = j;
  }
  free(keys);
  /* node correspondence across each interior face */
  for (int c = 0; c < o->ncell; ++c)
    for (int f = 0; f < nf; ++f) {
      size_t cf = (size_t)c * nf + f;
      for (int a = 0; a < nd; ++a) o->nbr_node[cf * MAXDOF + a] = -1;
      int nb = o->nbr[cf];
      if (nb < 0) continue;
      for (int k = 0; k < o->fdof; ++k) {
        int a = o->face_nodes[f * o->fdof + k], ida[2], idb[2];
        node_identity(o, c, a, ida);
        for (int b = 0; b < nd; ++b) {
          node_identity(o, nb, b, idb);
          if (ida[0] == idb[0] && ida[1] == idb[1]) { o->nbr_node[cf * MAXDOF + a] = b; break; }
        }
        if (o->nbr_node[cf * MAXDOF + a] < 0) return ORC_E_INVALID;
      }
    }
  return ORC_OK;
}

/* ------------------------------------------------------------------- sweep graphs */

/* sign of v_j . n on face f of cell c (R1): +1 outflow, -1 inflow, 0 none */
static int face_sign(const orc_t *o, int j, int c, int f) {
  size_t cf = (size_t)c * o->nface + f;
  double s = vdotN(o->v + (size_t)j * o->dim, o->ncan + cf * o->dim, o->dim);
  if (s == 0.0) return 0;
  return (s > 0.0 ? 1 : -1) * o->orient[cf];
}

/* Sweep graph G_j (Sec. 4.1): edge (a, b) when a is adjacent to and upwind of b, i.e.
 * face f of a has v_j . n > 0 and a neighbour b across it.  Successors of a are listed
 * in ascending cell id.  Back edges found by the DFS of R2 are lagged; generations are
 * longest-path levels of the remaining DAG. */
typedef struct { int *idx, *adj, *adj_face; } csr_t;

static void build_graph(const orc_t *o, int j, csr_t *g) {
  int nf = o->nface;
  for (int c = 0; c <= o->ncell; ++c) g->idx[c] = 0;
  for (int c = 0; c < o->ncell; ++c)
    for (int f = 0; f < nf; ++f)
      if (o->nbr[(size_t)c * nf + f] >= 0 && face_sign(o, j, c, f) > 0) g->idx[c + 1]++;
  for (int c = 0; c < o->ncell; ++c) g->idx[c + 1] += g->idx[c];
  for (int c = 0; c < o->ncell; ++c) {
    int p = g->idx[c];
    for (int f = 0; f < nf; ++f) {
      size_t cf = (size_t)c * nf + f;
      if (o->nbr[cf] >= 0 && face_sign(o, j, c, f) > 0) { g->adj[p] = o->nbr[cf]; g->adj_face[p] = o->nbr_face[cf]; ++p; }
    }
    /* ascending successor id */
    for (int a = g->idx[c] + 1; a < g->idx[c + 1]; ++a) {
      int x = g->adj[a], xf = g->adj_face[a], b = a - 1;
      while (b >= g->idx[c] && g->adj[b] > x) { g->adj[b + 1] = g->adj[b]; g->adj_face[b + 1] = g->adj_face[b]; --b; }
      g->adj[b + 1] = x; g->adj_face[b + 1] = xf;
    }
  }
}

/* Tarjan's strongly connected components, iterative. comp[c] = component id;
 * returns the number of components. */
static int tarjan(int n, const csr_t *g, int *comp, int *work) {
  int *index = work, *low = work + n, *stack = work + 2 * n, *cstack = work + 3 * n, *iter = work + 4 * n;
  unsigned char *on = (unsigned char *)(work + 5 * n);
  for (int i = 0; i < n; ++i) { index[i] = -1; on[i] = 0; }
  int counter = 0, sp = 0, csp = 0, ncomp = 0;
  for (int r = 0; r < n; ++r) {
    if (index[r] >= 0) continue;
    cstack[csp++] = r; iter[r] = g->idx[r];
    index[r] = low[r] = counter++; stack[sp++] = r; on[r] = 1;
    while (csp > 0) {
      int v = cstack[csp - 1];
      if (iter[v] < g->idx[v + 1]) {
        int w = g->adj[iter[v]++];
        if (index[w] < 0) {
          index[w] = low[w] = counter++; stack[sp++] = w; on[w] = 1;
          iter[w] = g->idx[w]; cstack[csp++] = w;
        } else if (on[w] && index[w] < low[v]) {
          low[v] = index[w];
        }
      } else {
        if (low[v] == index[v]) {
          int w;
          do { w = stack[--sp]; on[w] = 0; comp[w] = ncomp; } while (w != v);
          ++ncomp;
        }
        --csp;
        if (csp > 0) { int u = cstack[csp - 1]; if (low[v] < low[u]) low[u] = low[v]; }
      }
    }
  }
  return ncomp;
}

static int build_dag(orc_t *o, int j, csr_t *g, int *work, int *comp, int *state, int *stk, int *it, int *indeg) {
  int n = o->ncell, nf = o->nface;
  unsigned char *lag = o->lagged + (size_t)j * n * nf;
  memset(lag, 0, (size_t)n * nf);
  build_graph(o, j, g);
  int ncomp = tarjan(n, g, comp, work);
  int nlag = 0;
  if (ncomp < n) {
    /* component sizes; DFS inside every non-trivial component from its minimum id */
    int *csize = calloc((size_t)ncomp, sizeof(int));
    for (int c = 0; c < n; ++c) csize[comp[c]]++;
    for (int c = 0; c < n; ++c) state[c] = 0; /* 0 white, 1 on stack, 2 done */
    for (int r = 0; r < n; ++r) {            /* ascending id: first visit of a comp is its min */
      if (csize[comp[r]] < 2 || state[r] != 0) continue;
      int sp = 0; stk[sp++] = r; it[r] = g->idx[r]; state[r] = 1;
      while (sp > 0) {
        int v = stk[sp - 1];
        if (it[v] < g->idx[v + 1]) {
          int e = it[v]++, w = g->adj[e];
          if (comp[w] != comp[v]) continue;
          if (state[w] == 1) {               /* back edge v -> w: lag inflow of w */
            lag[(size_t)w * nf + g->adj_face[e]] = 1; ++nlag;
          } else if (state[w] == 0) {
            state[w] = 1; it[w] = g->idx[w]; stk[sp++] = w;
          }
        } else {
          state[v] = 2; --sp;
        }
      }
    }
    free(csize);
  }
  /* generations: longest path from the sources over non-lagged edges (Kahn levels) */
  int *gen = o->gen + (size_t)j * n, *ord = o->order + (size_t)j * n;
  for (int c = 0; c < n; ++c) indeg[c] = 0;
  for (int c = 0; c < n; ++c)
    for (int e = g->idx[c]; e < g->idx[c + 1]; ++e)
      if (!lag[(size_t)g->adj[e] * nf + g->adj_face[e]]) indeg[g->adj[e]]++;
  int head = 0, tail = 0;
  for (int c = 0; c < n; ++c) if (indeg[c] == 0) { gen[c] = 0; stk[tail++] = c; }
  while (head < tail) {
    int c = stk[head++];
    for (int e = g->idx[c]; e < g->idx[c + 1]; ++e) {
      int b = g->adj[e];
      if (lag[(size_t)b * nf + g->adj_face[e]]) continue;
      if (--indeg[b] == 0) {
        int mx = -1;
        /* gen(b) = 1 + max over non-lagged upwind a of gen(a) */
        for (int f = 0; f < nf; ++f) {
          size_t bf = (size_t)b * nf + f;
          int a = o->nbr[bf];
          if (a < 0 || lag[bf] || face_sign(o, j, b, f) >= 0) continue;
          if (gen[a] > mx) mx = gen[a];
        }
        gen[b] = mx + 1;
        stk[tail++] = b;
      }
    }
  }
  if (tail != n) return -1;
  /* order: ascending (gen, id) -- counting sort */
  int G = 0;
  for (int c = 0; c < n; ++c) if (gen[c] + 1 > G) G = gen[c] + 1;
  int *cnt = calloc((size_t)G + 1, sizeof(int));
  for (int c = 0; c < n; ++c) cnt[gen[c] + 1]++;
  for (int k = 0; k < G; ++k) cnt[k + 1] += cnt[k];
  for (int c = 0; c < n; ++c) ord[cnt[gen[c]]++] = c;
  free(cnt);
  o->ngen[j] = G;
  return nlag;
}

/* ------------------------------------------------------- Maxwellian projection */

/* Standard normal partial moments I_k = int_a^b t^k phi(t) dt, k = 0..kmax, with
 * phi(t) = exp(-t^2/2)/sqrt(2 pi); a = -inf / b = +inf allowed (ainf / binf). */
static void normal_moments(double a, int ainf, double b, int binf, int kmax, double *I) {
  const double rs2 = 0.70710678118654752440, rs2pi = 0.39894228040143267794;
  double pa = ainf ? 0.0 : rs2pi * exp(-0.5 * a * a), pb = binf ? 0.0 : rs2pi * exp(-0.5 * b * b);
  /* I_0 = Phi(b) - Phi(a), evaluated with erfc on the side that avoids cancellation */
  double I0;
  if (!ainf && a >= 0.0) {
    I0 = 0.5 * (erfc(a * rs2) - (binf ? 0.0 : erfc(b * rs2)));
  } else if (!binf && b <= 0.0) {
    I0 = 0.5 * (erfc(-b * rs2) - (ainf ? 0.0 : erfc(-a * rs2)));
  } else {
    double Pb = binf ? 1.0 : 1.0 - 0.5 * erfc(b * rs2);
    double Pa = ainf ? 0.0 : 0.5 * erfc(-a * rs2);
    I0 = Pb - Pa;
  }
  I[0] = I0;
  if (kmax >= 1) I[1] = pa - pb;
  double ak = 1.0, bk = 1.0; /* a^{k-1}, b^{k-1} */
  for (int k = 2; k <= kmax; ++k) {
    ak = ainf ? 0.0 : ak * a;
    bk = binf ? 0.0 : bk * b;
    I[k] = (k - 1) * I[k - 2] + (ainf ? 0.0 : ak * pa) - (binf ? 0.0 : bk * pb);
  }
}

/* 1D factors of the projected Maxwellian (App. B):
 *   c[m] = (1/w_m) int_R g(v) [E l_m](v) dv,   g = (2 pi theta)^{-1/2} exp(-(v-u)^2/(2 theta)),
 * where l_m is the Lagrange polynomial of node m on its velocity cell and E extends
 * the polynomial of the first / last cell to (-inf, -L) / (L, inf). */
static void project_1d(const orc_t *o, double u, double theta, double *c) {
  int np = o->kv + 1, ncl = o->n1d / np;
  double h = 2.0 * o->L / ncl, sig = sqrt(theta);
  for (int cl = 0; cl < ncl; ++cl) {
    double lo = -o->L + cl * h, hi = lo + h;
    int ainf = (cl == 0), binf = (cl == ncl - 1);
    double I[16];
    normal_moments((lo - u) / sig, ainf, (hi - u) / sig, binf, np - 1, I);
    for (int k = 0; k < np; ++k) {
      int m = cl * np + k;
      /* coefficients of l_m(u + sig t) as a polynomial in t */
      double p[16] = {0};
      p[0] = 1.0;
      int deg = 0;
      for (int i = 0; i < np; ++i) {
        if (i == k) continue;
        int mi = cl * np + i;
        double den = o->x1d[m] - o->x1d[mi];
        double c0 = (u - o->x1d[mi]) / den, c1 = sig / den; /* factor c0 + c1 t */
        for (int q = deg + 1; q >= 0; --q) p[q] = (q > 0 ? p[q - 1] * c1 : 0.0) + p[q] * c0;
        ++deg;
      }
      double s = 0.0;
      for (int q = 0; q <= deg; ++q) s += p[q] * I[q];
      c[m] = s / o->w1d[m];
    }
  }
}

/* nodal discrete Maxwellian M_j = n prod_alpha c_alpha[j_alpha] (Sec. 3.3 + App. B) */
static void maxwellian_at_node(const orc_t *o, const double *nut, double *out, size_t stride) {
  int d = o->dim, N = o->n1d;
  double c[3][128];
  for (int al = 0; al < d; ++al) project_1d(o, nut[1 + al], nut[1 + d], c[al]);
  for (int j = 0; j < o->nv; ++j) {
    int jj = j, ja[3];
    for (int al = d - 1; al >= 0; --al) { ja[al] = jj % N; jj /= N; }
    double m = nut[0];
    for (int al = 0; al < d; ++al) m *= c[al][ja[al]];
    out[(size_t)j * stride] = m;
  }
}

/* ------------------------------------------------------------------- moments */

/* U_i = sum_j w_j e(v_j) f_{j,i}, e = (1, v, |v|^2/2), summed in ascending j (Sec. 2, Eq. moments) */
static void moments(const orc_t *o, const double *f, double *U) {
  int d = o->dim, nm = d + 2;
  for (int i = 0; i < o->nnode; ++i) {
    double s[5] = {0, 0, 0, 0, 0};
    for (int j = 0; j < o->nv; ++j) {
      double fj = f[(size_t)j * o->nnode + i], wj = o->w[j];
      const double *v = o->v + (size_t)j * d;
      double e2 = 0.0;
      for (int al = 0; al < d; ++al) e2 += v[al] * v[al];
      s[0] += wj * fj;
      for (int al = 0; al < d; ++al) s[1 + al] += wj * v[al] * fj;
      s[1 + d] += wj * 0.5 * e2 * fj;
    }
    for (int m = 0; m < nm; ++m) U[(size_t)i * nm + m] = s[m];
  }
}

/* primitive (n, u, theta) from U: u = (n u)/n, theta = (2E/n - |u|^2)/d (Eq. moments) */
static int primitive(int d, const double *U, double *nut) {
  double n = U[0];
  nut[0] = n;
  double u2 = 0.0;
  for (int al = 0; al < d; ++al) { nut[1 + al] = U[1 + al] / n; u2 += nut[1 + al] * nut[1 + al]; }
  nut[1 + d] = (2.0 * U[1 + d] / n - u2) / d;
  if (!(n > 0.0) || !(nut[1 + d] > 0.0)) return ORC_E_NONPHYSICAL;
  return ORC_OK;
}

/* ----------------------------------------------------------------- local solve */

/* Gaussian elimination with partial pivoting, A is n x n row-major (overwritten). */
static void dense_solve(int n, double *A, double *b) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i) if (fabs(A[i * n + k]) > fabs(A[p * n + k])) p = i;
    if (p != k) {
      for (int c = 0; c < n; ++c) { double t = A[k * n + c]; A[k * n + c] = A[p * n + c]; A[p * n + c] = t; }
      double t = b[k]; b[k] = b[p]; b[p] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      double l = A[i * n + k] / A[k * n + k];
      for (int c = k; c < n; ++c) A[i * n + c] -= l * A[k * n + c];
      b[i] -= l * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int c = i + 1; c < n; ++c) s -= A[i * n + c] * b[c];
    b[i] = s / A[i * n + i];
  }
}

/* One transport sweep of the Picard iteration, Eq. (bgk-ss-picard) with R3:
 *  -(f, v.grad z)_K + (f, v.n z)_{d+K} + nu_s (f, z)_K
 *     = nu (M, z)_K + (q, z)_K - (f_up^{l+1}, v.n z)_{d-K up} - (f_up^{l}, v.n z)_{d-K down}
 *       - (f_bc, v.n z)_{d-K on dX}
 * for every ordinate j, cells visited in ascending (generation, id).  fold = f^l,
 * fnew = f^{l+1}; Mn = nodal Maxwellian; q = stage source; fbc = boundary values,
 * all [j][cell][node]. */
static void sweep_ordinate(const orc_t *o, int j, const double *fold, const double *Mn, const double *q,
                           const double *fbc, double nu, double nu_s, double *fnew, const double *fall) {
  int d = o->dim, nd = o->ndof, nf = o->nface;
  {
    const double *v = o->v + (size_t)j * d;
    size_t base = 0; /* every array argument is the row of ordinate j */
    const unsigned char *lag = o->lagged + (size_t)j * o->ncell * nf;
    for (int k = 0; k < o->ncell; ++k) {
      int c = o->order[(size_t)j * o->ncell + k];
      const double *M = o->M + (size_t)c * nd * nd;
      const double *G = o->G + (size_t)c * d * nd * nd;
      double A[MAXDOF * MAXDOF], b[MAXDOF];
      for (int a = 0; a < nd; ++a) {
        double rhs = 0.0;
        for (int bb = 0; bb < nd; ++bb) {
          double vg = 0.0;
          for (int al = 0; al < d; ++al) vg += v[al] * G[((size_t)al * nd + a) * nd + bb];
          A[a * nd + bb] = -vg + nu_s * M[a * nd + bb];
          size_t ib = base + (size_t)c * nd + bb;
          rhs += nu * M[a * nd + bb] * Mn[ib] + M[a * nd + bb] * q[ib];
        }
        b[a] = rhs;
      }
      for (int f = 0; f < nf; ++f) {
        int sg = face_sign(o, j, c, f);
        if (sg == 0) continue;
        size_t cf = (size_t)c * nf + f;
        const double *un = o->unit_n + cf * d;
        double vn = 0.0;
        for (int al = 0; al < d; ++al) vn += v[al] * un[al];
        const double *Fm = o->Fm + cf * nd * nd;
        if (sg > 0) {         /* outflow: interior trace */
          for (int a = 0; a < nd; ++a)
            for (int bb = 0; bb < nd; ++bb) A[a * nd + bb] += vn * Fm[a * nd + bb];
        } else {              /* inflow: upwind trace, new / lagged / boundary */
          int nb = o->nbr[cf];
          double y[MAXDOF] = {0};
          for (int k = 0; k < o->fdof; ++k) {
            int bb = o->face_nodes[f * o->fdof + k]; /* nodes off the face have zero face mass */
            if (nb < 0 && o->wmirror && o->wmirror[cf] >= 0) {
              /* wall: the mirror ordinate's interior trace at the same node, from f^l */
              int jm = o->mirror[(size_t)o->wmirror[cf] * o->nv + j];
              y[bb] = fall[(size_t)jm * o->nnode + (size_t)c * nd + bb];
            } else if (nb < 0) y[bb] = fbc[base + (size_t)c * nd + bb];
            else {
              size_t iu = base + (size_t)nb * nd + o->nbr_node[cf * MAXDOF + bb];
              y[bb] = lag[cf] ? fold[iu] : fnew[iu];
            }
          }
          for (int a = 0; a < nd; ++a)
            for (int bb = 0; bb < nd; ++bb) b[a] -= vn * Fm[a * nd + bb] * y[bb];
        }
      }
      dense_solve(nd, A, b);
      for (int a = 0; a < nd; ++a) fnew[base + (size_t)c * nd + a] = b[a];
    }
  }
}

/* The ordinates of one sweep are independent (each reads only its own rows, and f^l for
 * walls), so the loop over them may run on several threads: the timed CPU baseline is this
 * source built with -fopenmp; the parity build ignores the pragma and runs in order.  Each
 * ordinate's arithmetic is the same either way. */
static void sweep_range(const orc_t *o, const double *fold, const double *Mn, const double *q, const double *fbc,
                        double nu, double nu_s, double *fnew, int j0, int j1) {
  size_t nn = (size_t)o->nnode;
#pragma omp parallel for schedule(dynamic, 1)
  for (int j = j0; j < j1; ++j)
    sweep_ordinate(o, j, fold + (size_t)j * nn, Mn + (size_t)j * nn, q + (size_t)j * nn, fbc + (size_t)j * nn, nu,
                   nu_s, fnew + (size_t)j * nn, fold);
}

static void sweep(const orc_t *o, const double *fold, const double *Mn, const double *q, const double *fbc,
                  double nu, double nu_s, double *fnew) {
  sweep_range(o, fold, Mn, q, fbc, nu, nu_s, fnew, 0, o->nv);
}

/* ============================================================ public interface */

void orc_destroy(orc_t *o) {
  if (!o) return;
  free(o->xyz); free(o->cells); free(o->x1d); free(o->w1d); free(o->v); free(o->w);
  free(o->vol); free(o->M); free(o->G); free(o->Fm); free(o->ncan); free(o->orient); free(o->unit_n);
  free(o->farea); free(o->nbr); free(o->nbr_face); free(o->nbr_node); free(o->face_nodes);
  free(o->gen); free(o->order); free(o->lagged); free(o->ngen);
  free(o->wmirror); free(o->mirror);
  free(o);
}

/* Geometry and velocity grid of a simplex or (quad = 1) quadrilateral mesh. */
static orc_t *create_impl(int dim, int kx, int quad, int nvert, const double *xyz, int ncell, const int *cells,
                          int n1d, int kv, double L) {
  if ((dim != 2 && dim != 3) || (kx != 1 && kx != 2) || (kx == 2 && dim != 2)) return NULL;
  if (quad && (dim != 2 || kx != 1)) return NULL;
  if (kv < 1 || kv > 4 || n1d % (kv + 1) != 0 || n1d > 128 || !(L > 0.0)) return NULL;
  orc_t *o = calloc(1, sizeof(orc_t));
  o->dim = dim; o->kx = kx; o->nvert = nvert; o->ncell = ncell;
  o->quad = quad;
  o->nvc = quad ? 4 : dim + 1;
  o->ndof = quad ? 4 : kx == 1 ? dim + 1 : 6;
  o->nface = quad ? 4 : dim + 1;
  o->fdof = kx == 1 ? dim : 3;
  o->nnode = ncell * o->ndof;
  o->xyz = malloc(sizeof(double) * (size_t)nvert * dim);
  memcpy(o->xyz, xyz, sizeof(double) * (size_t)nvert * dim);
  o->cells = malloc(sizeof(int) * (size_t)ncell * o->nvc);
  memcpy(o->cells, cells, sizeof(int) * (size_t)ncell * o->nvc);
  o->n1d = n1d; o->kv = kv; o->L = L;
  o->nv = 1;
  for (int i = 0; i < dim; ++i) o->nv *= n1d;
  /* velocity grid: n1d/(kv+1) uniform cells on [-L, L], Gauss points in each */
  int np = kv + 1, ncl = n1d / np;
  double xg[8], wg[8], h = 2.0 * L / ncl;
  gauss_legendre(np, xg, wg);
  o->x1d = malloc(sizeof(double) * n1d);
  o->w1d = malloc(sizeof(double) * n1d);
  for (int cl = 0; cl < ncl; ++cl)
    for (int k = 0; k < np; ++k) {
      double mid = -L + (cl + 0.5) * h;
      o->x1d[cl * np + k] = mid + 0.5 * h * xg[k];
      o->w1d[cl * np + k] = 0.5 * h * wg[k];
    }
  o->v = malloc(sizeof(double) * (size_t)o->nv * dim);
  o->w = malloc(sizeof(double) * (size_t)o->nv);
  for (int j = 0; j < o->nv; ++j) {
    int jj = j, ja[3];
    for (int al = dim - 1; al >= 0; --al) { ja[al] = jj % n1d; jj /= n1d; }
    double w = 1.0;
    for (int al = 0; al < dim; ++al) { o->v[(size_t)j * dim + al] = o->x1d[ja[al]]; w *= o->w1d[ja[al]]; }
    o->w[j] = w;
  }
  size_t nd = o->ndof, nf = o->nface;
  o->vol = malloc(sizeof(double) * ncell);
  o->M = malloc(sizeof(double) * ncell * nd * nd);
  o->G = malloc(sizeof(double) * ncell * dim * nd * nd);
  o->Fm = malloc(sizeof(double) * ncell * nf * nd * nd);
  o->ncan = malloc(sizeof(double) * ncell * nf * dim);
  o->orient = malloc(sizeof(int) * ncell * nf);
  o->unit_n = malloc(sizeof(double) * ncell * nf * dim);
  o->farea = malloc(sizeof(double) * ncell * nf);
  o->nbr = malloc(sizeof(int) * ncell * nf);
  o->nbr_face = malloc(sizeof(int) * ncell * nf);
  o->nbr_node = malloc(sizeof(int) * ncell * nf * MAXDOF);
  o->face_nodes = malloc(sizeof(int) * nf * o->fdof);
  for (int c = 0; c < ncell; ++c)
    for (int k = 0; k < o->nvc; ++k) {
      int g = cells[(size_t)c * o->nvc + k];
      if (g < 0 || g >= nvert) { orc_destroy(o); return NULL; }
    }
  if (build_geometry(o) != ORC_OK) { orc_destroy(o); return NULL; }
  o->nu = 0.0; o->dt = 1.0; o->tau = 1e-8; o->integrator = INT_BE; o->lmax = 1000;
  return o;
}

/* Build mesh geometry and the velocity grid.  n1d points per dimension, kv+1 Gauss
 * points per velocity cell, V = [-L, L]^dim. Returns NULL on invalid input. */
orc_t *orc_create(int dim, int kx, int nvert, const double *xyz, int ncell, const int *cells, int n1d, int kv,
                  double L) {
  return create_impl(dim, kx, 0, nvert, xyz, ncell, cells, n1d, kv, L);
}

/* The same on Q1 quadrilaterals: cells [ncell][4], vertices in order around each cell. */
orc_t *orc_create_quad(int nvert, const double *xyz, int ncell, const int *cells, int n1d, int kv, double L) {
  return create_impl(2, 1, 1, nvert, xyz, ncell, cells, n1d, kv, L);
}

int orc_info(const orc_t *o, int *out) {
  out[0] = o->nv; out[1] = o->nnode; out[2] = o->ndof; out[3] = o->nface; out[4] = o->ncell;
  return ORC_OK;
}

void orc_velocity(const orc_t *o, double *v, double *w, double *x1d, double *w1d) {
  memcpy(v, o->v, sizeof(double) * (size_t)o->nv * o->dim);
  memcpy(w, o->w, sizeof(double) * (size_t)o->nv);
  memcpy(x1d, o->x1d, sizeof(double) * o->n1d);
  memcpy(w1d, o->w1d, sizeof(double) * o->n1d);
}

void orc_cell(const orc_t *o, int c, double *vol, double *M, double *G, double *Fm, double *unit_n, double *area,
              int *nbr, int *nbr_node) {
  size_t nd = o->ndof, nf = o->nface, d = o->dim;
  *vol = o->vol[c];
  memcpy(M, o->M + c * nd * nd, sizeof(double) * nd * nd);
  memcpy(G, o->G + c * d * nd * nd, sizeof(double) * d * nd * nd);
  memcpy(Fm, o->Fm + c * nf * nd * nd, sizeof(double) * nf * nd * nd);
  memcpy(unit_n, o->unit_n + c * nf * d, sizeof(double) * nf * d);
  memcpy(area, o->farea + c * nf, sizeof(double) * nf);
  memcpy(nbr, o->nbr + c * nf, sizeof(int) * nf);
  for (size_t f = 0; f < nf; ++f)
    for (size_t a = 0; a < nd; ++a) nbr_node[f * nd + a] = o->nbr_node[((size_t)c * nf + f) * MAXDOF + a];
}

void orc_project_1d(const orc_t *o, double u, double theta, double *c) { project_1d(o, u, theta, c); }

/* f[j][node] = projected Maxwellian of the nodal state (R4) */
void orc_maxwellian(const orc_t *o, const double *nut, double *out) {
  int nm = o->dim + 2;
  for (int i = 0; i < o->nnode; ++i) maxwellian_at_node(o, nut + (size_t)i * nm, out + i, (size_t)o->nnode);
}

void orc_moments(const orc_t *o, const double *f, double *U) { moments(o, f, U); }

/* Build the DAGs of the listed ordinates (all when js == NULL); returns the total of
 * lagged edges, or -1 on failure.  Ordinates not listed are left unbuilt. */
long orc_build_dags_for(orc_t *o, const int *js, int nj) {
  int n = o->ncell;
  size_t nv = o->nv;
  free(o->gen); free(o->order); free(o->lagged); free(o->ngen);
  o->gen = malloc(sizeof(int) * nv * n);
  o->order = malloc(sizeof(int) * nv * n);
  o->lagged = malloc(nv * n * o->nface);
  o->ngen = malloc(sizeof(int) * nv);
  csr_t g;
  g.idx = malloc(sizeof(int) * (n + 1));
  g.adj = malloc(sizeof(int) * (size_t)n * o->nface);
  g.adj_face = malloc(sizeof(int) * (size_t)n * o->nface);
  int *work = malloc(sizeof(int) * (size_t)n * 6 + 16);
  int *comp = malloc(sizeof(int) * n), *state = malloc(sizeof(int) * n), *stk = malloc(sizeof(int) * n);
  int *it = malloc(sizeof(int) * n), *indeg = malloc(sizeof(int) * n);
  long total = 0;
  size_t cnt = js ? (size_t)nj : nv;
  for (size_t k = 0; k < cnt; ++k) {
    int j = js ? js[k] : (int)k;
    int r = build_dag(o, j, &g, work, comp, state, stk, it, indeg);
    if (r < 0) { total = -1; break; }
    total += r;
  }
  free(g.idx); free(g.adj); free(g.adj_face); free(work); free(comp); free(state); free(stk); free(it); free(indeg);
  o->n_lagged_total = total;
  return total;
}

long orc_build_dags(orc_t *o) { return orc_build_dags_for(o, NULL, 0); }

int orc_generations(const orc_t *o, int j, int *gen, unsigned char *lagged) {
  memcpy(gen, o->gen + (size_t)j * o->ncell, sizeof(int) * o->ncell);
  if (lagged) memcpy(lagged, o->lagged + (size_t)j * o->ncell * o->nface, (size_t)o->ncell * o->nface);
  return o->ngen[j];
}

/* face signs (R1) for ordinate j: [cell][face] in {-1, 0, 1} */
void orc_face_signs(const orc_t *o, int j, int *s) {
  for (int c = 0; c < o->ncell; ++c)
    for (int f = 0; f < o->nface; ++f) s[c * o->nface + f] = face_sign(o, j, c, f);
}

void orc_sweep(const orc_t *o, const double *fold, const double *Mn, const double *q, const double *fbc, double nu,
               double nu_s, double *fnew) {
  sweep(o, fold, Mn, q, fbc, nu, nu_s, fnew);
}

/* the same sweep restricted to ordinates j0 <= j < j1 (used to time a bounded sample) */
void orc_sweep_range(const orc_t *o, const double *fold, const double *Mn, const double *q, const double *fbc,
                     double nu, double nu_s, double *fnew, int j0, int j1) {
  sweep_range(o, fold, Mn, q, fbc, nu, nu_s, fnew, j0, j1);
}

/* Projected Maxwellian of the nodal states for the listed ordinates only:
 * out[r][node] for j = js[r], r < nj. */
void orc_maxwellian_rows(const orc_t *o, const double *nut, const int *js, int nj, double *out) {
  int d = o->dim, N = o->n1d, nm = d + 2;
  double c[3][128];
  for (int i = 0; i < o->nnode; ++i) {
    const double *p = nut + (size_t)i * nm;
    for (int al = 0; al < d; ++al) project_1d(o, p[1 + al], p[1 + d], c[al]);
    for (int r = 0; r < nj; ++r) {
      int jj = js[r], ja[3];
      for (int al = d - 1; al >= 0; --al) { ja[al] = jj % N; jj /= N; }
      double m = p[0];
      for (int al = 0; al < d; ++al) m *= c[al][ja[al]];
      out[(size_t)r * o->nnode + i] = m;
    }
  }
}

/* One sweep for the listed ordinates only (in parallel in the OpenMP build, see
 * sweep_range); all arrays hold just those rows
 * ([nj][nnode]); the graphs must have been built.  Inflow boundaries only (a wall needs
 * the mirror ordinates' rows): with walls set it returns ORC_E_INVALID and sweeps nothing. */
int orc_sweep_rows(const orc_t *o, const int *js, int nj, const double *fold, const double *Mn, const double *q,
                    const double *fbc, double nu, double nu_s, double *fnew) {
  size_t nn = (size_t)o->nnode;
  if (o->wmirror) return ORC_E_INVALID;
#pragma omp parallel for schedule(dynamic, 1)
  for (int r = 0; r < nj; ++r)
    sweep_ordinate(o, js[r], fold + (size_t)r * nn, Mn + (size_t)r * nn, q + (size_t)r * nn, fbc + (size_t)r * nn, nu,
                   nu_s, fnew + (size_t)r * nn, NULL);
  return ORC_OK;
}

/* explicit time-step bound (Sec. 5): dt_e = (1/d) (1/(2 kx + 1)) h_min / max_j |v_j|,
 * h_min = (min cell volume)^(1/d) */
double orc_dt_explicit(const orc_t *o) {
  double vmin = o->vol[0], vmax = 0.0;
  for (int c = 1; c < o->ncell; ++c) if (o->vol[c] < vmin) vmin = o->vol[c];
  for (int j = 0; j < o->nv; ++j) {
    double s = 0.0;
    for (int al = 0; al < o->dim; ++al) s += o->v[(size_t)j * o->dim + al] * o->v[(size_t)j * o->dim + al];
    if (sqrt(s) > vmax) vmax = sqrt(s);
  }
  return (1.0 / o->dim) * (1.0 / (2 * o->kx + 1)) * pow(vmin, 1.0 / o->dim) / vmax;
}

/* Butcher tableaus (App. A); R7 for DIRK3. Returns S. */
int orc_tableau(int integ, double *A, double *b, double *c) {
  memset(A, 0, sizeof(double) * 9); memset(b, 0, sizeof(double) * 3); memset(c, 0, sizeof(double) * 3);
  if (integ == INT_BE || integ == INT_BDF2) { A[0] = 1.0; b[0] = 1.0; c[0] = 1.0; return 1; }
  if (integ == INT_DIRK2) {
    double g = 1.0 - sqrt(2.0) / 2.0;
    A[0] = g; A[3] = sqrt(2.0) / 2.0; A[4] = g;
    b[0] = sqrt(2.0) / 2.0; b[1] = g; c[0] = g; c[1] = 1.0;
    return 2;
  }
  if (integ == INT_DIRK3) {
    /* gamma: root in (0,1) of 6x^3 - 18x^2 + 9x - 1 closest to 0.4358665, by Newton */
    double g = 0.4358665;
    for (int it = 0; it < 50; ++it) g -= (6 * g * g * g - 18 * g * g + 9 * g - 1) / (18 * g * g - 36 * g + 9);
    double b1 = -1.5 * g * g + 4.0 * g - 0.25, b2 = 1.5 * g * g - 5.0 * g + 1.25;
    A[0] = g;
    A[3] = 0.5 * (1.0 - g); A[4] = g;
    A[6] = b1; A[7] = b2; A[8] = g;
    b[0] = b1; b[1] = b2; b[2] = g;
    c[0] = g; c[1] = 0.5 * (1.0 + g); c[2] = 1.0;
    return 3;
  }
  if (integ == INT_BSTABLE2) {
    double g = (3.0 + sqrt(3.0)) / 6.0;
    A[0] = g; A[3] = 1.0 - 2.0 * g; A[4] = g;
    b[0] = 0.5; b[1] = 0.5; c[0] = g; c[1] = 1.0 - g;
    return 2;
  }
  return 0;
}

/* Convergence measure of Eq. (convergence-criteria) with R5:
 * max_m |U^{l+1,m} - U^{l,m}| / |U^{l,m}| over all nodes (l2 over nodes, Euclidean in m=1). */
double orc_conv_measure(const orc_t *o, const double *Unew, const double *Uold) {
  int d = o->dim, nm = d + 2;
  double dn[3] = {0, 0, 0}, no[3] = {0, 0, 0};
  for (int i = 0; i < o->nnode; ++i) {
    const double *a = Unew + (size_t)i * nm, *b = Uold + (size_t)i * nm;
    dn[0] += (a[0] - b[0]) * (a[0] - b[0]);
    no[0] += b[0] * b[0];
    for (int al = 0; al < d; ++al) { dn[1] += (a[1 + al] - b[1 + al]) * (a[1 + al] - b[1 + al]); no[1] += b[1 + al] * b[1 + al]; }
    dn[2] += (a[1 + d] - b[1 + d]) * (a[1 + d] - b[1 + d]);
    no[2] += b[1 + d] * b[1 + d];
  }
  double r0 = sqrt(dn[0]) / sqrt(no[0]);
  double den1 = sqrt(no[1]) > sqrt(no[0]) ? sqrt(no[1]) : sqrt(no[0]);
  double r1 = sqrt(dn[1]) / den1;
  double r2 = sqrt(dn[2]) / sqrt(no[2]);
  double r = r0 > r1 ? r0 : r1;
  return r > r2 ? r : r2;
}

/* One Picard iteration loop for one stage: starts from f (in place), returns iterations
 * used, writes the last convergence measure. fbc, q as in sweep. */
static int picard(orc_t *o, double *f, const double *q, const double *fbc, double nu, double nu_s, double tol,
                  int lmax, double *meas, int *status) {
  size_t nn = (size_t)o->nv * o->nnode;
  int nm = o->dim + 2;
  double *fnew = malloc(sizeof(double) * nn), *Mn = malloc(sizeof(double) * nn);
  double *Uo = malloc(sizeof(double) * o->nnode * nm), *Un = malloc(sizeof(double) * o->nnode * nm);
  double *nut = malloc(sizeof(double) * o->nnode * nm);
  moments(o, f, Uo);
  int l = 0;
  *status = ORC_E_NOCONV;
  for (l = 0; l < lmax; ++l) {
    int bad = 0;
    if (o->collision == 1) {
      /* Eq. linear-Maxwellian: the same value n / |V| at every ordinate, |V| = (2L)^d */
      double vol = 1.0;
      for (int al = 0; al < o->dim; ++al) vol *= 2.0 * o->L;
      for (int i = 0; i < o->nnode; ++i) {
        double n = Uo[(size_t)i * nm];
        if (!(n > 0.0) || !isfinite(n)) bad = 1;
        for (int j = 0; j < o->nv; ++j) Mn[(size_t)j * o->nnode + i] = n / vol;
      }
      if (bad) { *status = ORC_E_NONPHYSICAL; break; }
    } else if (o->collision == 2) {
      /* Sec. 5.1.1's alternative: the Maxwellian M_{n,u,theta} (Eq. Maxwellian) evaluated
       * at each grid velocity v_j, n (2 pi theta)^(-d/2) exp(-|v_j - u|^2 / (2 theta)) */
      for (int i = 0; i < o->nnode; ++i) bad |= primitive(o->dim, Uo + (size_t)i * nm, nut + (size_t)i * nm);
      if (bad) { *status = ORC_E_NONPHYSICAL; break; }
      for (int i = 0; i < o->nnode; ++i) {
        const double *p = nut + (size_t)i * nm;
        double th = p[1 + o->dim];
        for (int j = 0; j < o->nv; ++j) {
          double r2 = 0.0;
          for (int al = 0; al < o->dim; ++al) {
            double dv = o->v[(size_t)j * o->dim + al] - p[1 + al];
            r2 += dv * dv;
          }
          Mn[(size_t)j * o->nnode + i] = p[0] * pow(2.0 * acos(-1.0) * th, -0.5 * o->dim) * exp(-r2 / (2.0 * th));
        }
      }
    } else {
      for (int i = 0; i < o->nnode; ++i) bad |= primitive(o->dim, Uo + (size_t)i * nm, nut + (size_t)i * nm);
      if (bad) { *status = ORC_E_NONPHYSICAL; break; }
      orc_maxwellian(o, nut, Mn);
    }
    sweep(o, f, Mn, q, fbc, nu, nu_s, fnew);
    moments(o, fnew, Un);
    *meas = orc_conv_measure(o, Un, Uo);
    memcpy(f, fnew, sizeof(double) * nn);
    double *t = Uo; Uo = Un; Un = t;
    if (*meas < tol) { *status = ORC_OK; ++l; break; }
  }
  free(fnew); free(Mn); free(Uo); free(Un); free(nut);
  return l;
}

/* Set physics: nu = collision frequency, dt = time step, integrator id, tau, l_max. */
void orc_set_physics(orc_t *o, double nu, double dt, int integrator, double tau, int lmax) {
  o->nu = nu; o->dt = dt; o->integrator = integrator; o->tau = tau; o->lmax = lmax;
}

/* Collision model: 0 = the projected Maxwellian (App. B), 1 = the simplified Maxwellian of
 * Eq. linear-Maxwellian (Prop. Linear Stability). */
void orc_set_collision(orc_t *o, int kind) { o->collision = kind; }

/* Boundary conditions of Sec. 4.2 per side of a box: kinds[2a + s] for the side whose unit
 * outward normal is -e_a (s = 0) or +e_a (s = 1); 0 inflow, 1 bounce-back
 * f^bc(x, v) = f(x, -v), 2 reflection f^bc(x, v) = f(x, R_n v), R_n v = v - 2 (v.n) n.
 * A face is on a side when its unit normal's other components are below 1e-10.  The
 * mirror ordinate of each transform is found by searching the grid for the transformed
 * velocity (the paper assumes it is a grid point; ORC_E_INVALID if it is not, within
 * 1e-12 L).  Walls read the mirror's trace from the previous Picard iterate (lagged). */
int orc_set_walls(orc_t *o, const int *kinds) {
  int d = o->dim, nf = o->nface, any = 0;
  free(o->wmirror); free(o->mirror);
  o->wmirror = NULL; o->mirror = NULL;
  for (int k = 0; k < 2 * d; ++k) {
    if (kinds[k] < 0 || kinds[k] > 2) return ORC_E_INVALID;
    if (kinds[k]) any = 1;
  }
  if (!any) return ORC_OK;
  int *mir = malloc(sizeof(int) * (size_t)(1 + d) * o->nv);
  for (int t = 0; t <= d; ++t)
    for (int j = 0; j < o->nv; ++j) {
      double tv[3];
      for (int al = 0; al < d; ++al) {
        double vj = o->v[(size_t)j * d + al];
        tv[al] = (t == 0 || t == 1 + al) ? -vj : vj;
      }
      int found = -1;
      for (int jj = 0; jj < o->nv && found < 0; ++jj) {
        double dmax = 0.0;
        for (int al = 0; al < d; ++al) {
          double e = fabs(o->v[(size_t)jj * d + al] - tv[al]);
          if (e > dmax) dmax = e;
        }
        if (dmax <= 1e-12 * o->L) found = jj;
      }
      if (found < 0) { free(mir); return ORC_E_INVALID; }
      mir[(size_t)t * o->nv + j] = found;
    }
  int *wm = malloc(sizeof(int) * (size_t)o->ncell * nf);
  for (int cf = 0; cf < o->ncell * nf; ++cf) {
    wm[cf] = -1;
    if (o->nbr[cf] >= 0) continue;
    const double *un = o->unit_n + (size_t)cf * d;
    for (int al = 0; al < d; ++al) {
      int aligned = 1;
      for (int be = 0; be < d; ++be)
        if (be != al && !(fabs(un[be]) <= 1e-10)) aligned = 0;
      if (!aligned) continue;
      int kind = kinds[2 * al + (un[al] > 0.0 ? 1 : 0)];
      if (kind == 1) wm[cf] = 0;
      else if (kind == 2) wm[cf] = 1 + al;
    }
  }
  o->wmirror = wm;
  o->mirror = mir;
  return ORC_OK;
}

/* Advance one time step (Sec. 3.5 + Sec. 4).  f: in f^k, out f^{k+1}.  fprev: f^{k-1}
 * (BDF2 only; NULL -> backward Euler start).  fbc: boundary values [j][cell][node].
 * iters[s]: Picard iterations of stage s; meas[s]: final convergence measure. */
int orc_step(orc_t *o, double *f, const double *fprev, const double *fbc, int *iters, double *meas) {
  size_t nn = (size_t)o->nv * o->nnode;
  double A[9], b[3], c[3];
  int S = orc_tableau(o->integrator, A, b, c);
  if (S == 0) return ORC_E_INVALID;
  double dt = o->dt, nu = o->nu;
  double tol = o->tau / (nu * dt > 1.0 ? nu * dt : 1.0);
  int status = ORC_OK;
  if (o->integrator == INT_BDF2 && fprev) {
    /* R6: nu' = nu + 3/(2 dt), q = (4 f^n - f^{n-1}) / (2 dt) */
    double *q = malloc(sizeof(double) * nn);
    for (size_t i = 0; i < nn; ++i) q[i] = (4.0 * f[i] - fprev[i]) / (2.0 * dt);
    iters[0] = picard(o, f, q, fbc, nu, nu + 3.0 / (2.0 * dt), tol, o->lmax, &meas[0], &status);
    free(q);
    return status;
  }
  double *fk = malloc(sizeof(double) * nn), *fs = malloc(sizeof(double) * nn), *q = malloc(sizeof(double) * nn);
  double *F = malloc(sizeof(double) * nn * S);
  memcpy(fk, f, sizeof(double) * nn);
  memcpy(fs, f, sizeof(double) * nn); /* stage 1 starts from f^k; later stages from f^{(s-1)} */
  for (int s = 0; s < S && status == ORC_OK; ++s) {
    double ass = A[s * 3 + s];
    /* Eq. (q-stages): q = (f^k + dt sum_{r<s} A_sr F_r) / (dt A_ss) */
    for (size_t i = 0; i < nn; ++i) {
      double acc = fk[i];
      for (int r = 0; r < s; ++r) acc += dt * A[s * 3 + r] * F[(size_t)r * nn + i];
      q[i] = acc / (dt * ass);
    }
    iters[s] = picard(o, fs, q, fbc, nu, nu + 1.0 / (dt * ass), tol, o->lmax, &meas[s], &status);
    /* Eq. (dirk-recursive-def): F_s = (f^(s) - f^k - dt sum_{r<s} A_sr F_r) / (dt A_ss) */
    for (size_t i = 0; i < nn; ++i) {
      double acc = fs[i] - fk[i];
      for (int r = 0; r < s; ++r) acc -= dt * A[s * 3 + r] * F[(size_t)r * nn + i];
      F[(size_t)s * nn + i] = acc / (dt * ass);
    }
  }
  /* Eq. (dirk-n): f^{k+1} = f^k + dt sum_s b_s F_s */
  for (size_t i = 0; i < nn; ++i) {
    double acc = fk[i];
    for (int s = 0; s < S; ++s) acc += dt * b[s] * F[(size_t)s * nn + i];
    f[i] = acc;
  }
  free(fk); free(fs); free(q); free(F);
  return status;
}
