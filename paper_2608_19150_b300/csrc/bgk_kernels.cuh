// Device kernels of the B300 sweep solver.  All arithmetic of the hot path lives here.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "bgk_internal.h"
#include "bgk_tables.h"

namespace bgk {

// Device-resident iteration state of one handle.
struct DevState {
  int it;            // Picard iterations since creation (parity selects the moment buffer)
  int stage_it;      // iterations of the current stage
  int status;        // BGK_OK or an error of the running step
  int err;           // non-physical moments seen (bit set by the Maxwellian kernel)
  int iters[4];
  double meas[4];
  int iters32[4];    // mixed precision: FP32-phase iterations of each stage
  int total_sweeps;
  int cont;          // the stage loop continues (read by the host in eager mode)
  int done;          // the stage loop of this problem has ended (batched runs skip it)
  int cf_fresh;      // the Maxwellian factors were rebuilt from the current moments by the
                     // moment kernel itself (the factor pass then has nothing to do)
};

__device__ __forceinline__ void ordinate(const VGrid& g, int j, double (&v)[3]) {
  if (g.dim == 2) {
    v[0] = g.x[j / g.N];
    v[1] = g.x[j % g.N];
    v[2] = 0.0;
  } else {
    v[0] = g.x[j / (g.N * g.N)];
    v[1] = g.x[(j / g.N) % g.N];
    v[2] = g.x[j % g.N];
  }
}

// Face code of cell c for velocity v: 2 bits per face, 01 = v.N > 0 (outflow),
// 10 = v.N < 0 (inflow), 00 = no flux.  v.N is evaluated in FP64 with one rounding
// per operation (no contraction), exactly like the host evaluation.
template <int D, int NF>
__device__ __forceinline__ uint32_t face_code(const double* __restrict__ G, const double (&v)[3]) {
  uint32_t code = 0;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    double s = __dmul_rn(v[0], G[f * D + 0]);
    s = __dadd_rn(s, __dmul_rn(v[1], G[f * D + 1]));
    if (D == 3) s = __dadd_rn(s, __dmul_rn(v[2], G[f * D + 2]));
    code |= (s > 0.0 ? 1u : (s < 0.0 ? 2u : 0u)) << (2 * f);
  }
  return code;
}

// ---------------------------------------------------------------------------------
// Conservative projection of a Maxwellian onto the velocity space (App. B):
// c[m] = (1/w_m) int g(v) [E l_m](v) dv, g the 1D Gaussian of mean u, variance theta,
// l_m the Lagrange basis of node m on its velocity cell, extended polynomially beyond
// [-L, L] on the first and last cells.  Exact up to rounding via erfc and the Gaussian
// partial-moment recurrence, in arithmetic R; writes scale * c[m] to out[m * stride].
// grid constants in the projection's arithmetic type (floats precomputed on the host)
template <typename R>
struct GridVals;
template <>
struct GridVals<double> {
  const VGrid& g;
  __device__ double bnd(int c) const { return -g.L + c * g.h; }
  __device__ double mid(int c) const { return -g.L + (c + 0.5) * g.h; }
  __device__ double iw(int m) const { return 1.0 / g.w[m]; }
  __device__ double lag(int k, int p) const { return g.lag[k][p]; }
  __device__ double hh() const { return 0.5 * g.h; }
};
template <>
struct GridVals<float> {
  const VGrid& g;
  __device__ float bnd(int c) const { return g.bnd_f[c]; }
  __device__ float mid(int c) const { return g.mid_f[c]; }
  __device__ float iw(int m) const { return g.iw_f[m]; }
  __device__ float lag(int k, int p) const { return g.lag_f[k][p]; }
  __device__ float hh() const { return g.hh_f; }
};

// KV: the velocity degree k_v as a compile-time constant, so the per-cell arrays below
// stay in registers (proj_factors_t dispatches on g.kv).
// Velocity cells [cl0, cl1) only: the boundary values at cell cl0's left edge are
// evaluated directly (the same expressions the loop carries from cell to cell), so
// disjoint ranges computed separately give the whole projection's values bit for bit.
template <typename R, typename TO, int KV>
__device__ __forceinline__ void proj_factors_cells(const VGrid& g, R u, R theta, TO* out, size_t stride, R scale,
                                                   int cl0, int cl1) {
  constexpr int NP = KV + 1;
  const R rs2 = (R)0.70710678118654752440, rs2pi = (R)0.39894228040143267794;
  const R sig = sqrt(theta), isig = R(1) / sig;
  const GridVals<R> gv{g};
  const R hh = gv.hh();
  // the point weights repeat from cell to cell (uniform grid, the same expression per
  // cell): their reciprocals once per call instead of a division per point (FP64 division
  // is a multi-instruction sequence on B300's narrow FP64 pipe); the same values
  R iwk[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) iwk[k] = gv.iw(k);
  R tprev = -(R)INFINITY, phiprev = 0, Eprev = 0;
  if (cl0 > 0) {
    tprev = (gv.bnd(cl0) - u) * isig;
    phiprev = rs2pi * exp(R(-0.5) * tprev * tprev);
    Eprev = R(0.5) * erfc(fabs(tprev) * rs2);
  }
  for (int cl = cl0; cl < cl1; ++cl) {
    R tb, phib, Eb;
    if (cl == g.ncl - 1) {
      tb = (R)INFINITY;
      phib = 0;
      Eb = 0;
    } else {
      tb = (gv.bnd(cl + 1) - u) * isig;
      phib = rs2pi * exp(R(-0.5) * tb * tb);
      Eb = R(0.5) * erfc(fabs(tb) * rs2);
    }
    const R ta = tprev, phia = phiprev, Ea = Eprev;
    R I[KV + 1];
    // I_0 = Phi(tb) - Phi(ta) from the tails that avoid cancellation
    if (ta >= 0)
      I[0] = Ea - Eb;
    else if (tb <= 0)
      I[0] = Eb - Ea;
    else
      I[0] = (R(1) - Eb) - Ea;
    // I_k = int t^k phi: I_1 = phi(a) - phi(b); I_k = (k-1) I_{k-2} + a^{k-1}phi(a) - b^{k-1}phi(b)
    if (KV >= 1) I[1] = phia - phib;
    R ap = 1, bp = 1;
#pragma unroll
    for (int k = 2; k <= KV; ++k) {
      ap = isinf(ta) ? R(0) : ap * ta;
      bp = isinf(tb) ? R(0) : bp * tb;
      I[k] = (R)(k - 1) * I[k - 2] + (isinf(ta) ? R(0) : ap * phia) - (isinf(tb) ? R(0) : bp * phib);
    }
    // local variable xi = (v - mid)/(h/2) = alpha + beta t
    const R mid = gv.mid(cl);
    const R alpha = (u - mid) / hh, beta = sig / hh;
    R J[KV + 1];  // J_p = int phi (alpha + beta t)^p dt
    R binom[KV + 1];
    binom[0] = 1;
#pragma unroll
    for (int q = 1; q <= KV; ++q) binom[q] = 0;
#pragma unroll
    for (int p = 0; p <= KV; ++p) {
      if (p > 0)
#pragma unroll
        for (int q = p; q >= 1; --q) binom[q] += binom[q - 1];
      R apow[KV + 1];
      apow[0] = 1;
#pragma unroll
      for (int q = 1; q <= p; ++q) apow[q] = apow[q - 1] * alpha;
      R sacc = 0, ab = 1;
#pragma unroll
      for (int q = 0; q <= p; ++q) {
        sacc += binom[q] * apow[p - q] * ab * I[q];
        ab *= beta;
      }
      J[p] = sacc;
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      R sacc = 0;
#pragma unroll
      for (int p = 0; p < NP; ++p) sacc += gv.lag(k, p) * J[p];
      const int m = cl * NP + k;
      out[(size_t)m * stride] = (TO)(scale * sacc * iwk[k]);
    }
    tprev = tb;
    phiprev = phib;
    Eprev = Eb;
  }
}

// First-order change of the projected 1D factors (App. B) of all velocity cells along a
// change (du, dth) of the node's velocity component and temperature, in arithmetic R.
// With t = (v - u)/sigma the Gaussian's mass per dt is phi(t); under the change it moves
// by phi(t) (a t + b (t^2 - 1)) dt, a = du/sigma, b = dth/(2 theta) (the derivatives of
// log G in u and theta), so each projection integral J_p = int xi^p phi dt changes by the
// same combination of partial moments with I_q replaced by
// K_q = a I_{q+1} + b (I_{q+2} - I_q): the recurrence of proj_factors_cells taken two
// orders further.  Writes outd[m] = scale dc[m] + dscale c[m] (the change of scale c[m])
// and outc[m] = scale c[m] + cw outd[m] (cw = 1/2 at the midpoint of a change: the factor
// after the change, to second order).
template <typename R, int KV>
__device__ __forceinline__ void proj_dfactors_cells(const VGrid& g, R u, R theta, R du, R dth, R scale, R dscale,
                                                    R cw, float* outc, float* outd, size_t stride) {
  constexpr int NP = KV + 1, NI = KV + 3;
  const R rs2 = (R)0.70710678118654752440, rs2pi = (R)0.39894228040143267794;
  const R sig = sqrt(theta), isig = R(1) / sig;
  const R ca = du * isig, cb = dth / (R(2) * theta);
  const GridVals<R> gv{g};
  const R hh = gv.hh();
  R iwk[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) iwk[k] = gv.iw(k);
  R tprev = -(R)INFINITY, phiprev = 0, Eprev = 0;
  for (int cl = 0; cl < g.ncl; ++cl) {
    R tb, phib, Eb;
    if (cl == g.ncl - 1) {
      tb = (R)INFINITY;
      phib = 0;
      Eb = 0;
    } else {
      tb = (gv.bnd(cl + 1) - u) * isig;
      phib = rs2pi * exp(R(-0.5) * tb * tb);
      Eb = R(0.5) * erfc(fabs(tb) * rs2);
    }
    const R ta = tprev, phia = phiprev, Ea = Eprev;
    R I[NI];
    if (ta >= 0)
      I[0] = Ea - Eb;
    else if (tb <= 0)
      I[0] = Eb - Ea;
    else
      I[0] = (R(1) - Eb) - Ea;
    I[1] = phia - phib;
    R ap = 1, bp = 1;
#pragma unroll
    for (int k = 2; k < NI; ++k) {
      ap = isinf(ta) ? R(0) : ap * ta;
      bp = isinf(tb) ? R(0) : bp * tb;
      I[k] = (R)(k - 1) * I[k - 2] + (isinf(ta) ? R(0) : ap * phia) - (isinf(tb) ? R(0) : bp * phib);
    }
    R K[NP];
#pragma unroll
    for (int q = 0; q <= KV; ++q) K[q] = ca * I[q + 1] + cb * (I[q + 2] - I[q]);
    const R mid = gv.mid(cl);
    const R alpha = (u - mid) / hh, beta = sig / hh;
    R J[NP], dJ[NP], binom[NP];
    binom[0] = 1;
#pragma unroll
    for (int q = 1; q <= KV; ++q) binom[q] = 0;
#pragma unroll
    for (int p = 0; p <= KV; ++p) {
      if (p > 0)
#pragma unroll
        for (int q = p; q >= 1; --q) binom[q] += binom[q - 1];
      R apow[NP];
      apow[0] = 1;
#pragma unroll
      for (int q = 1; q <= p; ++q) apow[q] = apow[q - 1] * alpha;
      R sj = 0, sd = 0, ab = 1;
#pragma unroll
      for (int q = 0; q <= p; ++q) {
        const R w = binom[q] * apow[p - q] * ab;
        sj += w * I[q];
        sd += w * K[q];
        ab *= beta;
      }
      J[p] = sj;
      dJ[p] = sd;
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      R sc = 0, sd = 0;
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        sc += gv.lag(k, p) * J[p];
        sd += gv.lag(k, p) * dJ[p];
      }
      const R c = sc * iwk[k], d = scale * (sd * iwk[k]) + dscale * c;
      const size_t m = (size_t)(cl * NP + k) * stride;
      outd[m] = (float)d;
      outc[m] = (float)(scale * c + cw * d);
    }
    tprev = tb;
    phiprev = phib;
    Eprev = Eb;
  }
}

template <typename R, typename TO>
__device__ __forceinline__ void proj_factors_range(const VGrid& g, R u, R theta, TO* out, size_t stride, R scale,
                                                   int cl0, int cl1) {
  switch (g.kv) {
    case 1: proj_factors_cells<R, TO, 1>(g, u, theta, out, stride, scale, cl0, cl1); break;
    case 2: proj_factors_cells<R, TO, 2>(g, u, theta, out, stride, scale, cl0, cl1); break;
    case 3: proj_factors_cells<R, TO, 3>(g, u, theta, out, stride, scale, cl0, cl1); break;
    default: proj_factors_cells<R, TO, 4>(g, u, theta, out, stride, scale, cl0, cl1); break;
  }
}

template <typename R, typename TO>
__device__ __forceinline__ void proj_factors_t(const VGrid& g, R u, R theta, TO* out, size_t stride, R scale) {
  proj_factors_range<R, TO>(g, u, theta, out, stride, scale, 0, g.ncl);
}

__device__ __forceinline__ void proj_factors(const VGrid& g, double u, double theta, double* c, int stride) {
  proj_factors_t<double, double>(g, u, theta, c, (size_t)stride, 1.0);
}

// out[j * ostride + p] = coef * n_p * prod_a c_a[j_a](u_p, theta_p) + qscale * q[j * ostride + p]
// for p < npos.  States: mode 0 -> st0 holds (n, u, theta) per node; mode 1 -> moment
// buffers U[it & 1] (n, n u, E), converted to primitives (Eq. moments) with a
// non-physical check.  nodemap (optional) maps output position -> state node.
template <typename T>
__global__ void k_maxwell(VGrid g, int npos, int nm, const double* __restrict__ st0, const double* __restrict__ st1,
                          int mode, const DevState* __restrict__ dsr, DevState* ds, const int32_t* __restrict__ nodemap,
                          T* __restrict__ out, size_t ostride, double coef, const T* __restrict__ q, double qscale) {
  extern __shared__ double csm[];  // [dim*N][blockDim]
  if (ds && ds->status != BGK_OK) return;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int tid = threadIdx.x, bd = blockDim.x;
  if (p >= npos) return;
  const int node = nodemap ? nodemap[p] : p;
  const double* S = (mode == 0) ? st0 : (((dsr->it & 1) == 0) ? st0 : st1);
  const double* Un = S + (size_t)node * nm;
  double n, u[3] = {0, 0, 0}, th;
  if (mode == 0) {
    n = Un[0];
    for (int a = 0; a < g.dim; ++a) u[a] = Un[1 + a];
    th = Un[1 + g.dim];
  } else {
    n = Un[0];
    double u2 = 0.0;
    for (int a = 0; a < g.dim; ++a) {
      u[a] = Un[1 + a] / n;
      u2 += u[a] * u[a];
    }
    th = (2.0 * Un[1 + g.dim] / n - u2) / g.dim;
  }
  if (!(n > 0.0) || !(th > 0.0) || !isfinite(n) || !isfinite(th)) {
    if (ds) atomicOr(&ds->err, 1);
    n = 0.0;
    th = 1.0;
    for (int a = 0; a < g.dim; ++a) u[a] = 0.0;
  }
  for (int a = 0; a < g.dim; ++a) proj_factors(g, u[a], th, csm + (size_t)(a * g.N) * bd + tid, bd);
  const double cn = coef * n;
  if (g.dim == 2) {
    for (int j0 = 0; j0 < g.N; ++j0) {
      const double c0 = cn * csm[(size_t)j0 * bd + tid];
      for (int j1 = 0; j1 < g.N; ++j1) {
        const size_t j = (size_t)j0 * g.N + j1;
        double val = c0 * csm[(size_t)(g.N + j1) * bd + tid];
        if (q) val += qscale * (double)q[j * ostride + p];
        out[j * ostride + p] = (T)val;
      }
    }
  } else {
    for (int j0 = 0; j0 < g.N; ++j0) {
      const double c0 = cn * csm[(size_t)j0 * bd + tid];
      for (int j1 = 0; j1 < g.N; ++j1) {
        const double c01 = c0 * csm[(size_t)(g.N + j1) * bd + tid];
        for (int j2 = 0; j2 < g.N; ++j2) {
          const size_t j = ((size_t)j0 * g.N + j1) * g.N + j2;
          double val = c01 * csm[(size_t)(2 * g.N + j2) * bd + tid];
          if (q) val += qscale * (double)q[j * ostride + p];
          out[j * ostride + p] = (T)val;
        }
      }
    }
  }
}

// Primitive variables of one node from its moments (n, n u, E) (Eq. moments) and the
// scale coef * n of the collision term's first factor.  ok = false for n <= 0, theta <= 0
// or a non-finite value (the simplified Maxwellian needs only n); the factors are then
// written as those of (0, 0, 1) and the caller raises the non-physical flag.
struct NodePrim {
  double n, u[3], th, scale;
  bool ok;
};
__device__ __forceinline__ NodePrim node_prim(const double* U, int dim, double coef, int kind) {
  NodePrim P;
  P.n = U[0];
  P.u[0] = P.u[1] = P.u[2] = 0.0;
  if (kind == BGK_COLL_LINEAR) {
    P.ok = P.n > 0.0 && isfinite(P.n);
    P.th = 1.0;
    P.scale = P.ok ? coef * P.n : 0.0;
    return P;
  }
  double u2 = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (a < dim) {
      P.u[a] = U[1 + a] / P.n;
      u2 += P.u[a] * P.u[a];
    }
  P.th = (2.0 * U[1 + dim] / P.n - u2) / dim;
  P.scale = coef * P.n;
  P.ok = P.n > 0.0 && P.th > 0.0 && isfinite(P.n) && isfinite(P.th);
  if (!P.ok) {
    P.scale = 0.0;
    P.th = 1.0;
    P.u[0] = P.u[1] = P.u[2] = 0.0;
  }
  return P;
}

// Factors of one node along velocity dimension a, for the velocity cells [cl0, cl1):
// out[m * stride], m the 1D points of those cells.  Projected Maxwellian (App. B): c_a[m]
// in the storage type T, with the scale in a = 0; simplified Maxwellian (Eq.
// linear-Maxwellian): scale / (2L)^d in a = 0 and 1 elsewhere; interpolated Maxwellian
// (Sec. 5.1.1): the 1D Gaussian's values at the points.
template <typename T>
__device__ __forceinline__ void node_factors(const VGrid& g, int kind, const NodePrim& P, int a, T* out,
                                             size_t stride, int cl0, int cl1) {
  const int np = g.kv + 1;
  if (kind == BGK_COLL_LINEAR) {
    double vol = 1.0;
    for (int b = 0; b < g.dim; ++b) vol *= 2.0 * g.L;
    const double val = a == 0 ? P.scale / vol : 1.0;
    for (int m = cl0 * np; m < cl1 * np; ++m) out[(size_t)m * stride] = (T)val;
    return;
  }
  if (kind == BGK_COLL_INTERP) {
    const double rs = rsqrt(2.0 * 3.14159265358979323846 * P.th), h = 0.5 / P.th;
    for (int m = cl0 * np; m < cl1 * np; ++m) {
      const double dv = g.x[m] - P.u[a];
      out[(size_t)m * stride] = (T)((a == 0 ? P.scale : 1.0) * rs * exp(-h * dv * dv));
    }
    return;
  }
  proj_factors_range<T, T>(g, (T)P.u[a], (T)P.th, out, stride, (T)(a == 0 ? P.scale : 1.0), cl0, cl1);
}

// ---------------------------------------------------------------------------------
// Inner moment sums over the last velocity dimension: S_k = sum_m W_k[m] f_m with
// W = (w, w x, w x^2), by the compensated dot product of Ogita, Rump and Oishi (2005) in
// FP32 (error-free TwoProduct by fma and TwoSum), with each FP64 weight split into two
// floats (and FP64 data into float pairs), so the sums carry about 48 significant bits --
// FP64 accuracy at FP32 instruction rate.
template <typename T>
struct InnerSums;

// Both storage types are summed with FP32 error-free transformations (TwoProd by FMA,
// TwoSum; the compensated dot product of Ogita, Rump and Oishi), which on B300 run on
// the FP32 pipes at ~58x the FP64 rate: the weights are float pairs wh + wl, FP32 data
// enter as f, FP64 data as a float pair fh + fl split with integer operations.  The
// sums keep ~2^-47 relative accuracy (FP64 rounding is 2^-53; the tolerance of the
// Picard criterion is 1e-8).

// Split a double into floats hi + lo with integer operations only: hi = sign, exponent
// and the leading 23 stored mantissa bits; lo = the remaining 29 bits rounded to float.
// |f - hi - lo| <= 2^-47 |f| for 2^-126 <= |f| < 2^128; smaller magnitudes contribute
// at most 2^-97 absolute; larger ones and non-finite values convert directly.
__device__ __forceinline__ void split_double(double f, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(f);
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ffu);
  const int ef = e - 1023 + 127;  // biased float exponent of hi
  if (ef >= 255) {
    hi = (float)f;
    lo = 0.f;
    return;
  }
  if (ef <= 0) {
    hi = __int_as_float((int)sign);
    lo = hi;
    return;
  }
  const unsigned long long m = b & 0xfffffffffffffull;  // 52 stored mantissa bits
  hi = __int_as_float((int)(sign | ((unsigned int)ef << 23) | (unsigned int)(m >> 29)));
  // lo = (m mod 2^29) * 2^(e - 1075)
  const int pe = e - 1075 + 127;  // biased exponent of 2^(e - 1075)
  const float r = (float)(unsigned int)(m & 0x1fffffffu);
  const float sc = pe >= 1 ? __int_as_float(pe << 23) : 0.f;
  lo = __int_as_float(__float_as_int(r * sc) | (int)sign);
}

// ---------------------------------------------------------------------------------
// Float-pair arithmetic for the FP64-data sweeps of the mixed precision's FP64 phase (PAIR):
// B300 runs FP64 at about 1/62 of its FP32 rate, so the FP64-data sweep forms its
// right-hand side and its product with the cached inverse in pairs of floats hi + lo
// (error-free transformations: TwoProduct by fma, TwoSum, Dekker's renormalisation),
// about 2^-44..2^-47 relative per operation instead of FP64's 2^-53: eight orders below
// the Picard tolerance, at FP32 instruction rates.  The data in memory stay FP64 (split
// with integer operations on load, rebuilt exactly from the pair on store).
struct fpair {
  float h, l;
  __host__ __device__ constexpr fpair() : h(0.f), l(0.f) {}
  __host__ __device__ constexpr fpair(float hi, float lo) : h(hi), l(lo) {}
  // compile-time constants of the element tables (folded by the compiler; runtime FP64
  // values go through fp_split)
  __host__ __device__ constexpr explicit fpair(double d) : h((float)d), l((float)(d - (double)(float)d)) {}
};
__device__ __forceinline__ fpair fp_split(double d) {
  fpair r;
  split_double(d, r.h, r.l);
  return r;
}
__device__ __forceinline__ fpair operator*(fpair a, fpair b) {
  const float p = a.h * b.h;
  const float e = fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p)));
  const float s = p + e;
  return fpair(s, e - (s - p));
}
__device__ __forceinline__ fpair operator+(fpair a, fpair b) {
  const float s = a.h + b.h;  // TwoSum(a.h, b.h), then the low parts, renormalised
  const float v = s - a.h;
  const float e = ((a.h - (s - v)) + (b.h - v)) + (a.l + b.l);
  const float t = s + e;
  return fpair(t, e - (t - s));
}
__device__ __forceinline__ fpair& operator+=(fpair& a, fpair b) {
  a = a + b;
  return a;
}
// scaling by a signed power of two k (the integer face-mass entries of inflow_int): exact
__device__ __forceinline__ fpair operator*(fpair a, float k) { return fpair(a.h * k, a.l * k); }

// The double of a float by integer operations (no FP64 conversion instruction): exact for
// normal floats, zero for zeros and subnormals (at most 2^-126 absolute), infinities and
// NaNs kept non-finite.
__device__ __forceinline__ double float_to_double(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned s = u & 0x80000000u;
  if (e == 0u) return __hiloint2double((int)s, 0);
  const unsigned ed = e == 0xffu ? 0x7ffu : e + 896u;  // 1023 - 127
  return __hiloint2double((int)(s | (ed << 20) | ((u & 0x7fffffu) >> 3)), (int)(u << 29));
}
// a pair stored in the 8 bytes of one double (hi at the lower address) and back
__device__ __forceinline__ fpair fp_from_bits(double d) {
  return fpair(__int_as_float(__double2loint(d)), __int_as_float(__double2hiint(d)));
}
__device__ __forceinline__ double fp_to_bits(fpair a) {
  return __hiloint2double(__float_as_int(a.l), __float_as_int(a.h));
}


template <>
struct InnerSums<float> {
  float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f};
  // accumulate (wh + wl)(fh + fl) for the three weights of point m
  __device__ __forceinline__ void add2(const VGrid& g, int m, float fh, float fl) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float wh = g.wh[k][m], wl = g.wl[k][m];
      const float p = wh * fh;
      const float ep = fmaf(wh, fh, -p) + fmaf(wh, fl, wl * fh);  // p + ep = (wh + wl)(fh + fl) - wl fl
      const float t = hi[k] + p;                                  // TwoSum(hi, p)
      const float z = t - hi[k];
      const float es = (hi[k] - (t - z)) + (p - z);
      hi[k] = t;
      lo[k] += es + ep;
    }
  }
  __device__ __forceinline__ void add(const VGrid& g, int m, float f) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float wh = g.wh[k][m];
      const float p = wh * f;
      const float ep = fmaf(wh, f, -p) + g.wl[k][m] * f;  // p + ep = (wh + wl) f
      const float t = hi[k] + p;                          // TwoSum(hi, p)
      const float z = t - hi[k];
      const float es = (hi[k] - (t - z)) + (p - z);
      hi[k] = t;
      lo[k] += es + ep;
    }
  }
  __device__ __forceinline__ double get(int k) const { return (double)hi[k] + (double)lo[k]; }
  __device__ __forceinline__ fpair pair(int k) const { return fpair(hi[k], lo[k]); }
};

template <>
struct InnerSums<double> {
  InnerSums<float> S;
  __device__ __forceinline__ void add(const VGrid& g, int m, double f) {
    float fh, fl;
    split_double(f, fh, fl);
    S.add2(g, m, fh, fl);
  }
  __device__ __forceinline__ double get(int k) const { return S.get(k); }
  __device__ __forceinline__ fpair pair(int k) const { return S.pair(k); }
};

// The outer levels of the moment sums in the same compensated FP32 arithmetic: acc +=
// (wh + wl) s for a weight pair (the grid's float pairs of w, w x, w x^2, optionally
// halved, which is exact) and a partial sum s carried as an unevaluated pair -- TwoProduct
// and TwoSum with every error term gathered in lo, as in the inner sums, so no FP64
// instruction runs per velocity point (B300 issues FP64 at a small fraction of FP32).
struct MomAcc {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float wh, float wl, fpair v) {
    const float p = wh * v.h;
    const float ep = fmaf(wh, v.h, -p) + fmaf(wh, v.l, wl * v.h);
    const float t = hi + p;
    const float z = t - hi;
    lo += ((hi - (t - z)) + (p - z)) + ep;
    hi = t;
  }
  __device__ __forceinline__ fpair pair() const { return fpair(hi, lo); }
  __device__ __forceinline__ double get() const { return (double)hi + (double)lo; }
};

// Velocity moments U_i = sum_j w_j (1, v_j, |v_j|^2/2) f_{j,i} (Eq. moments), FP64
// accuracy for either storage type.  A block of 128 threads covers 128 / PARTS nodes;
// PARTS thread groups split the outermost velocity index into ranges (more loads in
// flight per node: 4 for FP64 data, 2 for FP32) and their partial sums are added in a
// fixed order.  mode 0: write U[it&1].  mode 1: write U[(it+1)&1] and per-block partial
// sums of |dU_m|^2 and |U_old,m|^2, m = 0, 1, 2, for the criterion of Eq.
// (convergence-criteria).  Launch: 128 threads, ceil(nnode * PARTS / 128) blocks.
template <typename T>
struct MomentParts {
  static constexpr int value = sizeof(T) == 8 ? 4 : 2;
};

//
// Fused with the Maxwellian rebuild (cf != nullptr, mode 1): the block then also writes the
// collision-term factors cf[a][m][i] of its nodes from the new moments (node_factors; the
// work of every (node, dimension, half of the velocity cells) spread over the block's
// threads) and marks them current (ds->cf_fresh), so the next iteration needs no factor
// pass; non-physical moments raise ds->err.  Mode 0 marks the factors stale.
//
// conv: each value read is also written there in the other storage type (FP32 data: its
// double; FP64 data: the float nearest to it), at the same index -- the states handed
// between the FP32 and the FP64 phases of the mixed precision in the same pass that takes
// the moments.  gate: the kernel runs only when gate's loop succeeded (gate_when 1) or
// only when it failed (gate_when 2; failed = non-physical, as k_convert_gated skips).
// fupd, addin (f then unused): the pass first updates fupd += addin in place (the change of
// a Picard iterate, FP32) and sums the updated values.
template <typename T>
__global__ void __launch_bounds__(128) k_moments(VGrid g, const T* __restrict__ f, int nnode, double* U0,
                                                 double* U1, DevState* ds, int mode,
                                                 double* __restrict__ partial, T* __restrict__ cf, double coef,
                                                 int kind, void* __restrict__ conv = nullptr,
                                                 const DevState* __restrict__ gate = nullptr, int gate_when = 0,
                                                 T* fupd = nullptr, const float* __restrict__ addin = nullptr) {
  using TC = typename std::conditional<sizeof(T) == 4, double, float>::type;
  if (ds->status != BGK_OK || ds->done) return;
  if (gate) {
    const bool failed = gate->err || gate->status == BGK_E_NONPHYSICAL;
    if ((gate_when == 1 && failed) || (gate_when == 2 && !failed)) return;
  }
  if (mode == 0 && blockIdx.x == 0 && threadIdx.x == 0) ds->cf_fresh = 0;
  constexpr int PARTS = MomentParts<T>::value, NPB = 128 / PARTS;
  const int nl = threadIdx.x % NPB, part = threadIdx.x / NPB;
  const int i = blockIdx.x * NPB + nl;
  const int nm = g.dim + 2;
  const int ja = part * g.N / PARTS, jb = (part + 1) * g.N / PARTS;
  double acc[5] = {0, 0, 0, 0, 0};
  MomAcc A[5];
  if (i < nnode) {
    if (g.dim == 2) {
      for (int j0 = ja; j0 < jb; ++j0) {
        InnerSums<T> S;
        const size_t o0 = (size_t)j0 * g.N * nnode + i;
        const T* fr = addin ? nullptr : f + o0;
        if (addin) {
          T* fw = fupd + o0;
          const float* dr = addin + o0;
#pragma unroll 8
          for (int j1 = 0; j1 < g.N; ++j1) {
            const T v = fw[(size_t)j1 * nnode] + (T)float_to_double(dr[(size_t)j1 * nnode]);
            fw[(size_t)j1 * nnode] = v;
            S.add(g, j1, v);
          }
        } else if (conv) {
          TC* cr = static_cast<TC*>(conv) + o0;
#pragma unroll 8
          for (int j1 = 0; j1 < g.N; ++j1) {
            const T v = fr[(size_t)j1 * nnode];
            cr[(size_t)j1 * nnode] = (TC)v;
            S.add(g, j1, v);
          }
        }
        // the plain pass: two independent compensated sums (even and odd points) for more
        // loads and arithmetic in flight, added at the end
        InnerSums<T> S2;
        if (!addin && !conv) {
          int j1 = 0;
#pragma unroll 4
          for (; j1 + 1 < g.N; j1 += 2) {
            const T a0 = fr[(size_t)j1 * nnode], a1 = fr[(size_t)(j1 + 1) * nnode];
            S.add(g, j1, a0);
            S2.add(g, j1 + 1, a1);
          }
          if (j1 < g.N) S.add(g, j1, fr[(size_t)j1 * nnode]);
        }
        const fpair s0 = S.pair(0) + S2.pair(0), s1 = S.pair(1) + S2.pair(1), s2 = S.pair(2) + S2.pair(2);
        // acc += w0 (s0, x0 s0, s1, (x0^2 s0 + s2) / 2)
        A[0].add(g.wh[0][j0], g.wl[0][j0], s0);
        A[1].add(g.wh[1][j0], g.wl[1][j0], s0);
        A[2].add(g.wh[0][j0], g.wl[0][j0], s1);
        A[3].add(0.5f * g.wh[2][j0], 0.5f * g.wl[2][j0], s0);
        A[3].add(0.5f * g.wh[0][j0], 0.5f * g.wl[0][j0], s2);
      }
    } else {
      for (int j0 = ja; j0 < jb; ++j0) {
        MomAcc t[4];
        for (int j1 = 0; j1 < g.N; ++j1) {
          InnerSums<T> S;
          const size_t o1 = ((size_t)j0 * g.N + j1) * g.N * nnode + i;
          const T* fr = addin ? nullptr : f + o1;
          if (addin) {
            T* fw = fupd + o1;
            const float* dr = addin + o1;
#pragma unroll 8
            for (int j2 = 0; j2 < g.N; ++j2) {
              const T v = fw[(size_t)j2 * nnode] + (T)float_to_double(dr[(size_t)j2 * nnode]);
              fw[(size_t)j2 * nnode] = v;
              S.add(g, j2, v);
            }
          } else if (conv) {
            TC* cr = static_cast<TC*>(conv) + o1;
#pragma unroll 8
            for (int j2 = 0; j2 < g.N; ++j2) {
              const T v = fr[(size_t)j2 * nnode];
              cr[(size_t)j2 * nnode] = (TC)v;
              S.add(g, j2, v);
            }
          } else {
#pragma unroll 8
            for (int j2 = 0; j2 < g.N; ++j2) S.add(g, j2, fr[(size_t)j2 * nnode]);
          }
          const fpair s0 = S.pair(0), s1 = S.pair(1), s2 = S.pair(2);
          // t += w1 (s0, x1 s0, s1, x1^2 s0 + s2)
          t[0].add(g.wh[0][j1], g.wl[0][j1], s0);
          t[1].add(g.wh[1][j1], g.wl[1][j1], s0);
          t[2].add(g.wh[0][j1], g.wl[0][j1], s1);
          t[3].add(g.wh[2][j1], g.wl[2][j1], s0);
          t[3].add(g.wh[0][j1], g.wl[0][j1], s2);
        }
        // acc += w0 (t0, x0 t0, t1, t2, (x0^2 t0 + t3) / 2)
        const fpair t0 = t[0].pair(), t1 = t[1].pair(), t2 = t[2].pair(), t3 = t[3].pair();
        A[0].add(g.wh[0][j0], g.wl[0][j0], t0);
        A[1].add(g.wh[1][j0], g.wl[1][j0], t0);
        A[2].add(g.wh[0][j0], g.wl[0][j0], t1);
        A[3].add(g.wh[0][j0], g.wl[0][j0], t2);
        A[4].add(0.5f * g.wh[2][j0], 0.5f * g.wl[2][j0], t0);
        A[4].add(0.5f * g.wh[0][j0], 0.5f * g.wl[0][j0], t3);
      }
    }
#pragma unroll
    for (int m = 0; m < 5; ++m) acc[m] = A[m].get();
  }
  if constexpr (PARTS > 1) {
    __shared__ double accp[PARTS][5][NPB];
#pragma unroll
    for (int m = 0; m < 5; ++m) accp[part][m][nl] = acc[m];
    __syncthreads();
    if (part == 0)
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        double t = accp[0][m][nl];
#pragma unroll
        for (int q = 1; q < PARTS; ++q) t += accp[q][m][nl];
        acc[m] = t;
      }
  }
  const bool owner = part == 0 && i < nnode;
  const int cur = ds->it & 1;
  double* Uw = (mode == 0) ? (cur == 0 ? U0 : U1) : (cur == 0 ? U1 : U0);
  if (owner)
#pragma unroll
    for (int m = 0; m < 5; ++m)
      if (m < nm) Uw[(size_t)i * nm + m] = acc[m];
  if (mode == 0) return;
  // partial sums for the convergence measure over the block's nodes
  const double* Uo = cur == 0 ? U0 : U1;
  double r[6] = {0, 0, 0, 0, 0, 0};
  if (owner) {
    const double* o = Uo + (size_t)i * nm;
    r[0] = (acc[0] - o[0]) * (acc[0] - o[0]);
    r[1] = o[0] * o[0];
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (a < g.dim) {
        r[2] += (acc[1 + a] - o[1 + a]) * (acc[1 + a] - o[1 + a]);
        r[3] += o[1 + a] * o[1 + a];
      }
    const double aE = g.dim == 2 ? acc[3] : acc[4];
    r[4] = (aE - o[nm - 1]) * (aE - o[nm - 1]);
    r[5] = o[nm - 1] * o[nm - 1];
  }
  __shared__ double red[6][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double x = r[k];
    for (int o2 = 16; o2 > 0; o2 >>= 1) x += __shfl_down_sync(0xffffffffu, x, o2);
    if (lane == 0) red[k][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < 6)
    partial[(size_t)blockIdx.x * 6 + threadIdx.x] =
        ((red[threadIdx.x][0] + red[threadIdx.x][1]) + red[threadIdx.x][2]) + red[threadIdx.x][3];
  if (!cf) return;
  // the Maxwellian of the new moments (Sec. 3.3, App. B) for the next iteration
  __shared__ NodePrim prim[NPB];
  if (part == 0) {
    double Uc[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) Uc[m] = acc[m];
    prim[nl] = node_prim(Uc, g.dim, coef, kind);
    if (i < nnode && !prim[nl].ok) atomicOr(&ds->err, 1);
  }
  __syncthreads();
  const int H = (128 / NPB) / g.dim > 1 ? 2 : 1;
  const int tasks = NPB * g.dim * H;
  for (int t = threadIdx.x; t < tasks; t += 128) {
    const int q = t % NPB, r = t / NPB, a = r % g.dim, hh = r / g.dim;
    const int iq = blockIdx.x * NPB + q;
    if (iq < nnode)
      node_factors<T>(g, kind, prim[q], a, cf + (size_t)a * g.N * nnode + iq, (size_t)nnode, hh * g.ncl / H,
                      (hh + 1) * g.ncl / H);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ds->cf_fresh = 1;
}

// Partial moments over the ordinates whose outermost velocity index lies in [ja, jb) (one
// shard of an ordinate-sharded sweep): out[i][m] = sum over those j of w_j e_m(v_j) f_j,i.
// The shards' partial moments add up to Eq. (moments).
template <typename T>
__global__ void k_moments_range(VGrid g, const T* __restrict__ f, int nnode, int ja, int jb,
                                double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nnode) return;
  const int nm = g.dim + 2;
  const size_t inner = g.dim == 2 ? (size_t)g.N : (size_t)g.N * g.N;  // ordinates per outer index
  double acc[5] = {0, 0, 0, 0, 0};
  for (int j0 = ja; j0 < jb; ++j0) {
    double t0 = 0, t1 = 0, t2 = 0, t3 = 0;
    const int nmid = g.dim == 2 ? 1 : g.N;
    for (int j1 = 0; j1 < nmid; ++j1) {
      InnerSums<T> S;
      const T* fr = f + ((size_t)j0 * inner + (size_t)j1 * g.N) * nnode + i;
      for (int j2 = 0; j2 < g.N; ++j2) S.add(g, j2, fr[(size_t)j2 * nnode]);
      const double s0 = S.get(0), s1 = S.get(1), s2 = S.get(2);
      const double w1 = g.dim == 2 ? 1.0 : g.w[j1], x1 = g.dim == 2 ? 0.0 : g.x[j1];
      t0 += w1 * s0;
      t1 += w1 * x1 * s0;
      t2 += w1 * s1;
      t3 += w1 * (x1 * x1 * s0 + s2);
    }
    const double w0 = g.w[j0], x0 = g.x[j0];
    acc[0] += w0 * t0;
    acc[1] += w0 * x0 * t0;
    if (g.dim == 2) {
      acc[2] += w0 * t2;
      acc[3] += 0.5 * w0 * (x0 * x0 * t0 + t3);
    } else {
      acc[2] += w0 * t1;
      acc[3] += w0 * t2;
      acc[4] += 0.5 * w0 * (x0 * x0 * t0 + t3);
    }
  }
#pragma unroll
  for (int m = 0; m < 5; ++m)
    if (m < nm) out[(size_t)i * nm + m] = acc[m];
}

// Collision-term factors of every node from the current moments U[it & 1]: cf[a][m][i]
// (node_factors), coef * n_i folded into a = 0.  The moments and primitive variables are
// FP64; the projection runs in the storage type T (FP64 for FP64 states, FP32 for FP32
// sweeps, whose source is FP32 anyway).  Non-physical moments set the error flag (the
// stage loop then stops).  Nothing to do when the moment kernel has already rebuilt the
// factors from these moments (ds->cf_fresh).
// pairs (T = double, float-pair sweeps): each factor is stored as its float pair in the
// 8 bytes of its double (fp_to_bits), split once here for the pair source pass.
template <typename T>
__global__ void k_factors(VGrid g, int nnode, const double* __restrict__ U0, const double* __restrict__ U1,
                          DevState* ds, double coef, T* __restrict__ cf, int kind, int pairs) {
  if (ds->status != BGK_OK || ds->done || ds->cf_fresh) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nnode) return;
  const int nm = g.dim + 2;
  const NodePrim P = node_prim((((ds->it & 1) == 0) ? U0 : U1) + (size_t)i * nm, g.dim, coef, kind);
  if (!P.ok) atomicOr(&ds->err, 1);
  for (int a = 0; a < g.dim; ++a) {
    T* out = cf + (size_t)a * g.N * nnode + i;
    node_factors<T>(g, kind, P, a, out, (size_t)nnode, 0, g.ncl);
    if constexpr (sizeof(T) == 8) {
      if (pairs)
        for (int m = 0; m < g.N; ++m) out[(size_t)m * nnode] = fp_to_bits(fp_split(out[(size_t)m * nnode]));
    }
  }
}
// src[j][i] = prod_a cf[a][j_a][i] + qscale * q[j][i]  (nu M^l + q of Eq. bgk-ss-picard)
// Launch: 2D grid, blockIdx.y (and its strides) over ordinates, x over nodes (k_source_grid),
// so no thread divides a flat index.
template <typename T, typename TQ = T>
__global__ void k_source(VGrid g, int nnode, const T* __restrict__ cf, const TQ* __restrict__ q, T qscale,
                         T* __restrict__ src, const DevState* ds) {
  if (ds->status != BGK_OK || ds->done) return;
  for (int j = blockIdx.y; j < g.nv; j += gridDim.y) {
    const T* c1;
    const T* c2;
    const T* c3 = nullptr;
    if (g.dim == 2) {
      c1 = cf + (size_t)(j / g.N) * nnode;
      c2 = cf + (size_t)(g.N + j % g.N) * nnode;
    } else {
      c1 = cf + (size_t)(j / (g.N * g.N)) * nnode;
      c2 = cf + (size_t)(g.N + (j / g.N) % g.N) * nnode;
      c3 = cf + (size_t)(2 * g.N + j % g.N) * nnode;
    }
    const TQ* qj = q + (size_t)j * nnode;
    T* sj = src + (size_t)j * nnode;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nnode; i += gridDim.x * blockDim.x) {
      T m = c1[i] * c2[i];
      if (c3) m = m * c3[i];
      sj[i] = fma(qscale, (T)qj[i], m);
    }
  }
}

// Picard refinement of the mixed precision (2D): the change of the collision-term factors
// between two FP64-phase iterates.  C32 = the new factors as floats, D32 = new - old as
// floats of the difference taken in the stored precision (FP64 values, or float pairs:
// (hi - hi') + (lo - lo'), exact to about 2^-48 of the factors).  n = rows x nodes.
__global__ void k_delta_factors(size_t n, const double* __restrict__ cf, const double* __restrict__ cf_prev,
                                int pairs, float* __restrict__ C32, float* __restrict__ D32, const DevState* ds) {
  if (ds->status != BGK_OK || ds->done) return;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    if (pairs) {
      const fpair a = fp_from_bits(cf[t]), b = fp_from_bits(cf_prev[t]);
      C32[t] = a.h;
      D32[t] = (a.h - b.h) + (a.l - b.l);
    } else {
      C32[t] = (float)cf[t];
      D32[t] = (float)(cf[t] - cf_prev[t]);
    }
  }
}

// Picard refinement with the projected Maxwellian: the same C32 and D32 as k_delta_factors
// (the new factors and their change, rows x nodes) without the FP64 factors of either
// iterate stored.  Per node the primitive variables of the last two iterates' moments
// (U[it & 1] new, the other buffer old) and their change dP in FP64; where the largest
// relative change (|dn|/n, |du_a|/sqrt(theta), |dtheta|/theta) is below lin_max, the
// factors' change is the derivative at the midpoint of the two states along dP
// (proj_dfactors_cells in FP32: the neglected terms are of third order in dP, the FP32
// rounding about 1e-6 of the change), otherwise the difference of the two states' FP64
// factors (node_factors, through the scratch rows Wn and Wo: rows x nodes).  The rounding
// of the derivatives adds up over the stage's corrections, so they serve only when the
// stage's FP32 phase (state gate, stage st) ended normally within phase_max (its last
// measure): the FP64 phase then moves the moments by about that much in all.
__global__ void k_delta_factors_lin(VGrid g, int nnode, const double* __restrict__ U0, const double* __restrict__ U1,
                                    DevState* ds, double coef, float* __restrict__ C32, float* __restrict__ D32,
                                    double lin_max, double* __restrict__ Wn, double* __restrict__ Wo,
                                    const DevState* __restrict__ gate, int st, double phase_max) {
  if (ds->status != BGK_OK || ds->done) return;
  const bool phase_ok = !gate->err && gate->status == BGK_OK && gate->meas[st] <= phase_max;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nnode) return;
  const int nm = g.dim + 2;
  const bool cur0 = (ds->it & 1) == 0;
  const NodePrim Pn = node_prim((cur0 ? U0 : U1) + (size_t)i * nm, g.dim, coef, BGK_COLL_MAXWELLIAN);
  const NodePrim Po = node_prim((cur0 ? U1 : U0) + (size_t)i * nm, g.dim, coef, BGK_COLL_MAXWELLIAN);
  if (!Pn.ok || !Po.ok) atomicOr(&ds->err, 1);
  double rel = fabs(Pn.n - Po.n) / Po.n;
  rel = fmax(rel, fabs(Pn.th - Po.th) / Po.th);
  const double isg = rsqrt(Po.th);
  for (int a = 0; a < g.dim; ++a) rel = fmax(rel, fabs(Pn.u[a] - Po.u[a]) * isg);
  if (phase_ok && rel < lin_max) {
    const double thm = 0.5 * (Po.th + Pn.th);
    const float th = (float)thm, dth = (float)(Pn.th - Po.th);
    for (int a = 0; a < g.dim; ++a) {
      const float u = (float)(0.5 * (Po.u[a] + Pn.u[a])), du = (float)(Pn.u[a] - Po.u[a]);
      const float sc = a == 0 ? (float)(0.5 * (Po.scale + Pn.scale)) : 1.0f;
      const float dsc = a == 0 ? (float)(Pn.scale - Po.scale) : 0.0f;
      float* oc = C32 + (size_t)a * g.N * nnode + i;
      float* od = D32 + (size_t)a * g.N * nnode + i;
      switch (g.kv) {
        case 1: proj_dfactors_cells<float, 1>(g, u, th, du, dth, sc, dsc, 0.5f, oc, od, (size_t)nnode); break;
        case 2: proj_dfactors_cells<float, 2>(g, u, th, du, dth, sc, dsc, 0.5f, oc, od, (size_t)nnode); break;
        case 3: proj_dfactors_cells<float, 3>(g, u, th, du, dth, sc, dsc, 0.5f, oc, od, (size_t)nnode); break;
        default: proj_dfactors_cells<float, 4>(g, u, th, du, dth, sc, dsc, 0.5f, oc, od, (size_t)nnode); break;
      }
    }
  } else {
    // both states' factors in FP64 (each thread reads back only its own node's values)
    for (int a = 0; a < g.dim; ++a) {
      const size_t r = (size_t)a * g.N * nnode + i;
      node_factors<double>(g, BGK_COLL_MAXWELLIAN, Pn, a, Wn + r, (size_t)nnode, 0, g.ncl);
      node_factors<double>(g, BGK_COLL_MAXWELLIAN, Po, a, Wo + r, (size_t)nnode, 0, g.ncl);
      for (int m = 0; m < g.N; ++m) {
        const double cn = Wn[r + (size_t)m * nnode], co = Wo[r + (size_t)m * nnode];
        C32[r + (size_t)m * nnode] = (float)cn;
        D32[r + (size_t)m * nnode] = (float)(cn - co);
      }
    }
  }
}

// The change of the source nu M between two iterates (2D: M = c_1[j_1] c_2[j_2]), from the
// factors' change: c1' c2' - c1 c2 = c1' (c2' - c2) + (c1' - c1) c2, in FP32 (it is the
// source of a correction sweep whose result is a small change of f).  dM[j][i].
// Launch: 2D grid, blockIdx.y (and its strides) over ordinates, x over nodes.
__global__ void k_delta_source(VGrid g, int nnode, const float* __restrict__ C32, const float* __restrict__ D32,
                               float* __restrict__ dM, const DevState* ds) {
  if (ds->status != BGK_OK || ds->done) return;
  for (int j = blockIdx.y; j < g.nv; j += gridDim.y) {
    float* out = dM + (size_t)j * nnode;
    if (g.dim == 2) {
      const size_t r1 = (size_t)(j / g.N) * nnode, r2 = (size_t)(g.N + j % g.N) * nnode;
      for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nnode; i += gridDim.x * blockDim.x) {
        const float c2old = C32[r2 + i] - D32[r2 + i];
        out[i] = fmaf(C32[r1 + i], D32[r2 + i], D32[r1 + i] * c2old);
      }
    } else {
      // c1'c2'c3' - c1c2c3 = (c1'-c1) c2'c3' + c1 (c2'-c2) c3' + c1 c2 (c3'-c3)
      const size_t r1 = (size_t)(j / (g.N * g.N)) * nnode, r2 = (size_t)(g.N + (j / g.N) % g.N) * nnode,
                   r3 = (size_t)(2 * g.N + j % g.N) * nnode;
      for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nnode; i += gridDim.x * blockDim.x) {
        const float a1 = C32[r1 + i], a2 = C32[r2 + i], a3 = C32[r3 + i];
        const float d1 = D32[r1 + i], d2 = D32[r2 + i], d3 = D32[r3 + i];
        const float o1 = a1 - d1, o2 = a2 - d2;
        out[i] = fmaf(d1, a2 * a3, fmaf(o1, d2 * a3, o1 * o2 * d3));
      }
    }
  }
}

// k_delta_source for 2D grids: a block of blockDim.x nodes first stages the second
// velocity dimension's rows for its nodes in shared memory (c2 = c2' - (c2' - c2) and
// c2' - c2: 2 N blockDim.x floats), then each thread loops over j_1 (c1' and c1' - c1 of
// its node in registers) and j_2, so the loads are a small fraction of the stores (the
// same FP32 expression per element).  Launch: x over node blocks, dynamic shared memory
// 8 N blockDim.x bytes.
__global__ void k_delta_source_2d(VGrid g, int nnode, const float* __restrict__ C32, const float* __restrict__ D32,
                                  float* __restrict__ dM, const DevState* ds) {
  extern __shared__ float rows2[];  // [2][N][blockDim.x]: c2, then c2' - c2
  if (ds->status != BGK_OK || ds->done) return;
  const int nb = (int)blockDim.x, t = (int)threadIdx.x, N = g.N;
  for (int i0 = blockIdx.x * nb; i0 < nnode; i0 += gridDim.x * nb) {
    const int i = i0 + t;
    __syncthreads();
    if (i < nnode)
      for (int j2 = 0; j2 < N; ++j2) {
        const size_t r2 = (size_t)(N + j2) * nnode + i;
        const float d2 = D32[r2];
        rows2[j2 * nb + t] = C32[r2] - d2;
        rows2[(N + j2) * nb + t] = d2;
      }
    __syncthreads();
    if (i >= nnode) continue;
    for (int j1 = 0; j1 < N; ++j1) {
      const size_t r1 = (size_t)j1 * nnode + i;
      const float a1 = C32[r1], d1 = D32[r1];
      float* out = dM + (size_t)j1 * N * nnode + i;
      for (int j2 = 0; j2 < N; ++j2)
        out[(size_t)j2 * nnode] = fmaf(a1, rows2[(N + j2) * nb + t], d1 * rows2[j2 * nb + t]);
    }
  }
}

// The change of f made by the FP64 phase's full sweep of a stage, as the FP32 start of the
// refinement's corrections (their wall data and lagged inflow read the previous change):
// d = f - f_prev with f_prev the state the sweep started from -- the FP32 phase's result
// (exactly the double of d's own buffer), or, when that phase failed and left the FP64
// state as it was, the copy taken before the sweep.
__global__ void k_delta0(size_t n, const double* __restrict__ f, float* d, const double* __restrict__ fsave,
                         const DevState* __restrict__ gate, const DevState* ds) {
  if (ds->status != BGK_OK || ds->done) return;
  const bool failed = gate->err || gate->status == BGK_E_NONPHYSICAL;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    d[t] = (float)(f[t] - (failed ? fsave[t] : (double)d[t]));
}

// out <- in when gate reports that its loop failed (the state the FP64 phase starts from
// is then not the FP32 phase's result)
__global__ void k_copy_if_failed(size_t n, const double* __restrict__ in, double* __restrict__ out,
                                 const DevState* __restrict__ gate) {
  if (!(gate->err || gate->status == BGK_E_NONPHYSICAL)) return;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    out[t] = in[t];
}

// grid of k_source: about four nodes per thread of 256, at most 65535 ordinate rows
inline dim3 k_source_grid(int nnode, int nv) {
  const int bx = (nnode + 1023) / 1024;
  return dim3((unsigned)(bx > 0 ? bx : 1), (unsigned)(nv < 65535 ? nv : 65535));
}

// Reduce the partials in a fixed order, evaluate Eq. (convergence-criteria) (m = 1
// denominator max(|U^1|, |U^0|)), advance the iteration counters and set the while
// condition of the stage loop.
// stall_stop (FP32 phase of the mixed mode): also stop once the measure is below 1e-5
// and has decreased by less than 10% over the last iteration (FP32 rounding floor).
// stall_stop (the FP32 phase of the mixed precision): also stop once the measure is below
// 1e-5 and fell by less than 10% (stagnation), or once two more iterations at the observed
// contraction rate rho = meas / prev would bring it below half the next phase's tolerance
// tol_next (rho^2 meas < tol_next / 2): the FP64 phase then needs its two iterations
// whatever further FP32 iterations do.
__global__ void k_finalize(DevState* ds, const double* __restrict__ partial, int nblk, double tol, int lmax, int stage,
                           cudaGraphConditionalHandle cond, int use_cond, int stall_stop = 0,
                           double tol_next = 0.0) {
  __shared__ double red[6][256];
  double s[6] = {0, 0, 0, 0, 0, 0};
  const bool skip = ds->status != BGK_OK || ds->done;
  if (!skip)
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
      for (int k = 0; k < 6; ++k) s[k] += partial[(size_t)b * 6 + k];
  for (int k = 0; k < 6; ++k) red[k][threadIdx.x] = s[k];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < 6; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  int cont = 0;
  if (!skip) {
    const double r0 = sqrt(red[0][0]) / sqrt(red[1][0]);
    const double r1 = sqrt(red[2][0]) / fmax(sqrt(red[3][0]), sqrt(red[1][0]));
    const double r2 = sqrt(red[4][0]) / sqrt(red[5][0]);
    const double meas = fmax(r0, fmax(r1, r2));
    const double prev = ds->meas[stage];
    ds->it += 1;
    ds->stage_it += 1;
    ds->total_sweeps += 1;
    ds->iters[stage] = ds->stage_it;
    ds->meas[stage] = meas;
    const bool stalled = stall_stop && ds->stage_it > 2 && meas < 1e-5 && meas > 0.9 * prev;
    const double rho = prev > 0.0 ? meas / prev : 1.0;
    const bool enough = stall_stop && ds->stage_it > 1 && rho < 1.0 && rho * rho * meas < 0.5 * tol_next;
    if (ds->err) {
      ds->status = BGK_E_NONPHYSICAL;
    } else if (!(meas < tol) && !stalled && !enough) {
      if (ds->stage_it >= lmax)
        ds->status = BGK_E_NOCONV;
      else
        cont = 1;
    }
  }
  ds->cont = cont;
  ds->done = !cont;
  if (use_cond) cudaGraphSetConditional(cond, cont);
}

// U = sum_p parts[p] in part order p = 0, 1, ... (elementwise; the same bits for the same
// inputs on every device), n values per part.
__global__ void k_sum_parts(const double* __restrict__ parts, int nparts, size_t n, double* __restrict__ U) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double s = parts[i];
    for (int p = 1; p < nparts; ++p) s += parts[(size_t)p * n + i];
    U[i] = s;
  }
}

// Per-block sums of the convergence measure's squares (Eq. convergence-criteria): for
// U_new, U_old [node][d+2]: |dU_0|^2, |U_0|^2, |dU_1..d|^2, |U_1..d|^2, |dU_d+1|^2, |U_d+1|^2
// into partial[block][6]; one fixed block size and grid, so the sums are deterministic.
__global__ void __launch_bounds__(256) k_measure_parts(const double* __restrict__ Un, const double* __restrict__ Uo,
                                                       int nnode, int dim, double* __restrict__ partial) {
  __shared__ double red[6][256];
  const int nm = dim + 2;
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nnode; i += gridDim.x * blockDim.x) {
    const double* a = Un + (size_t)i * nm;
    const double* b = Uo + (size_t)i * nm;
    double d = a[0] - b[0];
    s[0] += d * d;
    s[1] += b[0] * b[0];
    for (int al = 1; al <= dim; ++al) {
      d = a[al] - b[al];
      s[2] += d * d;
      s[3] += b[al] * b[al];
    }
    d = a[dim + 1] - b[dim + 1];
    s[4] += d * d;
    s[5] += b[dim + 1] * b[dim + 1];
  }
  for (int k = 0; k < 6; ++k) red[k][threadIdx.x] = s[k];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < 6; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 6; ++k) partial[(size_t)blockIdx.x * 6 + k] = red[k][0];
}

__global__ void k_stage_begin(DevState* ds, int stage) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ds->stage_it = 0;
    ds->done = 0;
    ds->cont = 1;
    ds->iters[stage] = 0;
    ds->meas[stage] = 0.0;
  }
}

__global__ void k_reset_state(DevState* ds) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ds->status = BGK_OK;
    ds->err = 0;
    ds->done = 0;
    ds->cf_fresh = 0;
    for (int s = 0; s < 4; ++s) {
      ds->iters[s] = 0;
      ds->meas[s] = 0.0;
      ds->iters32[s] = 0;
    }
  }
}

// ---------------------------------------------------------------------------------
// Generations of every ordinate's sweep graph (Sec. 4.1): Kahn's peel, one CTA per
// ordinate.  In-degrees are packed bytes in shared memory.  Level g of the list is the
// set Gen_j(g): cells whose longest path from a source has length g.  Lagged inflow
// faces (bit f of lag[c]) are not edges.  Writes glist[j][*] (packed entries, level
// by level), lvl[j][g] (level starts), ngen[j], nproc[j] (cells reached).
template <int D, int NF>
__global__ void k_peel(const double* __restrict__ geo, int gs, const int32_t* __restrict__ nbr,
                       const int32_t* __restrict__ nbr_face, int ncell, VGrid g, const int32_t* __restrict__ jlist,
                       const uint8_t* __restrict__ lag, uint32_t* __restrict__ glist, int32_t* __restrict__ lvl,
                       int32_t* __restrict__ ngen, int32_t* __restrict__ nproc) {
  extern __shared__ uint32_t indeg[];
  __shared__ int cnt;
  const int j = jlist ? jlist[blockIdx.x] : blockIdx.x;
  const uint8_t* lj = lag ? lag + (size_t)blockIdx.x * ncell : nullptr;
  double v[3];
  ordinate(g, j, v);
  uint32_t* gl = glist + (size_t)j * ncell;
  int32_t* lv = lvl + (size_t)j * (ncell + 1);
  const int nw = (ncell + 3) >> 2;
  for (int w = threadIdx.x; w < nw; w += blockDim.x) indeg[w] = 0u;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
    const uint32_t code = face_code<D, NF>(geo + (size_t)c * gs, v);
    uint32_t deg = 0;
    const uint32_t lb = lj ? lj[c] : 0u;
#pragma unroll
    for (int f = 0; f < NF; ++f)
      if (((code >> (2 * f)) & 3u) == 2u && nbr[(size_t)c * 4 + f] >= 0 && !((lb >> f) & 1u)) ++deg;
    if (deg)
      atomicAdd(&indeg[c >> 2], deg << (8 * (c & 3)));
    else
      gl[atomicAdd(&cnt, 1)] = (uint32_t)c | (code << kCellBits);
  }
  __syncthreads();
  int start = 0, end = cnt, gen = 0;
  while (start < end) {
    if (threadIdx.x == 0) lv[gen] = start;
    for (int k = start + threadIdx.x; k < end; k += blockDim.x) {
      const uint32_t e = gl[k];
      const int c = (int)(e & kCellMask);
      const uint32_t code = e >> kCellBits;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        if (((code >> (2 * f)) & 3u) != 1u) continue;
        const int nb = nbr[(size_t)c * 4 + f];
        if (nb < 0) continue;
        if (lag) {
          const int f2 = nbr_face[(size_t)c * 4 + f];
          if ((lj[nb] >> f2) & 1u) continue;
        }
        const uint32_t old = atomicSub(&indeg[nb >> 2], 1u << (8 * (nb & 3)));
        if (((old >> (8 * (nb & 3))) & 0xFFu) == 1u) {
          const uint32_t cb = face_code<D, NF>(geo + (size_t)nb * gs, v);
          gl[atomicAdd(&cnt, 1)] = (uint32_t)nb | (cb << kCellBits);
        }
      }
    }
    __syncthreads();
    start = end;
    end = cnt;
    ++gen;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    lv[gen] = start;
    ngen[j] = gen;
    nproc[j] = start;
  }
}

// Order of the cells inside each generation (Sec. 4.1: the cells of one generation are
// independent, so any order gives the same sweep): counting sort by the packed face code,
// so that the threads of a warp, which take consecutive positions, mostly share one
// inflow/outflow pattern and the face-dependent code of the local solve does not diverge.
// One CTA per ordinate; generations longer than cap entries keep their order.
__global__ void k_sort_gen(uint32_t* __restrict__ glist, const int32_t* __restrict__ lvl,
                           const int32_t* __restrict__ ngen, int ncell, int cap) {
  extern __shared__ uint32_t sbuf[];  // cap entries
  __shared__ int hist[256];
  const int j = blockIdx.x;
  uint32_t* gl = glist + (size_t)j * ncell;
  const int32_t* lv = lvl + (size_t)j * (ncell + 1);
  const int G = ngen[j];
  for (int gg = 0; gg < G; ++gg) {
    const int a = lv[gg], n = lv[gg + 1] - a;
    if (n <= 1 || n > cap) continue;  // (uniform over the block)
    for (int t = threadIdx.x; t < 256; t += blockDim.x) hist[t] = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const uint32_t e = gl[a + k];
      sbuf[k] = e;
      atomicAdd(&hist[e >> kCellBits], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int t = 0; t < 256; ++t) {
        const int c = hist[t];
        hist[t] = acc;
        acc += c;
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const uint32_t e = sbuf[k];
      gl[a + atomicAdd(&hist[e >> kCellBits], 1)] = e;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------
// LU without pivoting: the local matrix has a positive definite symmetric part
// (nu_s M + upwind transport), so elimination in natural order is stable.
template <int N, typename T>
__device__ __forceinline__ void lu_solve(T (&A)[N][N], T (&b)[N]) {
  T inv[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    // FP32 sweeps take the fast reciprocal (2 ulp): the FP32 phase is refined in FP64
    if constexpr (sizeof(T) == 4)
      inv[k] = __fdividef(1.0f, A[k][k]);
    else
      inv[k] = T(1) / A[k][k];
#pragma unroll
    for (int i = k + 1; i < N; ++i) {
      const T l = A[i][k] * inv[k];
#pragma unroll
      for (int c = k + 1; c < N; ++c) A[i][c] -= l * A[k][c];
      b[i] -= l * b[k];
    }
  }
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    T s = b[i];
#pragma unroll
    for (int c = i + 1; c < N; ++c) s -= A[i][c] * b[c];
    b[i] = s * inv[i];
  }
}

// Sweep schedule of one ordinate, as the kernels see it.
struct SweepArgs {
  const double* geo;
  const float* geof;   // the same geometry as floats (FP32 sweeps)
  int gs;
  const int32_t* nbr;
  const uint64_t* perm;
  const uint32_t* glist;
  const int32_t* lvl;
  const int32_t* ngen;
  int ncell, nnode, nbface;
};

// Local operator of one (cell, ordinate) from its packed schedule entry (Sec. 3.3):
// r_i = s_i / |K| with the sign taken from the entry's face code.
template <class E, typename T>
__device__ __forceinline__ void face_rates(const double* __restrict__ Gc, uint32_t code, T v0, T v1, T v2,
                                           T (&r)[E::NF], unsigned& outm, int gstride = 1) {
  constexpr int D = E::D, NF = E::NF;
  const T invK = (T)Gc[(NF * D) * gstride];
  outm = 0;
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    const uint32_t fl = (code >> (2 * i)) & 3u;
    T s = v0 * (T)Gc[(i * D) * gstride] + v1 * (T)Gc[(i * D + 1) * gstride];
    if (D == 3) s += v2 * (T)Gc[(i * D + 2) * gstride];
    s = fabs(s) * invK;
    r[i] = fl == 1u ? s : (fl == 2u ? -s : T(0));
    outm |= (fl == 1u ? 1u : 0u) << i;
  }
}

// Elements per cached local inverse: ND*ND rounded up to a 16-byte multiple, so every
// inverse starts on a 16-byte boundary (vector loads, 16-byte asynchronous copies).
template <class E, typename T>
__host__ __device__ constexpr int ainv_stride() {
  return (E::NDOF * E::NDOF + (int)(16 / sizeof(T)) - 1) / (int)(16 / sizeof(T)) * (int)(16 / sizeof(T));
}

// face_rates with the geometry already held in registers as T
template <class E, typename T>
__device__ __forceinline__ void face_rates_t(const T (&Gc)[E::NF * E::D + 1], uint32_t code, T v0, T v1, T v2,
                                             T (&r)[E::NF], unsigned& outm) {
  constexpr int D = E::D, NF = E::NF;
  const T invK = Gc[NF * D];
  outm = 0;
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    const uint32_t fl = (code >> (2 * i)) & 3u;
    T s = v0 * Gc[i * D] + v1 * Gc[i * D + 1];
    if (D == 3) s += v2 * Gc[i * D + 2];
    s = fabs(s) * invK;
    r[i] = fl == 1u ? s : (fl == 2u ? -s : T(0));
    outm |= (fl == 1u ? 1u : 0u) << i;
  }
}

// Inverse of the local matrix of every (ordinate, schedule position), computed in FP64
// by Gauss-Jordan elimination in natural order and stored as T in schedule order:
// Ainv[(j * ncell + k) * S + a * ND + b], S = ainv_stride.  Valid for one nu_s; a sweep with that
// nu_s then needs only the right-hand side and one matrix-vector product per cell.
// PAIR (T = double): each FP64 entry is stored as a float pair hi + lo (split_double,
// |X - hi - lo| <= 2^-47 |X|) in the same S * 8 bytes: the S hi floats, then the S lo
// floats, for the float-pair product of the sweep (sweep_ordinate, PAIR).
template <class E, typename T, bool PAIR = false>
__global__ void k_local_inverse(SweepArgs sa, VGrid g, double nus, T* __restrict__ Ainv) {
  constexpr int ND = E::NDOF, NF = E::NF;
  const size_t total = (size_t)g.nv * sa.ncell;
  for (size_t it = (size_t)blockIdx.x * blockDim.x + threadIdx.x; it < total; it += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(it / sa.ncell);
    const int k = (int)(it % sa.ncell);
    double vd[3];
    ordinate(g, j, vd);
    const uint32_t e = sa.glist[(size_t)j * sa.ncell + k];
    const int c = (int)(e & kCellMask);
    double r[NF];
    unsigned outm;
    face_rates<E, double>(sa.geo + (size_t)c * sa.gs, e >> kCellBits, vd[0], vd[1], vd[2], r, outm);
    double A[ND][ND], X[ND][ND];
    E::assemble(nus, r, outm, A);
#pragma unroll
    for (int a = 0; a < ND; ++a)
#pragma unroll
      for (int bb = 0; bb < ND; ++bb) X[a][bb] = a == bb ? 1.0 : 0.0;
#pragma unroll
    for (int p = 0; p < ND; ++p) {
      const double inv = 1.0 / A[p][p];
#pragma unroll
      for (int cc = 0; cc < ND; ++cc) {
        A[p][cc] *= inv;
        X[p][cc] *= inv;
      }
#pragma unroll
      for (int i = 0; i < ND; ++i) {
        if (i == p) continue;
        const double l = A[i][p];
#pragma unroll
        for (int cc = 0; cc < ND; ++cc) {
          A[i][cc] -= l * A[p][cc];
          X[i][cc] -= l * X[p][cc];
        }
      }
    }
    T* out = Ainv + it * ainv_stride<E, T>();
    if constexpr (PAIR) {
      static_assert(sizeof(T) == 8, "float pairs replace FP64 entries");
      constexpr int AS = ainv_stride<E, T>();
      float* o = reinterpret_cast<float*>(out);
#pragma unroll
      for (int a = 0; a < ND; ++a)
#pragma unroll
        for (int bb = 0; bb < ND; ++bb) split_double(X[a][bb], o[a * ND + bb], o[AS + a * ND + bb]);
    } else {
#pragma unroll
      for (int a = 0; a < ND; ++a)
#pragma unroll
        for (int bb = 0; bb < ND; ++bb) out[a * ND + bb] = (T)X[a][bb];
    }
  }
}

// Asynchronous global -> shared copies (cp.async, 4 or 8 bytes), per-thread groups.
__device__ __forceinline__ void cp_async_bytes(void* smem, const void* gmem, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
// Asynchronous prefetch of `bytes` (a multiple of 16, 16-byte aligned) into L2.
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

// Shared-memory slots of one thread for the prefetched geometry and local inverse: two
// slots, each the cell's gs geometry doubles followed by the padded inverse, stored
// contiguously per thread and filled with 16-byte asynchronous copies.
template <class E, typename T>
struct PrefetchSlots {
  unsigned char* base;
  int nt, tid, gs;
  static constexpr int AS = ainv_stride<E, T>();
  __device__ __forceinline__ size_t per_thread() const { return (size_t)gs * sizeof(double) + AS * sizeof(T); }
  __device__ __forceinline__ unsigned char* slot(int s) const { return base + ((size_t)s * nt + tid) * per_thread(); }
  __device__ __forceinline__ const double* geo(int s) const { return (const double*)slot(s); }
  __device__ __forceinline__ const T* ainv(int s) const { return (const T*)(slot(s) + (size_t)gs * sizeof(double)); }
  // issue the copies of item k (cell c) into slot s and commit them as one group
  __device__ __forceinline__ void issue(int s, const double* __restrict__ geo_g, const T* __restrict__ ainv_g,
                                        int c, int k) const {
    unsigned char* d = slot(s);
    const unsigned char* gsrc = (const unsigned char*)(geo_g + (size_t)c * gs);
    for (int q = 0; q < gs * (int)sizeof(double) / 16; ++q) cp_async16(d + 16 * q, gsrc + 16 * q);
    d += (size_t)gs * sizeof(double);
    const unsigned char* asrc = (const unsigned char*)(ainv_g + (size_t)k * AS);
#pragma unroll
    for (int q = 0; q < AS * (int)sizeof(T) / 16; ++q) cp_async16(d + 16 * q, asrc + 16 * q);
    cp_async_commit();
  }
};

// Per-item data that does not depend on values written during the sweep, so the next
// item's copy can be loaded while the current item is processed.
// REG: the item also carries its geometry (converted to T), loaded one item ahead in
// registers (FP32 sweeps; FP64 sweeps are bound by FP64 arithmetic, not by latency).
// FUSED: the item carries the stage source q and the Maxwellian factors of its nodes
// instead of src, and the solve forms src = prod_a cf[a][j_a] + qscale q itself (the
// product of k_source, in the same order), so no src array is written or read.
template <class E, typename T, bool REG = false, bool FUSED = false>
struct SweepItem {
  uint32_t e;
  int4 nb;
  uint64_t pm;
  T src[E::NDOF];  // src, or q when FUSED
  T geo[REG ? E::NF * E::D + 1 : 1];
  T c1[FUSED ? E::NDOF : 1], c2[FUSED ? E::NDOF : 1], c3[(FUSED && E::D == 3) ? E::NDOF : 1];
};

// Values per cell of the geometry rows (face normals N_i, 1/|K|, padding): the layout of
// the host set-up, checked when a handle is created.
template <class E>
__host__ __device__ constexpr int geo_stride() {
  return E::D == 3 ? 16 : (E::NF == 4 ? 10 : 8);
}

// Source of one sweep launch: src = nu M^l + qscale q precomputed (src), or its factors
// (FUSED: cf[a][m][node] of k_factors, q and qscale).
template <typename T>
struct SrcArgs {
  const T* src;
  const T* cf;
  const T* q;
  T qscale;
};

// Per-ordinate pointers of the source: sj = src or q; c1..c3 the factor rows of j's
// velocity indices (j lexicographic, last dimension fastest).
template <typename T>
struct SrcRows {
  const T* sj;
  const T* c1;
  const T* c2;
  const T* c3;
};

template <typename T, bool FUSED>
__device__ __forceinline__ SrcRows<T> src_rows(const SrcArgs<T>& sr, const VGrid& g, int j, int nnode) {
  SrcRows<T> r{};
  if constexpr (FUSED) {
    r.sj = sr.q + (size_t)j * nnode;
    if (g.dim == 2) {
      r.c1 = sr.cf + (size_t)(j / g.N) * nnode;
      r.c2 = sr.cf + (size_t)(g.N + j % g.N) * nnode;
    } else {
      r.c1 = sr.cf + (size_t)(j / (g.N * g.N)) * nnode;
      r.c2 = sr.cf + (size_t)(g.N + (j / g.N) % g.N) * nnode;
      r.c3 = sr.cf + (size_t)(2 * g.N + j % g.N) * nnode;
    }
  } else {
    r.sj = sr.src + (size_t)j * nnode;
  }
  return r;
}

// Load the N values of T at p with the widest vector loads that p's alignment (ALIGN
// bytes, a compile-time fact of the layout) allows.
// (the vector types are read as such and unpacked by value: no type-punned stores into v)
template <typename T, int N, int ALIGN>
__device__ __forceinline__ void load_vec(const T* __restrict__ p, T (&v)[N]) {
  constexpr int BYTES = N * (int)sizeof(T);
  if constexpr (sizeof(T) == 4 && ALIGN % 16 == 0 && BYTES % 16 == 0) {
#pragma unroll
    for (int q = 0; q < N / 4; ++q) {
      const float4 t = reinterpret_cast<const float4*>(p)[q];
      v[4 * q] = t.x;
      v[4 * q + 1] = t.y;
      v[4 * q + 2] = t.z;
      v[4 * q + 3] = t.w;
    }
  } else if constexpr (sizeof(T) == 4 && ALIGN % 8 == 0 && BYTES % 8 == 0) {
#pragma unroll
    for (int q = 0; q < N / 2; ++q) {
      const float2 t = reinterpret_cast<const float2*>(p)[q];
      v[2 * q] = t.x;
      v[2 * q + 1] = t.y;
    }
  } else if constexpr (sizeof(T) == 8 && ALIGN % 16 == 0 && BYTES % 16 == 0) {
#pragma unroll
    for (int q = 0; q < N / 2; ++q) {
      const double2 t = reinterpret_cast<const double2*>(p)[q];
      v[2 * q] = t.x;
      v[2 * q + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] = p[q];
  }
}

// Read-only global data (not written while the kernel runs) in 256-bit loads when p is
// 32-byte aligned and the size a multiple of 32 bytes (sm_100 and later); otherwise as
// load_vec.  A warp's scattered loads cost one L1 wavefront per distinct line and
// instruction: a cell's data in half as many instructions.
template <typename T, int N, int ALIGN>
__device__ __forceinline__ void load_ro(const T* __restrict__ p, T (&v)[N]) {
  constexpr int BYTES = N * (int)sizeof(T);
  if constexpr (ALIGN % 32 == 0 && BYTES % 32 == 0 && sizeof(T) == 4) {
#pragma unroll
    for (int q = 0; q < N / 8; ++q)
      asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
          : "=f"(v[8 * q]), "=f"(v[8 * q + 1]), "=f"(v[8 * q + 2]), "=f"(v[8 * q + 3]), "=f"(v[8 * q + 4]),
            "=f"(v[8 * q + 5]), "=f"(v[8 * q + 6]), "=f"(v[8 * q + 7])
          : "l"(p + 8 * q));
  } else if constexpr (ALIGN % 32 == 0 && BYTES % 32 == 0 && sizeof(T) == 8) {
#pragma unroll
    for (int q = 0; q < N / 4; ++q)
      asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
          : "=d"(v[4 * q]), "=d"(v[4 * q + 1]), "=d"(v[4 * q + 2]), "=d"(v[4 * q + 3])
          : "l"(p + 4 * q));
  } else {
    load_vec<T, N, ALIGN>(p, v);
  }
}

// alignment in bytes of a cell's node values (cell * NDOF * sizeof(T) from a 256-byte
// aligned array whose ordinate rows are NDOF * n_cells values long)
template <class E, typename T>
__host__ __device__ constexpr int cell_align() {
  return (E::NDOF * (int)sizeof(T)) % 16 == 0 ? 16 : (E::NDOF * (int)sizeof(T)) % 8 == 0 ? 8 : 4;
}

// Loads of an item whose schedule entry e is already known.
template <class E, typename T, bool REG, bool FUSED>
__device__ __forceinline__ void fetch_item_e(const SweepArgs& sa, uint32_t e, const SrcRows<T>& rw,
                                             SweepItem<E, T, REG, FUSED>& it) {
  it.e = e;
  const int c = (int)(it.e & kCellMask);
  it.nb = *reinterpret_cast<const int4*>(sa.nbr + (size_t)c * 4);
  it.pm = sa.perm[c];
  const size_t o = (size_t)c * E::NDOF;
  constexpr int AL = cell_align<E, T>();
  load_vec<T, E::NDOF, AL>(rw.sj + o, it.src);
  if constexpr (FUSED) {
    load_vec<T, E::NDOF, AL>(rw.c1 + o, it.c1);
    load_vec<T, E::NDOF, AL>(rw.c2 + o, it.c2);
    if constexpr (E::D == 3) load_vec<T, E::NDOF, AL>(rw.c3 + o, it.c3);
  }
  if constexpr (REG) {
    // the cell's whole geometry row (padding included) in the widest aligned vector loads:
    // a warp's scattered loads cost one L1 wavefront per distinct line and instruction
    constexpr int GS = geo_stride<E>(), GA = (GS * 4) % 32 == 0 ? 32 : (GS * 4) % 16 == 0 ? 16 : 8;
    float gr[GS];
    load_ro<float, GS, GA>(sa.geof + (size_t)c * GS, gr);
#pragma unroll
    for (int q = 0; q <= E::NF * E::D; ++q) it.geo[q] = gr[q];
  }
}

template <class E, typename T, bool REG, bool FUSED>
__device__ __forceinline__ void fetch_item(const SweepArgs& sa, const uint32_t* __restrict__ gl,
                                           const SrcRows<T>& rw, int k, SweepItem<E, T, REG, FUSED>& it) {
  fetch_item_e<E, T, REG, FUSED>(sa, gl[k], rw, it);
}

// FUSED: replace q by src = prod c + qscale q (as k_source forms it) once the item
// becomes the current one, so only src stays live while it waits to be solved.
template <class E, typename T, bool REG, bool FUSED>
__device__ __forceinline__ void resolve_src(SweepItem<E, T, REG, FUSED>& it, T qscale) {
  if constexpr (FUSED) {
#pragma unroll
    for (int a = 0; a < E::NDOF; ++a) {
      T m = it.c1[a] * it.c2[a];
      if constexpr (E::D == 3) m = m * it.c3[a];
      it.src[a] = fma(qscale, it.src[a], m);
    }
  }
}

// Barrier of the threads that share one ordinate's sweep: the whole CTA, or a named
// barrier over a sub-group of `count` threads (a multiple of 32).
struct CtaBarrier {
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};
// No barrier: a single thread sweeps its ordinate alone (TS).
struct NoBarrier {
  __device__ __forceinline__ void sync() const {}
};
struct NamedBarrier {
  int id, count;
  __device__ __forceinline__ void sync() const {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
  }
};

// |v . N_i| / |K| of face i in FP64 for the pair sweeps, with explicit roundings so that
// every pair kernel forms the same value
template <class E>
__device__ __forceinline__ double inflow_rate64(const double* __restrict__ Gc, int i, double v0, double v1,
                                                double v2) {
  double sf = __dmul_rn(v0, Gc[i * E::D]);
  sf = __fma_rn(v1, Gc[i * E::D + 1], sf);
  if constexpr (E::D == 3) sf = __fma_rn(v2, Gc[i * E::D + 2], sf);
  return __dmul_rn(fabs(sf), Gc[E::NF * E::D]);
}

// x = Ainv b of one cell in pairs: Ainv as the float pairs of k_local_inverse<E, double,
// true> (hi at Ap[0 .. S), lo at Ap[S .. 2S)); each x_a = sum_b (Ah + Al)(bh + bl) is the
// compensated dot product of Ogita, Rump and Oishi (TwoProduct by fma, TwoSum) with the
// cross terms Ah bl + Al bh in the error term and Al bl (2^-48 of the product) left out:
// about 2^-47 of the sum of |terms|.  x is returned as FP64 (hi + lo, one FP64 add).
template <int ND, int S>
__device__ __forceinline__ void inverse_product_pair_r(const float (&Ah)[S], const float (&Al)[S],
                                                       const fpair (&b)[ND], double (&x)[ND]) {
#pragma unroll
  for (int a = 0; a < ND; ++a) {
    const float* ah = Ah + a * ND;
    const float* al = Al + a * ND;
    float hi = ah[0] * b[0].h;
    float lo = fmaf(ah[0], b[0].h, -hi) + fmaf(ah[0], b[0].l, al[0] * b[0].h);
#pragma unroll
    for (int q = 1; q < ND; ++q) {
      const float p = ah[q] * b[q].h;
      const float ep = fmaf(ah[q], b[q].h, -p) + fmaf(ah[q], b[q].l, al[q] * b[q].h);
      const float t = hi + p;  // TwoSum(hi, p)
      const float z = t - hi;
      const float es = (hi - (t - z)) + (p - z);
      hi = t;
      lo += es + ep;
    }
    x[a] = float_to_double(hi) + float_to_double(lo);
  }
}
template <int S>
__device__ __forceinline__ void load_inverse_pair(const float* __restrict__ Ap, float (&Ah)[S], float (&Al)[S]) {
  if constexpr (S % 8 == 4) {
    // 32-byte aligned inverses of 2 S floats (S = 8 m + 4): hi = m 32-byte loads and a
    // 16-byte tail; lo = a 16-byte head, then m 32-byte loads from a 32-byte boundary
    float h1[S - 4], t1[4], t2[4], l2[S - 4];
    load_ro<float, S - 4, 32>(Ap, h1);
    load_vec<float, 4, 16>(Ap + S - 4, t1);
    load_vec<float, 4, 16>(Ap + S, t2);
    load_ro<float, S - 4, 32>(Ap + S + 4, l2);
#pragma unroll
    for (int q = 0; q < S - 4; ++q) {
      Ah[q] = h1[q];
      Al[4 + q] = l2[q];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      Ah[S - 4 + q] = t1[q];
      Al[q] = t2[q];
    }
  } else if constexpr (S % 8 == 0) {
    load_ro<float, S, 32>(Ap, Ah);
    load_ro<float, S, 32>(Ap + S, Al);
  } else {
    load_vec<float, S, 16>(Ap, Ah);
    load_vec<float, S, (S % 4 == 0 ? 16 : 8)>(Ap + S, Al);
  }
}
template <int ND, int S>
__device__ __forceinline__ void inverse_product_pair(const float* __restrict__ Ap, const fpair (&b)[ND],
                                                     double (&x)[ND]) {
  float Ah[S], Al[S];
  load_inverse_pair<S>(Ap, Ah, Al);
  inverse_product_pair_r<ND, S>(Ah, Al, b, x);
}

// PAIR source pass (cf as float pairs from k_factors<double> with pairs set):
// b0[j][cell] = Mh (prod_a cf[a][j_a] + qscale q[j]) over the cell's
// nodes, in pairs, stored as pairs in the 8 bytes of each node's double (fp_to_bits), so
// the PAIR sweep starts from the mass-weighted source (the FP64 sweep applies Mh itself).
// Launch: 2D grid, blockIdx.y (and its strides) over ordinates, x over cells.
template <class E>
__global__ void k_source_pair(VGrid g, int ncell, const double* __restrict__ cf, const double* __restrict__ q,
                              double qscale, double* __restrict__ b0, const DevState* ds) {
  if (ds->status != BGK_OK || ds->done) return;
  constexpr int ND = E::NDOF;
  const size_t nnode = (size_t)ncell * ND;
  const fpair qs = fp_split(qscale);
  for (int j = blockIdx.y; j < g.nv; j += gridDim.y) {
    const double* c1;
    const double* c2;
    const double* c3 = nullptr;
    if (g.dim == 2) {
      c1 = cf + (size_t)(j / g.N) * nnode;
      c2 = cf + (size_t)(g.N + j % g.N) * nnode;
    } else {
      c1 = cf + (size_t)(j / (g.N * g.N)) * nnode;
      c2 = cf + (size_t)(g.N + (j / g.N) % g.N) * nnode;
      c3 = cf + (size_t)(2 * g.N + j % g.N) * nnode;
    }
    const double* qj = q + (size_t)j * nnode;
    double* bj = b0 + (size_t)j * nnode;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
      const size_t o = (size_t)c * ND;
      fpair sv[ND], bv[ND];
#pragma unroll
      for (int a = 0; a < ND; ++a) {
        fpair m = fp_from_bits(c1[o + a]) * fp_from_bits(c2[o + a]);
        if (c3) m = m * fp_from_bits(c3[o + a]);
        sv[a] = m + qs * fp_split(qj[o + a]);
      }
      E::mass(sv, bv);
#pragma unroll
      for (int a = 0; a < ND; ++a) bj[o + a] = fp_to_bits(bv[a]);
    }
  }
}

// One ordinate's transport sweep (Sec. 4, Eq. bgk-ss-picard) by a group of `nt` threads
// (thread `tid` of the group) walking the ordinate's generations; the cells of one
// generation are independent and share the group's threads.  For cell K and ordinate j
// (s_i = v_j . N_i, r_i = s_i/|K|):
//   (nu_s Mh + sum_i r_i (Dd_i + [s_i>0] Eh_i)) f_K = Mh src_K + sum_{s_i<0} (-r_i) Eh_i y_i
// where src = nu M^l + q and y_i is the upwind trace: the neighbour's value in f,
// updated in place.  An upwind cell reached by a lagged (cycle) edge has a higher
// generation, so it still holds f^l when read; boundary faces read fbc.
// CACHED: the local inverse comes from k_local_inverse (schedule order, coalesced);
// otherwise the matrix is assembled and factorised in place.  PAIR (FP64 data, cached
// float-pair inverse): src holds the pairs of Mh src (k_source_pair) and the inflow terms
// and the product with the inverse run in float pairs (fpair).  The schedule entry, the
// neighbour ids, the node permutation and src of the thread's next item are loaded
// before the current item is solved (they are not written during the sweep).
template <class E, typename T, bool CACHED, class Bar, bool PF = false, bool FUSED = false, bool PAIR = false>
__device__ __forceinline__ void sweep_ordinate(const SweepArgs& sa, const VGrid& g, int j, T nus,
                                               const SrcArgs<T>& sr, const T* __restrict__ fbc,
                                               const T* __restrict__ Ainv, T* f, int tid, int nt, const Bar& bar,
                                               unsigned char* pf_smem = nullptr) {
  constexpr int ND = E::NDOF, NF = E::NF, FD = E::FD;
  double vd[3];
  ordinate(g, j, vd);
  const T v0 = (T)vd[0], v1 = (T)vd[1], v2 = (T)vd[2];
  const uint32_t* gl = sa.glist + (size_t)j * sa.ncell;
  const int32_t* lv = sa.lvl + (size_t)j * (sa.ncell + 1);
  const T* Aj = CACHED ? Ainv + (size_t)j * sa.ncell * ainv_stride<E, T>() : nullptr;
  const int G = sa.ngen[j];
  T* fj = f + (size_t)j * sa.nnode;
  const SrcRows<T> rw = src_rows<T, FUSED>(sr, g, j, sa.nnode);
  const T* bj = fbc + (size_t)j * sa.nbface * FD;
  constexpr bool REG = !PF && sizeof(T) == 4;
  SweepItem<E, T, REG, FUSED> cur, nxt;
  // prefetch slots (PF): item data of cur in slot `slot`, of nxt in slot ^ 1
  const PrefetchSlots<E, T> pfs{pf_smem, nt, tid, sa.gs};
  int slot = 0;
  // The thread's items are the positions lv[g] + tid + m nt of each generation g, in
  // order.  The one being solved (k), the next (kn: its data is loaded while k is
  // solved) and the one after (kn2: its schedule entry is loaded while k is solved), so
  // no load of item data waits on the entry load before it.
  auto seek = [&](int g2, int& kq, int& gq) {
    for (; g2 < G; ++g2) {
      const int k2 = lv[g2] + tid;
      if (k2 < lv[g2 + 1]) {
        kq = k2;
        gq = g2;
        return;
      }
    }
    kq = -1;
    gq = G;
  };
  auto advance = [&](int kq, int gq, int& kr, int& gr) {
    if (kq < 0) {
      kr = -1;
      gr = G;
    } else if (kq + nt < lv[gq + 1]) {
      kr = kq + nt;
      gr = gq;
    } else {
      seek(gq + 1, kr, gr);
    }
  };
  int k, gk, kn, gn, kn2, gn2;
  seek(0, k, gk);
  advance(k, gk, kn, gn);
  advance(kn, gn, kn2, gn2);
  if (k >= 0) {
    fetch_item<E, T, REG, FUSED>(sa, gl, rw, k, cur);
    resolve_src(cur, sr.qscale);
    if (PF) pfs.issue(slot, sa.geo, Aj, (int)(cur.e & kCellMask), k);
  }
  uint32_t en = kn >= 0 ? gl[kn] : 0u;
  for (int gg = 0; gg < G; ++gg) {
    while (k >= 0 && gk == gg) {
      if (kn >= 0) {
        // the next item's cached inverse streams from HBM into L2 while this one is solved
        if constexpr (CACHED && !PF) prefetch_l2_bulk(Aj + (size_t)kn * ainv_stride<E, T>(),
                                                      ainv_stride<E, T>() * (uint32_t)sizeof(T));
        fetch_item_e<E, T, REG, FUSED>(sa, en, rw, nxt);
        if (PF) pfs.issue(slot ^ 1, sa.geo, Aj, (int)(nxt.e & kCellMask), kn);
      }
      const uint32_t en2 = kn2 >= 0 ? gl[kn2] : 0u;
      if (PF) {
        if (kn >= 0)
          cp_async_wait<1>();
        else
          cp_async_wait<0>();
      }
      // ---- solve item k
      const int c = (int)(cur.e & kCellMask);
      const uint32_t code = cur.e >> kCellBits;
      // face rates r_i (all faces for the assembly; with a cached inverse only the inflow
      // faces' |r_i| are needed and are formed below, face by face)
      T r[NF];
      unsigned outm = 0;
      if constexpr (!CACHED) {
        if constexpr (REG)
          face_rates_t<E, T>(cur.geo, code, v0, v1, v2, r, outm);
        else
          face_rates<E, T>(sa.geo + (size_t)c * sa.gs, code, v0, v1, v2, r, outm);
      }
      T b[ND];
      fpair bp[PAIR ? ND : 1];  // PAIR: the right-hand side in pairs, from Mh src
      if constexpr (PAIR) {
#pragma unroll
        for (int a = 0; a < ND; ++a) bp[a] = fp_from_bits(cur.src[a]);
      } else {
        E::mass(cur.src, b);
      }
      const int nbs[4] = {cur.nb.x, cur.nb.y, cur.nb.z, cur.nb.w};
      // upwind traces of all faces in one round of loads (no branch between them): an
      // inflow face reads its neighbour's values (or the boundary data), any other face
      // reads this cell's own old values, which are not used
      T y[NF][FD];
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        const bool in = ((code >> (2 * i)) & 3u) == 2u;
        const int nb = nbs[i];
#pragma unroll
        for (int kk = 0; kk < FD; ++kk) {
          const T* p = !in ? fj + (size_t)c * ND
                           : (nb >= 0 ? fj + (size_t)nb * ND + (int)((cur.pm >> (16 * i + 4 * kk)) & 15u)
                                      : bj + (size_t)(-nb - 1) * FD + kk);
          y[i][kk] = *p;
        }
      }
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        if (((code >> (2 * i)) & 3u) != 2u) continue;
        T ci;
        if constexpr (CACHED) {
          // |v . N_i| / |K| of inflow face i, as face_rates forms it
          if constexpr (REG) {
            T sf = v0 * cur.geo[i * E::D] + v1 * cur.geo[i * E::D + 1];
            if (E::D == 3) sf += v2 * cur.geo[i * E::D + 2];
            ci = fabs(sf) * cur.geo[NF * E::D];
          } else if constexpr (PAIR) {
            ci = inflow_rate64<E>(sa.geo + (size_t)c * sa.gs, i, v0, v1, v2);
          } else {
            const double* Gc = PF ? pfs.geo(slot) : sa.geo + (size_t)c * sa.gs;
            T sf = v0 * (T)Gc[i * E::D] + v1 * (T)Gc[i * E::D + 1];
            if (E::D == 3) sf += v2 * (T)Gc[i * E::D + 2];
            ci = fabs(sf) * (T)Gc[NF * E::D];
          }
        } else {
          ci = -r[i];
        }
        if constexpr (PAIR) {
          fpair yp[FD];
#pragma unroll
          for (int kk = 0; kk < FD; ++kk) yp[kk] = fp_split(y[i][kk]);
          E::inflow_int(i, fp_split(ci) * fpair(1.0 / E::inflow_den), yp, bp);
        } else {
          E::inflow(i, ci, y[i], b);
        }
      }
      T x[ND];
      if constexpr (CACHED && PAIR) {
        static_assert(sizeof(T) == 8 && !PF && !REG, "pair sweep: FP64 data, inverse read in place");
        inverse_product_pair<ND, ainv_stride<E, T>()>(
            reinterpret_cast<const float*>(Aj + (size_t)k * ainv_stride<E, T>()), bp, x);
      } else if (CACHED) {
        // the inverse is 16-byte aligned and padded: read it with 128-bit loads
        constexpr int AS = ainv_stride<E, T>(), NV = AS * (int)sizeof(T) / 16;
        static_assert(AS * (int)sizeof(T) == NV * 16, "padded inverse");
        const T* Ap = PF ? pfs.ainv(slot) : Aj + (size_t)k * AS;
        {
          T Ar[AS];
          load_vec<T, AS, 16>(Ap, Ar);
#pragma unroll
          for (int a = 0; a < ND; ++a) {
            T s = T(0);
#pragma unroll
            for (int bb = 0; bb < ND; ++bb) s += Ar[a * ND + bb] * b[bb];
            x[a] = s;
          }
        }
      } else {
        T A[ND][ND];
        E::assemble(nus, r, outm, A);
        lu_solve<ND, T>(A, b);
#pragma unroll
        for (int a = 0; a < ND; ++a) x[a] = b[a];
      }
#pragma unroll
      for (int a = 0; a < ND; ++a) fj[(size_t)c * ND + a] = x[a];
      // ---- advance
      if (kn >= 0) {
        cur = nxt;
        resolve_src(cur, sr.qscale);
        slot ^= 1;
      }
      k = kn;
      gk = gn;
      kn = kn2;
      gn = gn2;
      en = en2;
      advance(kn, gn, kn2, gn2);
    }
    bar.sync();
  }
  if (PF) cp_async_wait<0>();
}

// The FP64-data sweep in float pairs (PAIR): at most 128 registers, so that every CTA of
// the launch is resident at once.
template <class E>
__global__ void __launch_bounds__(128, 4) k_sweep_pair(SweepArgs sa, VGrid g, double nus, SrcArgs<double> sr,
                                                     const double* __restrict__ fbc,
                                                     const double* __restrict__ Ainv, double* f,
                                                     const DevState* ds, int jofs) {
  if (ds && (ds->status != BGK_OK || ds->done)) return;
  sweep_ordinate<E, double, true, CtaBarrier, false, false, true>(sa, g, jofs + (int)blockIdx.x, nus, sr, fbc,
                                                                  Ainv, f, (int)threadIdx.x, (int)blockDim.x,
                                                                  CtaBarrier());
}

// One sweep of every ordinate of one problem: one CTA per ordinate.  PF: the cached
// local inverse and the geometry of each thread's next cell are copied to shared memory
// asynchronously while the current cell is solved (dynamic shared memory).
// Topological sweep (TS, Sec. 4.1): one thread per ordinate walks that ordinate's whole
// schedule alone, cell after cell in generation order, with no barrier; the concurrent
// work is the number of ordinates (the generation sweep's is ordinates x generation
// width).  Same operations per cell as the generation sweep.
template <class E, typename T, bool CACHED, bool FUSED = false, bool PAIR = false>
__global__ void __launch_bounds__(64) k_sweep_ts(SweepArgs sa, VGrid g, T nus, SrcArgs<T> sr,
                                                 const T* __restrict__ fbc, const T* __restrict__ Ainv, T* f,
                                                 const DevState* ds, int jb, int je) {
  if (ds && (ds->status != BGK_OK || ds->done)) return;
  const int j = jb + (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (j >= je) return;
  sweep_ordinate<E, T, CACHED, NoBarrier, false, FUSED, PAIR>(sa, g, j, nus, sr, fbc, Ainv, f, 0, 1, NoBarrier());
}

// (ordinates jofs + blockIdx.x: all of them, or one shard's range)
template <class E, typename T, bool CACHED, bool PF = false, bool FUSED = false>
__global__ void __launch_bounds__(256) k_sweep(SweepArgs sa, VGrid g, T nus, SrcArgs<T> sr,
                                               const T* __restrict__ fbc, const T* __restrict__ Ainv, T* f,
                                               const DevState* ds, int jofs) {
  extern __shared__ __align__(16) unsigned char pf_smem[];
  if (ds && (ds->status != BGK_OK || ds->done)) return;
  sweep_ordinate<E, T, CACHED, CtaBarrier, PF, FUSED>(sa, g, jofs + (int)blockIdx.x, nus, sr, fbc, Ainv, f,
                                                      (int)threadIdx.x, (int)blockDim.x, CtaBarrier(), pf_smem);
}

// ---------------------------------------------------------------------------------
// Shared-memory front of the FP32 generation sweep.  The trace of a cell on one of its
// outflow faces is read by the neighbour across that face, in a later generation of the
// same ordinate when the edge is not lagged (Sec. 4.1), so it only has to live from the
// cell's generation to the neighbour's.  Per ordinate, every such (cell, outflow face)
// gets a 16-byte slot of a shared-memory buffer by greedy interval colouring in generation
// order (a slot is free again one generation after its reader), and every schedule
// position records per face either the slot it writes (outflow) or the slot it reads
// (non-lagged inflow) plus whether the two cells list the face's vertices in opposite
// order.  The sweep then reads those upwind traces with one shared-memory load per face;
// lagged upwind cells (their global values are still f^l) and boundary faces read global
// memory as before.  Packed per position: 12 bits per face (kFrontNone: none), then one
// reversal bit per face from bit 48.
constexpr unsigned kFrontNone = 0xFFFu;
constexpr int kFrontMaxSlots = 4000;
constexpr int kFrontSmemMax = 96 * 1024;  // dynamic shared memory of one front-sweep CTA

// genc[j][c] = generation of cell c for ordinate j (one CTA per ordinate)
__global__ void k_front_gen(const uint32_t* __restrict__ glist, const int32_t* __restrict__ lvl,
                            const int32_t* __restrict__ ngen, int ncell, int32_t* __restrict__ genc) {
  const int j = blockIdx.x;
  const uint32_t* gl = glist + (size_t)j * ncell;
  const int32_t* lv = lvl + (size_t)j * (ncell + 1);
  int32_t* gc = genc + (size_t)j * ncell;
  const int G = ngen[j];
  for (int gg = 0; gg < G; ++gg)
    for (int k = lv[gg] + threadIdx.x; k < lv[gg + 1]; k += blockDim.x) gc[gl[k] & kCellMask] = gg;
}

// Greedy slot allocation, one CTA per ordinate, in generation order.  A face that is
// outflow for cell c is inflow for its neighbour, which reads c's trace in this sweep
// exactly when its generation is higher (a lagged edge points the other way).  At the
// start of generation g the slots whose reader ran in generation g-1 go back to the free
// stack (one thread walks that release list); then the generation's cells take slots
// concurrently (free stack first, else a new slot) and each slot joins the release list of
// its reader's generation + 1.  The slot count equals the largest number of traces alive
// at a generation boundary, whatever the order inside a generation.  fslot[j][c][f]
// receives the slot of (c, f) or -1; head holds (ncell + 1) ints per ordinate; *nslots the
// largest slot count, *overflow set when an ordinate needs more than kFrontMaxSlots.
template <int NF>
__global__ void __launch_bounds__(256) k_front_alloc(const uint32_t* __restrict__ glist, const int32_t* __restrict__ lvl,
                                                     const int32_t* __restrict__ ngen, const int32_t* __restrict__ nbr,
                                                     int ncell, const int32_t* __restrict__ genc,
                                                     int16_t* __restrict__ fslot, int32_t* __restrict__ head,
                                                     int* nslots, int* overflow) {
  __shared__ int16_t stk[kFrontMaxSlots], nxt[kFrontMaxSlots];
  __shared__ int nfree, top, over;
  const int j = blockIdx.x;
  const uint32_t* gl = glist + (size_t)j * ncell;
  const int32_t* lv = lvl + (size_t)j * (ncell + 1);
  const int32_t* gc = genc + (size_t)j * ncell;
  int16_t* fs = fslot + (size_t)j * ncell * 4;
  int32_t* hd = head + (size_t)j * (ncell + 1);  // hd[g]: slots released at the start of generation g
  const int G = ngen[j];
  for (int gg = threadIdx.x; gg <= G; gg += blockDim.x) hd[gg] = -1;
  if (threadIdx.x == 0) {
    nfree = 0;
    top = 0;
    over = 0;
  }
  __syncthreads();
  for (int gg = 0; gg < G; ++gg) {
    if (threadIdx.x == 0) {
      int nf = max(nfree, 0);
      for (int sl = hd[gg]; sl >= 0; sl = nxt[sl]) stk[nf++] = (int16_t)sl;
      nfree = nf;
    }
    __syncthreads();
    for (int k = lv[gg] + threadIdx.x; k < lv[gg + 1]; k += blockDim.x) {
      const uint32_t e = gl[k];
      const int c = (int)(e & kCellMask);
      const uint32_t code = e >> kCellBits;
      for (int i = 0; i < 4; ++i) {
        int sl = -1;
        if (i < NF && ((code >> (2 * i)) & 3u) == 1u) {
          const int nb = nbr[(size_t)c * 4 + i];
          const int gr = nb >= 0 ? gc[nb] : -1;
          if (gr > gg) {
            const int p = atomicSub(&nfree, 1) - 1;
            if (p >= 0) {
              sl = stk[p];
            } else {
              const int t = atomicAdd(&top, 1);
              if (t < kFrontMaxSlots)
                sl = t;
              else
                over = 1;
            }
            if (sl >= 0) nxt[sl] = (int16_t)atomicExch(&hd[gr + 1], sl);
          }
        }
        fs[(size_t)c * 4 + i] = (int16_t)sl;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicMax(nslots, min(top, kFrontMaxSlots));
    if (over) atomicOr(overflow, 1);
  }
}

// Packed front slots of every schedule position (see above).
template <class E>
__global__ void k_front_pack(const uint32_t* __restrict__ glist, const int32_t* __restrict__ nbr,
                             const int32_t* __restrict__ nbr_face, const uint64_t* __restrict__ perm, int ncell,
                             const int32_t* __restrict__ genc, const int16_t* __restrict__ fslot,
                             uint64_t* __restrict__ fslots) {
  constexpr int NF = E::NF;
  const int j = blockIdx.x;
  const uint32_t* gl = glist + (size_t)j * ncell;
  const int32_t* gc = genc + (size_t)j * ncell;
  const int16_t* fs = fslot + (size_t)j * ncell * 4;
  for (int k = threadIdx.x; k < ncell; k += blockDim.x) {
    const uint32_t e = gl[k];
    const int c = (int)(e & kCellMask);
    const uint32_t code = e >> kCellBits;
    uint64_t w = 0;
#pragma unroll
    for (int i = 0; i < NF; ++i) {
      uint64_t sl = kFrontNone, rev = 0;
      const uint32_t fl = (code >> (2 * i)) & 3u;
      if (fl == 1u) {
        const int s0 = fs[(size_t)c * 4 + i];
        if (s0 >= 0) sl = (uint64_t)s0;
      } else if (fl == 2u) {
        const int nb = nbr[(size_t)c * 4 + i];
        if (nb >= 0 && gc[nb] < gc[c]) {
          const int f2 = nbr_face[(size_t)c * 4 + i];
          const int s0 = fs[(size_t)nb * 4 + f2];
          if (s0 >= 0) {
            sl = (uint64_t)s0;
            // the neighbour wrote its face-node values in its own face order
            const int p0 = (int)((perm[c] >> (16 * i)) & 15u);
            rev = p0 == E::fn(f2, 0) ? 0u : 1u;
          }
        }
      }
      w |= sl << (12 * i);
      w |= rev << (48 + i);
    }
    fslots[(size_t)j * ncell + k] = w;
  }
}

// Store the N values of T at p with the widest vector stores the alignment allows.
template <typename T, int N, int ALIGN>
__device__ __forceinline__ void store_vec(T* __restrict__ p, const T (&v)[N]) {
  constexpr int BYTES = N * (int)sizeof(T);
  if constexpr (sizeof(T) == 4 && ALIGN % 16 == 0 && BYTES % 16 == 0) {
#pragma unroll
    for (int q = 0; q < N / 4; ++q)
      reinterpret_cast<float4*>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else if constexpr (sizeof(T) == 4 && ALIGN % 8 == 0 && BYTES % 8 == 0) {
#pragma unroll
    for (int q = 0; q < N / 2; ++q) reinterpret_cast<float2*>(p)[q] = make_float2(v[2 * q], v[2 * q + 1]);
  } else {
#pragma unroll
    for (int q = 0; q < N; ++q) p[q] = v[q];
  }
}

// One cell's N floats of an FP32 node row at p (N = 3: 4-byte aligned; N = 6: 8-byte
// aligned; otherwise 16-byte aligned) in at most two vector stores: the split between a
// 16-byte and an 8-byte part (N = 6) or an 8-byte and a 4-byte part (N = 3) follows the
// address.  A warp's scattered stores cost one L1 wavefront per distinct line and
// instruction.  (The same split for the loads measured slower: its selects cost more than
// the wavefronts they save.)
template <int N>
__device__ __forceinline__ void store_cell_f32(float* __restrict__ p, const float (&v)[N]) {
  if constexpr (N == 6) {
    const bool odd = (reinterpret_cast<uintptr_t>(p) & 15u) != 0;
    *reinterpret_cast<float4*>(p + (odd ? 2 : 0)) =
        odd ? make_float4(v[2], v[3], v[4], v[5]) : make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float2*>(p + (odd ? 0 : 4)) = odd ? make_float2(v[0], v[1]) : make_float2(v[4], v[5]);
  } else if constexpr (N == 3) {
    const bool odd = (reinterpret_cast<uintptr_t>(p) & 7u) != 0;
    *reinterpret_cast<float2*>(p + (odd ? 1 : 0)) = odd ? make_float2(v[1], v[2]) : make_float2(v[0], v[1]);
    p[odd ? 0 : 2] = odd ? v[0] : v[2];
  } else {
    static_assert((N * 4) % 16 == 0, "16-byte cells");
    store_vec<float, N, 16>(p, v);
  }
}

// FP32 generation sweep with the shared-memory front (one CTA per ordinate, the same
// operations per cell as sweep_ordinate with the fused source): Sec. 4, Eq. bgk-ss-picard,
//   (nu_s Mh + sum_i r_i (Dd_i + [s_i>0] Eh_i)) f_K = Mh src_K + sum_{s_i<0} (-r_i) Eh_i y_i,
// src = prod_a cf[a][j_a] + qscale q (FUSED; otherwise src is read as given: the
// corrections of the Picard refinement).  The generation offsets sit in shared memory; each
// thread takes positions lv[g] + tid + m nt of generation g and carries the next item's
// neighbours, permutation, geometry, q (src), factors and front slots in registers (loaded
// while the current item is solved; the schedule entry one item earlier still).
// Dynamic shared memory: the front (S float4), then the generation offsets (lvcap ints,
// G + 1 of the largest G rounded up to 4).  2D elements (P1/P2 triangles, Q1).
template <class E, bool FUSED = true>
__global__ void __launch_bounds__(128, 4) k_sweep_front(SweepArgs sa, VGrid g, float nus, SrcArgs<float> sr,
                                                       const float* __restrict__ fbc, float* f, const DevState* ds,
                                                       int jofs, const uint64_t* __restrict__ fslots, int S,
                                                       int lvcap) {
  using T = float;
  constexpr int ND = E::NDOF, NF = E::NF, FD = E::FD;
  static_assert(E::D == 2 && FD <= 4, "2D elements");
  extern __shared__ __align__(16) float fsm[];
  if (ds && (ds->status != BGK_OK || ds->done)) return;
  const int j = jofs + (int)blockIdx.x, tid = (int)threadIdx.x, nt = (int)blockDim.x;
  const int G = sa.ngen[j];
  float4* front = reinterpret_cast<float4*>(fsm);
  int* lv = reinterpret_cast<int*>(fsm + 4 * S);
  {
    const int32_t* lvg = sa.lvl + (size_t)j * (sa.ncell + 1);
    for (int i = tid; i <= G; i += nt) lv[i] = lvg[i];
  }
  double vd[3];
  ordinate(g, j, vd);
  const T v0 = (T)vd[0], v1 = (T)vd[1];
  const uint32_t* gl = sa.glist + (size_t)j * sa.ncell;
  const uint64_t* slj = fslots + (size_t)j * sa.ncell;
  T* fj = f + (size_t)j * sa.nnode;
  const SrcRows<T> rw = src_rows<T, FUSED>(sr, g, j, sa.nnode);
  const T* bj = fbc + (size_t)j * sa.nbface * FD;
  __syncthreads();
  auto seek = [&](int g2, int& kq, int& gq) {
    for (; g2 < G; ++g2) {
      const int k2 = lv[g2] + tid;
      if (k2 < lv[g2 + 1]) {
        kq = k2;
        gq = g2;
        return;
      }
    }
    kq = -1;
    gq = G;
  };
  auto advance = [&](int kq, int gq, int& kr, int& gr) {
    if (kq < 0) {
      kr = -1;
      gr = G;
    } else if (kq + nt < lv[gq + 1]) {
      kr = kq + nt;
      gr = gq;
    } else {
      seek(gq + 1, kr, gr);
    }
  };
  SweepItem<E, T, true, FUSED> cur, nxt;
  uint64_t scur = 0, snxt = 0;
  // current item k, next kn (its data is loaded while k is solved) and the one after,
  // kn2 (its schedule entry is loaded while k is solved)
  int k, gk, kn, gn, kn2, gn2;
  seek(0, k, gk);
  advance(k, gk, kn, gn);
  advance(kn, gn, kn2, gn2);
  if (k >= 0) {
    fetch_item<E, T, true, FUSED>(sa, gl, rw, k, cur);
    scur = slj[k];
    resolve_src(cur, sr.qscale);
  }
  uint32_t en = kn >= 0 ? gl[kn] : 0u;
  for (int gg = 0; gg < G; ++gg) {
    while (k >= 0 && gk == gg) {
      if (kn >= 0) {
        fetch_item_e<E, T, true, FUSED>(sa, en, rw, nxt);
        snxt = slj[kn];
      }
      const uint32_t en2 = kn2 >= 0 ? gl[kn2] : 0u;
      const int c = (int)(cur.e & kCellMask);
      const uint32_t code = cur.e >> kCellBits;
      T r[NF];
      unsigned outm = 0;
      face_rates_t<E, T>(cur.geo, code, v0, v1, T(0), r, outm);
      T b[ND];
      E::mass(cur.src, b);
      const int nbs[4] = {cur.nb.x, cur.nb.y, cur.nb.z, cur.nb.w};
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        if (((code >> (2 * i)) & 3u) != 2u) continue;
        const unsigned su = (unsigned)(scur >> (12 * i)) & kFrontNone;
        T y[FD];
        if (su != kFrontNone) {
          // non-lagged interior inflow: the upwind cell's face trace from the front
          const float4 t = front[su];
          const bool rv = (scur >> (48 + i)) & 1u;
          y[0] = rv ? t.y : t.x;
          y[1] = rv ? t.x : t.y;
          if constexpr (FD > 2) y[2] = t.z;
        } else if (nbs[i] < 0) {
#pragma unroll
          for (int kk = 0; kk < FD; ++kk) y[kk] = bj[(-nbs[i] - 1) * FD + kk];
        } else {
          // lagged upwind cell: its global values are still f^l
#pragma unroll
          for (int kk = 0; kk < FD; ++kk) y[kk] = fj[nbs[i] * ND + (int)((cur.pm >> (16 * i + 4 * kk)) & 15u)];
        }
        E::inflow(i, -r[i], y, b);
      }
      T A[ND][ND];
      E::assemble(nus, r, outm, A);
      lu_solve<ND, T>(A, b);
      store_cell_f32<ND>(fj + c * ND, b);
      // this cell's traces on its outflow faces, in its own face order, for the readers
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        const unsigned so = (unsigned)(scur >> (12 * i)) & kFrontNone;
        if (((code >> (2 * i)) & 3u) == 1u && so != kFrontNone)
          front[so] = make_float4(b[E::fn(i, 0)], b[E::fn(i, 1)], FD > 2 ? b[E::fn(i, 2 % FD)] : T(0), T(0));
      }
      if (kn >= 0) {
        cur = nxt;
        scur = snxt;
        resolve_src(cur, sr.qscale);
      }
      k = kn;
      gk = gn;
      kn = kn2;
      gn = gn2;
      en = en2;
      advance(kn, gn, kn2, gn2);
    }
    __syncthreads();
  }
}

// The float-pair FP64-data sweep (PAIR, see sweep_ordinate) with the shared-memory front
// of k_sweep_front: one CTA per ordinate, the generation offsets in shared memory, the
// next item's schedule entry, neighbours, permutation and mass-weighted source (pairs in
// FP64 words, k_source_pair) in registers, the next cached inverse prefetched into L2.
// A non-lagged interior upwind trace comes from the front as the float pairs of the
// upwind cell's FP64 values (split once by the writer, the same pairs the reader would
// split from global memory, so the results equal k_sweep_pair's bit for bit).  Front slot
// s holds FD pairs in FW float4: (h0 l0 h1 l1)(h2 l2 - -).  Dynamic shared memory: the
// front (S * FW float4), then the generation offsets (lvcap ints).  2D elements.
// (launched only with at most 64 threads per CTA; bounds for seven such CTAs per SM, which
// keep all 1,024 ordinates of the benchmark resident: measured 6.21 -> 6.09 ms against the
// bounds of four 128-thread CTAs, at the same 128 registers)
template <class E>
__global__ void __launch_bounds__(64, 7) k_sweep_front_pair(SweepArgs sa, VGrid g, SrcArgs<double> sr,
                                                            const double* __restrict__ fbc,
                                                            const double* __restrict__ Ainv, double* f,
                                                            const DevState* ds, int jofs,
                                                            const uint64_t* __restrict__ fslots, int S, int lvcap) {
  using T = double;
  constexpr int ND = E::NDOF, NF = E::NF, FD = E::FD, FW = FD > 2 ? 2 : 1, AS = ainv_stride<E, T>();
  static_assert(E::D == 2 && FD <= 4, "2D elements");
  extern __shared__ __align__(16) float fsm[];
  if (ds && (ds->status != BGK_OK || ds->done)) return;
  const int j = jofs + (int)blockIdx.x, tid = (int)threadIdx.x, nt = (int)blockDim.x;
  const int G = sa.ngen[j];
  float4* front = reinterpret_cast<float4*>(fsm);
  int* lv = reinterpret_cast<int*>(fsm + 4 * FW * S);
  {
    const int32_t* lvg = sa.lvl + (size_t)j * (sa.ncell + 1);
    for (int i = tid; i <= G; i += nt) lv[i] = lvg[i];
  }
  double vd[3];
  ordinate(g, j, vd);
  const T v0 = vd[0], v1 = vd[1];
  const uint32_t* gl = sa.glist + (size_t)j * sa.ncell;
  const uint64_t* slj = fslots + (size_t)j * sa.ncell;
  const T* Aj = Ainv + (size_t)j * sa.ncell * AS;
  T* fj = f + (size_t)j * sa.nnode;
  const SrcRows<T> rw = src_rows<T, false>(sr, g, j, sa.nnode);
  const T* bj = fbc + (size_t)j * sa.nbface * FD;
  __syncthreads();
  auto seek = [&](int g2, int& kq, int& gq) {
    for (; g2 < G; ++g2) {
      const int k2 = lv[g2] + tid;
      if (k2 < lv[g2 + 1]) {
        kq = k2;
        gq = g2;
        return;
      }
    }
    kq = -1;
    gq = G;
  };
  auto advance = [&](int kq, int gq, int& kr, int& gr) {
    if (kq < 0) {
      kr = -1;
      gr = G;
    } else if (kq + nt < lv[gq + 1]) {
      kr = kq + nt;
      gr = gq;
    } else {
      seek(gq + 1, kr, gr);
    }
  };
  SweepItem<E, T, false, false> cur, nxt;
  uint64_t scur = 0, snxt = 0;
  int k, gk, kn, gn, kn2, gn2;
  seek(0, k, gk);
  advance(k, gk, kn, gn);
  advance(kn, gn, kn2, gn2);
  if (k >= 0) {
    fetch_item<E, T, false, false>(sa, gl, rw, k, cur);
    scur = slj[k];
  }
  uint32_t en = kn >= 0 ? gl[kn] : 0u;
  for (int gg = 0; gg < G; ++gg) {
    while (k >= 0 && gk == gg) {
      if (kn >= 0) {
        prefetch_l2_bulk(Aj + (size_t)kn * AS, AS * (uint32_t)sizeof(T));
        fetch_item_e<E, T, false, false>(sa, en, rw, nxt);
        snxt = slj[kn];
      }
      const uint32_t en2 = kn2 >= 0 ? gl[kn2] : 0u;
      const int c = (int)(cur.e & kCellMask);
      const uint32_t code = cur.e >> kCellBits;
      fpair bp[ND];
#pragma unroll
      for (int a = 0; a < ND; ++a) bp[a] = fp_from_bits(cur.src[a]);
      const int nbs[4] = {cur.nb.x, cur.nb.y, cur.nb.z, cur.nb.w};
      const double* Gc = sa.geo + (size_t)c * sa.gs;
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        if (((code >> (2 * i)) & 3u) != 2u) continue;
        const T ci = inflow_rate64<E>(Gc, i, v0, v1, 0.0);
        const unsigned su = (unsigned)(scur >> (12 * i)) & kFrontNone;
        fpair yp[FD];
        if (su != kFrontNone) {
          // non-lagged interior inflow: the upwind cell's face trace from the front
          const float4 t0 = front[(size_t)FW * su];
          const bool rv = (scur >> (48 + i)) & 1u;
          yp[0] = rv ? fpair(t0.z, t0.w) : fpair(t0.x, t0.y);
          yp[1] = rv ? fpair(t0.x, t0.y) : fpair(t0.z, t0.w);
          if constexpr (FD > 2) {
            const float4 t1 = front[(size_t)FW * su + 1];
            yp[2] = fpair(t1.x, t1.y);
          }
        } else if (nbs[i] < 0) {
#pragma unroll
          for (int kk = 0; kk < FD; ++kk) yp[kk] = fp_split(bj[(-nbs[i] - 1) * FD + kk]);
        } else {
          // lagged upwind cell: its global values are still f^l
#pragma unroll
          for (int kk = 0; kk < FD; ++kk)
            yp[kk] = fp_split(fj[nbs[i] * ND + (int)((cur.pm >> (16 * i + 4 * kk)) & 15u)]);
        }
        E::inflow_int(i, fp_split(ci) * fpair(1.0 / E::inflow_den), yp, bp);
      }
      T x[ND];
      inverse_product_pair<ND, AS>(reinterpret_cast<const float*>(Aj + (size_t)k * AS), bp, x);
      store_vec<T, ND, cell_align<E, T>()>(fj + c * ND, x);
      // this cell's traces on its outflow faces, in its own face order, for the readers
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        const unsigned so = (unsigned)(scur >> (12 * i)) & kFrontNone;
        if (((code >> (2 * i)) & 3u) == 1u && so != kFrontNone) {
          const fpair p0 = fp_split(x[E::fn(i, 0)]), p1 = fp_split(x[E::fn(i, 1)]);
          front[(size_t)FW * so] = make_float4(p0.h, p0.l, p1.h, p1.l);
          if constexpr (FD > 2) {
            const fpair p2 = fp_split(x[E::fn(i, 2 % FD)]);
            front[(size_t)FW * so + 1] = make_float4(p2.h, p2.l, 0.f, 0.f);
          }
        }
      }
      if (kn >= 0) {
        cur = nxt;
        scur = snxt;
      }
      k = kn;
      gk = gn;
      kn = kn2;
      gn = gn2;
      en = en2;
      advance(kn, gn, kn2, gn2);
    }
    __syncthreads();
  }
}

// out = a_k * fk + a_f * f + sum_r cF[r] * F[r]   (stage bookkeeping of Sec. 3.5); out32
// (if given) also receives the float of each value written (the FP32 phase's copy of q)
template <typename T>
__global__ void k_combine(size_t n, T* __restrict__ out, double a_k, const T* __restrict__ fk, double a_f,
                          const T* __restrict__ f, int nF, double c0, const T* __restrict__ F0, double c1,
                          const T* __restrict__ F1, double c2, const T* __restrict__ F2, const DevState* ds,
                          float* __restrict__ out32 = nullptr) {
  if (ds && ds->status != BGK_OK) return;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    if (fk) s += a_k * (double)fk[i];
    if (f) s += a_f * (double)f[i];
    if (nF > 0) s += c0 * (double)F0[i];
    if (nF > 1) s += c1 * (double)F1[i];
    if (nF > 2) s += c2 * (double)F2[i];
    out[i] = (T)s;
    if (out32) out32[i] = (float)(T)s;
  }
}

// out <- in, skipped when gate (if given) reports that its loop failed
template <typename TI, typename TO>
__global__ void k_convert_gated(size_t n, const TI* __restrict__ in, TO* __restrict__ out,
                                const DevState* __restrict__ gate) {
  if (gate && (gate->err || gate->status == BGK_E_NONPHYSICAL)) return;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (TO)in[i];
}

// Copy the current moments of one state to another (parities from each state's counter).
__global__ void k_copy_moments(size_t n, const double* __restrict__ A0, const double* __restrict__ A1,
                               const DevState* __restrict__ da, double* B0, double* B1, DevState* db) {
  const double* A = (da->it & 1) == 0 ? A0 : A1;
  double* B = (db->it & 1) == 0 ? B0 : B1;
  if (blockIdx.x == 0 && threadIdx.x == 0) db->cf_fresh = 0;  // B's factors are not built yet
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    B[i] = A[i];
}

// Stage predictor (bgk_config.stage_predictor).  dst <- the current moments U[it & 1].
__global__ void k_save_moments(size_t n, const DevState* __restrict__ ds, const double* __restrict__ U0,
                               const double* __restrict__ U1, double* __restrict__ dst) {
  if (ds->status != BGK_OK) return;
  const double* U = (ds->it & 1) == 0 ? U0 : U1;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = U[i];
}
// The moments a stage starts from: U[it & 1] <- wk Uk + w0 S0 + w1 S1 per node (Uk the
// moments of f^k, S0 and S1 those the first two stages ended with; S1 unused when w1 = 0),
// where the result is physical (n > 0, theta > 0, finite); elsewhere the current moments
// (the previous stage's) stay.  The factors built from the old moments go stale.
__global__ void k_predict_moments(int nnode, int dim, DevState* ds, double* U0, double* U1,
                                  const double* __restrict__ Uk, const double* __restrict__ S0,
                                  const double* __restrict__ S1, double wk, double w0, double w1) {
  if (ds->status != BGK_OK) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) ds->cf_fresh = 0;
  double* U = (ds->it & 1) == 0 ? U0 : U1;
  const int nm = dim + 2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nnode; i += gridDim.x * blockDim.x) {
    double v[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      if (m >= nm) break;
      const size_t o = (size_t)i * nm + m;
      double x = wk * Uk[o] + w0 * S0[o];
      if (w1 != 0.0) x += w1 * S1[o];
      v[m] = x;
    }
    const double n = v[0];
    double u2 = 0.0;
    for (int a = 0; a < dim; ++a) u2 += (v[1 + a] / n) * (v[1 + a] / n);
    const double th = (2.0 * v[nm - 1] / n - u2) / dim;
    if (!(n > 0.0) || !(th > 0.0) || !isfinite(n) || !isfinite(th)) continue;
    for (int m = 0; m < nm; ++m) U[(size_t)i * nm + m] = v[m];
  }
}

// Record the FP32 phase's iteration count of stage st in the main state.
__global__ void k_record_fp32(const DevState* __restrict__ sh, DevState* main, int st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    main->iters32[st] = sh->stage_it;
    main->total_sweeps += sh->stage_it;
  }
}

// Wall boundary data of Sec. 4.2, refreshed before every sweep from the current iterate
// f^l: at boundary-face position p of a wall face, fbc[j][p] = f[j'][bnode[p]] with j' the
// mirror ordinate (wall code 1: -v_j, every velocity index i -> N-1-i; code 2+a: R_n v_j
// for the normal +/-e_a, index a mirrored).  Positions of inflow faces (code 0) keep
// their given data.  The 1D grid is symmetric about 0, so the mirrored index holds the
// mirrored velocity.
template <typename T>
__global__ void k_wall_bc(VGrid g, int npos, int fd, int nnode, const T* __restrict__ f,
                          const int32_t* __restrict__ bnode, const int8_t* __restrict__ wall,
                          T* __restrict__ fbc) {
  const size_t n = (size_t)g.nv * npos;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(i / npos), p = (int)(i - (size_t)j * npos);
    const int w = wall[p / fd];
    if (w == 0) continue;
    int jm = 0, stride = 1, jj = j;  // velocity component d-1 varies fastest in j
    for (int a = g.dim - 1; a >= 0; --a) {
      const int ia = jj % g.N;
      jj /= g.N;
      jm += ((w == 1 || w == 2 + a) ? g.N - 1 - ia : ia) * stride;
      stride *= g.N;
    }
    fbc[i] = f[(size_t)jm * nnode + bnode[p]];
  }
}

// Inflow data from nodal values: fbc[j][p] = fn[j][bnode[p]] (boundary-face positions p).
template <typename T>
__global__ void k_gather_inflow(int nv, int npos, int nnode, const double* __restrict__ fn,
                                const int32_t* __restrict__ bnode, T* __restrict__ fbc) {
  const size_t n = (size_t)nv * npos;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t j = i / npos, p = i - j * npos;
    fbc[i] = (T)fn[j * nnode + bnode[p]];
  }
}

template <typename TI, typename TO>
__global__ void k_convert(size_t n, const TI* __restrict__ in, TO* __restrict__ out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (TO)in[i];
}

}  // namespace bgk
