// Learned initial guess of the Picard iteration: a small MLP, trained on moment
// trajectories the solver generates, predicts each node's stage moments from the
// stage-start state; its prediction replaces the moments of iterate l = 0 (the Maxwellian
// parameters of the first sweep).  The plain iteration then runs to the same criterion,
// so the converged result is the solver's own; a non-physical prediction at a node falls
// back to that node's plain moments.  Included at the end of bgk_lib.cu.
//
// Network: F inputs -> H -> H -> H -> O (tanh on hidden layers), inputs and outputs
// normalised by per-column mean and standard deviation.  Training in FP32 (own forward,
// backward and Adam kernels); inference with BF16-stored weights and FP32 accumulation.
#include <cuda_bf16.h>

namespace bgk {

// ---------------------------------------------------------------------------------
// Features of node i (d = dimension, s = sqrt(theta), q = (log n, u, log theta)):
//   q (d+2) | s dt grad log n (d) | dt grad u (d x d) | s dt grad log theta (d) |
//   log10(nu dt) | change of q over the previous stage (d+2, zero without history)
// Gradients are those of the P1 interpolant of the cell's vertex values,
// grad l_a = -N_a / (d |K|).  Outputs: the stage's change of q at the node.
__host__ __device__ constexpr int guess_features(int d) { return (d + 2) + d + d * d + d + 1 + (d + 2); }

__device__ __forceinline__ void prim_log(const double* U, int d, double* q) {
  const double n = U[0];
  double u2 = 0.0;
  for (int a = 0; a < d; ++a) {
    q[1 + a] = U[1 + a] / n;
    u2 += q[1 + a] * q[1 + a];
  }
  const double th = (2.0 * U[1 + d] / n - u2) / d;
  q[0] = log(fmax(n, 1e-300));
  q[1 + d] = log(fmax(th, 1e-300));
}

__global__ void k_guess_features(int d, int ndof, int quad, int ncell, const double* __restrict__ geo, int gs,
                                 const double* __restrict__ U0, const double* __restrict__ U1,
                                 const DevState* __restrict__ ds, const double* __restrict__ Uhist,
                                 const int* __restrict__ have_hist, double dt, double nu, float* __restrict__ X) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int nm = d + 2, F = guess_features(d);
  const double* U = ((ds->it & 1) == 0) ? U0 : U1;
  const int nvx = quad ? 4 : d + 1;  // vertices (the first nodes of the cell)
  double qv[4][5];  // vertex values of q
  for (int a = 0; a < nvx; ++a) prim_log(U + (size_t)(c * ndof + a) * nm, d, qv[a]);
  const double* G = geo + (size_t)c * gs;
  const double invK = G[nvx * d];
  double grad[5][3] = {{0}};
  if (quad) {
    // mean gradient of the bilinear interpolant: (1/|K|) sum_faces N_f (q_f + q_f+1) / 2
    for (int f = 0; f < 4; ++f)
      for (int al = 0; al < d; ++al) {
        const double gl = 0.5 * G[f * d + al] * invK;
        for (int m = 0; m < nm; ++m) grad[m][al] += (qv[f][m] + qv[(f + 1) % 4][m]) * gl;
      }
  } else {
    for (int a = 0; a <= d; ++a)
      for (int al = 0; al < d; ++al) {
        const double gl = -G[a * d + al] * invK / d;
        for (int m = 0; m < nm; ++m) grad[m][al] += qv[a][m] * gl;
      }
  }
  const double lnd = log10(fmax(nu * dt, 1e-30));
  const bool hist = *have_hist != 0;
  for (int a = 0; a < ndof; ++a) {
    const int i = c * ndof + a;
    double q[5];
    prim_log(U + (size_t)i * nm, d, q);
    const double s = exp(0.5 * q[1 + d]);
    float* x = X + (size_t)i * F;
    int k = 0;
    for (int m = 0; m < nm; ++m) x[k++] = (float)q[m];
    for (int al = 0; al < d; ++al) x[k++] = (float)(s * dt * grad[0][al]);
    for (int b = 0; b < d; ++b)
      for (int al = 0; al < d; ++al) x[k++] = (float)(dt * grad[1 + b][al]);
    for (int al = 0; al < d; ++al) x[k++] = (float)(s * dt * grad[1 + d][al]);
    x[k++] = (float)lnd;
    double qh[5] = {0, 0, 0, 0, 0};
    if (hist) prim_log(Uhist + (size_t)i * nm, d, qh);
    for (int m = 0; m < nm; ++m) x[k++] = hist ? (float)(q[m] - qh[m]) : 0.f;
  }
}

// U_hist <- current moments; the history feature is available from now on.
__global__ void k_guess_history(int nnode, int nm, const double* __restrict__ U0, const double* __restrict__ U1,
                                const DevState* __restrict__ ds, double* __restrict__ Uhist, int* have_hist) {
  const double* U = ((ds->it & 1) == 0) ? U0 : U1;
  const size_t n = (size_t)nnode * nm;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    Uhist[t] = U[t];
  if (blockIdx.x == 0 && threadIdx.x == 0) *have_hist = 1;
}

// Training targets: change of q from the stage-start moments Ustart to the current ones,
// minus the previous stage's change (the last d+2 features X): the network learns the
// correction to extrapolating the previous change.
__global__ void k_guess_targets(int nnode, int d, const double* __restrict__ Ustart, const double* __restrict__ U0,
                                const double* __restrict__ U1, const DevState* __restrict__ ds,
                                const float* __restrict__ X, float* __restrict__ Y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nnode) return;
  const int nm = d + 2, F = guess_features(d);
  const double* U = ((ds->it & 1) == 0) ? U0 : U1;
  double a[5], b[5];
  prim_log(Ustart + (size_t)i * nm, d, a);
  prim_log(U + (size_t)i * nm, d, b);
  for (int m = 0; m < nm; ++m)
    Y[(size_t)i * nm + m] = (float)((b[m] - a[m]) - (double)X[(size_t)i * F + F - nm + m]);
}

// Guess applied to iterate 0: q + (previous change + network correction) -> (n, u,
// theta) -> U; nodes whose prediction is non-physical or non-finite keep their plain
// moments.  X: the stage's features (their last d+2 entries are the previous change).
__global__ void k_guess_apply(int nnode, int d, const float* __restrict__ dq, const float* __restrict__ X, double* U0,
                              double* U1, const DevState* __restrict__ ds) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nnode) return;
  const int nm = d + 2;
  double* U = (((ds->it & 1) == 0) ? U0 : U1) + (size_t)i * nm;
  double q[5];
  prim_log(U, d, q);
  double p[5];
  bool ok = true;
  const int F = guess_features(d);
  for (int m = 0; m < nm; ++m) {
    p[m] = q[m] + (double)dq[(size_t)i * nm + m] + (double)X[(size_t)i * F + F - nm + m];
    ok = ok && isfinite(p[m]);
  }
  if (!ok) return;
  const double n = exp(p[0]), th = exp(p[1 + d]);
  if (!(n > 0.0) || !(th > 0.0) || !isfinite(n) || !isfinite(th)) return;
  double u2 = 0.0;
  U[0] = n;
  for (int a = 0; a < d; ++a) {
    U[1 + a] = n * p[1 + a];
    u2 += p[1 + a] * p[1 + a];
  }
  U[1 + d] = 0.5 * n * u2 + 0.5 * d * n * th;
}

// ---------------------------------------------------------------------------------
// Dense layer Y[r][c] = act(sum_k X[r][k] Wt(k, c) + b[c]) for r < n, c < cols, where
// Wt(k, c) = W[c][k] (forward, W stored [out][in]) or W[k][c] (backward-data).  Inputs
// optionally normalised column-wise (layer 0).  Backward-data multiplies by tanh'
// from the layer's input activations A (1 - A^2).  One CTA: 32 rows x up to 128 cols.
template <typename WT, bool TRANS, int ACT>  // ACT: 0 none, 1 tanh, 2 times (1 - A^2)
__global__ void __launch_bounds__(256) k_dense(const float* __restrict__ X, int n, int kdim, const WT* __restrict__ W,
                                              const WT* __restrict__ b, int cols, float* __restrict__ Y,
                                              const float* __restrict__ mu, const float* __restrict__ sd,
                                              const float* __restrict__ A) {
  extern __shared__ float sm[];
  float* Xs = sm;               // [32][kdim]
  float* Ws = sm + 32 * kdim;   // [kdim][cols]
  const int r0 = blockIdx.x * 32;
  for (int t = threadIdx.x; t < kdim * cols; t += blockDim.x) {
    const int k = t / cols, c = t % cols;
    const WT w = TRANS ? W[(size_t)k * cols + c] : W[(size_t)c * kdim + k];
    Ws[t] = (float)w;
  }
  for (int t = threadIdx.x; t < 32 * kdim; t += blockDim.x) {
    const int r = t / kdim, k = t % kdim;
    float x = (r0 + r < n) ? X[(size_t)(r0 + r) * kdim + k] : 0.f;
    if (mu) x = (x - mu[k]) / sd[k];
    Xs[t] = x;
  }
  __syncthreads();
  const int r = threadIdx.x >> 3, c0 = threadIdx.x & 7;
  float acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.f;
  for (int k = 0; k < kdim; ++k) {
    const float x = Xs[r * kdim + k];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int c = c0 + 8 * q;
      if (c < cols) acc[q] = fmaf(x, Ws[k * cols + c], acc[q]);
    }
  }
  if (r0 + r >= n) return;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int c = c0 + 8 * q;
    if (c >= cols) continue;
    float y = acc[q] + (b ? (float)b[c] : 0.f);
    if (ACT == 1) y = tanhf(y);
    if (ACT == 2) {
      const float a = A[(size_t)(r0 + r) * cols + c];
      y *= 1.f - a * a;
    }
    Y[(size_t)(r0 + r) * cols + c] = y;
  }
}

// Weight gradients: partial[chunk][o][k] = sum over the chunk's 64 rows of dY[r][o] X[r][k]
// (k = kdim is the bias column, X = 1); inputs normalised if mu is given.
__global__ void __launch_bounds__(256) k_dense_wgrad(const float* __restrict__ X, const float* __restrict__ dY, int n,
                                                    int kdim, int odim, const float* __restrict__ mu,
                                                    const float* __restrict__ sd, float* __restrict__ partial) {
  extern __shared__ float sm[];
  const int kk = kdim + 1;
  float* Xs = sm;             // [64][kdim+1]
  float* Ds = sm + 64 * kk;   // [64][odim]
  const int r0 = blockIdx.x * 64;
  for (int t = threadIdx.x; t < 64 * kk; t += blockDim.x) {
    const int r = t / kk, k = t % kk;
    float x = 0.f;
    if (r0 + r < n) {
      if (k == kdim) {
        x = 1.f;
      } else {
        x = X[(size_t)(r0 + r) * kdim + k];
        if (mu) x = (x - mu[k]) / sd[k];
      }
    }
    Xs[t] = x;
  }
  for (int t = threadIdx.x; t < 64 * odim; t += blockDim.x) {
    const int r = t / odim, o = t % odim;
    Ds[t] = (r0 + r < n) ? dY[(size_t)(r0 + r) * odim + o] : 0.f;
  }
  __syncthreads();
  float* P = partial + (size_t)blockIdx.x * odim * kk;
  for (int t = threadIdx.x; t < odim * kk; t += blockDim.x) {
    const int o = t / kk, k = t % kk;
    float s = 0.f;
    for (int r = 0; r < 64; ++r) s = fmaf(Ds[r * odim + o], Xs[r * kk + k], s);
    P[t] = s;
  }
}

// Sum the chunk partials in chunk order into W-grad [o][kdim] and b-grad [o].
__global__ void k_dense_wreduce(const float* __restrict__ partial, int nchunk, int kdim, int odim,
                                float* __restrict__ gW, float* __restrict__ gb) {
  const int kk = kdim + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= odim * kk) return;
  float s = 0.f;
  for (int ch = 0; ch < nchunk; ++ch) s += partial[(size_t)ch * odim * kk + t];
  const int o = t / kk, k = t % kk;
  if (k == kdim)
    gb[o] = s;
  else
    gW[(size_t)o * kdim + k] = s;
}

// MSE on normalised outputs: d = 2 (yhat - (y - mu)/sd) / (n O); per-block loss sums.
__global__ void k_mse(const float* __restrict__ yhat, const float* __restrict__ y, int n, int O,
                      const float* __restrict__ mu, const float* __restrict__ sd, float* __restrict__ d,
                      double* __restrict__ part) {
  __shared__ double red[256];
  double acc = 0.0;
  const size_t tot = (size_t)n * O;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const int o = (int)(t % O);
    const float e = yhat[t] - (y[t] - mu[o]) / sd[o];
    d[t] = 2.f * e / (float)tot;
    acc += (double)e * e;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_adam(int np, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= np) return;
  const float gt = g[t];
  const float mt = b1 * m[t] + (1.f - b1) * gt;
  const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
  m[t] = mt;
  v[t] = vt;
  p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

// Column mean and standard deviation of A[n][cols] (FP64 sums, fixed order per column).
__global__ void k_colstats(const float* __restrict__ A, int64_t n, int cols, float* __restrict__ mu,
                           float* __restrict__ sd) {
  __shared__ double s1[256], s2[256];
  const int c = blockIdx.x;
  double a = 0.0, b = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    const double x = A[r * cols + c];
    a += x;
    b += x * x;
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s1[threadIdx.x] += s1[threadIdx.x + w];
      s2[threadIdx.x] += s2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double m = s1[0] / n;
    const double var = fmax(s2[0] / n - m * m, 0.0);
    mu[c] = (float)m;
    sd[c] = (float)fmax(sqrt(var), 1e-6);
  }
}

__global__ void k_to_bf16(int np, const float* __restrict__ p, __nv_bfloat16* __restrict__ q) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < np) q[t] = __float2bfloat16(p[t]);
}

// y = yhat * sd + mu (de-normalised network output)
__global__ void k_denorm(const float* __restrict__ yh, int64_t n, int O, const float* __restrict__ mu,
                         const float* __restrict__ sd, float* __restrict__ y) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * O) return;
  const int o = (int)(t % O);
  y[t] = yh[t] * sd[o] + mu[o];
}

}  // namespace bgk

struct bgk_mlp {
  int F = 0, H = 0, O = 0;
  int np = 0;
  int64_t off[8] = {0};  // W0 b0 W1 b1 W2 b2 W3 b3
  float* p = nullptr;    // parameters (FP32)
  float* g = nullptr;    // gradients
  float* m = nullptr;    // Adam moments
  float* v = nullptr;
  __nv_bfloat16* pb = nullptr;  // BF16 copy for inference
  bool pb_valid = false;
  float* norm = nullptr;  // mu_x [F], sd_x [F], mu_y [O], sd_y [O]
  int step = 0;
  // scratch sized for cap rows
  int64_t cap = 0;
  float* act[4] = {nullptr, nullptr, nullptr, nullptr};  // layer outputs [cap][H] x3, [cap][O]
  float* d0 = nullptr;                                   // gradient buffers [cap][H]
  float* d1 = nullptr;
  float* partial = nullptr;
  double* lpart = nullptr;
};

namespace {

void mlp_free(bgk_mlp* m) {
  void* ptrs[] = {m->p, m->g, m->m, m->v, m->pb, m->norm, m->act[0], m->act[1], m->act[2], m->act[3], m->d0, m->d1,
                  m->partial, m->lpart};
  for (void* q : ptrs)
    if (q) cudaFree(q);
}

int mlp_reserve(bgk_mlp* m, int64_t n) {
  if (n <= m->cap) return BGK_OK;
  for (int l = 0; l < 4; ++l)
    if (m->act[l]) cudaFree(m->act[l]);
  if (m->d0) cudaFree(m->d0);
  if (m->d1) cudaFree(m->d1);
  if (m->partial) cudaFree(m->partial);
  if (m->lpart) cudaFree(m->lpart);
  m->cap = n;
  const int64_t chunks = (n + 63) / 64;
  const int64_t wmax = (int64_t)std::max(m->H, m->O) * (std::max(m->F, m->H) + 1);
  int rc = BGK_OK;
  for (int l = 0; l < 3; ++l)
    if (rc == BGK_OK) rc = dalloc(m->act[l], sizeof(float) * n * m->H);
  if (rc == BGK_OK) rc = dalloc(m->act[3], sizeof(float) * n * m->O);
  if (rc == BGK_OK) rc = dalloc(m->d0, sizeof(float) * n * std::max(m->H, m->O));
  if (rc == BGK_OK) rc = dalloc(m->d1, sizeof(float) * n * std::max(m->H, m->O));
  if (rc == BGK_OK) rc = dalloc(m->partial, sizeof(float) * chunks * wmax);
  if (rc == BGK_OK) rc = dalloc(m->lpart, sizeof(double) * 1024);
  return rc;
}

template <typename WT, bool TRANS, int ACT>
void dense_t(cudaStream_t s, const float* X, int64_t n, int kdim, const WT* W, const WT* b, int cols, float* Y,
             const float* mu, const float* sd, const float* A) {
  const int blocks = (int)((n + 31) / 32);
  const size_t smem = sizeof(float) * (32 * kdim + kdim * cols);
  k_dense<WT, TRANS, ACT><<<blocks, 256, smem, s>>>(X, (int)n, kdim, W, b, cols, Y, mu, sd, A);
}

// Forward pass: hidden activations in act[0..2], normalised output in act[3].
template <typename WT>
void mlp_forward(bgk_mlp* m, cudaStream_t s, const float* X, int64_t n, const WT* P) {
  const float* mu = m->norm;
  const float* sd = m->norm + m->F;
  dense_t<WT, false, 1>(s, X, n, m->F, P + m->off[0], P + m->off[1], m->H, m->act[0], mu, sd, nullptr);
  dense_t<WT, false, 1>(s, m->act[0], n, m->H, P + m->off[2], P + m->off[3], m->H, m->act[1], nullptr, nullptr,
                        nullptr);
  dense_t<WT, false, 1>(s, m->act[1], n, m->H, P + m->off[4], P + m->off[5], m->H, m->act[2], nullptr, nullptr,
                        nullptr);
  dense_t<WT, false, 0>(s, m->act[2], n, m->H, P + m->off[6], P + m->off[7], m->O, m->act[3], nullptr, nullptr,
                        nullptr);
}

void wgrad(bgk_mlp* m, cudaStream_t s, const float* X, const float* dY, int64_t n, int kdim, int odim,
           const float* mu, const float* sd, float* gW, float* gb) {
  const int chunks = (int)((n + 63) / 64);
  const size_t smem = sizeof(float) * (64 * (kdim + 1) + 64 * odim);
  k_dense_wgrad<<<chunks, 256, smem, s>>>(X, dY, (int)n, kdim, odim, mu, sd, m->partial);
  const int t = odim * (kdim + 1);
  k_dense_wreduce<<<(t + 255) / 256, 256, 0, s>>>(m->partial, chunks, kdim, odim, gW, gb);
}

// Loss and gradients of all parameters for the batch (X, Y) (FP32).
int mlp_loss_grad(bgk_mlp* m, cudaStream_t s, const float* X, const float* Y, int64_t n, double* loss) {
  int rc = mlp_reserve(m, n);
  if (rc != BGK_OK) return rc;
  const float* mux = m->norm;
  const float* sdx = m->norm + m->F;
  const float* muy = m->norm + 2 * m->F;
  const float* sdy = m->norm + 2 * m->F + m->O;
  mlp_forward<float>(m, s, X, n, m->p);
  const int lb = 512;
  k_mse<<<lb, 256, 0, s>>>(m->act[3], Y, (int)n, m->O, muy, sdy, m->d0, m->lpart);
  float* g = m->g;
  // layer 3 (linear): dY = d0
  wgrad(m, s, m->act[2], m->d0, n, m->H, m->O, nullptr, nullptr, g + m->off[6], g + m->off[7]);
  dense_t<float, true, 2>(s, m->d0, n, m->O, m->p + m->off[6], (const float*)nullptr, m->H, m->d1, nullptr, nullptr,
                          m->act[2]);
  // layer 2
  wgrad(m, s, m->act[1], m->d1, n, m->H, m->H, nullptr, nullptr, g + m->off[4], g + m->off[5]);
  dense_t<float, true, 2>(s, m->d1, n, m->H, m->p + m->off[4], (const float*)nullptr, m->H, m->d0, nullptr, nullptr,
                          m->act[1]);
  // layer 1
  wgrad(m, s, m->act[0], m->d0, n, m->H, m->H, nullptr, nullptr, g + m->off[2], g + m->off[3]);
  dense_t<float, true, 2>(s, m->d0, n, m->H, m->p + m->off[2], (const float*)nullptr, m->H, m->d1, nullptr, nullptr,
                          m->act[0]);
  // layer 0 (inputs normalised on the fly)
  wgrad(m, s, X, m->d1, n, m->F, m->H, mux, sdx, g + m->off[0], g + m->off[1]);
  CK(cudaGetLastError());
  if (loss) {
    std::vector<double> part(lb);
    CK(cudaMemcpyAsync(part.data(), m->lpart, sizeof(double) * lb, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double t = 0.0;
    for (double x : part) t += x;
    *loss = t / ((double)n * m->O);
  }
  return BGK_OK;
}

// splitmix64 (Steele, Lea, Flood 2014) for the seeded initialisation
uint64_t smix(uint64_t& st) {
  uint64_t z = (st += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int bgk_mlp_create(int n_in, int n_hidden, int n_out, uint64_t seed, bgk_mlp** out) {
  if (!out || n_in <= 0 || n_in > 128 || n_hidden <= 0 || n_hidden > 128 || n_out <= 0 || n_out > 128)
    return BGK_E_INVALID;
  *out = nullptr;
  bgk_mlp* m = new (std::nothrow) bgk_mlp();
  if (!m) return BGK_E_OOM;
  m->F = n_in;
  m->H = n_hidden;
  m->O = n_out;
  const int dims[5] = {n_in, n_hidden, n_hidden, n_hidden, n_out};
  int64_t o = 0;
  for (int l = 0; l < 4; ++l) {
    m->off[2 * l] = o;
    o += (int64_t)dims[l + 1] * dims[l];
    m->off[2 * l + 1] = o;
    o += dims[l + 1];
  }
  m->np = (int)o;
  int rc = dalloc(m->p, sizeof(float) * o);
  if (rc == BGK_OK) rc = dalloc(m->g, sizeof(float) * o);
  if (rc == BGK_OK) rc = dalloc(m->m, sizeof(float) * o);
  if (rc == BGK_OK) rc = dalloc(m->v, sizeof(float) * o);
  if (rc == BGK_OK) rc = dalloc(m->pb, sizeof(__nv_bfloat16) * o);
  if (rc == BGK_OK) rc = dalloc(m->norm, sizeof(float) * (2 * n_in + 2 * n_out));
  if (rc != BGK_OK) {
    mlp_free(m);
    delete m;
    return rc;
  }
  // Glorot-uniform weights from splitmix64, zero biases, identity normalisation
  std::vector<float> hp(o, 0.f);
  uint64_t st = seed;
  for (int l = 0; l < 4; ++l) {
    const double a = std::sqrt(6.0 / (dims[l] + dims[l + 1]));
    for (int64_t t = m->off[2 * l]; t < m->off[2 * l + 1]; ++t) {
      const double u = (double)(smix(st) >> 11) * (1.0 / 9007199254740992.0);
      hp[t] = (float)((2.0 * u - 1.0) * a);
    }
  }
  const int big = 200 * 1024;
  cudaFuncSetAttribute(k_dense<float, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_dense<float, false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_dense<float, true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_dense<__nv_bfloat16, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_dense<__nv_bfloat16, false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_dense_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  std::vector<float> nrm(2 * n_in + 2 * n_out, 0.f);
  for (int k = 0; k < n_in; ++k) nrm[n_in + k] = 1.f;
  for (int k = 0; k < n_out; ++k) nrm[2 * n_in + n_out + k] = 1.f;
  cudaMemcpy(m->p, hp.data(), sizeof(float) * o, cudaMemcpyHostToDevice);
  cudaMemset(m->m, 0, sizeof(float) * o);
  cudaMemset(m->v, 0, sizeof(float) * o);
  cudaMemcpy(m->norm, nrm.data(), sizeof(float) * nrm.size(), cudaMemcpyHostToDevice);
  *out = m;
  return BGK_OK;
}

int bgk_mlp_destroy(bgk_mlp* m) {
  if (!m) return BGK_OK;
  cudaDeviceSynchronize();
  mlp_free(m);
  delete m;
  return BGK_OK;
}

int bgk_mlp_num_params(const bgk_mlp* m, int64_t* n) {
  if (!m || !n) return BGK_E_INVALID;
  *n = m->np;
  return BGK_OK;
}

int bgk_mlp_get_params(const bgk_mlp* m, float* h_params, float* h_norm) {
  if (!m) return BGK_E_INVALID;
  if (h_params) CK(cudaMemcpy(h_params, m->p, sizeof(float) * m->np, cudaMemcpyDeviceToHost));
  if (h_norm) CK(cudaMemcpy(h_norm, m->norm, sizeof(float) * (2 * m->F + 2 * m->O), cudaMemcpyDeviceToHost));
  return BGK_OK;
}

int bgk_mlp_set_params(bgk_mlp* m, const float* h_params, const float* h_norm) {
  if (!m) return BGK_E_INVALID;
  if (h_params) CK(cudaMemcpy(m->p, h_params, sizeof(float) * m->np, cudaMemcpyHostToDevice));
  if (h_norm) CK(cudaMemcpy(m->norm, h_norm, sizeof(float) * (2 * m->F + 2 * m->O), cudaMemcpyHostToDevice));
  m->pb_valid = false;
  return BGK_OK;
}

int bgk_mlp_fit_norm(bgk_mlp* m, const float* d_X, const float* d_Y, int64_t n) {
  if (!m || !d_X || !d_Y || n <= 0) return BGK_E_INVALID;
  k_colstats<<<m->F, 256>>>(d_X, n, m->F, m->norm, m->norm + m->F);
  k_colstats<<<m->O, 256>>>(d_Y, n, m->O, m->norm + 2 * m->F, m->norm + 2 * m->F + m->O);
  CK(cudaDeviceSynchronize());
  m->pb_valid = false;
  return BGK_OK;
}

int bgk_mlp_loss_grad(bgk_mlp* m, const float* d_X, const float* d_Y, int64_t n, double* loss, float* h_grad) {
  if (!m || !d_X || !d_Y || n <= 0) return BGK_E_INVALID;
  int rc = mlp_loss_grad(m, 0, d_X, d_Y, n, loss);
  if (rc != BGK_OK) return rc;
  if (h_grad) CK(cudaMemcpy(h_grad, m->g, sizeof(float) * m->np, cudaMemcpyDeviceToHost));
  CK(cudaDeviceSynchronize());
  return BGK_OK;
}

int bgk_mlp_train_step(bgk_mlp* m, const float* d_X, const float* d_Y, int64_t n, float lr, double* loss) {
  if (!m || !d_X || !d_Y || n <= 0) return BGK_E_INVALID;
  int rc = mlp_loss_grad(m, 0, d_X, d_Y, n, loss);
  if (rc != BGK_OK) return rc;
  m->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
  k_adam<<<(m->np + 255) / 256, 256>>>(m->np, m->p, m->g, m->m, m->v, lr, b1, b2, 1e-8f, c1, c2);
  m->pb_valid = false;
  CK(cudaGetLastError());
  return BGK_OK;
}

// Network output (de-normalised) for n rows; bf16 != 0 uses BF16-stored weights.
int bgk_mlp_predict(bgk_mlp* m, const float* d_X, int64_t n, float* d_Y, int bf16) {
  if (!m || !d_X || !d_Y || n <= 0) return BGK_E_INVALID;
  int rc = mlp_reserve(m, n);
  if (rc != BGK_OK) return rc;
  if (bf16) {
    if (!m->pb_valid) {
      k_to_bf16<<<(m->np + 255) / 256, 256>>>(m->np, m->p, m->pb);
      m->pb_valid = true;
    }
    mlp_forward<__nv_bfloat16>(m, 0, d_X, n, m->pb);
  } else {
    mlp_forward<float>(m, 0, d_X, n, m->p);
  }
  k_denorm<<<(int)((n * m->O + 255) / 256), 256>>>(m->act[3], n, m->O, m->norm + 2 * m->F, m->norm + 2 * m->F + m->O,
                                                   d_Y);
  CK(cudaDeviceSynchronize());
  return BGK_OK;
}

}  // extern "C"
