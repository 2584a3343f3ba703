// Moments and convergence measure without device allocation.
//
// Some callers cannot call cudaMalloc: programs that have handed all device memory to
// their own pool allocator up front (a further cudaMalloc would fail, or fragment the
// pool they manage), and programs that must never synchronize the device, which
// cudaMalloc and cudaFree may do.  This file gives them bgk_moments_measure_noalloc:
// the same computation as the handle's moment reduction plus the convergence measure,
// with its scratch (one row of partial sums per thread block) in a file-scope device
// array of fixed size.  The caller passes inputs and outputs; nothing is allocated.
#include <cuda_runtime.h>

#include <mutex>

#include "bgk_internal.h"

namespace {

// One block reduces 128 spatial nodes; each block leaves 6 partial sums.
constexpr int kThreads = 128;
constexpr int kMaxBlocks = 16384;                        // up to 2,097,152 nodes
constexpr int64_t kMaxNodes = (int64_t)kMaxBlocks * kThreads;

// Scratch shared by every call in the process: 16384 x 6 doubles = 768 KiB, held by
// every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_partial_scratch[kMaxBlocks * 6];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once per device.
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BGK_E_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_partial_scratch) != cudaSuccess) {
      cudaGetLastError();
      return BGK_E_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return BGK_OK;
}

// U_i = sum_j w_j (1, v_j, |v_j|^2/2) f_{j,i} accumulated in FP64, and per-block sums of
// |U_new,m - U_old,m|^2 and |U_old,m|^2 for m = density, momentum, energy.
template <typename T>
__global__ void k_moments_noalloc(bgk::VGrid g, const T* __restrict__ f, int nnode, const double* __restrict__ Uold,
                                  double* __restrict__ Unew, double* __restrict__ partial) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int nm = g.dim + 2;
  double acc[5] = {0, 0, 0, 0, 0};
  if (i < nnode) {
    if (g.dim == 2) {
      for (int j0 = 0; j0 < g.N; ++j0) {
        double s0 = 0, s1 = 0, s2 = 0;
        const T* fr = f + (size_t)j0 * g.N * nnode + i;
        for (int j1 = 0; j1 < g.N; ++j1) {
          const double wf = g.w[j1] * (double)fr[(size_t)j1 * nnode];
          s0 += wf;
          s1 += g.x[j1] * wf;
          s2 += g.x[j1] * g.x[j1] * wf;
        }
        const double w0 = g.w[j0], x0 = g.x[j0];
        acc[0] += w0 * s0;
        acc[1] += w0 * x0 * s0;
        acc[2] += w0 * s1;
        acc[3] += 0.5 * w0 * (x0 * x0 * s0 + s2);
      }
    } else {
      for (int j0 = 0; j0 < g.N; ++j0) {
        double t0 = 0, t1 = 0, t2 = 0, t3 = 0;
        for (int j1 = 0; j1 < g.N; ++j1) {
          double s0 = 0, s1 = 0, s2 = 0;
          const T* fr = f + ((size_t)j0 * g.N + j1) * g.N * nnode + i;
          for (int j2 = 0; j2 < g.N; ++j2) {
            const double wf = g.w[j2] * (double)fr[(size_t)j2 * nnode];
            s0 += wf;
            s1 += g.x[j2] * wf;
            s2 += g.x[j2] * g.x[j2] * wf;
          }
          const double w1 = g.w[j1], x1 = g.x[j1];
          t0 += w1 * s0;
          t1 += w1 * x1 * s0;
          t2 += w1 * s1;
          t3 += w1 * (x1 * x1 * s0 + s2);
        }
        const double w0 = g.w[j0], x0 = g.x[j0];
        acc[0] += w0 * t0;
        acc[1] += w0 * x0 * t0;
        acc[2] += w0 * t1;
        acc[3] += w0 * t2;
        acc[4] += 0.5 * w0 * (x0 * x0 * t0 + t3);
      }
    }
  }
  double r[6] = {0, 0, 0, 0, 0, 0};
  if (i < nnode) {
    for (int m = 0; m < nm; ++m) Unew[(size_t)i * nm + m] = acc[m];
    const double* o = Uold + (size_t)i * nm;
    r[0] = (acc[0] - o[0]) * (acc[0] - o[0]);
    r[1] = o[0] * o[0];
    for (int a = 0; a < g.dim; ++a) {
      r[2] += (acc[1 + a] - o[1 + a]) * (acc[1 + a] - o[1 + a]);
      r[3] += o[1 + a] * o[1 + a];
    }
    r[4] = (acc[nm - 1] - o[nm - 1]) * (acc[nm - 1] - o[nm - 1]);
    r[5] = o[nm - 1] * o[nm - 1];
  }
  __shared__ double red[6][kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double x = r[k];
    for (int o2 = 16; o2 > 0; o2 >>= 1) x += __shfl_down_sync(0xffffffffu, x, o2);
    if (lane == 0) red[k][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[threadIdx.x][w];
    partial[(size_t)blockIdx.x * 6 + threadIdx.x] = s;
  }
}

// Sum the block partials in a fixed order and write the measure
// max(|dU_0|/|U_0|, |dU_1|/max(|U_1|, |U_0|), |dU_2|/|U_2|).
__global__ void k_measure_noalloc(const double* __restrict__ partial, int nblk, double* __restrict__ measure) {
  __shared__ double red[6][256];
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x)
    for (int k = 0; k < 6; ++k) s[k] += partial[(size_t)b * 6 + k];
  for (int k = 0; k < 6; ++k) red[k][threadIdx.x] = s[k];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < 6; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double r0 = sqrt(red[0][0]) / sqrt(red[1][0]);
    const double r1 = sqrt(red[2][0]) / fmax(sqrt(red[3][0]), sqrt(red[1][0]));
    const double r2 = sqrt(red[4][0]) / sqrt(red[5][0]);
    *measure = fmax(r0, fmax(r1, r2));
  }
}

}  // namespace

extern "C" int bgk_moments_measure_noalloc(const bgk_vgrid* vgrid, int dim, int64_t n_nodes, const void* d_f,
                                           int dtype, const double* d_U_old, double* d_U_new, double* d_measure,
                                           void* stream) {
  if (!vgrid || !d_f || !d_U_old || !d_U_new || !d_measure) return BGK_E_INVALID;
  if (n_nodes <= 0 || n_nodes > kMaxNodes) return BGK_E_INVALID;
  if (dtype != BGK_DTYPE_F64 && dtype != BGK_DTYPE_F32) return BGK_E_INVALID;
  bgk::VGrid g;
  if (bgk::build_vgrid(dim, vgrid->n_points, vgrid->k_v, vgrid->L, g) != BGK_OK) return BGK_E_INVALID;
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != BGK_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int nblk = (int)((n_nodes + kThreads - 1) / kThreads);
  if (dtype == BGK_DTYPE_F64)
    k_moments_noalloc<double><<<nblk, kThreads, 0, s>>>(g, (const double*)d_f, (int)n_nodes, d_U_old, d_U_new,
                                                        scratch);
  else
    k_moments_noalloc<float><<<nblk, kThreads, 0, s>>>(g, (const float*)d_f, (int)n_nodes, d_U_old, d_U_new,
                                                       scratch);
  k_measure_noalloc<<<1, 256, 0, s>>>(scratch, nblk, d_measure);
  return cudaGetLastError() == cudaSuccess ? BGK_OK : BGK_E_CUDA;
}
