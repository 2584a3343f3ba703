// Internal declarations shared by the host (C++) and device (CUDA) parts of the library.
#pragma once
#include <stdint.h>

#include <vector>

#include "../../include/bgk.h"

namespace bgk {

constexpr int kMaxN1D = 128;  // velocity points per dimension (the paper runs up to 128)
constexpr int kMaxKv = 4;     // velocity polynomial degree

// Velocity grid of Sec. 3.2 (passed by value to kernels).
struct VGrid {
  int dim, N, kv, np, ncl, nv;
  double L, h;
  double x[kMaxN1D], w[kMaxN1D];
  // moment weights w, w x, w x^2 per 1D point; and each split into two floats (hi + lo)
  // for the compensated FP32 reduction of FP32 distributions
  double wx[kMaxN1D], wxx[kMaxN1D];
  float wh[3][kMaxN1D], wl[3][kMaxN1D];
  // Lagrange basis of one velocity cell in its local variable xi in [-1, 1]:
  // l_k(xi) = sum_p lag[k][p] xi^p  (same for every cell of the uniform grid).
  double lag[kMaxKv + 1][kMaxKv + 1];
  // the same grid constants as floats, for projections computed in FP32
  float bnd_f[kMaxN1D + 1];   // cell boundaries -L + c h
  float mid_f[kMaxN1D];       // cell midpoints
  float iw_f[kMaxN1D];        // 1 / w_m
  float lag_f[kMaxKv + 1][kMaxKv + 1];
  float hh_f;                 // h / 2
};

// Geometry of the mesh as the sweep needs it (Sec. 3.1 / 3.3).  Per cell: the d+1
// outward area-weighted face normals N_i (face i opposite vertex i) and 1/|K|.
struct HostMesh {
  int dim = 0, kx = 0, ndof = 0, nf = 0, fd = 0, ncell = 0, nvert = 0, nbface = 0, geo_stride = 0;
  bool quad = false;              // Q1 parallelograms (2D, 4 vertices per cell) instead of simplices
  std::vector<double> geo;        // [cell][geo_stride]: N_0 .. N_d (dim each), 1/|K|
  std::vector<int32_t> nbr;       // [cell][4]: neighbour id, or -(boundary face + 1)
  std::vector<int32_t> nbr_face;  // [cell][4]: face index of this face in the neighbour
  std::vector<uint64_t> perm;     // [cell]: 16 bits per face, 4 bits per face-local node:
                                  //   the neighbour's local node matching face node k
  std::vector<int32_t> bnode;     // [bface][fd]: node index (cell*ndof+local) of face node k
  std::vector<int8_t> bside;      // [bface]: side 2a + (n_a > 0) of the box when the unit
                                  //   outward normal is +/-e_a, else -1
  double min_vol = 0.0;
};

// Builds HostMesh from the C-ABI mesh; returns BGK_OK or BGK_E_INVALID.
int build_host_mesh(const bgk_mesh* m, HostMesh& hm);
// Gauss-Legendre velocity grid and the cell Lagrange basis.
int build_vgrid(int dim, int N, int kv, double L, VGrid& g);
// Sign of v_j . N for face f of cell c, evaluated in FP64 without contraction:
// +1 outflow, -1 inflow, 0 none.  Bit-identical to the device evaluation.
int host_face_sign(const HostMesh& hm, const VGrid& g, int j, int c, int f);
// For one ordinate: break the cycles of the sweep graph (SCCs; DFS from the smallest
// id of each non-trivial SCC, successors in ascending id; back edges are lagged) and
// set bit f of lag[c] when the inflow of cell c through face f is lagged.
// Returns the number of lagged edges.
int host_break_cycles(const HostMesh& hm, const VGrid& g, int j, uint8_t* lag);

// Packed generation-list entry: cell id in bits 0..23, then 2 bits per face
// (01 outflow, 10 inflow, 00 no flux) in bits 24..31.
constexpr int kCellBits = 24;
constexpr uint32_t kCellMask = (1u << kCellBits) - 1u;

}  // namespace bgk
