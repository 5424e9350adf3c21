// Internal state of the learned preconditioner (pcnet.cu) and the entry points the
// Krylov solver uses.
#pragma once
#include <cstdint>
#include <vector>

#include "internal.h"

namespace fsi {
namespace pcn {
constexpr int NLAYER = 15;
constexpr int NLEVEL = 4;

struct Grid3 {
  int nx, ny, nz;
  __host__ __device__ int64_t nv() const { return (int64_t)nx * ny * nz; }
};
// a channel-octet-planar bf16 tensor: voxel (x, y, z) of octet o at
// p + (((oct0 + o) * nz + z) * ny + y) * nx + x) * 8
struct TView {
  uint16_t* p;
  int noct, oct0;
  int nx, ny, nz;
};
}  // namespace pcn
}  // namespace fsi

struct fsi_pc {
  fsi_mesh* m = nullptr;
  int ncomp = 4, cout = 4, nph = 0;
  bool linear = false;    // no ReLU: the network is a linear operator
  bool modulate = false;  // input s_c (1 + phi_s) / 2 for the solids instead of phi
  bool smooth = false;    // apply y <- P R y to the output
  fsi::pcn::Grid3 lv[fsi::pcn::NLEVEL];
  int lcin[fsi::pcn::NLAYER], lcout[fsi::pcn::NLAYER];
  int64_t woff[fsi::pcn::NLAYER];
  int64_t nw = 0;
  float *w = nullptr, *mo = nullptr, *vo = nullptr, *grad = nullptr;  // master weights, Adam moments, gradient
  uint16_t* wpk = nullptr;                                            // packed bf16 B operands
  uint16_t* wf[fsi::pcn::NLAYER];                                     // forward
  uint16_t* wb[fsi::pcn::NLAYER];                                     // data gradient
  int64_t adam_t = 0;
  // activations per level: x (input of the level), a, [e | P d] concatenation, b, d
  uint16_t *x[fsi::pcn::NLEVEL] = {}, *a[fsi::pcn::NLEVEL] = {}, *b[fsi::pcn::NLEVEL] = {},
           *d[fsi::pcn::NLEVEL] = {}, *cat[fsi::pcn::NLEVEL] = {};
  // their gradients
  uint16_t *gd[fsi::pcn::NLEVEL] = {}, *ga[fsi::pcn::NLEVEL] = {}, *gb[fsi::pcn::NLEVEL] = {},
           *gcat[fsi::pcn::NLEVEL] = {}, *ge[fsi::pcn::NLEVEL] = {}, *gx[fsi::pcn::NLEVEL] = {};
  uint16_t* xin = nullptr;    // packed network input of an apply
  float* y32 = nullptr;       // network output [cout][V0]
  float* ys1 = nullptr;       // its restriction to level 1 [cout][V1] (smoothing)
  double* tmp = nullptr;      // [ncomp][nn]
  double* lpart = nullptr;    // reduction partials
  double* loss_dev = nullptr; // per-iteration training losses
  int* err = nullptr;         // device flag: a completion wait gave up
  float* wpart = nullptr;     // weight-gradient partials
  int64_t wpart_n = 0;
  const uint8_t* dmask = nullptr;  // Dirichlet bits of the mesh (bit c: component c)
  double valid_rows = 1.0;
  // training pairs (ring buffer)
  int cap = 0, count = 0, head = 0;
  int64_t in_stride = 0, t_stride = 0;
  uint16_t* ds_in = nullptr;  // packed inputs
  uint16_t* ds_t = nullptr;   // targets, planar bf16 [ncomp][nn]
  std::vector<double> pair_ss; // per stored pair and component: sum of target^2 (valid rows)
  double dbar[4] = {1, 1, 1, 1}, kc[4] = {1, 1, 1, 1};
  bool have_dbar = false;
  // solve checkpoints for harvesting pairs
  double* ck = nullptr;       // [2][CKMAX][n]: x_k, r_k
  int ck_n = 0;
  double flops = 0.0;         // tensor-core flops issued (measurement)
};

namespace fsi {
namespace pcn {
constexpr int CKMAX = 32;
int apply(fsi_pc* pc, const double* r, double rnorm, const double* dinv, double* z);
int add_pair(fsi_pc* pc, const double* ra, const double* rb, const double* ea, const double* eb, const double* dinv);
int check_err(fsi_pc* pc);
int ensure_checkpoints(fsi_pc* pc);
}  // namespace pcn
}  // namespace fsi
