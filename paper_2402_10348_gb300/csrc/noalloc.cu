// fsi_gamma_beta_noalloc: the mobility gamma and the multiplier beta of one phase
// indicator without any device allocation.
//
// This is the same element reduction that fsi_update_ac_coeffs runs (the tile
// kernel over Q1 elements with one partial sum per CTA, then a fixed-order final
// sum), but its per-CTA partial sums live in a file-scope __device__ array instead
// of memory the library allocates.  It exists for callers that cannot call
// cudaMalloc: code that must not synchronise the device (cudaMalloc and cudaFree
// may), and code running inside a framework whose allocator owns all device memory.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "internal.h"

namespace fsi {
namespace {

// Capacity: one {sum val^2, n_band, int F', int sqrt F} slot per CTA of the launch.
constexpr int64_t NOALLOC_MAX_CTAS = 16384;  // 16384 x 4 doubles = 512 KiB per device
static __device__ __align__(256) double g_coef_scratch[4 * NOALLOC_MAX_CTAS];

constexpr int MAX_DEVICES = 64;
// Per-device set-up state, written and read only under g_setup_mu: a host thread
// making its first call on a device either finds both fields set or sets them itself.
static std::mutex g_setup_mu;
static double* g_scratch_ptr[MAX_DEVICES];   // device address of g_coef_scratch, per device
static bool g_ready[MAX_DEVICES];

// Once per device, with that device current: the device address of the scratch
// array (in host code its name is only a host-side stand-in) and the tile kernel's
// shared-memory limit (through the library's locked per-(kernel, device) helper).
int setup_device(int dev, double** ptr) {
  if (dev < 0 || dev >= MAX_DEVICES) return set_error(FSI_EINVAL, "fsi_gamma_beta_noalloc: device ordinal too large");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_ready[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_coef_scratch);
    if (e != cudaSuccess) return cuda_check(e, "cudaGetSymbolAddress(g_coef_scratch)");
    if (!p) return set_error(FSI_ECUDA, "fsi_gamma_beta_noalloc: null scratch address");
    int rc = ensure_smem_attr((const void*)tile_kernel<CoefOp>, tile_smem_bytes<CoefOp>(4));
    if (rc) return rc;
    g_scratch_ptr[dev] = static_cast<double*>(p);
    g_ready[dev] = true;
  }
  *ptr = g_scratch_ptr[dev];
  return FSI_OK;
}

}  // namespace
}  // namespace fsi

using namespace fsi;

extern "C" int fsi_gamma_beta_noalloc(int32_t nx, int32_t ny, int32_t nz, double lx, double ly, double lz,
                                      double eta, const double* v, const double* phi, double* gamma_beta,
                                      void* stream) {
  if (!v || !phi || !gamma_beta) return set_error(FSI_EINVAL, "fsi_gamma_beta_noalloc: null pointer");
  if (nx < 1 || ny < 1 || nz < 1 || !(lx > 0) || !(ly > 0) || !(lz > 0) || !(eta > 0))
    return set_error(FSI_EINVAL, "fsi_gamma_beta_noalloc: need n >= 1, lengths > 0, eta > 0");
  Geom g{};
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.nn = ((int64_t)nx + 1) * ((int64_t)ny + 1) * ((int64_t)nz + 1);
  g.hx = lx / nx; g.hy = ly / ny; g.hz = lz / nz;
  g.ncx = (int)(((int64_t)nx + OX) / OX);
  g.ncy = (int)(((int64_t)ny + OY) / OY);
  const int64_t cols = (int64_t)g.ncx * g.ncy;
  const int64_t planes = (int64_t)nz + 1;
  const int64_t chunks = std::max<int64_t>(1, std::min<int64_t>(planes, (152 + cols / 2) / cols));
  const int64_t zc = (planes + chunks - 1) / chunks;
  const int64_t nchunk = (planes + zc - 1) / zc;
  const int64_t ncta = cols * nchunk;
  if (ncta > NOALLOC_MAX_CTAS) {
    char msg[160];
    snprintf(msg, sizeof msg,
             "fsi_gamma_beta_noalloc: mesh needs %lld partial sums, the static scratch holds %lld",
             (long long)ncta, (long long)NOALLOC_MAX_CTAS);
    return set_error(FSI_EINVAL, msg);
  }
  if (zc > INT32_MAX) return set_error(FSI_EINVAL, "fsi_gamma_beta_noalloc: too many node planes per CTA");
  g.zc = (int)zc;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_check(e, "cudaGetDevice");
  double* scratch = nullptr;
  int rc = setup_device(dev, &scratch);
  if (rc) return rc;

  CoefOp op;
  memset(&op, 0, sizeof(op));
  const int64_t nn = g.nn;
  for (int k = 0; k < 3; ++k) { op.F.d[k] = v + k * nn; op.F.f[k] = nullptr; }
  op.F.d[3] = phi;
  op.nf = 4;
  op.rh[0] = 1.0 / g.hx; op.rh[1] = 1.0 / g.hy; op.rh[2] = 1.0 / g.hz;
  op.W = g.hx * g.hy * g.hz / 8.0;
  op.phi_node = phi;
  op.ncta_xy[0] = g.ncx;
  op.ncta_xy[1] = g.ncy;
  op.partials = scratch;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // every CTA writes its own four slots before the final sum reads them: nothing
  // in the scratch has to start at zero
  tile_kernel<CoefOp><<<dim3(g.ncx, g.ncy, (unsigned)nchunk), NTHREADS, tile_smem_bytes<CoefOp>(4), s>>>(op, g);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(e, "gamma/beta tile kernel launch");
  coef_finalize<<<1, NTHREADS, 0, s>>>(scratch, ncta, eta, gamma_beta);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(e, "gamma/beta final sum launch");
  return FSI_OK;
}
