// fsi_gamma_beta_noalloc: the mobility gamma and the multiplier beta of one phase
// indicator without any device allocation.
//
// This is the same element reduction that fsi_update_ac_coeffs runs (the tile
// kernel over Q1 elements with one partial sum per CTA, then a fixed-order final
// sum), but its per-CTA partial sums live in a file-scope __device__ array instead
// of memory the library allocates.  It exists for callers that cannot call
// cudaMalloc: code that must not synchronise the device (cudaMalloc and cudaFree
// may), and code running inside a framework whose allocator owns all device memory.
#include <cstdio>

#include "internal.h"

namespace fsi {
namespace {

// Capacity: one {sum val^2, n_band, int F', int sqrt F} slot per CTA of the launch.
constexpr int64_t NOALLOC_MAX_CTAS = 16384;  // 16384 x 4 doubles = 512 KiB per device
static __device__ __align__(256) double g_coef_scratch[4 * NOALLOC_MAX_CTAS];

constexpr int MAX_DEVICES = 64;
static double* g_scratch_ptr[MAX_DEVICES];   // device address of g_coef_scratch, per device
static bool g_ready[MAX_DEVICES];

__global__ void noalloc_finalize(const double* partials, int64_t n, double eta, double* out) {
  __shared__ double s[4][NTHREADS];
  double a[4] = {0, 0, 0, 0};
  for (int64_t i = threadIdx.x; i < n; i += NTHREADS)
    for (int c = 0; c < 4; ++c) a[c] += partials[4 * i + c];
  for (int c = 0; c < 4; ++c) s[c][threadIdx.x] = a[c];
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[4] = {0, 0, 0, 0};
    for (int i = 0; i < NTHREADS; ++i)
      for (int c = 0; c < 4; ++c) t[c] += s[c][i];
    out[0] = t[1] > 0.0 ? sqrt(t[0] / t[1]) / eta : 0.0;
    out[1] = t[3] != 0.0 ? t[2] / t[3] : 0.0;
  }
}

// Once per device, with that device current: the device address of the scratch
// array (in host code its name is only a host-side stand-in) and the kernel's
// shared-memory limit.
int setup_device(int dev, double** ptr) {
  if (dev < 0 || dev >= MAX_DEVICES) return set_error(FSI_EINVAL, "fsi_gamma_beta_noalloc: device ordinal too large");
  if (!g_ready[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_coef_scratch);
    if (e != cudaSuccess) return cuda_check(e, "cudaGetSymbolAddress(g_coef_scratch)");
    e = cudaFuncSetAttribute(tile_kernel<CoefOp>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tile_smem_bytes<CoefOp>(4));
    if (e != cudaSuccess) return cuda_check(e, "cudaFuncSetAttribute");
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
  g.nn = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  g.hx = lx / nx; g.hy = ly / ny; g.hz = lz / nz;
  g.ncx = (nx + 1 + OX - 1) / OX;
  g.ncy = (ny + 1 + OY - 1) / OY;
  const int64_t cols = (int64_t)g.ncx * g.ncy;
  const int planes = nz + 1;
  const int chunks = (int)std::max<int64_t>(1, std::min<int64_t>(planes, (152 + cols / 2) / cols));
  g.zc = (planes + chunks - 1) / chunks;
  const int nchunk = (planes + g.zc - 1) / g.zc;
  const int64_t ncta = cols * nchunk;
  if (ncta > NOALLOC_MAX_CTAS) {
    char msg[160];
    snprintf(msg, sizeof msg,
             "fsi_gamma_beta_noalloc: mesh needs %lld partial sums, the static scratch holds %lld",
             (long long)ncta, (long long)NOALLOC_MAX_CTAS);
    return set_error(FSI_EINVAL, msg);
  }
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
  tile_kernel<CoefOp><<<dim3(g.ncx, g.ncy, nchunk), NTHREADS, tile_smem_bytes<CoefOp>(4), s>>>(op, g);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(e, "gamma/beta tile kernel launch");
  noalloc_finalize<<<1, NTHREADS, 0, s>>>(scratch, ncta, eta, gamma_beta);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(e, "gamma/beta final sum launch");
  return FSI_OK;
}
