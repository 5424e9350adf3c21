// Diagnostics of a computed state: the centre of mass of a solid (Section 5.2) and
// the tracking of material points (Appendix C).
//
// Centre of mass, x_c = int x alpha^s / int alpha^s with alpha^s = (1 + phi^s)/2: per
// element, with N_a the trilinear shape functions and x = x0 + h t on [0,1]^3,
//     int alpha    = vol/8  sum_a alpha_a
//     int x_d alpha = vol sum_a alpha_a (x0_d / 8 + h_d I(a_d) / 4),
// I(0) = int (1 - t) t dt = 1/6, I(1) = int t^2 dt = 1/3 -- the values the 2x2x2 Gauss
// rule of the operators gives (it is exact for these integrands).  One thread per
// element (grid-stride), per-CTA sums in a fixed tree order, then one fixed-order sum
// over the CTAs: deterministic.
//
// Tracking: the element of a point follows from its coordinates (clamped onto the
// box), the velocity is the trilinear interpolant of the nodal velocity, and the point
// moves by one forward-Euler step p += dt v(p).
#include <cmath>

#include "internal.h"

namespace fsi {

constexpr int DB = 256;        // threads per CTA
constexpr int DG = 152;        // CTAs of the centre-of-mass reduction
constexpr int DOUT = 1016;     // offset of the four results in the mesh's reduction scratch

__global__ void __launch_bounds__(DB) com_kernel(const double* __restrict__ phi, Geom g, double* part) {
  const int64_t ne = (int64_t)g.nx * g.ny * g.nz;
  const double vol = g.hx * g.hy * g.hz;
  const double h[3] = {g.hx, g.hy, g.hz};
  const int64_t sy = g.nx + 1, sz = (int64_t)(g.nx + 1) * (g.ny + 1);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t e = blockIdx.x * (int64_t)DB + threadIdx.x; e < ne; e += (int64_t)gridDim.x * DB) {
    const int ex = (int)(e % g.nx), ey = (int)((e / g.nx) % g.ny), ez = (int)(e / ((int64_t)g.nx * g.ny));
    const double x0[3] = {ex * g.hx, ey * g.hy, ez * g.hz};
    const int64_t n0 = ex + sy * ey + sz * ez;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int s0 = a & 1, s1 = (a >> 1) & 1, s2 = (a >> 2) & 1;
      const double al = 0.5 * (1.0 + phi[n0 + s0 + sy * s1 + sz * s2]);
      const int s[3] = {s0, s1, s2};
      acc[0] += al;
#pragma unroll
      for (int d = 0; d < 3; ++d) acc[1 + d] += al * (x0[d] / 8.0 + h[d] * (s[d] ? 1.0 / 3.0 : 1.0 / 6.0) / 4.0);
    }
  }
  acc[0] *= vol / 8.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) acc[1 + d] *= vol;
  __shared__ double sm[4][DB / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    double v = acc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sm[i][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int w = 0; w < DB / 32; ++w) s += sm[threadIdx.x][w];
    part[threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void com_finish(const double* __restrict__ part, int G, double* out) {
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int c = 0; c < G; ++c) s += part[threadIdx.x * G + c];
    out[threadIdx.x] = s;
  }
}

__global__ void __launch_bounds__(DB) track_kernel(const double* __restrict__ v, Geom g, double lx, double ly,
                                                   double lz, double dt, int64_t npts, double* __restrict__ pts) {
  const int64_t i = blockIdx.x * (int64_t)DB + threadIdx.x;
  if (i >= npts) return;
  const double L[3] = {lx, ly, lz}, h[3] = {g.hx, g.hy, g.hz};
  const int nc[3] = {g.nx, g.ny, g.nz};
  int cell[3];
  double xi[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double p = fmin(fmax(pts[3 * i + d], 0.0), L[d]);
    int c = (int)floor(p / h[d]);
    c = c < 0 ? 0 : (c > nc[d] - 1 ? nc[d] - 1 : c);
    cell[d] = c;
    xi[d] = (p - c * h[d]) / h[d];
  }
  double vel[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int s0 = a & 1, s1 = (a >> 1) & 1, s2 = (a >> 2) & 1;
    const double w = (s0 ? xi[0] : 1.0 - xi[0]) * (s1 ? xi[1] : 1.0 - xi[1]) * (s2 ? xi[2] : 1.0 - xi[2]);
    const int64_t n = (cell[0] + s0) + (int64_t)(g.nx + 1) * ((cell[1] + s1) + (int64_t)(g.ny + 1) * (cell[2] + s2));
#pragma unroll
    for (int k = 0; k < 3; ++k) vel[k] += w * v[(int64_t)k * g.nn + n];
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) pts[3 * i + d] += dt * vel[d];
}

}  // namespace fsi

using namespace fsi;

int fsi_center_of_mass(fsi_mesh* m, const double* x, int32_t solid, double* out) {
  if (m && m->tet) return set_error(FSI_EINVAL, "diagnostics: not on tetrahedral meshes");
  if (!m || !x || !out) return set_error(FSI_EINVAL, "fsi_center_of_mass: null argument");
  if (solid < 0 || solid >= m->ns) return set_error(FSI_EINVAL, "fsi_center_of_mass: bad solid index");
  const double* phi = x + (int64_t)(4 + m->P.solid_phase[solid]) * m->nn;
  double* part = m->red;
  double* res = m->red + DOUT;
  FSI_LAUNCH(m, P_INIT, com_kernel<<<DG, DB, 0, m->stream>>>(phi, m->g, part));
  FSI_LAUNCH(m, P_INIT, com_finish<<<1, 32, 0, m->stream>>>(part, DG, res));
  FSI_CUDA(cudaMemcpyAsync(m->red_host, res, sizeof(double) * 4, cudaMemcpyDeviceToHost, m->stream));
  FSI_CUDA(cudaStreamSynchronize(m->stream));
  const double mass = m->red_host[0];
  if (!(mass > 0.0) || !std::isfinite(mass))
    return set_error(FSI_EINVAL, "fsi_center_of_mass: the solid's indicator has no positive mass");
  for (int d = 0; d < 3; ++d) out[d] = m->red_host[1 + d] / mass;
  return FSI_OK;
}

int fsi_track_points(fsi_mesh* m, const double* x, int64_t n, double* points) {
  if (m && m->tet) return set_error(FSI_EINVAL, "diagnostics: not on tetrahedral meshes");
  if (!m || n < 0) return set_error(FSI_EINVAL, "fsi_track_points: bad argument");
  if (n == 0) return FSI_OK;
  if (!x || !points) return set_error(FSI_EINVAL, "fsi_track_points: null argument");
  const unsigned grid = (unsigned)((n + DB - 1) / DB);
  FSI_LAUNCH(m, P_INIT, track_kernel<<<grid, DB, 0, m->stream>>>(x, m->g, m->lx, m->ly, m->lz, m->P.dt, n, points));
  return FSI_OK;
}
