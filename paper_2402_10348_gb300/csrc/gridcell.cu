// Phase-indicator initialisation from triangulated surfaces (Section 3): grid-cell
// nearest-vertex distance (Algorithm 1) and +x ray casting with non-duplicated
// plane partitioning (Algorithm 2).
//
// This unit is compiled with -fmad=false: every float64 operation below rounds
// separately, in the order written, so integer results (cells, nearest vertices,
// crossing numbers) are bit-identical to any other IEEE evaluation of the same
// expressions:
//   node x = i*hx, cell size hc = (nx*hx - 0)/gx, cell = min(floor(x/hc), gx-1),
//   triangle cells floor(((min - 3eps) - 0)/hc) .. floor(((max + 3eps) - 0)/hc),
//   d^2 = (dx*dx + dy*dy) + dz*dz, area = 0.5*|(b_y-a_y)*(c_z-a_z) - (b_z-a_z)*(c_y-a_y)|,
//   x_c = ((A1*x1 + A2*x2) + A3*x3)/A0.
// Each triangle of a row of cells is tested once, in the first cell of the row
// segment [i, gx) that lists it; element crossings of distinct triangles are
// distinct keys, edge and node keys are de-duplicated in a per-ray list.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace fsi {

struct GCGeom {
  int nx, ny, nz;
  double hx, hy, hz;
  int g[3];
  double hc[3];
  double eps3;   // 3 eps
  double chi;
  double scale;  // sqrt(2) eps
};

__device__ __forceinline__ int cell_of(double x, double hc, int g) {
  const int c = (int)floor(x / hc);
  return c < g - 1 ? c : g - 1;
}

__global__ void tri_ranges(const double* __restrict__ V, const int* __restrict__ T, int nt, GCGeom G, int* range,
                           int* counts) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  int r[6];
  for (int d = 0; d < 3; ++d) {
    const double a = V[3 * T[3 * t + 0] + d], b = V[3 * T[3 * t + 1] + d], c = V[3 * T[3 * t + 2] + d];
    const double lo = fmin(fmin(a, b), c), hi = fmax(fmax(a, b), c);
    int i0 = (int)floor(((lo - G.eps3) - 0.0) / G.hc[d]);
    int i1 = (int)floor(((hi + G.eps3) - 0.0) / G.hc[d]);
    i0 = min(max(i0, 0), G.g[d] - 1);
    i1 = min(max(i1, 0), G.g[d] - 1);
    r[2 * d] = i0;
    r[2 * d + 1] = i1;
    range[6 * t + 2 * d] = i0;
    range[6 * t + 2 * d + 1] = i1;
  }
  if (counts)
    for (int cz = r[4]; cz <= r[5]; ++cz)
      for (int cy = r[2]; cy <= r[3]; ++cy)
        for (int cx = r[0]; cx <= r[1]; ++cx) atomicAdd(&counts[cx + G.g[0] * (cy + G.g[1] * cz)], 1);
}

__global__ void tri_fill(const int* __restrict__ range, int nt, GCGeom G, const int* __restrict__ offs, int* cursor,
                         int* list) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const int* r = range + 6 * t;
  for (int cz = r[4]; cz <= r[5]; ++cz)
    for (int cy = r[2]; cy <= r[3]; ++cy)
      for (int cx = r[0]; cx <= r[1]; ++cx) {
        const int c = cx + G.g[0] * (cy + G.g[1] * cz);
        const int p = atomicAdd(&cursor[c], 1);
        list[offs[c] + p] = t;
      }
}

__device__ __forceinline__ double area2d(double ay, double az, double by, double bz, double cy, double cz) {
  return 0.5 * fabs((by - ay) * (cz - az) - (bz - az) * (cy - ay));
}

constexpr int MAXKEYS = 64;

// Crossing number of the +x ray from (xp, yp, zp) in cell (cx, cy, cz); -1 on key overflow.
__device__ int ray_cross(double xp, double yp, double zp, int cx, int cy, int cz, const double* __restrict__ V,
                         const int* __restrict__ T, const int* __restrict__ range, const int* __restrict__ offs,
                         const int* __restrict__ counts, const int* __restrict__ list, const GCGeom& G) {
  int n_elem = 0, n_keys = 0;
  int ka[MAXKEYS], kb[MAXKEYS];  // edge (a<b) or node (a, -1) keys
  for (int c = cx; c < G.g[0]; ++c) {
    const int cell = c + G.g[0] * (cy + G.g[1] * cz);
    const int o = offs[cell], cnt = counts[cell];
    for (int q = 0; q < cnt; ++q) {
      const int t = list[o + q];
      const int i0 = range[6 * t], i1 = range[6 * t + 1];
      const int first = i0 > cx ? i0 : cx;
      if (first != c) continue;  // tested in an earlier cell of this row
      const int v1 = T[3 * t], v2 = T[3 * t + 1], v3 = T[3 * t + 2];
      const double x1 = V[3 * v1], y1 = V[3 * v1 + 1], z1 = V[3 * v1 + 2];
      const double x2 = V[3 * v2], y2 = V[3 * v2 + 1], z2 = V[3 * v2 + 2];
      const double x3 = V[3 * v3], y3 = V[3 * v3 + 1], z3 = V[3 * v3 + 2];
      const double A0 = area2d(y1, z1, y2, z2, y3, z3);
      if (!(A0 > G.chi)) continue;
      const double A1 = area2d(yp, zp, y2, z2, y3, z3);
      const double A2 = area2d(yp, zp, y3, z3, y1, z1);
      const double A3 = area2d(yp, zp, y1, z1, y2, z2);
      if (!(((A1 + A2) + A3) - A0 <= 2.0 * G.chi)) continue;
      const double xc = ((A1 * x1 + A2 * x2) + A3 * x3) / A0;
      if (!(xc > xp)) continue;
      // in the node's own cell only triangles with a vertex beyond the node count,
      // unless the triangle is listed again further along the row
      if (c == cx && !(x1 > xp || x2 > xp || x3 > xp) && !(i1 > cx)) continue;
      const bool s1 = A1 < G.chi, s2 = A2 < G.chi, s3 = A3 < G.chi;
      const int ns = (int)s1 + (int)s2 + (int)s3;
      int a = -1, b = -1;
      if (ns == 1) {
        if (s1) { a = v2; b = v3; } else if (s2) { a = v3; b = v1; } else { a = v1; b = v2; }
        if (a > b) { const int tmp = a; a = b; b = tmp; }
      } else if (ns == 2) {
        a = !s1 ? v1 : (!s2 ? v2 : v3);
        b = -1;
      } else {
        ++n_elem;
        continue;
      }
      bool dup = false;
      for (int k = 0; k < n_keys; ++k) dup |= (ka[k] == a && kb[k] == b);
      if (!dup) {
        if (n_keys == MAXKEYS) return -1;
        ka[n_keys] = a;
        kb[n_keys] = b;
        ++n_keys;
      }
    }
  }
  return n_elem + n_keys;
}

// Representative (lowest-index) node of every cell without triangles: its crossing number.
__global__ void empty_cells(const double* __restrict__ V, const int* __restrict__ T, const int* __restrict__ range,
                            const int* __restrict__ offs, const int* __restrict__ counts, const int* __restrict__ list,
                            GCGeom G, const int* __restrict__ first_node /*[3][gmax]*/, int gmax, int* cell_cross,
                            int* err) {
  const int ncell = G.g[0] * G.g[1] * G.g[2];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  cell_cross[c] = 0;
  if (counts[c] != 0) return;
  const int cx = c % G.g[0], cy = (c / G.g[0]) % G.g[1], cz = c / (G.g[0] * G.g[1]);
  const int i = first_node[cx], j = first_node[gmax + cy], k = first_node[2 * gmax + cz];
  if (i < 0 || j < 0 || k < 0) return;  // the cell holds no node
  const int r = ray_cross(i * G.hx, j * G.hy, k * G.hz, cx, cy, cz, V, T, range, offs, counts, list, G);
  if (r < 0) atomicExch(err, 1);
  cell_cross[c] = r;
}

__global__ void node_phi(const double* __restrict__ V, const int* __restrict__ T, const int* __restrict__ range,
                         const int* __restrict__ offs, const int* __restrict__ counts, const int* __restrict__ list,
                         const int* __restrict__ cell_cross, GCGeom G, double* phi, int* tags, int64_t nn,
                         int* err) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const int i = (int)(n % (G.nx + 1));
  const int j = (int)((n / (G.nx + 1)) % (G.ny + 1));
  const int k = (int)(n / ((int64_t)(G.nx + 1) * (G.ny + 1)));
  const double xp = i * G.hx, yp = j * G.hy, zp = k * G.hz;
  const int cx = cell_of(xp, G.hc[0], G.g[0]), cy = cell_of(yp, G.hc[1], G.g[1]), cz = cell_of(zp, G.hc[2], G.g[2]);
  const int cell = cx + G.g[0] * (cy + G.g[1] * cz);
  int nearest = -1, cross;
  double mag = 1.0;
  if (counts[cell] > 0) {
    double best = INFINITY;
    const int o = offs[cell], cnt = counts[cell];
    for (int q = 0; q < cnt; ++q) {
      const int t = list[o + q];
      for (int e = 0; e < 3; ++e) {
        const int v = T[3 * t + e];
        const double dx = xp - V[3 * v], dy = yp - V[3 * v + 1], dz = zp - V[3 * v + 2];
        const double d2 = (dx * dx + dy * dy) + dz * dz;
        if (d2 < best || (d2 == best && v < nearest)) {
          best = d2;
          nearest = v;
        }
      }
    }
    mag = tanh(sqrt(best) / G.scale);
    cross = ray_cross(xp, yp, zp, cx, cy, cz, V, T, range, offs, counts, list, G);
    if (cross < 0) {
      atomicExch(err, 1);
      cross = 0;
    }
  } else {
    cross = cell_cross[cell];
  }
  const bool inside = (cross & 1) == 1;
  phi[n] = inside ? mag : -mag;
  if (tags) {
    tags[n] = cell;
    tags[nn + n] = nearest;
    tags[2 * nn + n] = cross;
    tags[3 * nn + n] = inside ? 1 : 0;
  }
}

struct RuleDev {
  int kind, surface, side;
  double plane_z;
};

__global__ void apply_rules_kernel(const double* __restrict__ phis /*[n_surf][nn]*/, const RuleDev* rules, int nrules,
                                   double* out, int64_t nn, int nx, int ny, double hz, double scale) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= nn) return;
  double solid = 0.0;
  for (int r = 0; r < nrules; ++r)
    if (rules[r].kind == FSI_RULE_SURFACE) {
      const double p = phis[(int64_t)rules[r].surface * nn + n];
      out[(int64_t)r * nn + n] = p;
      solid = solid + (1.0 + p) / 2.0;
    }
  const int k = (int)(n / ((int64_t)(nx + 1) * (ny + 1)));
  const double z = k * hz;
  for (int r = 0; r < nrules; ++r)
    if (rules[r].kind == FSI_RULE_COMPLEMENT) {
      double a = fmax(0.0, 1.0 - solid);
      if (rules[r].side != 0) {
        const double pp = tanh((rules[r].plane_z - z) / scale);
        a = a * (rules[r].side > 0 ? (1.0 + pp) / 2.0 : (1.0 - pp) / 2.0);
      }
      out[(int64_t)r * nn + n] = 2.0 * a - 1.0;
    }
}

template <typename T>
struct DevBuf {
  T* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
  cudaError_t alloc(size_t n) { return cudaMalloc(&p, sizeof(T) * std::max<size_t>(n, 1)); }
};

static int cell_index_host(double x, double hc, int g) {
  const int c = (int)std::floor(x / hc);
  return c < g - 1 ? c : g - 1;
}

}  // namespace fsi

using namespace fsi;

extern "C" int fsi_init_phases(fsi_mesh* m, const fsi_surface* surfs, int32_t n_surf, const fsi_phase_rule* rules,
                               int32_t gx, int32_t gy, int32_t gz, double* phi_out, int32_t* tags_out) {
  if (m && m->tet) return set_error(FSI_EINVAL, "fsi_init_phases: not on tetrahedral meshes");
  if (!m || !phi_out || (n_surf > 0 && !surfs) || !rules) return set_error(FSI_EINVAL, "fsi_init_phases: null argument");
  if (gx < 1 || gy < 1 || gz < 1) return set_error(FSI_EINVAL, "fsi_init_phases: grid cells must be >= 1");
  for (int r = 0; r < m->N; ++r)
    if (rules[r].kind == FSI_RULE_SURFACE && (rules[r].surface < 0 || rules[r].surface >= n_surf))
      return set_error(FSI_EINVAL, "fsi_init_phases: rule names a missing surface");
  GCGeom G;
  G.nx = m->g.nx; G.ny = m->g.ny; G.nz = m->g.nz;
  G.hx = m->g.hx; G.hy = m->g.hy; G.hz = m->g.hz;
  G.g[0] = gx; G.g[1] = gy; G.g[2] = gz;
  const double xmax[3] = {m->g.nx * m->g.hx, m->g.ny * m->g.hy, m->g.nz * m->g.hz};
  for (int d = 0; d < 3; ++d) G.hc[d] = (xmax[d] - 0.0) / G.g[d];
  G.eps3 = 3.0 * m->P.eps;
  G.chi = 1e-12 * (m->lx * m->lx + m->ly * m->ly + m->lz * m->lz);
  G.scale = std::sqrt(2.0) * m->P.eps;
  const int64_t nn = m->nn;
  const int ncell = gx * gy * gz;
  // lowest node index of every cell row/column/layer: first i with cell(i) == c
  const int gmax = std::max(gx, std::max(gy, gz));
  std::vector<int> first(3 * gmax, -1);
  const int nmax[3] = {m->g.nx, m->g.ny, m->g.nz};
  const double h[3] = {m->g.hx, m->g.hy, m->g.hz};
  for (int d = 0; d < 3; ++d)
    for (int i = nmax[d]; i >= 0; --i) first[d * gmax + cell_index_host(i * h[d], G.hc[d], G.g[d])] = i;
  DevBuf<double> phis;
  DevBuf<int> dfirst, dcounts, doffs, dcursor, dcellx, derr;
  cudaStream_t s = m->stream;
  FSI_CUDA(phis.alloc((size_t)std::max(1, (int)n_surf) * nn));
  FSI_CUDA(dfirst.alloc(3 * gmax));
  FSI_CUDA(dcounts.alloc(ncell));
  FSI_CUDA(doffs.alloc(ncell));
  FSI_CUDA(dcursor.alloc(ncell));
  FSI_CUDA(dcellx.alloc(ncell));
  FSI_CUDA(derr.alloc(1));
  FSI_CUDA(cudaMemcpyAsync(dfirst.p, first.data(), sizeof(int) * 3 * gmax, cudaMemcpyHostToDevice, s));
  FSI_CUDA(cudaMemsetAsync(derr.p, 0, sizeof(int), s));
  std::vector<int> counts(ncell), offs(ncell);
  for (int si = 0; si < n_surf; ++si) {
    const fsi_surface& S = surfs[si];
    if (S.n_verts < 1 || S.n_tris < 1 || !S.verts || !S.tris) return set_error(FSI_EINVAL, "surface: empty");
    for (int t = 0; t < 3 * S.n_tris; ++t)
      if (S.tris[t] < 0 || S.tris[t] >= S.n_verts) return set_error(FSI_EINVAL, "surface: vertex index out of range");
    DevBuf<double> dV;
    DevBuf<int> dT, drange, dlist;
    FSI_CUDA(dV.alloc(3 * (size_t)S.n_verts));
    FSI_CUDA(dT.alloc(3 * (size_t)S.n_tris));
    FSI_CUDA(drange.alloc(6 * (size_t)S.n_tris));
    FSI_CUDA(cudaMemcpyAsync(dV.p, S.verts, sizeof(double) * 3 * S.n_verts, cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemcpyAsync(dT.p, S.tris, sizeof(int) * 3 * S.n_tris, cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemsetAsync(dcounts.p, 0, sizeof(int) * ncell, s));
    const int tb = 128, tg = (S.n_tris + tb - 1) / tb;
    FSI_LAUNCH(m, P_INIT, tri_ranges<<<tg, tb, 0, s>>>(dV.p, dT.p, S.n_tris, G, drange.p, dcounts.p));
    FSI_CUDA(cudaMemcpyAsync(counts.data(), dcounts.p, sizeof(int) * ncell, cudaMemcpyDeviceToHost, s));
    FSI_CUDA(cudaStreamSynchronize(s));
    int64_t total = 0;
    for (int c = 0; c < ncell; ++c) {
      offs[c] = (int)total;
      total += counts[c];
    }
    if (total > (int64_t)1 << 31) return set_error(FSI_EINVAL, "surface: too many cell entries");
    FSI_CUDA(dlist.alloc((size_t)total));
    FSI_CUDA(cudaMemcpyAsync(doffs.p, offs.data(), sizeof(int) * ncell, cudaMemcpyHostToDevice, s));
    FSI_CUDA(cudaMemsetAsync(dcursor.p, 0, sizeof(int) * ncell, s));
    FSI_LAUNCH(m, P_INIT, tri_fill<<<tg, tb, 0, s>>>(drange.p, S.n_tris, G, doffs.p, dcursor.p, dlist.p));
    FSI_LAUNCH(m, P_INIT, empty_cells<<<(ncell + 127) / 128, 128, 0, s>>>(dV.p, dT.p, drange.p, doffs.p, dcounts.p, dlist.p, G, dfirst.p,
                                                   gmax, dcellx.p, derr.p));
    FSI_LAUNCH(m, P_INIT, node_phi<<<(unsigned)((nn + 127) / 128), 128, 0, s>>>(dV.p, dT.p, drange.p, doffs.p, dcounts.p, dlist.p,
                                                          dcellx.p, G, phis.p + (int64_t)si * nn,
                                                          tags_out ? tags_out + (int64_t)si * 4 * nn : nullptr, nn,
                                                          derr.p));
    FSI_CUDA(cudaStreamSynchronize(s));  // the surface buffers are freed at scope exit
  }
  std::vector<RuleDev> rd(m->N);
  for (int r = 0; r < m->N; ++r) rd[r] = RuleDev{rules[r].kind, rules[r].surface, rules[r].plane_side, rules[r].plane_z};
  DevBuf<RuleDev> drules;
  FSI_CUDA(drules.alloc(m->N));
  FSI_CUDA(cudaMemcpyAsync(drules.p, rd.data(), sizeof(RuleDev) * m->N, cudaMemcpyHostToDevice, s));
  FSI_LAUNCH(m, P_INIT, apply_rules_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(phis.p, drules.p, m->N, phi_out, nn, m->g.nx,
                                                                   m->g.ny, m->g.hz, G.scale));
  int herr = 0;
  FSI_CUDA(cudaMemcpyAsync(&herr, derr.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FSI_CUDA(cudaStreamSynchronize(s));
  if (herr) return set_error(FSI_EINVAL, "fsi_init_phases: more than 64 distinct edge/node crossings on one ray");
  return FSI_OK;
}
