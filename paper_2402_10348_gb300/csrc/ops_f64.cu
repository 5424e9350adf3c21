// Float64 instantiations of the element operators and the gamma/beta reduction.
#include "ops_impl.cuh"

namespace fsi {

template int launch_ns<double>(fsi_mesh*, int, const double*, double*, unsigned);
template int launch_nsq<double>(fsi_mesh*, const double*, double*, unsigned);

// Builds the quadrature-point coefficients of the NS product at the staged state, in
// float64, with their float32 copy; solids beyond one pass's shared memory are added
// by further passes.
int ns_build(fsi_mesh* m, unsigned flags) {
  const int nxp = cq_pitch(m);
  const int64_t len = (int64_t)m->g.nz * 8 * NCQ * nxp * m->g.ny;
  if (m->cq_len < len) {
    cudaFree(m->cq64);
    cudaFree(m->cq32);
    m->cq64 = nullptr;
    m->cq32 = nullptr;
    m->cq_len = 0;
    FSI_CUDA(cudaMalloc(&m->cq64, sizeof(double) * (size_t)len));
    FSI_CUDA(cudaMalloc(&m->cq32, sizeof(float) * (size_t)len));
    m->cq_len = len;
  }
  const bool aug = (flags & FSI_ELASTIC_AUG) != 0;
  const int ns = aug ? m->ns : 0;
  const int fixed = 9;
  const int per = std::min(solids_per_pass<double>(fixed), (MAXF - fixed) / 7);
  if (per < 1 && ns > 0) return set_error(FSI_EINVAL, "NS coefficients: shared memory too small for one solid");
  const double* xa = m->staged_xa;
  const int64_t nn = m->nn;
  int s0 = 0;
  bool first = true;
  do {
    const int s1 = ns == 0 ? 0 : std::min(ns, s0 + per);
    NSBuildOp op;
    memset(&op, 0, sizeof(op));
    int f = 0;
    for (int k = 0; k < 3; ++k) put<double>(op.F, f++, xa + k * nn);  // v
    put<double>(op.F, f++, xa + 3 * nn);                                 // p^{n+1}
    for (int k = 0; k < 3; ++k) put<double>(op.F, f++, m->xd + k * nn); // dv/dt
    put<double>(op.F, f++, m->mat);                                      // rho
    put<double>(op.F, f++, m->mat + nn);                                 // mu
    for (int s = s0; s < s1; ++s) {
      put<double>(op.F, f++, m->mat + (2 + s) * nn);                     // alpha^s
      const int c0 = 4 + m->N + 6 * s;
      for (int c = 0; c < 6; ++c) put<double>(op.F, f++, xa + (c0 + c) * nn);
    }
    op.nf = f;
    op.s0 = s0;
    op.s1 = s1;
    op.fluid = first ? 1 : 0;
    op.elastic_aug = aug ? 1 : 0;
    op.P = m->P;
    fill_common(m, op.rh, &op.W);
    op.C.c64 = m->cq64;
    op.C.c32 = m->cq32;
    op.C.nxp = nxp;
    op.C.nxyp = (int64_t)nxp * m->g.ny;
    if (int rc = run_tile(m, op, P_NS_BUILD)) return rc;
    first = false;
    s0 = s1;
  } while (s0 < ns);
  m->cq_gen = m->stage_gen;
  m->cq_flags = flags & FSI_ELASTIC_AUG;
  ++m->cq_builds;
  return FSI_OK;
}

// Build: one thread per (element, column); threadIdx.x runs along x (coalesced
// coefficient loads and matrix stores), threadIdx.y and blockIdx.z over columns.
__global__ void __launch_bounds__(256) nse_build_kernel(const double* __restrict__ cq, double* __restrict__ K,
                                                        int nx, int ny, int nz, int nxp, int64_t nxyp, int elastic,
                                                        double alpha, double cm, double rhx, double rhy, double rhz) {
  const int ex = blockIdx.x * 32 + threadIdx.x;
  const int eyz = blockIdx.y;
  const int ey = eyz % ny, ez = eyz / ny;
  const int j = blockIdx.z * 8 + threadIdx.y;  // column: field j / 8, corner j % 8
  if (ex >= nx || ez >= nz) return;
  const int f = j >> 3, a = j & 7;
  const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
  const double* e0 = cq + (int64_t)ez * 8 * NCQ * nxyp + (int64_t)ey * nxp + ex;
  double c[4][8];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int b = 0; b < 8; ++b) c[q][b] = 0.0;
#pragma unroll 1
  for (int q = 0; q < 8; ++q) {
    QW<double> w;
    w.set(q);
    // the unit increment at corner a, interpolated: N_a and grad N_a at the point
    const double N = w.wx[ax] * w.wy[ay] * w.wz[az];
    const double g[3] = {(ax ? 1.0 : -1.0) * rhx * w.wy[ay] * w.wz[az], (ay ? 1.0 : -1.0) * rhy * w.wx[ax] * w.wz[az],
                         (az ? 1.0 : -1.0) * rhz * w.wx[ax] * w.wy[ay]};
    double dv[3], gd[3][3], dgp[3];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
      const bool on = f == kk;
      dv[kk] = on ? N : 0.0;
#pragma unroll
      for (int b = 0; b < 3; ++b) gd[kk][b] = on ? g[b] : 0.0;
      dgp[kk] = f == 3 ? g[kk] : 0.0;
    }
    const double dp = f == 3 ? N : 0.0;
    nsq_point<double>(CoefRef<double>{e0 + (int64_t)q * NCQ * nxyp, nxyp}, elastic != 0, dv, gd, dp, dgp, alpha, cm,
                      w, rhx, rhy, rhz, c);
  }
  double* out = K + ((int64_t)ez * NKE + j) * nxyp + (int64_t)ey * nxp + ex;
#pragma unroll
  for (int i = 0; i < 32; ++i) out[(int64_t)i * 32 * nxyp] = c[i >> 3][i & 7];
}

// Element-centric products of the Allen-Cahn element matrices and the B split operator:
// one thread per element (x fastest) gathers its increment values, applies the stored
// operator and writes its 8 (AC) or 48 (B) corner contributions into E[slot][element];
// em_node_kernel then sums, per node, the slots of its up to 8 elements in a fixed order
// (z, y, x).  Each element is evaluated once (no halo recomputation); deterministic.
// Allen-Cahn: c[b] = sum_a K[b][a] x[a]
__global__ void __launch_bounds__(128) ace_elem_kernel(const double* __restrict__ K, const double* __restrict__ dx,
                                                       double* __restrict__ E, int nx, int ny, int nz, int nxp,
                                                       int64_t nxyp) {
  ElemIdx I;
  if (!I.set(nx, ny, nz, nxp, nxyp)) return;
  double x[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) x[a] = __ldg(dx + I.n0 + I.off[a]);
  const double* k = K + (int64_t)I.ez * 64 * nxyp + (int64_t)I.ey * nxp + I.ex;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) acc += __ldg(k + (int64_t)(b * 8 + a) * nxyp) * x[a];
    E[b * I.es + I.e] = acc;
  }
}

// B split operator of one solid: c[cc][a] = sum_b S[a][b] dB_cc[b]
//   - sum_q Ta_q[a] (L_q dB_q + dB_q L_q^T)_cc   (the stretching coupling at point q)
__global__ void __launch_bounds__(128) be_elem_kernel(const double* __restrict__ K, const double* __restrict__ dx,
                                                      double* __restrict__ E, int nx, int ny, int nz, int nxp,
                                                      int64_t nxyp, int64_t nn) {
  ElemIdx I;
  if (!I.set(nx, ny, nz, nxp, nxyp)) return;
  double x[6][8];
#pragma unroll
  for (int cc = 0; cc < 6; ++cc)
#pragma unroll
    for (int a = 0; a < 8; ++a) x[cc][a] = __ldg(dx + cc * nn + I.n0 + I.off[a]);
  const double* k = K + (int64_t)I.ez * NBK * nxyp + (int64_t)I.ey * nxp + I.ex;
  double c[6][8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    double s[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) s[b] = __ldg(k + (int64_t)(a * 8 + b) * nxyp);
#pragma unroll
    for (int cc = 0; cc < 6; ++cc) {
      double acc = 0.0;
#pragma unroll
      for (int b = 0; b < 8; ++b) acc += s[b] * x[cc][b];
      c[cc][a] = acc;
    }
  }
#pragma unroll 1
  for (int q = 0; q < 8; ++q) {
    QW<double> w;
    w.set(q);
    const double* kq = k + (int64_t)(64 + 17 * q) * nxyp;
    double dB[6];
#pragma unroll
    for (int cc = 0; cc < 6; ++cc) dB[cc] = interp_v(x[cc], w);
    double L[3][3];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk)
#pragma unroll
      for (int mm = 0; mm < 3; ++mm) L[kk][mm] = __ldg(kq + (int64_t)(8 + 3 * kk + mm) * nxyp);
    double st[6];
#pragma unroll
    for (int cc = 0; cc < 6; ++cc) {
      const int kk = sym_k(cc), l = sym_l(cc);
      double t = 0.0;
#pragma unroll
      for (int mm = 0; mm < 3; ++mm) t += L[kk][mm] * dB[sym_idx(mm, l)] + dB[sym_idx(kk, mm)] * L[l][mm];
      st[cc] = t;
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const double ta = __ldg(kq + (int64_t)a * nxyp);
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) c[cc][a] -= ta * st[cc];
    }
  }
#pragma unroll
  for (int cc = 0; cc < 6; ++cc)
#pragma unroll
    for (int a = 0; a < 8; ++a) E[(8 * cc + a) * I.es + I.e] = c[cc][a];
}

template <int NC>
__global__ void __launch_bounds__(128) em_node_kernel(const double* __restrict__ E, int nx, int ny, int nz, int nxp,
                                                      int64_t nxyp, int64_t nn, double* __restrict__ y) {
  int i;
  const int64_t jk = row_index(nx + 1, &i);
  if (i > nx || jk >= (int64_t)(ny + 1) * (nz + 1)) return;
  const int j = (int)(jk % (ny + 1)), k = (int)(jk / (ny + 1));
  const int64_t n = i + (int64_t)(nx + 1) * (j + (int64_t)(ny + 1) * k);
  const int64_t es = (int64_t)nz * nxyp;
  double s[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) s[c] = 0.0;
  for (int az = 1; az >= 0; --az) {
    const int ez = k - az;
    if (ez < 0 || ez >= nz) continue;
    for (int ay = 1; ay >= 0; --ay) {
      const int ey = j - ay;
      if (ey < 0 || ey >= ny) continue;
      for (int ax = 1; ax >= 0; --ax) {
        const int ex = i - ax;
        if (ex < 0 || ex >= nx) continue;
        const int64_t e = (int64_t)ez * nxyp + (int64_t)ey * nxp + ex;
        const int a = ax + 2 * ay + 4 * az;
#pragma unroll
        for (int c = 0; c < NC; ++c) s[c] += E[(8 * c + a) * es + e];
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) y[c * nn + n] = s[c];
}

// E[slots][nz * nxyp] scratch of the element-centric products (NS, AC and B in turn)
int ensure_elem_scratch(fsi_mesh* m, int slots, int64_t nxyp) {
  const int64_t elen = (int64_t)slots * m->g.nz * nxyp;
  if (m->ke_e_len < elen) {
    cudaFree(m->ke_e);
    m->ke_e = nullptr;
    m->ke_e_len = 0;
    FSI_CUDA(cudaMalloc(&m->ke_e, sizeof(double) * (size_t)elen));
    m->ke_e_len = elen;
  }
  return FSI_OK;
}

int launch_ace(fsi_mesh* m, int phase, const double* dx, double* y) {
  const int nxp = cq_pitch(m);
  const int64_t nxyp = (int64_t)nxp * m->g.ny;
  const int64_t nn = m->nn;
  if (!m->ake_built) {
    const int64_t len = (int64_t)m->g.nz * 64 * nxyp;
    if (m->ake_len < len) {
      cudaFree(m->ake64);
      m->ake64 = nullptr;
      m->ake_len = 0;
      FSI_CUDA(cudaMalloc(&m->ake64, sizeof(double) * (size_t)len));
      m->ake_len = len;
    }
    ACEBuildOp b;
    memset(&b, 0, sizeof(b));
    const double* xa = m->staged_xa;
    for (int k = 0; k < 3; ++k) put<double>(b.F, k, xa + k * nn);
    put<double>(b.F, 3, xa + (4 + phase) * nn);
    b.nf = 4;
    b.P = m->P;
    fill_common(m, b.rh, &b.W);
    b.gamma = m->gamma[phase];
    b.beta = m->beta[phase];
    b.K = m->ake64;
    b.nxp = nxp;
    b.nxyp = nxyp;
    if (int rc = run_tile(m, b, P_NS_BUILD)) return rc;
    m->ake_built = 1;
  }
  if (int rc = ensure_elem_scratch(m, 8, nxyp)) return rc;
  const Geom& g = m->g;
  const int64_t ne = (int64_t)g.nx * g.ny * g.nz;
  prof_bytes(m, P_AC_JVP64, (double)ne * (64 * 8.0 + 8 * 8.0) + (double)nn * 8.0);
  prof_bytes(m, P_NODE_SUM, (double)ne * 8 * 8.0 + (double)nn * 8.0);
  const RowLaunch el = elem_launch(g), nl = node_launch(g);
  FSI_LAUNCH(m, P_AC_JVP64,
             ace_elem_kernel<<<el.grid, el.block, 0, m->stream>>>(m->ake64, dx, m->ke_e, g.nx, g.ny, g.nz, nxp, nxyp));
  FSI_LAUNCH(m, P_NODE_SUM,
             em_node_kernel<1><<<nl.grid, nl.block, 0, m->stream>>>(m->ke_e, g.nx, g.ny, g.nz, nxp, nxyp, nn, y));
  return FSI_OK;
}

// Product with element matrices, element-centric: one thread per element (x fastest)
// gathers its 32 increment values, applies its matrix and writes the 32 products into
// E[i][element] (each element evaluated once: no halo recomputation); ns_node_kernel then
// sums, per node, the slots of its up to 8 elements in a fixed order (z, y, x) and applies
// the Dirichlet rows (deterministic, no atomics).
__global__ void __launch_bounds__(128) nse_elem_kernel(const double* __restrict__ K, const double* __restrict__ dx,
                                                       double* __restrict__ E, int nx, int ny, int nz, int nxp,
                                                       int64_t nxyp, int64_t nn) {
  int ex;
  const int64_t eyz = row_index(nx, &ex);
  if (ex >= nx || eyz >= (int64_t)ny * nz) return;
  const int ey = (int)(eyz % ny), ez = (int)(eyz / ny);
  const int64_t sx = 1, sy = nx + 1, sz = (int64_t)(nx + 1) * (ny + 1);
  const int64_t n0 = ex + sy * ey + sz * ez;
  const int64_t off[8] = {0, sx, sy, sx + sy, sz, sz + sx, sz + sy, sz + sx + sy};
  double x[32];
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int a = 0; a < 8; ++a) x[8 * f + a] = __ldg(dx + f * nn + n0 + off[a]);
  const int64_t e = (int64_t)ez * nxyp + (int64_t)ey * nxp + ex;
  const double* k = K + (int64_t)ez * NKE * nxyp + (int64_t)ey * nxp + ex;
  const int64_t es = (int64_t)nz * nxyp;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const double* row = k + (int64_t)i * 32 * nxyp;
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < 32; ++j) acc += __ldg(row + j * nxyp) * x[j];
    E[i * es + e] = acc;
  }
}

int launch_be(fsi_mesh* m, int solid, const double* dx, double* y) {
  const int nxp = cq_pitch(m);
  const int64_t nxyp = (int64_t)nxp * m->g.ny;
  const int64_t nn = m->nn;
  if (!m->bke_built) {
    const int64_t len = (int64_t)m->g.nz * NBK * nxyp;
    if (m->bke_len < len) {
      cudaFree(m->bke64);
      m->bke64 = nullptr;
      m->bke_len = 0;
      FSI_CUDA(cudaMalloc(&m->bke64, sizeof(double) * (size_t)len));
      m->bke_len = len;
    }
    BEBuildOp b;
    memset(&b, 0, sizeof(b));
    const double* xa = m->staged_xa;
    for (int k = 0; k < 3; ++k) put<double>(b.F, k, xa + k * nn);
    put<double>(b.F, 3, m->mat + (2 + solid) * nn);
    b.nf = 4;
    b.P = m->P;
    fill_common(m, b.rh, &b.W);
    b.K = m->bke64;
    b.nxp = nxp;
    b.nxyp = nxyp;
    if (int rc = run_tile(m, b, P_NS_BUILD)) return rc;
    m->bke_built = 1;
  }
  if (int rc = ensure_elem_scratch(m, 48, nxyp)) return rc;
  const Geom& g = m->g;
  const int64_t ne = (int64_t)g.nx * g.ny * g.nz;
  prof_bytes(m, P_B_JVP64, (double)ne * (NBK * 8.0 + 48 * 8.0) + (double)nn * 48.0);
  prof_bytes(m, P_NODE_SUM, (double)ne * 48 * 8.0 + (double)nn * 48.0);
  const RowLaunch el = elem_launch(g), nl = node_launch(g);
  FSI_LAUNCH(m, P_B_JVP64,
             be_elem_kernel<<<el.grid, el.block, 0, m->stream>>>(m->bke64, dx, m->ke_e, g.nx, g.ny, g.nz, nxp, nxyp,
                                                                nn));
  FSI_LAUNCH(m, P_NODE_SUM,
             em_node_kernel<6><<<nl.grid, nl.block, 0, m->stream>>>(m->ke_e, g.nx, g.ny, g.nz, nxp, nxyp, nn, y));
  return FSI_OK;
}

int launch_nse(fsi_mesh* m, const double* dx, double* y, unsigned flags) {
  const int nxp = cq_pitch(m);
  const int64_t nxyp = (int64_t)nxp * m->g.ny;
  const int elastic = ((flags & FSI_ELASTIC_AUG) && m->ns > 0) ? 1 : 0;
  if (m->ke_gen != m->cq_builds) {
    const int64_t len = (int64_t)m->g.nz * NKE * nxyp;
    if (m->ke_len < len) {
      cudaFree(m->ke64);
      m->ke64 = nullptr;
      m->ke_len = 0;
      FSI_CUDA(cudaMalloc(&m->ke64, sizeof(double) * (size_t)len));
      m->ke_len = len;
    }
    const dim3 grid((m->g.nx + 31) / 32, (unsigned)((int64_t)m->g.ny * m->g.nz), 4);
    FSI_LAUNCH(m, P_NS_BUILD,
               nse_build_kernel<<<grid, dim3(32, 8), 0, m->stream>>>(m->cq64, m->ke64, m->g.nx, m->g.ny, m->g.nz, nxp,
                                                                     nxyp, elastic, m->P.alpha, m->P.c_mass,
                                                                     1.0 / m->g.hx, 1.0 / m->g.hy, 1.0 / m->g.hz));
    m->ke_gen = m->cq_builds;
  }
  const int64_t nn = m->nn;
  if (int rc = ensure_elem_scratch(m, 32, nxyp)) return rc;
  const Geom& g = m->g;
  const int64_t ne = (int64_t)g.nx * g.ny * g.nz;
  // algorithmic bytes: the element kernel reads the matrices once and the increment once per
  // node and writes the 32 element products; the node kernel reads those back and writes
  // the product and reads the mask once per node
  prof_bytes(m, P_NS_JVP64E, (double)ne * (NKE * 8.0 + 32 * 8.0) + (double)nn * 32.0);
  prof_bytes(m, P_NODE_SUM, (double)ne * 32 * 8.0 + (double)nn * (32.0 + 1.0));
  const RowLaunch el = elem_launch(g), nl = node_launch(g);
  FSI_LAUNCH(m, P_NS_JVP64E,
             nse_elem_kernel<<<el.grid, el.block, 0, m->stream>>>(
                 m->ke64, dx, m->ke_e, g.nx, g.ny, g.nz, nxp, nxyp, nn));
  FSI_LAUNCH(m, P_NODE_SUM,
             ns_node_kernel<double><<<nl.grid, nl.block, 0, m->stream>>>(m->ke_e, g.nx, g.ny, g.nz, nxp, nxyp, nn,
                                                                         g.hx * g.hy * g.hz / 8.0, m->mask,
                                                                         m->pin_active, dx, nullptr, y));
  return FSI_OK;
}
template int launch_ac<double>(fsi_mesh*, int, int, const double*, double*);
template int launch_b<double>(fsi_mesh*, int, int, const double*, double*);

// Sums the per-CTA partials {sum val^2, n_band, int F', int sqrt F} in a fixed order.
__global__ void coef_finalize(const double* partials, int64_t n, double eta, double* out) {
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
    out[0] = t[1] > 0.0 ? sqrt(t[0] / t[1]) / eta : 0.0;  // gamma
    out[1] = t[3] != 0.0 ? t[2] / t[3] : 0.0;             // beta
  }
}

int op_coeffs(fsi_mesh* m, int i, double* gb) {
  static_assert(CoefOp::MINB == 1, "the partial sums are sized for the mesh's own tile grid");
  if (m->tet) return tet_coeffs(m, i, gb);
  CoefOp op;
  memset(&op, 0, sizeof(op));
  const int64_t nn = m->nn;
  for (int k = 0; k < 3; ++k) { op.F.d[k] = m->staged_xa + k * nn; op.F.f[k] = nullptr; }
  op.F.d[3] = m->staged_xa + (4 + i) * nn;
  op.nf = 4;
  fill_common(m, op.rh, &op.W);
  op.phi_node = m->staged_xa + (4 + i) * nn;
  dim3 grid;
  tile_grid(m, &grid);
  op.ncta_xy[0] = grid.x;
  op.ncta_xy[1] = grid.y;
  const int64_t ncta = (int64_t)grid.x * grid.y * grid.z;
  if (m->n_partials < ncta) {
    if (m->partials) cudaFree(m->partials);
    m->partials = nullptr;
    FSI_CUDA(cudaMalloc(&m->partials, sizeof(double) * 4 * ncta));
    m->n_partials = ncta;
  }
  op.partials = m->partials;
  int rc = run_tile(m, op, P_COEF);
  if (rc) return rc;
  FSI_LAUNCH(m, P_COEF, coef_finalize<<<1, NTHREADS, 0, m->stream>>>(m->partials, ncta, m->P.eta, m->red));
  FSI_CUDA(cudaMemcpyAsync(m->red_host, m->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  FSI_CUDA(cudaStreamSynchronize(m->stream));
  gb[0] = m->red_host[0];
  gb[1] = m->red_host[1];
  return FSI_OK;
}

}  // namespace fsi
