// Linear (P1) tetrahedral meshes: the paper's element for its falling-sphere and
// ship-ice meshes (Sections 5.3 and 6).  The momentum/continuity residual, Jacobian-
// vector product and Jacobi diagonal of Eq. PG_NS evaluated element by element through
// the mesh connectivity.
//
// Node set, node numbering and boundary conditions are those of the description's box
// grid; coordinates and connectivity are the caller's (any conforming tetrahedral mesh of
// those nodes).  Quadrature: the symmetric 4-point rule (barycentric points
// (a, b, b, b) and permutations, weights |T|/4), exact for quadratics.  Stabilisation
// metric per element: G = sum_k grad(xi_k) grad(xi_k)^T over the reference coordinates.
//
// Assembly is atomics-free and deterministic: the element kernel writes each element's
// 4 corners x 4 equations into E (one slot per element and corner), and the node kernel
// sums, for every node, the slots of its elements in increasing element order (a CSR
// list built once at creation), then applies the Dirichlet rows.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace fsi {

struct TetData {
  int64_t ne = 0;
  int32_t* conn = nullptr;  // [4][ne] node of corner a of element e at conn[a * ne + e]
  double* geo = nullptr;    // [TG][ne]: grad lambda_a (12, a-major), quadrature weight |T|/4, G (6 sym)
  int64_t* nptr = nullptr;  // [nn + 1]
  int32_t* nlist = nullptr; // 4 e + a of every (element, corner) at a node, by element
  double* E = nullptr;      // [24][ne] element contributions, slot (a * ncomp + eq)
  // float64 NS element matrices [256][ne], row a * 4 + eq, column b * 4 + f, built once a
  // solve has taken NSE_AFTER products on one staging (k_stage) with one elastic flag
  double* K = nullptr;
  int64_t k_stage = -1;
  int k_elastic = -1, k_count = 0, k_built = 0;
};

constexpr int TG = 19;
#define FSI_TA 0.58541019662496845446  // (5 + 3 sqrt5) / 20
#define FSI_TB 0.13819660112501051518  // (5 - sqrt5) / 20

void tet_free(TetData* t) {
  if (!t) return;
  cudaFree(t->conn);
  cudaFree(t->geo);
  cudaFree(t->nptr);
  cudaFree(t->nlist);
  cudaFree(t->E);
  cudaFree(t->K);
  delete t;
}

struct TetArgs {
  const int32_t* conn;
  const double* geo;
  int64_t ne;
  const double* xa;   // x^{n+alpha} (pressure plane: p^{n+1})
  const double* xd;   // dx/dt^{n+alpha_m}
  const double* mat;  // rho, mu, alpha^s
  const double* dx;   // JVP increment (dv, dp) [4][nn]
  double* E;
  int64_t nn;
  int elastic;
  Phys P;
};

// nodal values of field f at the 4 corners
__device__ __forceinline__ void tet_gather(const double* f, const int (&nd)[4], double (&u)[4]) {
#pragma unroll
  for (int a = 0; a < 4; ++a) u[a] = f[nd[a]];
}
__device__ __forceinline__ double tet_val(const double (&u)[4], int q) {
  const double wa = FSI_TA, wb = FSI_TB;
  double s = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a) s += (a == q ? wa : wb) * u[a];
  return s;
}
__device__ __forceinline__ void tet_grad(const double (&u)[4], const double (&dN)[4][3], double (&g)[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) g[d] = dN[0][d] * u[0] + dN[1][d] * u[1] + dN[2][d] * u[2] + dN[3][d] * u[3];
}

// The 44 frozen coefficients of the product at quadrature point q of one element
// (the layout of NSBuildOp: rho, mu, v, grad v, R_m, tau_m, tau_c rho, tau_m / rho,
// sum a_s B^s, sum a_s grad B^s), and for the residual the elastic stress sum.
struct TetPoint {
  double k[NCQ];
  double p;        // p^{n+1}
  double acc[3];   // dv/dt + v.grad v
  double E[6];     // sum_s alpha^s mu_L^s (B^s - I)
};

__device__ void tet_point(const TetArgs& A, const int (&nd)[4], const double (&dN)[4][3], const double (&G)[6], int q,
                          bool with_elastic, TetPoint& o) {
  const Phys& P = A.P;
  const int64_t nn = A.nn;
  double u[4], gr[3];
  double v[3], L[3][3];
  for (int kk = 0; kk < 3; ++kk) {
    tet_gather(A.xa + kk * nn, nd, u);
    v[kk] = tet_val(u, q);
    tet_grad(u, dN, gr);
    L[kk][0] = gr[0]; L[kk][1] = gr[1]; L[kk][2] = gr[2];
  }
  tet_gather(A.mat, nd, u);
  const double rho = tet_val(u, q);
  tet_gather(A.mat + nn, nd, u);
  const double mu = tet_val(u, q);
  tet_gather(A.xa + 3 * nn, nd, u);
  o.p = tet_val(u, q);
  double gp[3];
  tet_grad(u, dN, gp);
  double Rm[3];
  for (int kk = 0; kk < 3; ++kk) {
    tet_gather(A.xd + kk * nn, nd, u);
    o.acc[kk] = tet_val(u, q) + v[0] * L[kk][0] + v[1] * L[kk][1] + v[2] * L[kk][2];
    Rm[kk] = rho * o.acc[kk] + gp[kk] - rho * P.grav[kk];
  }
  // v.G v, G:G and tr G with the element's full metric
  const double Gm[3][3] = {{G[0], G[3], G[5]}, {G[3], G[1], G[4]}, {G[5], G[4], G[2]}};
  double vGv = 0.0, GG = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      vGv += v[i] * Gm[i][j] * v[j];
      GG += Gm[i][j] * Gm[i][j];
    }
  const double trG = G[0] + G[1] + G[2];
  const double nu = mu / rho;
  const double tau_m = 1.0 / sqrt(4.0 / (P.dt * P.dt) + vGv + P.c_i * nu * nu * GG);
  const double tau_c = 1.0 / (trG * tau_m);
  o.k[0] = rho;
  o.k[1] = mu;
  for (int kk = 0; kk < 3; ++kk) o.k[2 + kk] = v[kk];
  for (int kk = 0; kk < 3; ++kk)
    for (int j = 0; j < 3; ++j) o.k[5 + 3 * kk + j] = L[kk][j];
  for (int kk = 0; kk < 3; ++kk) o.k[14 + kk] = Rm[kk];
  o.k[17] = tau_m;
  o.k[18] = tau_c * rho;
  o.k[19] = tau_m / rho;
  for (int c = 0; c < 24; ++c) o.k[20 + c] = 0.0;
  for (int c = 0; c < 6; ++c) o.E[c] = 0.0;
  for (int s = 0; s < P.ns; ++s) {
    tet_gather(A.mat + (2 + s) * nn, nd, u);
    const double al = tet_val(u, q);
    const double muL = P.muL[P.solid_phase[s]];
    const double a = al * muL * P.c_el;
    const int c0 = 4 + P.N + 6 * s;
    for (int c = 0; c < 6; ++c) {
      tet_gather(A.xa + (int64_t)(c0 + c) * nn, nd, u);
      const double B = tet_val(u, q);
      o.E[c] += al * muL * (B - (c < 3 ? 1.0 : 0.0));
      if (with_elastic) {
        tet_grad(u, dN, gr);
        o.k[20 + c] += a * B;
        for (int d = 0; d < 3; ++d) o.k[26 + 3 * c + d] += a * gr[d];
      }
    }
  }
}

struct LocalCoef {
  const double* k;
  __device__ __forceinline__ double operator()(int i) const { return k[i]; }
};

__device__ __forceinline__ void tet_load_geo(const int32_t* conn, const double* geo, int64_t ne, int64_t e,
                                             int (&nd)[4], double (&dN)[4][3], double& w, double (&G)[6]) {
  for (int a = 0; a < 4; ++a) nd[a] = conn[a * ne + e];
  for (int a = 0; a < 4; ++a)
    for (int d = 0; d < 3; ++d) dN[a][d] = geo[(3 * a + d) * ne + e];
  w = geo[12 * ne + e];
  for (int c = 0; c < 6; ++c) G[c] = geo[(13 + c) * ne + e];
}

// MODE 0 residual, 1 product, 2 diagonal of the product: element contributions into E
template <int MODE>
__global__ void __launch_bounds__(128) tet_ns_elem(const TetArgs A) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= A.ne) return;
  int nd[4];
  double dN[4][3], w, G[6];
  tet_load_geo(A.conn, A.geo, A.ne, e, nd, dN, w, G);
  double c[4][4];  // [corner][equation]
  for (int a = 0; a < 4; ++a)
    for (int q = 0; q < 4; ++q) c[a][q] = 0.0;
  // the increment at the corners (product) and its constant gradient
  double du[4][4], dg[4][3];
  if (MODE == 1) {
    for (int f = 0; f < 4; ++f) {
      double u[4];
      tet_gather(A.dx + f * A.nn, nd, u);
      for (int a = 0; a < 4; ++a) du[f][a] = u[a];
      tet_grad(u, dN, dg[f]);
    }
  }
  for (int q = 0; q < 4; ++q) {
    TetPoint pt;
    tet_point(A, nd, dN, G, q, MODE != 0 && A.elastic, pt);
    double Nq[4];
    for (int a = 0; a < 4; ++a) Nq[a] = a == q ? FSI_TA : FSI_TB;
    if (MODE == 0) {
      const double* k = pt.k;
      const double rho = k[0], mu = k[1], tau_m = k[17], tc_rho = k[18], tm_rho = k[19];
      const double Rc = k[5] + k[9] + k[13];
      double f[4], g[4][3];
      for (int kk = 0; kk < 3; ++kk) {
        for (int j = 0; j < 3; ++j) {
          double s = pt.E[sym_idx(kk, j)] + mu * (k[5 + 3 * kk + j] + k[5 + 3 * j + kk]) + tau_m * k[2 + j] * k[14 + kk];
          if (j == kk) s += -pt.p + tc_rho * Rc;
          g[kk][j] = s;
        }
        f[kk] = rho * (pt.acc[kk] - A.P.grav[kk]);
      }
      f[3] = Rc;
      for (int j = 0; j < 3; ++j) g[3][j] = tm_rho * k[14 + j];
      for (int a = 0; a < 4; ++a)
        for (int eq = 0; eq < 4; ++eq)
          c[a][eq] += w * (Nq[a] * f[eq] + dN[a][0] * g[eq][0] + dN[a][1] * g[eq][1] + dN[a][2] * g[eq][2]);
    } else if (MODE == 1) {
      double dv[3], gd[3][3], dgp[3];
      for (int kk = 0; kk < 3; ++kk) {
        dv[kk] = Nq[0] * du[kk][0] + Nq[1] * du[kk][1] + Nq[2] * du[kk][2] + Nq[3] * du[kk][3];
        for (int d = 0; d < 3; ++d) gd[kk][d] = dg[kk][d];
        dgp[kk] = dg[3][kk];
      }
      const double dp = Nq[0] * du[3][0] + Nq[1] * du[3][1] + Nq[2] * du[3][2] + Nq[3] * du[3][3];
      double f[4], g[4][3];
      nsq_point_fg<double>(LocalCoef{pt.k}, A.elastic != 0, dv, gd, dp, dgp, A.P.alpha, A.P.c_mass, f, g);
      for (int a = 0; a < 4; ++a)
        for (int eq = 0; eq < 4; ++eq)
          c[a][eq] += w * (Nq[a] * f[eq] + dN[a][0] * g[eq][0] + dN[a][1] * g[eq][1] + dN[a][2] * g[eq][2]);
    } else {
      // diagonal: trial = test = (corner a, equation eq)
      for (int a = 0; a < 4; ++a)
        for (int fq = 0; fq < 4; ++fq) {
          double dv[3] = {0.0, 0.0, 0.0}, gd[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
          double dgp[3] = {0.0, 0.0, 0.0}, dp = 0.0;
          if (fq < 3) {
            dv[fq] = Nq[a];
            for (int d = 0; d < 3; ++d) gd[fq][d] = dN[a][d];
          } else {
            dp = Nq[a];
            for (int d = 0; d < 3; ++d) dgp[d] = dN[a][d];
          }
          double f[4], g[4][3];
          nsq_point_fg<double>(LocalCoef{pt.k}, A.elastic != 0, dv, gd, dp, dgp, A.P.alpha, A.P.c_mass, f, g);
          c[a][fq] += w * (Nq[a] * f[fq] + dN[a][0] * g[fq][0] + dN[a][1] * g[fq][1] + dN[a][2] * g[fq][2]);
        }
    }
  }
  for (int a = 0; a < 4; ++a)
    for (int eq = 0; eq < 4; ++eq) A.E[(int64_t)(a * 4 + eq) * A.ne + e] = c[a][eq];
}

// node sums in element order, then the Dirichlet rows (as the hexahedral operators)
template <int MODE>
__global__ void __launch_bounds__(256) tet_ns_node(const int64_t* __restrict__ nptr, const int32_t* __restrict__ nlist,
                                                   const double* __restrict__ E, int64_t ne, int64_t nn,
                                                   const uint8_t* mask, int pin, const double* x, const double* vD,
                                                   const double* dx, double* y) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= nn) return;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = nptr[n]; i < nptr[n + 1]; ++i) {
    const int32_t t = nlist[i];
    const int64_t e = t >> 2;
    const int a = t & 3;
    for (int eq = 0; eq < 4; ++eq) s[eq] += E[(int64_t)(a * 4 + eq) * ne + e];
  }
  const uint8_t m = mask[n];
  for (int k = 0; k < 4; ++k) {
    double v = s[k];
    if (((m >> k) & 1) && (k < 3 || pin)) {
      if (MODE == 0) v = x[(int64_t)k * nn + n] - (k < 3 ? vD[(int64_t)k * nn + n] : 0.0);
      else if (MODE == 1) v = dx[(int64_t)k * nn + n];
      else v = 1.0;
    }
    y[(int64_t)k * nn + n] = v;
  }
}

template <int MODE>
int tet_ns_run(fsi_mesh* m, const double* dx, double* y, unsigned flags) {
  TetData* t = m->tet;
  TetArgs A;
  A.conn = t->conn;
  A.geo = t->geo;
  A.ne = t->ne;
  A.xa = m->staged_xa;
  A.xd = m->xd;
  A.mat = m->mat;
  A.dx = dx;
  A.E = t->E;
  A.nn = m->nn;
  A.elastic = (MODE == 0) ? 0 : ((flags & FSI_ELASTIC_AUG) && m->ns > 0 ? 1 : 0);
  A.P = m->P;
  const int cls = MODE == 0 ? P_NS_RES : (MODE == 1 ? P_NS_JVP64 : P_NS_DIAG);
  FSI_LAUNCH(m, cls, tet_ns_elem<MODE><<<(unsigned)((t->ne + 127) / 128), 128, 0, m->stream>>>(A));
  FSI_LAUNCH(m, cls, tet_ns_node<MODE><<<(unsigned)((m->nn + 255) / 256), 256, 0, m->stream>>>(
                         t->nptr, t->nlist, t->E, t->ne, m->nn, m->mask, m->pin_active, m->staged_x, m->vD, dx, y));
  return FSI_OK;
}

// NS element matrices: one thread per element; per quadrature point the coefficients once,
// then the product's point arithmetic for each of the 16 unit increments (field f at corner
// b), added into column b * 4 + f of the element's matrix (the first point writes).  Same
// operator as tet_ns_elem<1> up to the order of the sums.
__global__ void __launch_bounds__(128) tet_nsk_build(const TetArgs A, double* __restrict__ K) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= A.ne) return;
  int nd[4];
  double dN[4][3], w, G[6];
  tet_load_geo(A.conn, A.geo, A.ne, e, nd, dN, w, G);
  for (int q = 0; q < 4; ++q) {
    TetPoint pt;
    tet_point(A, nd, dN, G, q, A.elastic, pt);
    double Nq[4];
    for (int a = 0; a < 4; ++a) Nq[a] = a == q ? FSI_TA : FSI_TB;
    for (int col = 0; col < 16; ++col) {
      const int b = col >> 2, f = col & 3;
      double dv[3], gd[3][3], dgp[3];
      for (int kk = 0; kk < 3; ++kk) {
        dv[kk] = kk == f ? Nq[b] : 0.0;
        for (int d = 0; d < 3; ++d) gd[kk][d] = kk == f ? dN[b][d] : 0.0;
        dgp[kk] = f == 3 ? dN[b][kk] : 0.0;
      }
      const double dp = f == 3 ? Nq[b] : 0.0;
      double fo[4], go[4][3];
      nsq_point_fg<double>(LocalCoef{pt.k}, A.elastic != 0, dv, gd, dp, dgp, A.P.alpha, A.P.c_mass, fo, go);
      for (int a = 0; a < 4; ++a)
        for (int eq = 0; eq < 4; ++eq) {
          const double v = w * (Nq[a] * fo[eq] + dN[a][0] * go[eq][0] + dN[a][1] * go[eq][1] + dN[a][2] * go[eq][2]);
          double* kp = K + (int64_t)((a * 4 + eq) * 16 + col) * A.ne + e;
          *kp = q == 0 ? v : *kp + v;
        }
    }
  }
}

// product through the element matrices: E slot a * 4 + eq = row of K times the element's
// increment values (column b * 4 + f = field f at corner b)
__global__ void __launch_bounds__(128) tet_nsk_apply(const int32_t* __restrict__ conn, const double* __restrict__ K,
                                                     const double* __restrict__ dx, double* __restrict__ E, int64_t ne,
                                                     int64_t nn) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= ne) return;
  double u[16];
  for (int b = 0; b < 4; ++b) {
    const int64_t node = conn[(int64_t)b * ne + e];
    for (int f = 0; f < 4; ++f) u[b * 4 + f] = __ldg(dx + (int64_t)f * nn + node);
  }
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    double acc = 0.0;
#pragma unroll
    for (int c = 0; c < 16; ++c) acc += __ldg(K + (int64_t)(r * 16 + c) * ne + e) * u[c];
    E[(int64_t)r * ne + e] = acc;
  }
}

int tet_ns(fsi_mesh* m, int mode, const double* dx, double* y, unsigned flags) {
  if (flags & FSI_FP32) return set_error(FSI_EINVAL, "tetrahedral meshes: float64 operators only");
  if (mode == 1 && !m->rec) {
    // a float64 solve on one staging: after NSE_AFTER products switch to element matrices
    TetData* t = m->tet;
    const int elastic = ((flags & FSI_ELASTIC_AUG) && m->ns > 0) ? 1 : 0;
    if (t->k_stage != m->stage_gen || t->k_elastic != elastic) {
      t->k_stage = m->stage_gen;
      t->k_elastic = elastic;
      t->k_count = 0;
      t->k_built = 0;
    }
    if (++t->k_count > NSE_AFTER) {
      const unsigned grid = (unsigned)((t->ne + 127) / 128);
      if (!t->k_built) {
        if (!t->K) FSI_CUDA(cudaMalloc(&t->K, sizeof(double) * 256 * (size_t)t->ne));
        TetArgs A;
        A.conn = t->conn;
        A.geo = t->geo;
        A.ne = t->ne;
        A.xa = m->staged_xa;
        A.xd = m->xd;
        A.mat = m->mat;
        A.dx = nullptr;
        A.E = t->E;
        A.nn = m->nn;
        A.elastic = elastic;
        A.P = m->P;
        FSI_LAUNCH(m, P_NS_BUILD, tet_nsk_build<<<grid, 128, 0, m->stream>>>(A, t->K));
        t->k_built = 1;
      }
      prof_bytes(m, P_NS_JVP64E, (double)t->ne * (256 * 8.0 + 16 * 4.0 + 16 * 8.0) + (double)m->nn * 32.0);
      FSI_LAUNCH(m, P_NS_JVP64E, tet_nsk_apply<<<grid, 128, 0, m->stream>>>(t->conn, t->K, dx, t->E, t->ne, m->nn));
      FSI_LAUNCH(m, P_NODE_SUM, tet_ns_node<1><<<(unsigned)((m->nn + 255) / 256), 256, 0, m->stream>>>(
                                    t->nptr, t->nlist, t->E, t->ne, m->nn, m->mask, m->pin_active, m->staged_x, m->vD,
                                    dx, y));
      return FSI_OK;
    }
  }
  if (mode == 0) return tet_ns_run<0>(m, dx, y, flags);
  if (mode == 1) return tet_ns_run<1>(m, dx, y, flags);
  return tet_ns_run<2>(m, dx, y, flags);
}

// ------------------------------------------------ Allen-Cahn, B and gamma/beta on tetrahedra
// The same weak forms as the hexahedral ACOp, BOp and CoefOp (Eq. PPV_AC, Eq. semiCGT,
// Sections 2.2.1-2.2.2), with the tetrahedral interpolation, the element's metric G and
// the 4-point rule; element kernels write their corner contributions, tet_node_sum adds
// them per node in element order.

struct TetACArgs {
  const int32_t* conn;
  const double* geo;
  int64_t ne, nn;
  const double* xa;
  const double* xd;
  const double* dx;
  double* E;
  int phase;
  double gamma, beta;
  Phys P;
};

__device__ __forceinline__ double tet_vGv(const double (&v)[3], const double (&G)[6], double* GG) {
  const double Gm[3][3] = {{G[0], G[3], G[5]}, {G[3], G[1], G[4]}, {G[5], G[4], G[2]}};
  double s = 0.0, g2 = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      s += v[i] * Gm[i][j] * v[j];
      g2 += Gm[i][j] * Gm[i][j];
    }
  if (GG) *GG = g2;
  return s;
}

template <int MODE>
__global__ void __launch_bounds__(128) tet_ac_elem(const TetACArgs A) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= A.ne) return;
  int nd[4];
  double dN[4][3], w, G[6];
  tet_load_geo(A.conn, A.geo, A.ne, e, nd, dN, w, G);
  const Phys& P = A.P;
  const int64_t nn = A.nn;
  double uv[3][4], uphi[4], ud[4], gphi[3], gd[3];
  for (int k = 0; k < 3; ++k) tet_gather(A.xa + k * nn, nd, uv[k]);
  tet_gather(A.xa + (4 + A.phase) * nn, nd, uphi);
  tet_grad(uphi, dN, gphi);
  if (MODE == 0) tet_gather(A.xd + (4 + A.phase) * nn, nd, ud);
  if (MODE == 1) {
    tet_gather(A.dx, nd, ud);
    tet_grad(ud, dN, gd);
  }
  const double gam = A.gamma, bet = A.beta, alpha = P.alpha, cm = P.c_mass;
  const double k_hat = gam * P.eps * P.eps;
  double c[4] = {0.0, 0.0, 0.0, 0.0};
  for (int q = 0; q < 4; ++q) {
    double Nq[4];
    for (int a = 0; a < 4; ++a) Nq[a] = a == q ? FSI_TA : FSI_TB;
    double v[3];
    for (int k = 0; k < 3; ++k) v[k] = tet_val(uv[k], q);
    const double phi = tet_val(uphi, q);
    double GG;
    const double vGv = tet_vGv(v, G, &GG);
    const double s_hat = gam * (3.0 * phi * phi - 1.0);
    const double tau = 1.0 / sqrt(4.0 / (P.dt * P.dt) + vGv + 9.0 * k_hat * k_hat * GG + s_hat * s_hat);
    if (MODE == 0) {
      const double R = tet_val(ud, q) + v[0] * gphi[0] + v[1] * gphi[1] + v[2] * gphi[2] +
                       gam * (phi * phi * phi - phi - bet * 0.5 * fabs(phi * phi - 1.0));
      for (int a = 0; a < 4; ++a) {
        const double vgN = v[0] * dN[a][0] + v[1] * dN[a][1] + v[2] * dN[a][2];
        c[a] += w * (Nq[a] * R + k_hat * (dN[a][0] * gphi[0] + dN[a][1] * gphi[1] + dN[a][2] * gphi[2]) +
                     tau * vgN * R);
      }
    } else {
      const double p2 = phi * phi - 1.0;
      const double dsF = p2 > 0.0 ? phi : (p2 < 0.0 ? -phi : 0.0);
      const double rp = gam * (3.0 * phi * phi - 1.0 - bet * dsF);
      for (int a = 0; a < 4; ++a) {
        const double vgN = v[0] * dN[a][0] + v[1] * dN[a][1] + v[2] * dN[a][2];
        if (MODE == 1) {
          const double d = tet_val(ud, q);
          const double dR = cm * d + alpha * (v[0] * gd[0] + v[1] * gd[1] + v[2] * gd[2]) + alpha * rp * d;
          c[a] += w * (Nq[a] * dR + k_hat * alpha * (dN[a][0] * gd[0] + dN[a][1] * gd[1] + dN[a][2] * gd[2]) +
                       tau * vgN * dR);
        } else {  // diagonal: trial = test = corner a
          const double dR = cm * Nq[a] + alpha * vgN + alpha * rp * Nq[a];
          c[a] += w * (Nq[a] * dR + k_hat * alpha * (dN[a][0] * dN[a][0] + dN[a][1] * dN[a][1] + dN[a][2] * dN[a][2]) +
                       tau * vgN * dR);
        }
      }
    }
  }
  for (int a = 0; a < 4; ++a) A.E[(int64_t)a * A.ne + e] = c[a];
}

struct TetBArgs {
  const int32_t* conn;
  const double* geo;
  int64_t ne, nn;
  const double* xa;
  const double* xd;
  const double* mat;
  const double* dx;
  double* E;
  int solid;
  Phys P;
};

template <int MODE>
__global__ void __launch_bounds__(128) tet_b_elem(const TetBArgs A) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= A.ne) return;
  int nd[4];
  double dN[4][3], w, G[6];
  tet_load_geo(A.conn, A.geo, A.ne, e, nd, dN, w, G);
  const Phys& P = A.P;
  const int64_t nn = A.nn;
  double uv[3][4], L[3][3], ual[4];
  for (int k = 0; k < 3; ++k) {
    tet_gather(A.xa + k * nn, nd, uv[k]);
    tet_grad(uv[k], dN, L[k]);
  }
  tet_gather(A.mat + (2 + A.solid) * nn, nd, ual);
  const int c0 = 4 + P.N + 6 * A.solid;
  double ub[6][4], gb[6][3], udot[6][4];
  for (int cc = 0; cc < 6; ++cc) {
    if (MODE == 1) tet_gather(A.dx + cc * nn, nd, ub[cc]);
    else tet_gather(A.xa + (int64_t)(c0 + cc) * nn, nd, ub[cc]);
    tet_grad(ub[cc], dN, gb[cc]);
    if (MODE == 0) tet_gather(A.xd + (int64_t)(c0 + cc) * nn, nd, udot[cc]);
  }
  const double alpha = P.alpha, cm = P.c_mass;
  double c[4][6];
  for (int a = 0; a < 4; ++a)
    for (int cc = 0; cc < 6; ++cc) c[a][cc] = 0.0;
  for (int q = 0; q < 4; ++q) {
    double Nq[4];
    for (int a = 0; a < 4; ++a) Nq[a] = a == q ? FSI_TA : FSI_TB;
    double v[3];
    for (int k = 0; k < 3; ++k) v[k] = tet_val(uv[k], q);
    const double al = tet_val(ual, q);
    const double tau = 1.0 / sqrt(4.0 / (P.dt * P.dt) + tet_vGv(v, G, nullptr));
    if (MODE == 2) {
      for (int a = 0; a < 4; ++a) {
        const double vgN = v[0] * dN[a][0] + v[1] * dN[a][1] + v[2] * dN[a][2];
        for (int cc = 0; cc < 6; ++cc) {
          const int k = sym_k(cc), l = sym_l(cc);
          const double dR = al * (cm * Nq[a] + alpha * vgN - alpha * Nq[a] * (L[k][k] + L[l][l])) +
                            (1.0 - al) * alpha * Nq[a];
          c[a][cc] += w * (Nq[a] + tau * vgN) * dR;
        }
      }
      continue;
    }
    double B[6], cv[6];
    for (int cc = 0; cc < 6; ++cc) {
      const double sc = MODE == 1 ? alpha : 1.0;
      B[cc] = sc * tet_val(ub[cc], q);
      cv[cc] = sc * (v[0] * gb[cc][0] + v[1] * gb[cc][1] + v[2] * gb[cc][2]);
      if (MODE == 1) cv[cc] += cm * tet_val(ub[cc], q);
      else cv[cc] += tet_val(udot[cc], q);
    }
    for (int cc = 0; cc < 6; ++cc) {
      const int k = sym_k(cc), l = sym_l(cc);
      double st = 0.0;
      for (int m = 0; m < 3; ++m) st += L[k][m] * B[sym_idx(m, l)] + B[sym_idx(k, m)] * L[l][m];
      const double rec = B[cc] - ((MODE == 0 && cc < 3) ? 1.0 : 0.0);
      const double R = al * (cv[cc] - st) + (1.0 - al) * rec;
      for (int a = 0; a < 4; ++a) {
        const double vgN = v[0] * dN[a][0] + v[1] * dN[a][1] + v[2] * dN[a][2];
        c[a][cc] += w * (Nq[a] + tau * vgN) * R;
      }
    }
  }
  for (int a = 0; a < 4; ++a)
    for (int cc = 0; cc < 6; ++cc) A.E[(int64_t)(a * 6 + cc) * A.ne + e] = c[a][cc];
}

// node sums of NCOMP components (no Dirichlet rows: the Allen-Cahn and B blocks have none)
template <int NCOMP>
__global__ void __launch_bounds__(256) tet_node_sum(const int64_t* __restrict__ nptr, const int32_t* __restrict__ nlist,
                                                    const double* __restrict__ E, int64_t ne, int64_t nn, double* y) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= nn) return;
  double s[NCOMP];
  for (int k = 0; k < NCOMP; ++k) s[k] = 0.0;
  for (int64_t i = nptr[n]; i < nptr[n + 1]; ++i) {
    const int32_t t = nlist[i];
    const int64_t e = t >> 2;
    const int a = t & 3;
    for (int k = 0; k < NCOMP; ++k) s[k] += E[(int64_t)(a * NCOMP + k) * ne + e];
  }
  for (int k = 0; k < NCOMP; ++k) y[(int64_t)k * nn + n] = s[k];
}

int tet_ac(fsi_mesh* m, int mode, int phase, const double* dx, double* y, unsigned flags) {
  if (flags & FSI_FP32) return set_error(FSI_EINVAL, "tetrahedral meshes: float64 operators only");
  TetData* t = m->tet;
  TetACArgs A{t->conn, t->geo, t->ne, m->nn, m->staged_xa, m->xd, dx, t->E, phase, m->gamma[phase], m->beta[phase], m->P};
  const int cls = mode == 0 ? P_AC_RES : (mode == 1 ? P_AC_JVP64 : P_AC_DIAG);
  const unsigned ge = (unsigned)((t->ne + 127) / 128);
  if (mode == 0) FSI_LAUNCH(m, cls, tet_ac_elem<0><<<ge, 128, 0, m->stream>>>(A));
  else if (mode == 1) FSI_LAUNCH(m, cls, tet_ac_elem<1><<<ge, 128, 0, m->stream>>>(A));
  else FSI_LAUNCH(m, cls, tet_ac_elem<2><<<ge, 128, 0, m->stream>>>(A));
  FSI_LAUNCH(m, cls, tet_node_sum<1><<<(unsigned)((m->nn + 255) / 256), 256, 0, m->stream>>>(t->nptr, t->nlist, t->E,
                                                                                           t->ne, m->nn, y));
  return FSI_OK;
}

int tet_b(fsi_mesh* m, int mode, int solid, const double* dx, double* y, unsigned flags) {
  if (flags & FSI_FP32) return set_error(FSI_EINVAL, "tetrahedral meshes: float64 operators only");
  TetData* t = m->tet;
  TetBArgs A{t->conn, t->geo, t->ne, m->nn, m->staged_xa, m->xd, m->mat, dx, t->E, solid, m->P};
  const int cls = mode == 0 ? P_B_RES : (mode == 1 ? P_B_JVP64 : P_B_DIAG);
  const unsigned ge = (unsigned)((t->ne + 127) / 128);
  if (mode == 0) FSI_LAUNCH(m, cls, tet_b_elem<0><<<ge, 128, 0, m->stream>>>(A));
  else if (mode == 1) FSI_LAUNCH(m, cls, tet_b_elem<1><<<ge, 128, 0, m->stream>>>(A));
  else FSI_LAUNCH(m, cls, tet_b_elem<2><<<ge, 128, 0, m->stream>>>(A));
  FSI_LAUNCH(m, cls, tet_node_sum<6><<<(unsigned)((m->nn + 255) / 256), 256, 0, m->stream>>>(t->nptr, t->nlist, t->E,
                                                                                           t->ne, m->nn, y));
  return FSI_OK;
}

// gamma and beta of one phase (Section 2.2.2 mobility by lumped L2 projection, Section
// 2.2.1 multiplier): element slots 0-3 int N_a q, 4-7 int N_a, 8 int F', 9 int sqrt F
__global__ void __launch_bounds__(128) tet_coef_elem(const TetArgs A, int phase) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= A.ne) return;
  int nd[4];
  double dN[4][3], w, G[6];
  tet_load_geo(A.conn, A.geo, A.ne, e, nd, dN, w, G);
  double L[3][3], u[4], uphi[4], g[3];
  for (int k = 0; k < 3; ++k) {
    tet_gather(A.xa + k * A.nn, nd, u);
    tet_grad(u, dN, L[k]);
  }
  tet_gather(A.xa + (4 + phase) * A.nn, nd, uphi);
  tet_grad(uphi, dN, g);
  const double n2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
  double num = 0.0;
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < 3; ++k) num += g[j] * L[j][k] * g[k];
  const double qv = n2 < 1e-30 ? 0.0 : num / n2;  // constant on the element
  double sq[4] = {0.0, 0.0, 0.0, 0.0}, s1[4] = {0.0, 0.0, 0.0, 0.0}, sFp = 0.0, ssF = 0.0;
  for (int q = 0; q < 4; ++q) {
    const double phi = tet_val(uphi, q);
    for (int a = 0; a < 4; ++a) {
      const double N = a == q ? FSI_TA : FSI_TB;
      sq[a] += w * N * qv;
      s1[a] += w * N;
    }
    sFp += w * (phi * phi * phi - phi);
    ssF += w * 0.5 * fabs(phi * phi - 1.0);
  }
  for (int a = 0; a < 4; ++a) {
    A.E[(int64_t)a * A.ne + e] = sq[a];
    A.E[(int64_t)(4 + a) * A.ne + e] = s1[a];
  }
  A.E[(int64_t)8 * A.ne + e] = sFp;
  A.E[(int64_t)9 * A.ne + e] = ssF;
}

// per-CTA partial sums {sum val^2 over band nodes, band nodes, int F', int sqrt F} in a
// fixed partition and order
__global__ void __launch_bounds__(256) tet_coef_reduce(const int64_t* __restrict__ nptr, const int32_t* __restrict__ nlist,
                                                       const double* __restrict__ E, int64_t ne, int64_t nn,
                                                       const double* phi, double* partials) {
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < nn; n += stride) {
    if (fabs(phi[n]) > 0.9) continue;
    double num = 0.0, den = 0.0;
    for (int64_t i = nptr[n]; i < nptr[n + 1]; ++i) {
      const int64_t e = nlist[i] >> 2;
      const int c = nlist[i] & 3;
      num += E[(int64_t)c * ne + e];
      den += E[(int64_t)(4 + c) * ne + e];
    }
    const double val = fabs(num / den);
    a[0] += val * val;
    a[1] += 1.0;
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += stride) {
    a[2] += E[(int64_t)8 * ne + e];
    a[3] += E[(int64_t)9 * ne + e];
  }
  __shared__ double sm[4][256];
  for (int k = 0; k < 4; ++k) sm[k][threadIdx.x] = a[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < 256; ++i)
      for (int k = 0; k < 4; ++k) t[k] += sm[k][i];
    for (int k = 0; k < 4; ++k) partials[4 * blockIdx.x + k] = t[k];
  }
}

int tet_coeffs(fsi_mesh* m, int phase, double* gb) {
  TetData* t = m->tet;
  constexpr int NB = 152;
  if (m->n_partials < NB) {
    cudaFree(m->partials);
    m->partials = nullptr;
    FSI_CUDA(cudaMalloc(&m->partials, sizeof(double) * 4 * NB));
    m->n_partials = NB;
  }
  TetArgs A{};
  A.conn = t->conn;
  A.geo = t->geo;
  A.ne = t->ne;
  A.xa = m->staged_xa;
  A.E = t->E;
  A.nn = m->nn;
  FSI_LAUNCH(m, P_COEF, tet_coef_elem<<<(unsigned)((t->ne + 127) / 128), 128, 0, m->stream>>>(A, phase));
  FSI_LAUNCH(m, P_COEF, tet_coef_reduce<<<NB, 256, 0, m->stream>>>(t->nptr, t->nlist, t->E, t->ne, m->nn,
                                                                   m->staged_xa + (4 + phase) * m->nn, m->partials));
  FSI_LAUNCH(m, P_COEF, coef_finalize<<<1, NTHREADS, 0, m->stream>>>(m->partials, NB, m->P.eta, m->red));
  FSI_CUDA(cudaMemcpyAsync(m->red_host, m->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  FSI_CUDA(cudaStreamSynchronize(m->stream));
  gb[0] = m->red_host[0];
  gb[1] = m->red_host[1];
  return FSI_OK;
}

}  // namespace fsi

using namespace fsi;

extern "C" int fsi_create_tet_mesh(const fsi_mesh_desc* d, const double* coords, const int32_t* conn, int64_t ne,
                                   fsi_mesh** out) {
  if (!out) return set_error(FSI_EINVAL, "fsi_create_tet_mesh: null output");
  *out = nullptr;
  if (!d || !coords || !conn || ne < 1) return set_error(FSI_EINVAL, "fsi_create_tet_mesh: null argument or no elements");
  if (ne > (int64_t)1 << 29) return set_error(FSI_EINVAL, "fsi_create_tet_mesh: at most 2^29 elements");
  fsi_mesh* m = nullptr;
  int rc = fsi_create_mesh(d, &m);
  if (rc) return rc;
  const int64_t nn = m->nn;
  std::vector<int32_t> cn((size_t)(4 * ne));
  std::vector<double> geo((size_t)(TG * ne));
  std::vector<int64_t> ptr(nn + 1, 0);
  for (int64_t e = 0; e < ne; ++e) {
    int n[4];
    for (int a = 0; a < 4; ++a) {
      n[a] = conn[4 * e + a];
      if (n[a] < 0 || n[a] >= nn) {
        fsi_destroy_mesh(m);
        return set_error(FSI_EINVAL, "fsi_create_tet_mesh: node index out of range");
      }
      cn[(size_t)(a * ne + e)] = n[a];
      ++ptr[n[a] + 1];
    }
    double J[3][3];  // columns x_a - x_0
    for (int a = 1; a < 4; ++a)
      for (int r = 0; r < 3; ++r) J[r][a - 1] = coords[(int64_t)r * nn + n[a]] - coords[(int64_t)r * nn + n[0]];
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    if (!(det > 0.0)) {
      fsi_destroy_mesh(m);
      return set_error(FSI_EINVAL, "fsi_create_tet_mesh: an element has non-positive volume (orientation)");
    }
    // inverse by cofactors: Jinv[k][j] = d xi_k / d x_j = grad(lambda_{k+1})_j
    double Ji[3][3];
    Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    double g[4][3];
    for (int j = 0; j < 3; ++j) {
      g[1][j] = Ji[0][j];
      g[2][j] = Ji[1][j];
      g[3][j] = Ji[2][j];
      g[0][j] = -(Ji[0][j] + Ji[1][j] + Ji[2][j]);
    }
    for (int a = 0; a < 4; ++a)
      for (int j = 0; j < 3; ++j) geo[(size_t)((3 * a + j) * ne + e)] = g[a][j];
    geo[(size_t)(12 * ne + e)] = det / 24.0;  // |T| / 4
    const int sym[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {1, 2}, {0, 2}};
    for (int c = 0; c < 6; ++c) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += Ji[k][sym[c][0]] * Ji[k][sym[c][1]];
      geo[(size_t)((13 + c) * ne + e)] = s;
    }
  }
  for (int64_t n = 0; n < nn; ++n) ptr[n + 1] += ptr[n];
  std::vector<int32_t> list((size_t)ptr[nn]);
  std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
  for (int64_t e = 0; e < ne; ++e)
    for (int a = 0; a < 4; ++a) list[(size_t)fill[conn[4 * e + a]]++] = (int32_t)(4 * e + a);
  auto* t = new TetData();
  t->ne = ne;
  m->tet = t;
  cudaError_t err = cudaSuccess;
  auto up = [&](void** p, const void* src, size_t bytes) {
    if (err != cudaSuccess) return;
    err = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (err == cudaSuccess && src) err = cudaMemcpy(*p, src, bytes, cudaMemcpyHostToDevice);
  };
  up((void**)&t->conn, cn.data(), sizeof(int32_t) * cn.size());
  up((void**)&t->geo, geo.data(), sizeof(double) * geo.size());
  up((void**)&t->nptr, ptr.data(), sizeof(int64_t) * ptr.size());
  up((void**)&t->nlist, list.data(), sizeof(int32_t) * list.size());
  up((void**)&t->E, nullptr, sizeof(double) * 24 * (size_t)ne);
  if (err != cudaSuccess) {
    rc = cuda_check(err, "fsi_create_tet_mesh: device arrays");
    fsi_destroy_mesh(m);
    return rc;
  }
  *out = m;
  return FSI_OK;
}
