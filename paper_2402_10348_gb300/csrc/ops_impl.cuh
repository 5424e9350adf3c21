// Host-side launchers of the element operators for one compute type T.
// Included by ops_f64.cu (T = double) and ops_f32.cu (T = float).
#pragma once
#include "internal.h"

namespace fsi {

template <typename T>
struct Staged;  // staged-state arrays of the compute type

template <>
struct Staged<double> {
  static const double* xa(const fsi_mesh* m) { return m->staged_xa; }
  static const double* xd(const fsi_mesh* m) { return m->xd; }
  static const double* mat(const fsi_mesh* m) { return m->mat; }
};
template <>
struct Staged<float> {
  static const float* xa(const fsi_mesh* m) { return m->xa32; }
  static const float* xd(const fsi_mesh* m) { return m->xd32; }
  static const float* mat(const fsi_mesh* m) { return m->mat32; }
};

template <typename T>
inline void put(Fields& F, int i, const T* p);
template <>
inline void put<double>(Fields& F, int i, const double* p) { F.d[i] = p; F.f[i] = nullptr; }
template <>
inline void put<float>(Fields& F, int i, const float* p) { F.f[i] = p; F.d[i] = nullptr; }

constexpr size_t SMEM_LIMIT = 232448;

inline void fill_common(const fsi_mesh* m, double rh[3], double* W) {
  rh[0] = 1.0 / m->g.hx; rh[1] = 1.0 / m->g.hy; rh[2] = 1.0 / m->g.hz;
  *W = m->g.hx * m->g.hy * m->g.hz / 8.0;
}

int batch_launch_tiles_impl(fsi_batch* b, const void* ops_dev, size_t smem, int cls, int use_active,
                            const void* kernel);

template <class Op>
int launch_batched(fsi_batch* b, const void* ops_dev, size_t smem, int cls, int use_active);

template <class Op>
void* upload_ops(const BatchRec& r) {
  void* d = nullptr;
  if (cudaMalloc(&d, r.bytes.size()) != cudaSuccess) return nullptr;
  if (cudaMemcpy(d, r.bytes.data(), r.bytes.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return nullptr;
  }
  return d;
}

template <class Op>
int record_op(BatchRec* r, const Op& op, int cls) {
  if (r->count > 0 && (r->op_size != sizeof(Op) || r->launch != &launch_batched<Op>))
    return set_error(FSI_EINVAL, "batch: instances need the same operator type (same block and pass count)");
  r->op_size = sizeof(Op);
  r->launch = &launch_batched<Op>;
  r->upload = &upload_ops<Op>;
  r->cls = cls;
  r->smem = std::max(r->smem, tile_smem_bytes<Op>(op.nf));
  const unsigned char* p = reinterpret_cast<const unsigned char*>(&op);
  r->bytes.insert(r->bytes.end(), p, p + sizeof(Op));
  ++r->count;
  return FSI_OK;
}

template <class Op>
int launch_batched(fsi_batch* b, const void* ops_dev, size_t smem, int cls, int use_active) {
  if (int rc = ensure_smem_attr(reinterpret_cast<const void*>(&tile_batch_kernel<Op>), smem)) return rc;
  return batch_launch_tiles_impl(b, ops_dev, smem, cls, use_active,
                                 reinterpret_cast<const void*>(&tile_batch_kernel<Op>));
}

// z-chunking of the tile grid for about `per_sm` x 152 CTAs (the mesh's own geometry
// targets one CTA per SM; operators that fit more CTAs per SM get shorter z-ranges)
inline Geom tile_geom(const fsi_mesh* m, int per_sm, dim3* grid) {
  Geom g = m->g;
  if (per_sm > 1) {
    const int cols = g.ncx * g.ncy;
    const int planes = g.nz + 1;
    const int chunks = std::max(1, std::min(planes, (152 * per_sm + cols / 2) / cols));
    g.zc = (planes + chunks - 1) / chunks;
  }
  *grid = dim3(g.ncx, g.ncy, (g.nz + 1 + g.zc - 1) / g.zc);
  return g;
}

template <class Op>
int run_tile(fsi_mesh* m, const Op& op, int cls) {
  if (m->rec) return record_op(m->rec, op, cls);
  const size_t smem = tile_smem_bytes<Op>(op.nf);
  if (int rc = ensure_smem_attr(reinterpret_cast<const void*>(&tile_kernel<Op>), smem)) return rc;
  dim3 grid;
  const Geom g = tile_geom(m, Op::MINB, &grid);
  FSI_LAUNCH(m, cls, tile_kernel<Op><<<grid, NTHREADS, smem, m->stream>>>(op, g));
  return FSI_OK;
}

template <typename T>
constexpr int jvp_class(int kind) {
  return kind == 0 ? (sizeof(T) == 8 ? P_NS_JVP64 : P_NS_JVP32)
                   : (kind == 1 ? (sizeof(T) == 8 ? P_AC_JVP64 : P_AC_JVP32) : (sizeof(T) == 8 ? P_B_JVP64 : P_B_JVP32));
}
template <typename T, int MODE>
constexpr int op_class(int kind) {
  return MODE == 1 ? jvp_class<T>(kind)
                   : (MODE == 0 ? (kind == 0 ? P_NS_RES : (kind == 1 ? P_AC_RES : P_B_RES))
                                : (kind == 0 ? P_NS_DIAG : (kind == 1 ? P_AC_DIAG : P_B_DIAG)));
}

// The increment of a product: float64 kernels read dx itself, float32 kernels the
// float copy the caller made (m->dx32, same layout).
template <typename T>
inline void put_dx(Fields& F, int i, const fsi_mesh* m, const double* dx, int64_t off) {
  if constexpr (sizeof(T) == 4) put<float>(F, i, m->dx32 + off);
  else put<double>(F, i, dx + off);
}

template <typename T>
inline int solids_per_pass(int nf_fixed) {
  // 3 ring slots x (nf_fixed + 7 s) fields + 4 x 8 x 256 contributions
  const size_t fixed = sizeof(T) * (size_t)(3 * nf_fixed * PP + 4 * 8 * NTHREADS);
  const size_t per = sizeof(T) * (size_t)(3 * 7 * PP);
  if (fixed >= SMEM_LIMIT) return 0;
  return (int)((SMEM_LIMIT - fixed) / per);
}

template <typename T, int MODE>
int ns_pass(fsi_mesh* m, const double* dx, double* y, unsigned flags, int s0, int s1, bool first) {
  NSOp<T, MODE> op;
  memset(&op, 0, sizeof(op));
  const T* xa = Staged<T>::xa(m);
  const T* xd = Staged<T>::xd(m);
  const T* mat = Staged<T>::mat(m);
  const int64_t nn = m->nn;
  if ((MODE == 1 ? 4 : 0) + 9 + 7 * (s1 - s0) > MAXF) return set_error(FSI_EINVAL, "NS operator: too many staged fields");
  int f = 0;
  if (MODE == 1) {
    for (int k = 0; k < 4; ++k) put_dx<T>(op.F, f++, m, dx, k * nn);
  }
  for (int k = 0; k < 3; ++k) put<T>(op.F, f++, xa + k * nn);   // v
  put<T>(op.F, f++, xa + 3 * nn);                                 // p^{n+1}
  for (int k = 0; k < 3; ++k) put<T>(op.F, f++, xd + k * nn);   // dv/dt
  put<T>(op.F, f++, mat);                                         // rho
  put<T>(op.F, f++, mat + nn);                                    // mu
  for (int s = s0; s < s1; ++s) {
    put<T>(op.F, f++, mat + (2 + s) * nn);                        // alpha^s
    const int c0 = 4 + m->N + 6 * s;
    for (int c = 0; c < 6; ++c) put<T>(op.F, f++, xa + (c0 + c) * nn);
  }
  op.nf = f;
  op.s0 = s0;
  op.s1 = s1;
  op.fluid = first ? 1 : 0;
  op.elastic_aug = (flags & FSI_ELASTIC_AUG) ? 1 : 0;
  op.P = m->P;
  fill_common(m, op.rh, &op.W);
  op.out.y = y;
  op.out.dx = dx;
  op.out.dx32 = sizeof(T) == 4 ? m->dx32 : nullptr;
  op.out.x = m->staged_x;
  op.out.mask = m->mask;
  op.out.vD = m->vD;
  op.out.accumulate = first ? 0 : 1;
  op.out.dirichlet = first ? 1 : 0;
  op.out.pin = m->pin_active;
  op.nn_ = nn;
  return run_tile(m, op, op_class<T, MODE>(0));
}

template <typename T>
int launch_ns(fsi_mesh* m, int mode, const double* dx, double* y, unsigned flags) {
  const bool need_solids = (mode == 0) || (flags & FSI_ELASTIC_AUG);
  const int ns = need_solids ? m->ns : 0;
  const int fixed = (mode == 1 ? 4 : 0) + 9;
  // bounded by shared memory and by the MAXF staged-field slots of Fields
  const int per = std::min(solids_per_pass<T>(fixed), (MAXF - fixed) / 7);
  if (per < 1 && ns > 0) return set_error(FSI_EINVAL, "NS operator: shared memory too small for one solid");
  int s0 = 0;
  bool first = true;
  do {
    const int s1 = ns == 0 ? 0 : std::min(ns, s0 + per);
    int rc;
    if (mode == 0) rc = ns_pass<T, 0>(m, dx, y, flags, s0, s1, first);
    else if (mode == 1) rc = ns_pass<T, 1>(m, dx, y, flags, s0, s1, first);
    else rc = ns_pass<T, 2>(m, dx, y, flags, s0, s1, first);
    if (rc) return rc;
    first = false;
    s0 = s1;
  } while (s0 < ns);
  return FSI_OK;
}

// x pitch of the coefficient planes: a multiple of 16 bytes for either compute type
inline int cq_pitch(const fsi_mesh* m) { return (m->g.nx + 3) & ~3; }

// ------------------------------------------------ element-centric products
// One thread per element (x fastest, one CTA row per (ey, ez)) gathers its corner values
// from the nodal vectors and writes its corner contributions into E[slot][element]
// (slot = 8 * component + corner, element index ez * nxyp + ey * nxp + ex); a node
// kernel then sums, per node, the slots of its up to 8 elements in a fixed order
// (z, y, x).  Each element is evaluated once (no halo recomputation); deterministic.
// the thread's position in a row_launch grid: x within the row (*x), row index returned
__device__ __forceinline__ int64_t row_index(int len, int* x) {
  const int nbx = (len + blockDim.x - 1) / blockDim.x;
  const int64_t bxi = blockIdx.x % nbx, byi = blockIdx.x / nbx;
  *x = (int)(bxi * blockDim.x + threadIdx.x);
  return byi * blockDim.y + threadIdx.y;
}

struct ElemIdx {
  int ex, ey, ez;
  int64_t n0, e, es;
  int64_t off[8];
  __device__ __forceinline__ bool set(int nx, int ny, int nz, int nxp, int64_t nxyp) {
    const int64_t eyz = row_index(nx, &ex);
    ey = (int)(eyz % ny);
    if (ex >= nx || eyz >= (int64_t)ny * nz) return false;
    ez = (int)(eyz / ny);
    const int64_t sy = nx + 1, sz = (int64_t)(nx + 1) * (ny + 1);
    n0 = ex + sy * ey + sz * ez;
    off[0] = 0; off[1] = 1; off[2] = sy; off[3] = sy + 1;
    off[4] = sz; off[5] = sz + 1; off[6] = sz + sy; off[7] = sz + sy + 1;
    e = (int64_t)ez * nxyp + (int64_t)ey * nxp + ex;
    es = (int64_t)nz * nxyp;
    return true;
  }
};

// Launch shape over rows of `len` items (elements or nodes along x), `rows` rows: CTAs of
// bx x by threads (bx the row length rounded up to a warp, at most 128; by = 128 / bx
// rows), numbered x-block fastest in a one-dimensional grid (no 65,535 limit on rows).
struct RowLaunch {
  dim3 grid, block;
};
inline RowLaunch row_launch(int len, int64_t rows) {
  const int bx = std::min(128, (len + 31) / 32 * 32), by = 128 / bx;
  const int64_t nbx = (len + bx - 1) / bx, nby = (rows + by - 1) / by;
  return RowLaunch{dim3((unsigned)(nbx * nby)), dim3(bx, by)};
}
inline RowLaunch elem_launch(const Geom& g) { return row_launch(g.nx, (int64_t)g.ny * g.nz); }
inline RowLaunch node_launch(const Geom& g) { return row_launch(g.nx + 1, (int64_t)(g.ny + 1) * (g.nz + 1)); }

// NS node sums: y = W * sum of the element slots, the Dirichlet rows (velocity; pressure
// at the pin node when pinned) take the increment itself (dx, or its float32 copy dx32)
template <typename T>
__global__ void __launch_bounds__(128) ns_node_kernel(const T* __restrict__ E, int nx, int ny, int nz, int nxp,
                                                      int64_t nxyp, int64_t nn, double W, const uint8_t* __restrict__ mask,
                                                      int pin, const double* __restrict__ dx,
                                                      const float* __restrict__ dx32, double* __restrict__ y) {
  int i;
  const int64_t jk = row_index(nx + 1, &i);
  if (i > nx || jk >= (int64_t)(ny + 1) * (nz + 1)) return;
  const int j = (int)(jk % (ny + 1)), k = (int)(jk / (ny + 1));
  const int64_t n = i + (int64_t)(nx + 1) * (j + (int64_t)(ny + 1) * k);
  const int64_t es = (int64_t)nz * nxyp;
  T s[4] = {T(0), T(0), T(0), T(0)};
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
        const int a = ax + 2 * ay + 4 * az;  // this node's corner in element (ex, ey, ez)
#pragma unroll
        for (int f = 0; f < 4; ++f) s[f] += E[(8 * f + a) * es + e];
      }
    }
  }
  const uint8_t mk = mask[n];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const bool dir = ((mk >> f) & 1) && (f < 3 || pin);
    y[f * nn + n] = dir ? (dx ? dx[f * nn + n] : (double)dx32[f * nn + n]) : W * (double)s[f];
  }
}

// NS product from the quadrature-point coefficients (see nsq_point) of element (ex, ey, ez)
// into its 32 contribution slots (element-centric)
template <typename T>
__device__ __forceinline__ void nsq_elem_body(const T* __restrict__ cq, const T* __restrict__ dx, T* __restrict__ E,
                                              int nx, int ny, int nz, int nxp, int64_t nxyp, int64_t nn, int elastic,
                                              T al, T cmass, T rhx, T rhy, T rhz, int ex, int ey, int ez) {
  const int64_t sy = nx + 1, sz = (int64_t)(nx + 1) * (ny + 1);
  const int64_t n0 = ex + sy * ey + sz * ez;
  const int64_t off[8] = {0, 1, sy, sy + 1, sz, sz + 1, sz + sy, sz + sy + 1};
  T x[4][8], c[4][8];
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      x[f][a] = __ldg(dx + f * nn + n0 + off[a]);
      c[f][a] = T(0);
    }
  const T* e0 = cq + (int64_t)ez * 8 * NCQ * nxyp + (int64_t)ey * nxp + ex;
#pragma unroll 1
  for (int q = 0; q < 8; ++q) {
    QW<T> w;
    w.set(q);
    T dv[3], gd[3][3];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
      const VG<T> r = interp_vg(x[kk], w, rhx, rhy, rhz);
      dv[kk] = r.v; gd[kk][0] = r.gx; gd[kk][1] = r.gy; gd[kk][2] = r.gz;
    }
    const VG<T> dpr = interp_vg(x[3], w, rhx, rhy, rhz);
    const T dgp[3] = {dpr.gx, dpr.gy, dpr.gz};
    nsq_point<T>(CoefRef<T>{e0 + (int64_t)q * NCQ * nxyp, nxyp}, elastic != 0, dv, gd, dpr.v, dgp, al, cmass, w, rhx,
                 rhy, rhz, c);
  }
  const int64_t e = (int64_t)ez * nxyp + (int64_t)ey * nxp + ex;
  const int64_t es = (int64_t)nz * nxyp;
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int a = 0; a < 8; ++a) E[(8 * f + a) * es + e] = c[f][a];
}

template <typename T>
__global__ void __launch_bounds__(128) nsq_elem_kernel(const T* __restrict__ cq, const T* __restrict__ dx,
                                                       T* __restrict__ E, int nx, int ny, int nz, int nxp, int64_t nxyp,
                                                       int64_t nn, int elastic, T al, T cmass, T rhx, T rhy, T rhz) {
  ElemIdx I;
  if (!I.set(nx, ny, nz, nxp, nxyp)) return;
  nsq_elem_body<T>(cq, dx, E, nx, ny, nz, nxp, nxyp, nn, elastic, al, cmass, rhx, rhy, rhz, I.ex, I.ey, I.ez);
}

template <typename T>
int launch_nsq(fsi_mesh* m, const double* dx, double* y, unsigned flags) {
  const unsigned eflags = flags & FSI_ELASTIC_AUG;
  if (m->cq_gen != m->stage_gen || m->cq_flags != eflags || !m->cq64) {
    if (int rc = ns_build(m, flags)) return rc;
  }
  if constexpr (sizeof(T) == 8) {
    // a float64 solve on this state: after NSE_AFTER products switch to element matrices
    if (m->f64_gen != m->cq_builds) {
      m->f64_gen = m->cq_builds;
      m->f64_count = 0;
    }
    if (++m->f64_count > NSE_AFTER) return launch_nse(m, dx, y, flags);
  }
  const Geom& g = m->g;
  const int64_t nn = m->nn;
  const int nxp = cq_pitch(m);
  const int64_t nxyp = (int64_t)nxp * g.ny;
  const int elastic = (eflags && m->ns > 0) ? 1 : 0;
  if (int rc = ensure_elem_scratch(m, 32, nxyp)) return rc;
  const T* cq;
  const T* xin;
  if constexpr (sizeof(T) == 8) {
    cq = reinterpret_cast<const T*>(m->cq64);
    xin = reinterpret_cast<const T*>(dx);
  } else {
    cq = reinterpret_cast<const T*>(m->cq32);
    xin = reinterpret_cast<const T*>(m->dx32);
  }
  T* E = reinterpret_cast<T*>(m->ke_e);
  // algorithmic bytes: the coefficient planes once per element, the increment once per
  // node, the 32 element contributions written; the node sums read them back and write
  // the product (the mask once per node)
  const int64_t ne = (int64_t)g.nx * g.ny * g.nz;
  prof_bytes(m, jvp_class<T>(0),
             (double)ne * (8.0 * (elastic ? NCQ : NCQ_FLUID) + 32.0) * sizeof(T) + (double)nn * 4.0 * sizeof(T));
  prof_bytes(m, P_NODE_SUM, (double)ne * 32.0 * sizeof(T) + (double)nn * (32.0 + 1.0));
  const RowLaunch el = elem_launch(g), nl = node_launch(g);
  if constexpr (sizeof(T) == 4) {
    (void)cq;
    (void)xin;
    if (int rc = launch_nsq_tma(m, elastic, E, dx, y)) return rc;
  } else {
    FSI_LAUNCH(m, jvp_class<T>(0),
               nsq_elem_kernel<T><<<el.grid, el.block, 0, m->stream>>>(
                   cq, xin, E, g.nx, g.ny, g.nz, nxp, nxyp, nn, elastic, T(m->P.alpha), T(m->P.c_mass),
                   T(1.0 / g.hx), T(1.0 / g.hy), T(1.0 / g.hz)));
  }
  FSI_LAUNCH(m, P_NODE_SUM,
             ns_node_kernel<T><<<nl.grid, nl.block, 0, m->stream>>>(
                 E, g.nx, g.ny, g.nz, nxp, nxyp, nn, g.hx * g.hy * g.hz / 8.0, m->mask, m->pin_active,
                 dx, sizeof(T) == 4 ? m->dx32 : nullptr, y));
  return FSI_OK;
}

template <typename T, int MODE>
int ac_run(fsi_mesh* m, int i, const double* dx, double* y) {
  ACOp<T, MODE> op;
  memset(&op, 0, sizeof(op));
  const T* xa = Staged<T>::xa(m);
  const T* xd = Staged<T>::xd(m);
  const int64_t nn = m->nn;
  int f = 0;
  if (MODE == 1) put_dx<T>(op.F, f++, m, dx, 0);
  for (int k = 0; k < 3; ++k) put<T>(op.F, f++, xa + k * nn);
  put<T>(op.F, f++, xa + (4 + i) * nn);
  if (MODE == 0) put<T>(op.F, f++, xd + (4 + i) * nn);
  op.nf = f;
  op.P = m->P;
  fill_common(m, op.rh, &op.W);
  op.gamma = m->gamma[i];
  op.beta = m->beta[i];
  op.out.y = y;
  op.nn_ = nn;
  return run_tile(m, op, op_class<T, MODE>(1));
}

template <typename T>
int launch_ac(fsi_mesh* m, int mode, int i, const double* dx, double* y) {
  if constexpr (sizeof(T) == 8) {
    // a float64 solve of this phase at this staging: after ACE_AFTER products switch to the
    // element matrices (not for recorded batched launches)
    if (mode == 1 && !m->rec) {
      if (m->ake_gen != m->stage_gen || m->ake_phase != i || m->ake_gamma != m->gamma[i] ||
          m->ake_beta != m->beta[i]) {
        m->ake_gen = m->stage_gen;
        m->ake_phase = i;
        m->ake_gamma = m->gamma[i];
        m->ake_beta = m->beta[i];
        m->ake_count = 0;
        m->ake_built = 0;
      }
      if (++m->ake_count > ACE_AFTER) return launch_ace(m, i, dx, y);
    }
  }
  if (mode == 0) return ac_run<T, 0>(m, i, dx, y);
  if (mode == 1) return ac_run<T, 1>(m, i, dx, y);
  return ac_run<T, 2>(m, i, dx, y);
}

template <typename T, int MODE>
int b_run(fsi_mesh* m, int s, const double* dx, double* y) {
  BOp<T, MODE> op;
  memset(&op, 0, sizeof(op));
  const T* xa = Staged<T>::xa(m);
  const T* xd = Staged<T>::xd(m);
  const T* mat = Staged<T>::mat(m);
  const int64_t nn = m->nn;
  const int c0 = 4 + m->N + 6 * s;
  int f = 0;
  if (MODE == 1)
    for (int c = 0; c < 6; ++c) put_dx<T>(op.F, f++, m, dx, c * nn);
  for (int k = 0; k < 3; ++k) put<T>(op.F, f++, xa + k * nn);
  put<T>(op.F, f++, mat + (2 + s) * nn);
  if (MODE == 0) {
    for (int c = 0; c < 6; ++c) put<T>(op.F, f++, xa + (c0 + c) * nn);
    for (int c = 0; c < 6; ++c) put<T>(op.F, f++, xd + (c0 + c) * nn);
  }
  op.nf = f;
  op.P = m->P;
  fill_common(m, op.rh, &op.W);
  op.out.y = y;
  op.nn_ = nn;
  return run_tile(m, op, op_class<T, MODE>(2));
}

template <typename T>
int launch_b(fsi_mesh* m, int mode, int s, const double* dx, double* y) {
  if constexpr (sizeof(T) == 8) {
    // a float64 solve of this solid at this staging: after BE_AFTER products switch to the
    // split operator (not for recorded batched launches)
    if (mode == 1 && !m->rec) {
      if (m->bke_gen != m->stage_gen || m->bke_solid != s) {
        m->bke_gen = m->stage_gen;
        m->bke_solid = s;
        m->bke_count = 0;
        m->bke_built = 0;
      }
      if (++m->bke_count > BE_AFTER) return launch_be(m, s, dx, y);
    }
  }
  if (mode == 0) return b_run<T, 0>(m, s, dx, y);
  if (mode == 1) return b_run<T, 1>(m, s, dx, y);
  return b_run<T, 2>(m, s, dx, y);
}

}  // namespace fsi
