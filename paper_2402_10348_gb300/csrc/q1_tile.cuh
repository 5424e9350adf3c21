// Q1 hexahedral element engine: z-marching column tiles with node-centric,
// atomics-free assembly through shared memory.
//
// Mesh: uniform box, node n = i + (nx+1)(j + (ny+1)k), element (ex,ey,ez) with
// corners a = ax + 2ay + 4az.  Quadrature: 2x2x2 Gauss (xi = +-1/sqrt3, weights 1,
// |det J| = hx hy hz / 8), exact for the trilinear mass and stiffness integrands.
//
// A CTA owns the node column [i0, i0+OX) x [j0, j0+OY) x [k0, k0+ZC).  It walks the
// element layers ez = k0-1 .. k0+ZC-1 of the (OX+1) x (OY+1) elements that touch its
// nodes (one thread per element, TX x TY = 16 x 16 threads).  Each layer needs the
// node planes ez and ez+1 (17 x 17 nodes, all staged fields) in shared memory; each
// element writes its 8 corner contributions to shared memory; each owned node then
// adds the 4 contributions of its lower-plane corners to the partial sum it carries
// from the layer below (complete -> written out) and starts the next plane's sum
// from its 4 upper-plane corners.  Every sum is taken in a fixed order: the result
// is deterministic and needs no atomics.  The one-element halo ring in x/y and the
// one extra layer below k0 are recomputed by neighbouring CTAs.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fsi {

constexpr int TX = 16, TY = 16;          // elements per layer tile = threads per CTA
constexpr int NTHREADS = TX * TY;
constexpr int OX = TX - 1, OY = TY - 1;  // owned nodes per CTA in x, y
constexpr int PX = TX + 1, PY = TY + 1;  // staged nodes per plane in x, y
constexpr int PP = PX * PY;

struct Geom {
  int nx, ny, nz;
  int64_t nn;
  double hx, hy, hz;
  int zc;       // owned node planes per CTA
  int ncx, ncy; // CTA columns in x, y
};

// 1D Gauss weights of the trilinear shape functions: the corner on the same side
// as the quadrature point gets G0 = (1 + 1/sqrt3)/2, the other G1 = (1 - 1/sqrt3)/2.
#define FSI_G0 0.78867513459481288225
#define FSI_G1 0.21132486540518711775

template <typename T>
struct QW {  // per-quadrature-point 1D weights
  T wx[2], wy[2], wz[2];
  __device__ __forceinline__ void set(int q) {
    const int qx = q & 1, qy = (q >> 1) & 1, qz = (q >> 2) & 1;
    wx[0] = qx == 0 ? T(FSI_G0) : T(FSI_G1); wx[1] = qx == 1 ? T(FSI_G0) : T(FSI_G1);
    wy[0] = qy == 0 ? T(FSI_G0) : T(FSI_G1); wy[1] = qy == 1 ? T(FSI_G0) : T(FSI_G1);
    wz[0] = qz == 0 ? T(FSI_G0) : T(FSI_G1); wz[1] = qz == 1 ? T(FSI_G0) : T(FSI_G1);
  }
};

template <typename T>
struct VG { T v, gx, gy, gz; };

// Value and physical gradient at one quadrature point from the 8 corner values,
// by passes along x, y, z (gradient along x = (u1 - u0)/hx interpolated in y, z).
template <typename T>
__device__ __forceinline__ VG<T> interp_vg(const T (&u)[8], const QW<T>& w, T rhx, T rhy, T rhz) {
  T ux[4], dx[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {  // r = ay + 2 az
    ux[r] = w.wx[0] * u[2 * r] + w.wx[1] * u[2 * r + 1];
    dx[r] = u[2 * r + 1] - u[2 * r];
  }
  T uxy[2], dxy[2], dyx[2];
#pragma unroll
  for (int az = 0; az < 2; ++az) {
    uxy[az] = w.wy[0] * ux[2 * az] + w.wy[1] * ux[2 * az + 1];
    dxy[az] = w.wy[0] * dx[2 * az] + w.wy[1] * dx[2 * az + 1];
    dyx[az] = ux[2 * az + 1] - ux[2 * az];
  }
  VG<T> o;
  o.v = w.wz[0] * uxy[0] + w.wz[1] * uxy[1];
  o.gx = (w.wz[0] * dxy[0] + w.wz[1] * dxy[1]) * rhx;
  o.gy = (w.wz[0] * dyx[0] + w.wz[1] * dyx[1]) * rhy;
  o.gz = (uxy[1] - uxy[0]) * rhz;
  return o;
}

template <typename T>
__device__ __forceinline__ T interp_v(const T (&u)[8], const QW<T>& w) {
  T uxy[2];
#pragma unroll
  for (int az = 0; az < 2; ++az) {
    const T a = w.wx[0] * u[4 * az] + w.wx[1] * u[4 * az + 1];
    const T b = w.wx[0] * u[4 * az + 2] + w.wx[1] * u[4 * az + 3];
    uxy[az] = w.wy[0] * a + w.wy[1] * b;
  }
  return w.wz[0] * uxy[0] + w.wz[1] * uxy[1];
}

// c[a] += N_a f + dN_a/dx gx + dN_a/dy gy + dN_a/dz gz  (transpose of interp_vg).
template <typename T>
__device__ __forceinline__ void scatter_vg(T (&c)[8], const QW<T>& w, T f, T gx, T gy, T gz,
                                           T rhx, T rhy, T rhz) {
  gx *= rhx; gy *= rhy; gz *= rhz;
  T uxy_b[2], dxy_b[2], dyx_b[2];
  uxy_b[0] = w.wz[0] * f - gz; uxy_b[1] = w.wz[1] * f + gz;
  dxy_b[0] = w.wz[0] * gx;     dxy_b[1] = w.wz[1] * gx;
  dyx_b[0] = w.wz[0] * gy;     dyx_b[1] = w.wz[1] * gy;
#pragma unroll
  for (int az = 0; az < 2; ++az) {
    const T ux0 = w.wy[0] * uxy_b[az] - dyx_b[az];
    const T ux1 = w.wy[1] * uxy_b[az] + dyx_b[az];
    const T dx0 = w.wy[0] * dxy_b[az];
    const T dx1 = w.wy[1] * dxy_b[az];
    c[4 * az + 0] += w.wx[0] * ux0 - dx0;
    c[4 * az + 1] += w.wx[1] * ux0 + dx0;
    c[4 * az + 2] += w.wx[0] * ux1 - dx1;
    c[4 * az + 3] += w.wx[1] * ux1 + dx1;
  }
}

// c[a] += N_a f
template <typename T>
__device__ __forceinline__ void scatter_v(T (&c)[8], const QW<T>& w, T f) {
#pragma unroll
  for (int a = 0; a < 8; ++a) c[a] += w.wx[a & 1] * w.wy[(a >> 1) & 1] * w.wz[(a >> 2) & 1] * f;
}

// Shared-memory view of the element's corners for the thread's element.
template <typename T>
struct Corners {
  const T* lo;  // plane ez: [NS][PP]
  const T* hi;  // plane ez+1
  int off;      // (ty)*PX + tx
  __device__ __forceinline__ void get(int f, T (&u)[8]) const {
    const T* a = lo + f * PP + off;
    const T* b = hi + f * PP + off;
    u[0] = a[0]; u[1] = a[1]; u[2] = a[PX]; u[3] = a[PX + 1];
    u[4] = b[0]; u[5] = b[1]; u[6] = b[PX]; u[7] = b[PX + 1];
  }
};

// Per-node context handed to Op::finish.
struct NodeCtx {
  int64_t n;
  int i, j, k;
};

// The engine.  Op provides:
//   using T (compute type), Red (per-thread reduction state); int nf (staged
//   fields); NC (output components);
//   T field(int f, int64_t node) const;                      staged nodal value
//   void element(const Corners<T>&, const ElemCtx&, T (&c)[NC][8], Red&) const;
//   void finish(const NodeCtx&, const T (&acc)[NC], Red&) const;
//   void begin_cta(Red&) const, end_cta(Red&) const.
struct ElemCtx {
  int ex, ey, ez;
  bool owned;  // this CTA is the one that counts the element in reductions
};

// cp.async of one element (4 or 8 bytes) global -> shared; src_bytes = 0 writes zeros.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src, bool valid) {
  const unsigned saddr = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  const int sz = valid ? (int)sizeof(T) : 0;
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(saddr), "l"(src), "r"(sz) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(saddr), "l"(src), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Node planes live in a ring of three shared-memory slots: while layer ez is
// computed from the planes ez and ez+1, the copies of plane ez+2 are in flight.
__host__ __device__ constexpr int plane_slot(int kz) { return ((kz % 3) + 3) % 3; }

// One CTA tile (bx, by, bz) of the z-marching element loop (the body of the single
// and the batched launches).
template <class Op>
__device__ __forceinline__ void tile_body(const Op& op, const Geom& g, int bx, int by, int bz,
                                          unsigned char* smem_raw) {
  using T = typename Op::T;
  constexpr int NC = Op::NC;
  const int NS = op.nf;
  T* planes = reinterpret_cast<T*>(smem_raw);       // [3][NS][PP]
  T* contrib = planes + 3 * NS * PP;                // [NC*8][NTHREADS]

  const int t = threadIdx.x;
  const int tx = t % TX, ty = t / TX;
  const int i0 = bx * OX, j0 = by * OY, k0 = bz * g.zc;
  const int ex = i0 - 1 + tx, ey = j0 - 1 + ty;
  const bool exy_ok = ex >= 0 && ex < g.nx && ey >= 0 && ey < g.ny;
  // owned node of this thread (local (tx+1, ty+1))
  const int ni = i0 + tx, nj = j0 + ty;
  const bool node_thread = tx < OX && ty < OY && ni <= g.nx && nj <= g.ny;
  // an element is counted by the CTA that owns its lower corner node
  const bool exy_owned = exy_ok && ex >= i0 && ey >= j0;

  T carry[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) carry[c] = T(0);
  typename Op::Red red;
  op.begin_cta(red);

  // issue the copies of node plane kz (all staged fields) into its ring slot
  auto issue_plane = [&](int kz) {
    T* dst = planes + plane_slot(kz) * NS * PP;
    for (int idx = t; idx < PP; idx += NTHREADS) {
      const int lx = idx % PX, ly = idx / PX;
      const int gi = i0 - 1 + lx, gj = j0 - 1 + ly;
      const bool ok = kz >= 0 && kz <= g.nz && gi >= 0 && gi <= g.nx && gj >= 0 && gj <= g.ny;
      const int64_t n = ok ? (int64_t)gi + (int64_t)(g.nx + 1) * ((int64_t)gj + (int64_t)(g.ny + 1) * kz) : 0;
      for (int f = 0; f < NS; ++f) {
        const T* src = op.fptr(f);
        cp_async_elem(dst + f * PP + idx, src + n, ok);
      }
    }
  };

  const int ez_begin = k0 - 1, ez_end = k0 + g.zc - 1;  // inclusive
  issue_plane(ez_begin);
  cp_async_commit();
  issue_plane(ez_begin + 1);
  cp_async_commit();
  for (int ez = ez_begin; ez <= ez_end; ++ez) {
    if (ez + 2 <= ez_end + 1) issue_plane(ez + 2);
    cp_async_commit();  // possibly empty: keeps one group per iteration
    cp_async_wait_1();  // this thread's copies of planes ez, ez+1 have landed
    __syncthreads();    // ... and everybody's
    {
      T c[NC][8];
#pragma unroll
      for (int q = 0; q < NC; ++q)
#pragma unroll
        for (int a = 0; a < 8; ++a) c[q][a] = T(0);
      if (exy_ok && ez >= 0 && ez < g.nz) {
        Corners<T> cr;
        cr.lo = planes + plane_slot(ez) * NS * PP;
        cr.hi = planes + plane_slot(ez + 1) * NS * PP;
        cr.off = ty * PX + tx;
        ElemCtx ec{ex, ey, ez, exy_owned && ez >= k0};
        op.element(cr, ec, c, red);
      }
#pragma unroll
      for (int q = 0; q < NC; ++q)
#pragma unroll
        for (int a = 0; a < 8; ++a) contrib[(q * 8 + a) * NTHREADS + t] = c[q][a];
    }
    // every read of plane ez is done after this barrier: the next iteration may
    // refill its slot with plane ez+3
    __syncthreads();
    if (node_thread) {
      const int e00 = ty * TX + tx;  // element (tx, ty) has this node as corner (1,1)
      const int e10 = ty * TX + tx + 1, e01 = (ty + 1) * TX + tx, e11 = (ty + 1) * TX + tx + 1;
      T lower[NC], upper[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        const T* C = contrib + q * 8 * NTHREADS;
        // node is corner (ax, ay) of element (tx+1-ax, ty+1-ay)
        lower[q] = C[3 * NTHREADS + e00] + C[2 * NTHREADS + e10] + C[1 * NTHREADS + e01] + C[0 * NTHREADS + e11];
        upper[q] = C[7 * NTHREADS + e00] + C[6 * NTHREADS + e10] + C[5 * NTHREADS + e01] + C[4 * NTHREADS + e11];
      }
      const int kz = ez;  // the plane completed by this layer
      if (kz >= k0 && kz <= g.nz) {
        T tot[NC];
#pragma unroll
        for (int q = 0; q < NC; ++q) tot[q] = carry[q] + lower[q];
        NodeCtx nc;
        nc.i = ni; nc.j = nj; nc.k = kz;
        nc.n = (int64_t)ni + (int64_t)(g.nx + 1) * ((int64_t)nj + (int64_t)(g.ny + 1) * kz);
        op.finish(nc, tot, red);
      }
#pragma unroll
      for (int q = 0; q < NC; ++q) carry[q] = upper[q];
    }
    // the contributions are rewritten only after the next iteration's first barrier
  }
  op.end_cta(red);
}

template <class Op>
__global__ void __launch_bounds__(NTHREADS, Op::MINB) tile_kernel(const __grid_constant__ Op op, const Geom g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  tile_body(op, g, blockIdx.x, blockIdx.y, blockIdx.z, smem_raw);
}

// Batched launch: persistent CTAs walk a list of (instance, bx, by, bz) tiles over
// many independent meshes; ops[i] and geoms[i] describe instance i.  Instances whose
// active flag is 0 are skipped.
template <class Op>
__global__ void __launch_bounds__(NTHREADS, Op::MINB)
    tile_batch_kernel(const Op* __restrict__ ops, const Geom* __restrict__ geoms, const int4* __restrict__ work,
                      int nwork, const int* __restrict__ active) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int4 it = work[w];
    if (active && !active[it.x]) continue;
    __syncthreads();  // the previous tile's shared-memory reads are done
    tile_body(ops[it.x], geoms[it.x], it.y, it.z, it.w, smem_raw);
  }
}

template <class Op>
inline size_t tile_smem_bytes(int nf) {
  using T = typename Op::T;
  return sizeof(T) * (size_t)(3 * nf * PP + Op::NC * 8 * NTHREADS);
}

struct NoRed {};

// Block-wide deterministic sum of one value per thread (fixed tree order).
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* scratch /* >= NTHREADS/32 */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  T s = T(0);
  if (threadIdx.x == 0)
    for (int i = 0; i < NTHREADS / 32; ++i) s += scratch[i];
  return s;  // valid in thread 0
}

}  // namespace fsi
