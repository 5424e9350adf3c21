// Batched solves over many independent meshes of uneven size (no counterpart in the
// paper, which treats one problem at a time).
//
// Operators: the per-instance operator structs are recorded by the ordinary
// launchers (fsi_mesh::rec) and replayed by one persistent launch whose CTAs walk a
// work list of (instance, tile) items (tile_batch_kernel), so an operator apply over
// 64 meshes is one launch instead of 64.
//
// Krylov: restarted GMRES(m) with Jacobi right preconditioning runs for all
// instances in lock-step.  Block vectors are concatenated (instance b owns
// [off_b, off_b + n_b)); each instance keeps its own chunk-interleaved basis (256
// elements per chunk, all m+1 vectors of a chunk contiguous).  Vector kernels walk a
// list of (instance, first chunk, last chunk) items that never cross an instance, so
// every reduction has per-item partial sums that one CTA per instance adds in a fixed
// order (bit-reproducible).  Arnoldi step j: precondition, one batched operator launch,
// classical Gram-Schmidt with the DGKS second pass where an instance needs it, Givens
// rotation per instance (one thread each); an instance whose residual estimate meets
// the tolerance deactivates itself on the device, and later launches skip its items.
// A whole restart cycle (m steps, the least-squares solution, x += D V y and the true
// residual) has no host decision in it: it is captured once as a CUDA graph and
// replayed; the host reads the per-instance residual norms once per cycle.
//
// Mixed precision as in the single-mesh solver: float32 operator inside float64
// iterative refinement (the outer residual is the float64 operator's).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include <sys/stat.h>

#include "internal.h"
#include "pcnet.h"

namespace fsi {

constexpr int BCH = 256;      // elements per basis chunk
constexpr int BMMAX = 64;     // largest restart length
constexpr int BITEM = 32;     // chunks per vector work item
constexpr int BVB = 256;      // threads per CTA of the vector kernels
constexpr int BKC = 16;       // dot products per CTA pass
constexpr int PSTRIDE = BMMAX + 2;

// Arnoldi/Givens state of one instance
struct BKry {
  double h[BMMAX + 2], h2[BMMAX + 2];
  double H[(BMMAX + 1) * BMMAX];
  double cs[BMMAX], sn[BMMAX], g[BMMAX + 1], y[BMMAX];
  double nrm_old, nrm_new, nrm_fin, bnorm, est, rn2;
  int reorth, jend;
};

struct OpSet {
  void* ops = nullptr;  // device array of operator structs (fixed address: graphs keep it)
  size_t bytes = 0;
  size_t smem = 0;
  int cls = 0;
  int (*launch)(fsi_batch*, const void*, size_t, int, int) = nullptr;
};

}  // namespace fsi

struct fsi_batch {
  std::vector<fsi_mesh*> meshes;  // per entry (a mesh may appear once per block of it)
  std::vector<int> blocks;        // per entry: the block id
  int n = 0;
  fsi::BlockInfo blk0{};
  int block = 0;
  float* dx32_own = nullptr;      // float increments of all entries (concatenated like the block vectors)
  cudaStream_t stream = nullptr;
  std::vector<int64_t> off;  // [n + 1]
  int64_t ntot = 0;
  // operator work list
  std::vector<fsi::Geom> geoms;
  fsi::Geom* geoms_dev = nullptr;
  int4* tiles_dev = nullptr;
  int ntiles = 0;
  int grid = 0;              // persistent CTAs of the batched operator launch
  int target_mult = 4;       // autotuned: total tiles ~ target_mult x 152
  int grid_mult = 2;         // autotuned: persistent CTAs = grid_mult x 152
  // vector work list
  int4* items_dev = nullptr; // (instance, first chunk, end chunk, 0)
  int nitems = 0;
  int* item_first_dev = nullptr;  // [n + 1] items of instance b: [first[b], first[b+1])
  std::vector<int> item_first;
  // Krylov
  int mm = 0, M1 = 0;
  double* V = nullptr;
  int64_t* vbase_dev = nullptr;   // per instance: offset of its basis in V
  int64_t* off_dev = nullptr;     // per instance: offset in concatenated vectors
  int64_t* nloc_dev = nullptr;    // per instance: block vector length
  float** dx32_dev = nullptr;     // per instance: its float copy of the increment
  double *w = nullptr, *z = nullptr, *r = nullptr, *t = nullptr, *dinv = nullptr, *d = nullptr;
  double *rin = nullptr, *rout = nullptr;  // inner right-hand side, outer residual
  double* part = nullptr;         // [nitems][PSTRIDE]
  fsi::BKry* K = nullptr;         // [n]
  int* act = nullptr;             // [n] instance iterating in the current cycle
  int* live = nullptr;            // [n] instance still solving (host-set per cycle)
  double* host_out = nullptr;     // pinned [2 n]: |r|^2 and iterations of the last cycle
  double* out_dev = nullptr;      // [2 n]
  int* host_live = nullptr;       // pinned [n]
  // recorded operator sets
  fsi::OpSet jvp_inner;   // z -> w (float32 or float64)
  fsi::OpSet jvp_d;       // d -> t (same precision as the inner solve)
  fsi::OpSet jvp_outer;   // x -> t (float64)
  fsi::OpSet jvp_user;    // fsi_batch_jvp
  unsigned inner_flags = 0;
  // graph of one restart cycle
  cudaGraphExec_t cycle = nullptr;
  double graph_rtol = -1.0;
  int graph_f32 = -1;
  int use_graph = 1;
  int64_t launches = 0;          // launches of this batch (graph replays count their nodes)
  int64_t launches_per_cycle = 0;
  // flexible GMRES with each instance's attached network (NS batches): the directions
  // Z [mm][ntot], set per solve
  double* Zb = nullptr;
  int64_t zb_len = 0;
  int use_pc = 0, pc_alternate = 0;
  // the network step of every instance as one captured graph: each instance's network on one
  // of a few side streams (parallel branches), output into zt [ntot]
  double* zt = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t net_graph = nullptr;
  int net_warm = 0;
  // work lists of the batched float32 NS coefficient product (built on first use)
  int4* nsq_eitems = nullptr;     // (instance, x block, y block, layer)
  int nsq_ne = 0;
  int4* nsq_nitems = nullptr;     // (instance, 128-node block, 0, 0)
  int nsq_nn = 0;
};

namespace fsi {

// ------------------------------------------------------------------ kernels
template <int K>
__device__ __forceinline__ void bsum_store(double (&acc)[K], int k, double* out) {
  __shared__ double sm[K][BVB / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    double v = acc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sm[i][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double s = 0.0;
    for (int wi = 0; wi < BVB / 32; ++wi) s += sm[threadIdx.x][wi];
    out[threadIdx.x] = s;
  }
}

template <typename T, int K>
__device__ __forceinline__ void bsum_store_t(T (&acc)[K], int k, double* out) {
  __shared__ T smt[K][BVB / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    T v = acc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) smt[i][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < k) {
    T s = T(0);
    for (int wi = 0; wi < BVB / 32; ++wi) s += smt[threadIdx.x][wi];
    out[threadIdx.x] = (double)s;
  }
}

// basis slot i of chunk c of instance b; the basis type VT is double for float64 solves and
// float for the inner solves of float32 refinement (the same allocation, element offsets)
template <typename VT>
__device__ __forceinline__ VT* bslot(VT* V, const int64_t* vbase, int b, int M1, int64_t c, int i) {
  return V + vbase[b] + c * (int64_t)M1 * BCH + (int64_t)i * BCH;
}

// z_b = dinv_b * V_b[j] (and the float copy for float32 operators)
template <typename VT>
__global__ void bk_precond(const int4* __restrict__ items, const int* __restrict__ act, VT* V,
                           const int64_t* vbase, const int64_t* off, const int64_t* nloc, int M1, int j,
                           const double* __restrict__ dinv, double* __restrict__ z, float* const* dx32,
                           double* __restrict__ zs) {
  const int4 it = items[blockIdx.x];
  const int b = it.x;
  if (!act[b]) return;
  for (int64_t c = it.y; c < it.z; ++c) {
    const int64_t e = c * BCH + threadIdx.x;
    if (e >= nloc[b]) break;
    const double v = dinv[off[b] + e] * (double)bslot(V, vbase, b, M1, c, j)[threadIdx.x];
    z[off[b] + e] = v;
    if (dx32) dx32[b][e] = (float)v;
    if (zs) zs[off[b] + e] = v;  // flexible GMRES keeps the direction
  }
}

// t = V_j (concatenated float64 copy of basis slot j of the active instances)
template <typename VT>
__global__ void bk_extract(const int4* __restrict__ items, const int* __restrict__ act, VT* V,
                           const int64_t* vbase, const int64_t* off, const int64_t* nloc, int M1, int j,
                           double* __restrict__ t) {
  const int4 it = items[blockIdx.x];
  const int b = it.x;
  if (!act[b]) return;
  for (int64_t c = it.y; c < it.z; ++c) {
    const int64_t e = c * BCH + threadIdx.x;
    if (e >= nloc[b]) break;
    t[off[b] + e] = (double)bslot(V, vbase, b, M1, c, j)[threadIdx.x];
  }
}

// the network's direction: Z_j = z = zt (with the float copy of z)
__global__ void bk_zfill(const int4* __restrict__ items, const int* __restrict__ act, const double* __restrict__ zt,
                         const int64_t* off, const int64_t* nloc, double* __restrict__ z, float* const* dx32,
                         double* __restrict__ zs) {
  const int4 it = items[blockIdx.x];
  const int b = it.x;
  if (!act[b]) return;
  for (int64_t c = it.y; c < it.z; ++c) {
    const int64_t e = c * BCH + threadIdx.x;
    if (e >= nloc[b]) break;
    const double v = zt[off[b] + e];
    z[off[b] + e] = v;
    zs[off[b] + e] = v;
    if (dx32) dx32[b][e] = (float)v;
  }
}

// x += sum_{i < jend} y_i Z_i (flexible GMRES)
__global__ void bk_zcombine(const int4* __restrict__ items, const BKry* __restrict__ K, const int* live,
                            const double* __restrict__ Z, int64_t ntot, const int64_t* off, const int64_t* nloc,
                            double* __restrict__ x) {
  const int4 it = items[blockIdx.x];
  const int b = it.x;
  if (!live[b]) return;
  __shared__ double ys[BMMAX];
  const int jend = K[b].jend;
  for (int i = threadIdx.x; i < jend; i += blockDim.x) ys[i] = K[b].y[i];
  __syncthreads();
  for (int64_t c = it.y; c < it.z; ++c) {
    const int64_t e = c * BCH + threadIdx.x;
    if (e >= nloc[b]) break;
    double s = 0.0;
    for (int i = 0; i < jend; ++i) s += ys[i] * Z[(int64_t)i * ntot + off[b] + e];
    x[off[b] + e] += s;
  }
}

// float copy of a concatenated vector into each instance's increment buffer
__global__ void bk_tofloat(const int4* __restrict__ items, const int* __restrict__ act, const int64_t* off,
                           const int64_t* nloc, const double* __restrict__ src, float* const* dx32, int gate) {
  const int4 it = items[blockIdx.x];
  const int b = it.x;
  if (gate && !act[b]) return;
  for (int64_t c = it.y; c < it.z; ++c) {
    const int64_t e = c * BCH + threadIdx.x;
    if (e >= nloc[b]) break;
    dx32[b][e] = (float)src[off[b] + e];
  }
}

// partials of V_b[i0 .. i0+kc) . w_b and (self) w_b . w_b; second pass only where reorth
template <bool SELF, typename VT>
__global__ void bk_mdot(const int4* __restrict__ items, const BKry* __restrict__ K, const int* __restrict__ act,
                        const VT* V,
                        const int64_t* vbase, const int64_t* off, const int64_t* nloc, int M1, int nvec,
                        const double* __restrict__ w, double* part, int second) {
  const int4 it = items[blockIdx.x];
  const int b = it.x;
  if (!act[b] || (second && !K[b].reorth)) return;
  const int i0 = blockIdx.y * BKC;
  const int kc = min(BKC, nvec - i0);
  if (kc <= 0 && !(SELF && blockIdx.y == 0)) return;
  VT acc[BKC + 1];  // per-thread sums in the basis type, the CTA's sums stored as double
#pragma unroll
  for (int i = 0; i <= BKC; ++i) acc[i] = VT(0);
  for (int64_t c = it.y; c < it.z; ++c) {
    const int64_t e = c * BCH + threadIdx.x;
    if (e >= nloc[b]) break;
    const VT wj = (VT)w[off[b] + e];
    const VT* blk = V + vbase[b] + c * (int64_t)M1 * BCH + (int64_t)i0 * BCH + threadIdx.x;
#pragma unroll
    for (int i = 0; i < BKC; ++i)
      if (i < kc) acc[i] += blk[i * BCH] * wj;
    if (SELF && blockIdx.y == 0) acc[BKC] += wj * wj;
  }
  double* out = part + (int64_t)blockIdx.x * PSTRIDE;
  __shared__ double res[BKC + 1];
  bsum_store_t<VT, BKC + 1>(acc, BKC + 1, res);
  __syncthreads();
  if ((int)threadIdx.x < kc) out[i0 + threadIdx.x] = res[threadIdx.x];
  if (SELF && blockIdx.y == 0 && threadIdx.x == 0) out[PSTRIDE - 1] = res[BKC];
}

// per instance: dst[i] = sum over its items of part[item][i], i < nv (fixed order);
// slot PSTRIDE-1 (|w|^2) goes to dst[nv] when self
__global__ void bk_reduce(const int* __restrict__ first, const double* __restrict__ part, BKry* K,
                          const int* __restrict__ act, int nv,
                          int self, int which, int second) {
  const int b = blockIdx.x;
  if (!act[b] || (second && !K[b].reorth)) return;
  double* dst = which == 0 ? K[b].h : K[b].h2;
  for (int i = threadIdx.x; i < nv + (self ? 1 : 0); i += blockDim.x) {
    const int src = i < nv ? i : PSTRIDE - 1;
    double s = 0.0;
    for (int it = first[b]; it < first[b + 1]; ++it) s += part[(int64_t)it * PSTRIDE + src];
    dst[i] = s;
  }
}

// w_b -= sum_i h_i V_b[i] and the partial |w_b|^2 (slot 0)
template <typename VT>
__global__ void bk_update(const int4* __restrict__ items, const BKry* __restrict__ K, const int* __restrict__ act,
                          const VT* V,
                          const int64_t* vbase, const int64_t* off, const int64_t* nloc, int M1, int nvec,
                          double* __restrict__ w, double* part, int which, int second) {
  const int4 it = items[blockIdx.x];
  const int b = it.x;
  if (!act[b] || (second && !K[b].reorth)) return;
  __shared__ VT hs[BMMAX + 1];
  const double* h = which == 0 ? K[b].h : K[b].h2;
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) hs[i] = (VT)h[i];
  __syncthreads();
  VT acc[1] = {VT(0)};
  for (int64_t c = it.y; c < it.z; ++c) {
    const int64_t e = c * BCH + threadIdx.x;
    if (e >= nloc[b]) break;
    const VT* blk = V + vbase[b] + c * (int64_t)M1 * BCH + threadIdx.x;
    VT s = VT(0);
    for (int i = 0; i < nvec; ++i) s += hs[i] * blk[(int64_t)i * BCH];
    const VT v = (VT)w[off[b] + e] - s;
    w[off[b] + e] = (double)v;
    acc[0] += v * v;
  }
  __shared__ double res[1];
  bsum_store_t<VT, 1>(acc, 1, res);
  __syncthreads();
  if (threadIdx.x == 0) part[(int64_t)blockIdx.x * PSTRIDE] = res[0];
}

__global__ void bk_norm_reduce(const int* __restrict__ first, const double* __restrict__ part, BKry* K,
                               const int* __restrict__ act, int nb,
                               int second) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb || !act[b] || (second && !K[b].reorth)) return;
  double s = 0.0;
  for (int it = first[b]; it < first[b + 1]; ++it) s += part[(int64_t)it * PSTRIDE];
  K[b].nrm_new = s;
}

// after pass 1: |w_old|^2 is h[j+1]; DGKS: a second pass when |w_new| < |w_old| / sqrt2
__global__ void bk_orth_decide(BKry* K, const int* __restrict__ act, int nb, int j) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb || !act[b]) return;
  K[b].nrm_old = sqrt(K[b].h[j + 1]);
  const double nn = sqrt(K[b].nrm_new);
  K[b].reorth = (nn < K[b].nrm_old * 0.70710678118654752) ? 1 : 0;
  K[b].nrm_fin = nn;
}

__global__ void bk_givens(BKry* K, int* act, int nb, int j, int mm, double rtol) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb || !act[b]) return;
  BKry& k = K[b];
  if (k.reorth) {
    for (int i = 0; i <= j; ++i) k.h[i] += k.h2[i];
    k.nrm_fin = sqrt(k.nrm_new);
  }
  double* col = k.H;
  for (int i = 0; i <= j; ++i) col[i * mm + j] = k.h[i];
  const double hn = k.nrm_fin;
  col[(j + 1) * mm + j] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = k.cs[i] * col[i * mm + j] + k.sn[i] * col[(i + 1) * mm + j];
    col[(i + 1) * mm + j] = -k.sn[i] * col[i * mm + j] + k.cs[i] * col[(i + 1) * mm + j];
    col[i * mm + j] = a;
  }
  const double den = hypot(col[j * mm + j], col[(j + 1) * mm + j]);
  k.cs[j] = den > 0.0 ? col[j * mm + j] / den : 1.0;
  k.sn[j] = den > 0.0 ? col[(j + 1) * mm + j] / den : 0.0;
  col[j * mm + j] = den;
  col[(j + 1) * mm + j] = 0.0;
  k.g[j + 1] = -k.sn[j] * k.g[j];
  k.g[j] = k.cs[j] * k.g[j];
  k.est = fabs(k.g[j + 1]) / k.bnorm;
  k.jend = j + 1;
  const bool breakdown = hn == 0.0 || den == 0.0 || !isfinite(hn);
  if (k.est <= rtol || breakdown || !isfinite(k.est)) act[b] = 0;  // converged (or stuck): stop this cycle
}

// V_b[j+1] = w_b / |w_b|
template <typename VT>
__global__ void bk_store(const int4* __restrict__ items, const BKry* __restrict__ K, const int* __restrict__ act,
                         VT* V, const int64_t* vbase,
                         const int64_t* off, const int64_t* nloc, int M1, int slot, const double* __restrict__ src,
                         int from_rn2) {
  const int4 it = items[blockIdx.x];
  const int b = it.x;
  if (!act[b]) return;
  const double nrm = from_rn2 ? sqrt(K[b].rn2) : K[b].nrm_fin;
  const double s = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (int64_t c = it.y; c < it.z; ++c) {
    const int64_t e = c * BCH + threadIdx.x;
    if (e >= nloc[b]) break;
    bslot(V, vbase, b, M1, c, slot)[threadIdx.x] = (VT)(s * src[off[b] + e]);
  }
}

// cycle start: instances still iterating (live) start a cycle with g = (|r|, 0, ...)
__global__ void bk_cycle_start(BKry* K, int* act, int nb, const int* live, int mm) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  act[b] = live[b];
  for (int i = 0; i <= mm; ++i) K[b].g[i] = 0.0;
  K[b].g[0] = sqrt(K[b].rn2);
  K[b].jend = 0;
  K[b].reorth = 0;
}

__global__ void bk_lsq(BKry* K, int nb, const int* live, int mm) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb || !live[b]) return;
  BKry& k = K[b];
  const int jend = k.jend;
  for (int i = jend - 1; i >= 0; --i) {
    double s = k.g[i];
    for (int q = i + 1; q < jend; ++q) s -= k.H[i * mm + q] * k.y[q];
    const double dd = k.H[i * mm + i];
    k.y[i] = dd != 0.0 ? s / dd : 0.0;
  }
}

// x_b += dinv_b * sum_{i < jend_b} y_i V_b[i]
template <typename VT>
__global__ void bk_combine(const int4* __restrict__ items, const BKry* __restrict__ K, const int* live,
                           const VT* V, const int64_t* vbase, const int64_t* off, const int64_t* nloc, int M1,
                           const double* __restrict__ dinv, double* __restrict__ x) {
  const int4 it = items[blockIdx.x];
  const int b = it.x;
  if (!live[b]) return;
  __shared__ double ys[BMMAX];
  const int jend = K[b].jend;
  for (int i = threadIdx.x; i < jend; i += blockDim.x) ys[i] = K[b].y[i];
  __syncthreads();
  for (int64_t c = it.y; c < it.z; ++c) {
    const int64_t e = c * BCH + threadIdx.x;
    if (e >= nloc[b]) break;
    const VT* blk = V + vbase[b] + c * (int64_t)M1 * BCH + threadIdx.x;
    double s = 0.0;
    for (int i = 0; i < jend; ++i) s += ys[i] * (double)blk[(int64_t)i * BCH];
    x[off[b] + e] += dinv[off[b] + e] * s;
  }
}

// r = b - t over live instances, with the partial |r|^2 (slot 0)
__global__ void bk_resid(const int4* __restrict__ items, const int* live, const int64_t* off, const int64_t* nloc,
                         const double* __restrict__ bv, const double* __restrict__ t, double* __restrict__ r,
                         double* part) {
  const int4 it = items[blockIdx.x];
  const int b = it.x;
  double acc[1] = {0.0};
  if (live[b]) {
    for (int64_t c = it.y; c < it.z; ++c) {
      const int64_t e = c * BCH + threadIdx.x;
      if (e >= nloc[b]) break;
      const double v = bv[off[b] + e] - t[off[b] + e];
      r[off[b] + e] = v;
      acc[0] += v * v;
    }
  }
  __shared__ double res[1];
  bsum_store<1>(acc, 1, res);
  __syncthreads();
  if (threadIdx.x == 0) part[(int64_t)blockIdx.x * PSTRIDE] = res[0];
}

__global__ void bk_rn2(const int* __restrict__ first, const double* __restrict__ part, BKry* K, const int* live,
                       int nb, double* out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  if (live && !live[b]) {
    out[b] = K[b].rn2;
    out[nb + b] = 0.0;
    return;
  }
  double s = 0.0;
  for (int it = first[b]; it < first[b + 1]; ++it) s += part[(int64_t)it * PSTRIDE];
  K[b].rn2 = s;
  out[b] = s;
  out[nb + b] = (double)K[b].jend;
}

// y = a * x + y over all elements (live instances)
__global__ void bk_axpy(const int4* __restrict__ items, const int* live, const int64_t* off, const int64_t* nloc,
                        double a, const double* __restrict__ xv, double* __restrict__ yv) {
  const int4 it = items[blockIdx.x];
  const int b = it.x;
  if (live && !live[b]) return;
  for (int64_t c = it.y; c < it.z; ++c) {
    const int64_t e = c * BCH + threadIdx.x;
    if (e >= nloc[b]) break;
    yv[off[b] + e] += a * xv[off[b] + e];
  }
}

__global__ void bk_set_bnorm(BKry* K, int nb, const double* bn) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nb) K[b].bnorm = bn[b];
}

__global__ void bk_recip(double* d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = 1.0 / d[i];
}

// ------------------------------------------------------------------ host
int batch_launch_tiles_impl(fsi_batch* b, const void* ops_dev, size_t smem, int cls, int use_active,
                            const void* kernel) {
  fsi_mesh* m = b->meshes[0];
  const int* active = nullptr;
  const void* ops = ops_dev;
  const Geom* geoms = b->geoms_dev;
  const int4* work = b->tiles_dev;
  int nwork = b->ntiles;
  // gate by the per-instance active flag of the Krylov state (int at a fixed offset)
  static_assert(sizeof(int) == 4, "int");
  const int* act_src = use_active == 1 ? b->act : (use_active == 2 ? b->live : nullptr);
  active = act_src;
  void* args[] = {const_cast<void**>(&ops), const_cast<Geom**>(&geoms), const_cast<int4**>(&work), &nwork,
                  const_cast<int**>(&active)};
  int rc = prof_begin(m, cls);
  if (rc) return rc;
  FSI_CUDA(cudaLaunchKernel(kernel, dim3(b->grid), dim3(NTHREADS), args, smem, b->stream));
  ++b->launches;
  return prof_end(m, cls);
}

}  // namespace fsi

// ------------------------------------------------------------------ host side
namespace fsi {
namespace {

// a norm-and-copy pass: dst = src over live instances, partial |src|^2 (slot 0)
__global__ void bk_copy_norm(const int4* __restrict__ items, const int* live, const int64_t* off,
                             const int64_t* nloc, const double* __restrict__ src, double* __restrict__ dst,
                             double* part) {
  const int4 it = items[blockIdx.x];
  const int b = it.x;
  double acc[1] = {0.0};
  if (!live || live[b]) {
    for (int64_t c = it.y; c < it.z; ++c) {
      const int64_t e = c * BCH + threadIdx.x;
      if (e >= nloc[b]) break;
      const double v = src[off[b] + e];
      if (dst) dst[off[b] + e] = v;
      acc[0] += v * v;
    }
  }
  __shared__ double res[1];
  bsum_store<1>(acc, 1, res);
  __syncthreads();
  if (threadIdx.x == 0) part[(int64_t)blockIdx.x * PSTRIDE] = res[0];
}

__global__ void bk_zero(const int4* __restrict__ items, const int* live, const int64_t* off, const int64_t* nloc,
                        double* __restrict__ v) {
  const int4 it = items[blockIdx.x];
  const int b = it.x;
  if (live && !live[b]) return;
  for (int64_t c = it.y; c < it.z; ++c) {
    const int64_t e = c * BCH + threadIdx.x;
    if (e >= nloc[b]) break;
    v[off[b] + e] = 0.0;
  }
}

int gx1(int n) { return (n + 127) / 128; }

// tiles: total ~ target_mult x 152; persistent CTAs: grid_mult x 152
int build_tiles(fsi_batch* b, int target_mult, int grid_mult) {
  int64_t work = 0;
  for (fsi_mesh* m : b->meshes) work += (int64_t)m->g.ncx * m->g.ncy * (m->g.nz + 1);
  const int zc0 = (int)std::max<int64_t>(1, (work + (int64_t)target_mult * 152 - 1) / ((int64_t)target_mult * 152));
  std::vector<int4> tiles;
  b->geoms.clear();
  for (int i = 0; i < b->n; ++i) {
    Geom g = b->meshes[i]->g;
    const int planes = g.nz + 1;
    const int chunks = std::max(1, (planes + zc0 - 1) / zc0);
    g.zc = (planes + chunks - 1) / chunks;
    b->geoms.push_back(g);
    for (int bz = 0; bz < chunks; ++bz)
      for (int by = 0; by < g.ncy; ++by)
        for (int bx = 0; bx < g.ncx; ++bx) tiles.push_back(make_int4(i, bx, by, bz));
  }
  cudaFree(b->tiles_dev);
  b->tiles_dev = nullptr;
  FSI_CUDA(cudaMalloc(&b->tiles_dev, sizeof(int4) * tiles.size()));
  FSI_CUDA(cudaMemcpy(b->tiles_dev, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice));
  FSI_CUDA(cudaMemcpy(b->geoms_dev, b->geoms.data(), sizeof(Geom) * b->n, cudaMemcpyHostToDevice));
  b->ntiles = (int)tiles.size();
  b->grid = std::max(1, std::min(b->ntiles, grid_mult * 152));
  b->target_mult = target_mult;
  b->grid_mult = grid_mult;
  // a captured cycle holds the old launch shape
  if (b->cycle) cudaGraphExecDestroy(b->cycle);
  b->cycle = nullptr;
  return FSI_OK;
}

// the batched float32 NS product from per-instance coefficients (nsq_tma.cu): element
// launch over every instance's 64 x 2-element tiles, node launch over its 128-node blocks
// work lists of the batched float32 NS product (built when the operator set is recorded,
// never inside a captured cycle)
int ensure_nsq_items(fsi_batch* b) {
  if (!b->nsq_eitems) {
    std::vector<int4> ei, ni;
    for (int i = 0; i < b->n; ++i) {
      const Geom& g = b->meshes[i]->g;
      const int nbx = (g.nx + NSQ_TBX - 1) / NSQ_TBX, nby = (g.ny + NSQ_TBY - 1) / NSQ_TBY;
      for (int ez = 0; ez < g.nz; ++ez)
        for (int by = 0; by < nby; ++by)
          for (int bx = 0; bx < nbx; ++bx) ei.push_back(make_int4(i, bx, by, ez));
      const int64_t nblk = (b->meshes[i]->nn + 127) / 128;
      for (int64_t k = 0; k < nblk; ++k) ni.push_back(make_int4(i, (int)k, 0, 0));
    }
    if (ei.size() > (size_t)INT32_MAX || ni.size() > (size_t)INT32_MAX)
      return set_error(FSI_EINVAL, "batch: too many tiles for one launch");
    FSI_CUDA(cudaMalloc(&b->nsq_eitems, sizeof(int4) * ei.size()));
    FSI_CUDA(cudaMalloc(&b->nsq_nitems, sizeof(int4) * ni.size()));
    FSI_CUDA(cudaMemcpy(b->nsq_eitems, ei.data(), sizeof(int4) * ei.size(), cudaMemcpyHostToDevice));
    FSI_CUDA(cudaMemcpy(b->nsq_nitems, ni.data(), sizeof(int4) * ni.size(), cudaMemcpyHostToDevice));
    b->nsq_ne = (int)ei.size();
    b->nsq_nn = (int)ni.size();
  }
  return FSI_OK;
}

int launch_nsq_batch_prec(fsi_batch* b, const void* ops_dev, int cls, int use_active, bool f64) {
  if (!b->nsq_eitems) return set_error(FSI_EINVAL, "batch: NS product work lists missing");
  fsi_mesh* m = b->meshes[0];
  const int* active = use_active == 1 ? b->act : (use_active == 2 ? b->live : nullptr);
  int rc = prof_begin(m, cls);
  if (rc) return rc;
  if ((rc = nsq_batch_launch(f64, static_cast<const NSQBatchRec*>(ops_dev), b->nsq_eitems, b->nsq_ne,
                             b->nsq_nitems, b->nsq_nn, active, b->stream)))
    return rc;
  b->launches += 2;
  return prof_end(m, cls);
}
int launch_nsq_batch32(fsi_batch* b, const void* ops_dev, size_t, int cls, int use_active) {
  return launch_nsq_batch_prec(b, ops_dev, cls, use_active, false);
}
int launch_nsq_batch64(fsi_batch* b, const void* ops_dev, size_t, int cls, int use_active) {
  return launch_nsq_batch_prec(b, ops_dev, cls, use_active, true);
}

// (re)allocates a set's device records for `bytes` (a captured cycle holding the old
// records is dropped)
int set_storage(fsi_batch* b, OpSet* set, size_t bytes) {
  if (set->ops && set->bytes == bytes) return FSI_OK;
  cudaFree(set->ops);
  set->ops = nullptr;
  FSI_CUDA(cudaMalloc(&set->ops, bytes));
  set->bytes = bytes;
  if (b->cycle) cudaGraphExecDestroy(b->cycle);
  b->cycle = nullptr;
  return FSI_OK;
}

// records the operator of every instance (dx = dx_base + off, y = y_base + off)
int record_set(fsi_batch* b, OpSet* set, unsigned flags, const double* dx_base, double* y_base) {
  BatchRec rec;
  const bool f32 = flags & FSI_FP32;
  bool all_ns = true;
  for (int i = 0; i < b->n; ++i) all_ns = all_ns && b->blocks[i] == FSI_BLOCK_NS;
  if (all_ns) {
    // NS products from each instance's frozen coefficients (built here, on the staged
    // states) in one element and one node launch: float32 TMA-staged, float64 read directly
    std::vector<NSQBatchRec> recs(b->n);
    for (int i = 0; i < b->n; ++i) {
      int rc = nsq_batch_record(b->meshes[i], flags, !f32, dx_base + b->off[i], y_base + b->off[i],
                                b->dx32_own + b->off[i], &recs[i]);
      if (rc) return rc;
    }
    const size_t bytes = sizeof(NSQBatchRec) * recs.size();
    if (int rc = ensure_nsq_items(b)) return rc;
    if (int rc = set_storage(b, set, bytes)) return rc;
    FSI_CUDA(cudaMemcpyAsync(set->ops, recs.data(), bytes, cudaMemcpyHostToDevice, b->stream));
    FSI_CUDA(cudaStreamSynchronize(b->stream));
    set->smem = 0;
    set->cls = f32 ? P_NS_JVP32 : P_NS_JVP64;
    set->launch = f32 ? &launch_nsq_batch32 : &launch_nsq_batch64;
    return FSI_OK;
  }
  for (int i = 0; i < b->n; ++i) {
    fsi_mesh* m = b->meshes[i];
    BlockInfo bi;
    int rc = block_info(m, b->blocks[i], &bi);
    if (rc) return rc;
    m->rec = &rec;
    // the entry's own float increment (a mesh with several entries must not share one)
    float* mesh_dx32 = m->dx32;
    m->dx32 = b->dx32_own + b->off[i];
    const double* dx = dx_base + b->off[i];
    double* y = y_base + b->off[i];
    if (bi.kind == 0) rc = f32 ? launch_ns<float>(m, 1, dx, y, flags) : launch_ns<double>(m, 1, dx, y, flags);
    else if (bi.kind == 1) rc = f32 ? launch_ac<float>(m, 1, bi.index, dx, y) : launch_ac<double>(m, 1, bi.index, dx, y);
    else rc = f32 ? launch_b<float>(m, 1, bi.index, dx, y) : launch_b<double>(m, 1, bi.index, dx, y);
    m->dx32 = mesh_dx32;
    m->rec = nullptr;
    if (rc) return rc;
  }
  if (rec.count != b->n)
    return set_error(FSI_EINVAL, "batch: an operator needs more than one pass (too many solids) for batching");
  if (int rc = set_storage(b, set, rec.bytes.size())) return rc;
  FSI_CUDA(cudaMemcpyAsync(set->ops, rec.bytes.data(), rec.bytes.size(), cudaMemcpyHostToDevice, b->stream));
  FSI_CUDA(cudaStreamSynchronize(b->stream));  // the host record is freed on return
  set->smem = rec.smem;
  set->cls = rec.cls;
  set->launch = rec.launch;
  return FSI_OK;
}

int run_set(fsi_batch* b, const OpSet& s, int gate) { return s.launch(b, s.ops, s.smem, s.cls, gate); }

#define BK_LAUNCH(b, cls, ...)                     \
  do {                                             \
    FSI_LAUNCH((b)->meshes[0], cls, __VA_ARGS__);  \
    ++(b)->launches;                               \
  } while (0)

// zt = M_i(t) for every instance (|t_i| = 1): the first time directly, one instance after
// another on the batch's stream; afterwards through a graph captured once per solve in which
// every instance's network runs on one of the side streams (independent branches the GPU
// runs side by side; the small grids of one instance's layers leave most SMs idle)
int net_step(fsi_batch* b) {
  cudaStream_t s = b->stream;
  const int nb = b->n;
  if (!b->net_warm || !b->use_graph || s == nullptr) {
    for (int i = 0; i < nb; ++i) {
      fsi_mesh* m = b->meshes[i];
      if (int rc = pcn::apply(m->pc, b->t + b->off[i], 1.0, b->dinv + b->off[i], b->zt + b->off[i])) return rc;
    }
    b->net_warm = 1;
    return FSI_OK;
  }
  if (!b->net_graph) {
    if (b->side.empty()) {
      // all side streams and events or none: a failure part-way releases what was made
      const int S = std::min(nb, 32);
      std::vector<cudaStream_t> side(S, nullptr);
      std::vector<cudaEvent_t> join(S, nullptr);
      cudaEvent_t fork = nullptr;
      cudaError_t ce = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
      for (int k = 0; k < S && ce == cudaSuccess; ++k) {
        ce = cudaStreamCreateWithFlags(&side[k], cudaStreamNonBlocking);
        if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming);
      }
      if (ce != cudaSuccess) {
        for (cudaStream_t x : side)
          if (x) cudaStreamDestroy(x);
        for (cudaEvent_t x : join)
          if (x) cudaEventDestroy(x);
        if (fork) cudaEventDestroy(fork);
        return cuda_check(ce, "batch network step: side streams");
      }
      b->side = std::move(side);
      b->join = std::move(join);
      b->fork = fork;
    }
    const int S = (int)b->side.size();
    std::vector<char> prof(nb);
    for (int i = 0; i < nb; ++i) prof[i] = b->meshes[i]->prof.on, b->meshes[i]->prof.on = false;
    cudaGraph_t g = nullptr;
    FSI_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaEventRecord(b->fork, s);
    for (int k = 0; k < S && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->side[k], b->fork, 0);
    int rc = FSI_OK;
    for (int i = 0; i < nb && e == cudaSuccess && !rc; ++i) {
      fsi_mesh* m = b->meshes[i];
      cudaStream_t saved = m->stream;
      m->stream = b->side[i % S];
      rc = pcn::apply(m->pc, b->t + b->off[i], 1.0, b->dinv + b->off[i], b->zt + b->off[i]);
      m->stream = saved;
    }
    for (int k = 0; k < S && e == cudaSuccess; ++k) {
      e = cudaEventRecord(b->join[k], b->side[k]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->join[k], 0);
    }
    const cudaError_t e2 = cudaStreamEndCapture(s, &g);
    for (int i = 0; i < nb; ++i) b->meshes[i]->prof.on = prof[i];
    if (rc || e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      if (rc) return rc;
      if (e != cudaSuccess) return cuda_check(e, "batch network step: capture");
      return cuda_check(e2, "batch network step: end capture");
    }
    e = cudaGraphInstantiate(&b->net_graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_check(e, "batch network step: instantiate");
  }
  FSI_CUDA(cudaGraphLaunch(b->net_graph, s));
  return FSI_OK;
}

// one Arnoldi step j of every active instance (basis type VT)
template <typename VT>
int enqueue_step_t(fsi_batch* b, int j, double rtol, bool f32) {
  VT* V = reinterpret_cast<VT*>(b->V);
  const int NI = b->nitems, nb = b->n, M1 = b->M1;
  cudaStream_t s = b->stream;
  double* Zj = b->use_pc ? b->Zb + (int64_t)j * b->ntot : nullptr;
  if (b->use_pc && !(b->pc_alternate && (j & 1))) {
    // flexible GMRES, network direction: z_j = M_i(v_j) per instance (|v_j| = 1)
    BK_LAUNCH(b, P_KRYLOV, bk_extract<VT><<<NI, BVB, 0, s>>>(b->items_dev, b->act, V, b->vbase_dev, b->off_dev,
                                                         b->nloc_dev, M1, j, b->t));
    if (int rc = net_step(b)) return rc;
    BK_LAUNCH(b, P_KRYLOV, bk_zfill<<<NI, BVB, 0, s>>>(b->items_dev, b->act, b->zt, b->off_dev, b->nloc_dev, b->z,
                                                       f32 ? b->dx32_dev : nullptr, Zj));
  } else {
    BK_LAUNCH(b, P_KRYLOV, bk_precond<VT><<<NI, BVB, 0, s>>>(b->items_dev, b->act, V, b->vbase_dev, b->off_dev,
                                                           b->nloc_dev, M1, j, b->dinv, b->z,
                                                           f32 ? b->dx32_dev : nullptr, Zj));
  }
  int rc = run_set(b, b->jvp_inner, 1);
  if (rc) return rc;
  const int nvec = j + 1;
  const dim3 g2(NI, (nvec + BKC - 1) / BKC);
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 0)
      BK_LAUNCH(b, P_KRY_DOT, bk_mdot<true, VT><<<g2, BVB, 0, s>>>(b->items_dev, b->K, b->act, V, b->vbase_dev,
                                                               b->off_dev, b->nloc_dev, M1, nvec, b->w, b->part, 0));
    else
      BK_LAUNCH(b, P_KRY_DOT, bk_mdot<false, VT><<<g2, BVB, 0, s>>>(b->items_dev, b->K, b->act, V, b->vbase_dev,
                                                                b->off_dev, b->nloc_dev, M1, nvec, b->w, b->part, 1));
    BK_LAUNCH(b, P_KRY_DOT, bk_reduce<<<nb, 128, 0, s>>>(b->item_first_dev, b->part, b->K, b->act, nvec,
                                                          pass == 0 ? 1 : 0, pass, pass));
    BK_LAUNCH(b, P_KRY_UPD, bk_update<VT><<<NI, BVB, 0, s>>>(b->items_dev, b->K, b->act, V, b->vbase_dev, b->off_dev,
                                                          b->nloc_dev, M1, nvec, b->w, b->part, pass, pass));
    BK_LAUNCH(b, P_KRY_UPD, bk_norm_reduce<<<gx1(nb), 128, 0, s>>>(b->item_first_dev, b->part, b->K, b->act, nb,
                                                                    pass));
    if (pass == 0) BK_LAUNCH(b, P_KRY_SMALL, bk_orth_decide<<<gx1(nb), 128, 0, s>>>(b->K, b->act, nb, j));
  }
  BK_LAUNCH(b, P_KRY_SMALL, bk_givens<<<gx1(nb), 128, 0, s>>>(b->K, b->act, nb, j, b->mm, rtol));
  BK_LAUNCH(b, P_KRYLOV, bk_store<VT><<<NI, BVB, 0, s>>>(b->items_dev, b->K, b->act, V, b->vbase_dev, b->off_dev,
                                                      b->nloc_dev, M1, j + 1, b->w, 0));
  return FSI_OK;
}

// one restart cycle of the inner solve: rhs b->rin, solution b->d, residual b->r; the
// float32 refinement's inner solves keep a float32 basis
template <typename VT>
int enqueue_cycle_t(fsi_batch* b, double rtol, bool f32);
int enqueue_cycle(fsi_batch* b, double rtol, bool f32) {
  if (f32) return enqueue_cycle_t<float>(b, rtol, f32);
  return enqueue_cycle_t<double>(b, rtol, f32);
}

template <typename VT>
int enqueue_cycle_t(fsi_batch* b, double rtol, bool f32) {
  VT* V = reinterpret_cast<VT*>(b->V);
  const int NI = b->nitems, nb = b->n, M1 = b->M1;
  cudaStream_t s = b->stream;
  BK_LAUNCH(b, P_KRY_SMALL, bk_cycle_start<<<gx1(nb), 128, 0, s>>>(b->K, b->act, nb, b->live, b->mm));
  BK_LAUNCH(b, P_KRYLOV, bk_store<VT><<<NI, BVB, 0, s>>>(b->items_dev, b->K, b->act, V, b->vbase_dev, b->off_dev,
                                                      b->nloc_dev, M1, 0, b->r, 1));
  for (int j = 0; j < b->mm; ++j) {
    int rc = enqueue_step_t<VT>(b, j, rtol, f32);
    if (rc) return rc;
  }
  BK_LAUNCH(b, P_KRY_SMALL, bk_lsq<<<gx1(nb), 128, 0, s>>>(b->K, nb, b->live, b->mm));
  if (b->use_pc)
    BK_LAUNCH(b, P_KRYLOV, bk_zcombine<<<NI, BVB, 0, s>>>(b->items_dev, b->K, b->live, b->Zb, b->ntot, b->off_dev,
                                                           b->nloc_dev, b->d));
  else
    BK_LAUNCH(b, P_KRYLOV, bk_combine<VT><<<NI, BVB, 0, s>>>(b->items_dev, b->K, b->live, V, b->vbase_dev, b->off_dev,
                                                          b->nloc_dev, M1, b->dinv, b->d));
  // true residual of the inner system: r = rin - A d (live instances)
  if (f32)
    BK_LAUNCH(b, P_KRY_CONV, bk_tofloat<<<NI, BVB, 0, s>>>(b->items_dev, b->live, b->off_dev, b->nloc_dev, b->d,
                                                           b->dx32_dev, 1));
  int rc = run_set(b, b->jvp_d, 2);
  if (rc) return rc;
  BK_LAUNCH(b, P_KRYLOV, bk_resid<<<NI, BVB, 0, s>>>(b->items_dev, b->live, b->off_dev, b->nloc_dev, b->rin, b->t,
                                                      b->r, b->part));
  BK_LAUNCH(b, P_KRYLOV, bk_rn2<<<gx1(nb), 128, 0, s>>>(b->item_first_dev, b->part, b->K, b->live, nb, b->out_dev));
  return FSI_OK;
}

int read_out(fsi_batch* b) {
  FSI_CUDA(cudaMemcpyAsync(b->host_out, b->out_dev, sizeof(double) * 2 * b->n, cudaMemcpyDeviceToHost, b->stream));
  FSI_CUDA(cudaStreamSynchronize(b->stream));
  return FSI_OK;
}

int upload_live(fsi_batch* b, const std::vector<int>& live) {
  memcpy(b->host_live, live.data(), sizeof(int) * b->n);
  FSI_CUDA(cudaMemcpyAsync(b->live, b->host_live, sizeof(int) * b->n, cudaMemcpyHostToDevice, b->stream));
  return FSI_OK;
}

// inner GMRES(m) of the live instances on b->rin -> b->d; iterations added to iters
int inner_solve(fsi_batch* b, std::vector<int> live, double rtol, int max_iter, bool f32, std::vector<int>& iters,
                std::vector<int>& restarts, std::vector<double>& rel, std::vector<int>& stalled) {
  const int NI = b->nitems, nb = b->n;
  cudaStream_t s = b->stream;
  int rc = upload_live(b, live);
  if (rc) return rc;
  BK_LAUNCH(b, P_KRYLOV, bk_zero<<<NI, BVB, 0, s>>>(b->items_dev, b->live, b->off_dev, b->nloc_dev, b->d));
  BK_LAUNCH(b, P_KRYLOV, bk_copy_norm<<<NI, BVB, 0, s>>>(b->items_dev, b->live, b->off_dev, b->nloc_dev, b->rin, b->r,
                                                          b->part));
  BK_LAUNCH(b, P_KRYLOV, bk_rn2<<<gx1(nb), 128, 0, s>>>(b->item_first_dev, b->part, b->K, b->live, nb, b->out_dev));
  if ((rc = read_out(b))) return rc;
  std::vector<double> bn(nb, 0.0), prev(nb, 1.0);
  for (int i = 0; i < nb; ++i) {
    bn[i] = std::sqrt(b->host_out[i]);
    if (!std::isfinite(bn[i])) return set_error(FSI_ENAN, "batch GMRES: right-hand side is not finite");
    if (bn[i] == 0.0) live[i] = 0;
    rel[i] = bn[i] > 0.0 ? 1.0 : 0.0;
  }
  FSI_CUDA(cudaMemcpyAsync(b->out_dev, bn.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, s));
  BK_LAUNCH(b, P_KRY_SMALL, bk_set_bnorm<<<gx1(nb), 128, 0, s>>>(b->K, nb, b->out_dev));
  FSI_CUDA(cudaStreamSynchronize(s));  // bn is a host temporary
  bool first = true;
  while (true) {
    int nlive = 0;
    for (int i = 0; i < nb; ++i) {
      if (!live[i]) continue;
      if (rel[i] <= rtol || iters[i] >= max_iter) live[i] = 0;
      else if (!first && rel[i] > 0.99 * prev[i]) live[i] = 0, stalled[i] = 1;
      nlive += live[i];
    }
    if (!nlive) break;
    for (int i = 0; i < nb; ++i) prev[i] = rel[i];
    first = false;
    if ((rc = upload_live(b, live))) return rc;
    // the legacy default stream cannot be captured: launch the cycle directly there
    if (b->use_graph && !b->use_pc && b->stream != nullptr) {
      if (!b->cycle || b->graph_rtol != rtol || b->graph_f32 != (int)f32) {
        if (b->cycle) cudaGraphExecDestroy(b->cycle);
        b->cycle = nullptr;
        fsi_mesh* m0 = b->meshes[0];
        const bool prof_on = m0->prof.on;
        m0->prof.on = false;  // no event records inside the capture
        const int64_t l0 = b->launches;
        cudaGraph_t g;
        FSI_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_cycle(b, rtol, f32);
        cudaError_t e = cudaStreamEndCapture(s, &g);
        m0->prof.on = prof_on;
        if (rc) return rc;
        if (e != cudaSuccess) return cuda_check(e, "batch GMRES: graph capture");
        e = cudaGraphInstantiate(&b->cycle, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_check(e, "batch GMRES: graph instantiate");
        b->launches_per_cycle = b->launches - l0;
        b->launches = l0;
        b->graph_rtol = rtol;
        b->graph_f32 = f32;
      }
      FSI_CUDA(cudaGraphLaunch(b->cycle, s));
      b->launches += b->launches_per_cycle;
    } else if ((rc = enqueue_cycle(b, rtol, f32))) {
      return rc;
    }
    if ((rc = read_out(b))) return rc;
    for (int i = 0; i < nb; ++i) {
      if (!live[i]) continue;
      const double r2 = b->host_out[i];
      if (!std::isfinite(r2)) return set_error(FSI_ENAN, "batch GMRES: residual is not finite");
      rel[i] = std::sqrt(r2) / bn[i];
      iters[i] += (int)b->host_out[nb + i];
      restarts[i] += 1;
    }
  }
  return FSI_OK;
}

int stage_all(fsi_batch* b, const fsi_state* states, bool f32) {
  for (int i = 0; i < b->n; ++i) {
    int rc = stage(b->meshes[i], &states[i], f32);
    if (rc) return rc;
  }
  return FSI_OK;
}

int ensure_dx32(fsi_batch* b) {
  if (!b->dx32_own) FSI_CUDA(cudaMalloc(&b->dx32_own, sizeof(float) * (size_t)std::max<int64_t>(b->ntot, 4)));
  std::vector<float*> p(b->n);
  for (int i = 0; i < b->n; ++i) {
    fsi_mesh* m = b->meshes[i];
    // the mesh's own copy is still needed by its single-mesh float32 launches
    if (!m->dx32) FSI_CUDA(cudaMalloc(&m->dx32, sizeof(float) * 6 * (size_t)m->nn));
    p[i] = b->dx32_own + b->off[i];
  }
  FSI_CUDA(cudaMemcpy(b->dx32_dev, p.data(), sizeof(float*) * b->n, cudaMemcpyHostToDevice));
  return FSI_OK;
}

// ------------------------------------------------------------------ autotuner cache
std::string cache_path() {
  if (const char* p = std::getenv("FSI_AUTOTUNE_CACHE")) return p;
  const char* home = std::getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/fsi_gb300_autotune.txt";
}

std::string tune_key(const fsi_batch* b, unsigned flags) {
  std::vector<std::string> parts;
  for (const fsi_mesh* m : b->meshes) {
    std::ostringstream o;
    o << m->g.nx << "x" << m->g.ny << "x" << m->g.nz << "s" << m->ns;
    parts.push_back(o.str());
  }
  std::sort(parts.begin(), parts.end());
  std::ostringstream k;
  k << "block" << b->block << "_f" << (flags & FSI_FP32 ? 32 : 64) << "_n" << b->n;
  uint64_t h = 1469598103934665603ull;  // FNV-1a of the sorted instance shapes
  for (const auto& p : parts)
    for (char c : p) h = (h ^ (unsigned char)c) * 1099511628211ull;
  k << "_" << std::hex << h;
  return k.str();
}

bool cache_lookup(const std::string& key, int* tm, int* gm) {
  std::ifstream f(cache_path());
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    std::istringstream is(line);
    std::string k;
    int a, c;
    double us;
    if (is >> k >> a >> c >> us && k == key) *tm = a, *gm = c, found = true;
  }
  return found;
}

void cache_store(const std::string& key, int tm, int gm, double us) {
  const std::string path = cache_path();
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos) {
    const std::string dir = path.substr(0, slash);
    mkdir(dir.c_str(), 0755);  // one level; an existing directory is fine
  }
  std::ofstream f(path, std::ios::app);
  if (f) f << key << " " << tm << " " << gm << " " << us << "\n";
}

}  // namespace
}  // namespace fsi

// ====================================================================== C ABI
using namespace fsi;

extern "C" {

int fsi_batch_destroy(fsi_batch* b) {
  if (!b) return FSI_OK;
  if (b->cycle) cudaGraphExecDestroy(b->cycle);
  if (b->net_graph) cudaGraphExecDestroy(b->net_graph);
  for (cudaStream_t st : b->side) cudaStreamDestroy(st);
  for (cudaEvent_t ev : b->join) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  cudaFree(b->zt);
  for (OpSet* s : {&b->jvp_inner, &b->jvp_d, &b->jvp_outer, &b->jvp_user}) cudaFree(s->ops);
  cudaFree(b->nsq_eitems);
  cudaFree(b->nsq_nitems);
  cudaFree(b->Zb);
  cudaFree(b->geoms_dev), cudaFree(b->tiles_dev), cudaFree(b->items_dev), cudaFree(b->item_first_dev);
  cudaFree(b->V), cudaFree(b->vbase_dev), cudaFree(b->off_dev), cudaFree(b->nloc_dev), cudaFree(b->dx32_dev);
  cudaFree(b->w), cudaFree(b->z), cudaFree(b->r), cudaFree(b->t), cudaFree(b->dinv), cudaFree(b->d);
  cudaFree(b->rin), cudaFree(b->rout), cudaFree(b->part), cudaFree(b->K), cudaFree(b->act), cudaFree(b->live);
  cudaFree(b->out_dev);
  cudaFree(b->dx32_own);
  if (b->host_out) cudaFreeHost(b->host_out);
  if (b->host_live) cudaFreeHost(b->host_live);
  delete b;
  return FSI_OK;
}

int fsi_batch_create(fsi_mesh* const* meshes, int32_t n, int32_t block, int32_t m, fsi_batch** out) {
  if (n < 1) return set_error(FSI_EINVAL, "fsi_batch_create: bad arguments");
  std::vector<int32_t> blocks(n, block);
  return fsi_batch_create_blocks(meshes, blocks.data(), n, m, out);
}

int fsi_batch_create_blocks(fsi_mesh* const* meshes, const int32_t* blocks, int32_t n, int32_t m, fsi_batch** out) {
  if (!meshes || !blocks || !out || n < 1) return set_error(FSI_EINVAL, "fsi_batch_create: bad arguments");
  if (m < 1 || m > BMMAX) return set_error(FSI_EINVAL, "fsi_batch_create: restart length must be in 1..64");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!meshes[i]) return set_error(FSI_EINVAL, "fsi_batch_create: null mesh");
    if (meshes[i]->tet) return set_error(FSI_EINVAL, "fsi_batch_create: not on tetrahedral meshes");
    if (meshes[i]->stream != meshes[0]->stream || meshes[i]->dev != meshes[0]->dev)
      return set_error(FSI_EINVAL, "fsi_batch_create: all instances need one device and one stream (fsi_set_stream)");
  }
  auto* b = new fsi_batch();
  auto fail = [&](int rc) {
    fsi_batch_destroy(b);
    return rc;
  };
  b->meshes.assign(meshes, meshes + n);
  b->blocks.assign(blocks, blocks + n);
  b->n = n;
  b->block = blocks[0];
  b->stream = meshes[0]->stream;
  b->mm = m;
  b->M1 = m + 1;
  b->off.assign(n + 1, 0);
  std::vector<int64_t> nloc(n), vbase(n);
  std::vector<int4> items;
  int64_t vtot = 0;
  for (int i = 0; i < n; ++i) {
    BlockInfo bi;
    int rc = block_info(meshes[i], blocks[i], &bi);
    if (rc) return fail(rc);
    if (i == 0) b->blk0 = bi;
    if (bi.kind != b->blk0.kind) return fail(set_error(FSI_EINVAL, "fsi_batch_create: block kinds differ"));
    nloc[i] = bi.n;
    b->off[i + 1] = b->off[i] + bi.n;
    const int64_t nch = (bi.n + BCH - 1) / BCH;
    vbase[i] = vtot;
    vtot += nch * b->M1 * BCH;
    b->item_first.push_back((int)items.size());
    for (int64_t c = 0; c < nch; c += BITEM) items.push_back(make_int4(i, (int)c, (int)std::min(nch, c + BITEM), 0));
  }
  b->item_first.push_back((int)items.size());
  b->ntot = b->off[n];
  b->nitems = (int)items.size();
  int rc;
  auto dmal = [&](auto** p, size_t bytes) -> int {
    FSI_CUDA(cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(bytes, 16)));
    FSI_CUDA(cudaMemset(*p, 0, std::max<size_t>(bytes, 16)));
    return FSI_OK;
  };
  const size_t vb = sizeof(double) * (size_t)b->ntot;
  if ((rc = dmal(&b->V, sizeof(double) * (size_t)vtot)) || (rc = dmal(&b->w, vb)) || (rc = dmal(&b->z, vb)) ||
      (rc = dmal(&b->r, vb)) || (rc = dmal(&b->t, vb)) || (rc = dmal(&b->dinv, vb)) || (rc = dmal(&b->d, vb)) ||
      (rc = dmal(&b->rin, vb)) || (rc = dmal(&b->rout, vb)) ||
      (rc = dmal(&b->part, sizeof(double) * (size_t)b->nitems * PSTRIDE)) || (rc = dmal(&b->K, sizeof(BKry) * n)) ||
      (rc = dmal(&b->act, sizeof(int) * n)) || (rc = dmal(&b->live, sizeof(int) * n)) ||
      (rc = dmal(&b->out_dev, sizeof(double) * 2 * n)) || (rc = dmal(&b->geoms_dev, sizeof(Geom) * n)) ||
      (rc = dmal(&b->items_dev, sizeof(int4) * items.size())) || (rc = dmal(&b->item_first_dev, sizeof(int) * (n + 1))) ||
      (rc = dmal(&b->vbase_dev, sizeof(int64_t) * n)) || (rc = dmal(&b->off_dev, sizeof(int64_t) * n)) ||
      (rc = dmal(&b->nloc_dev, sizeof(int64_t) * n)) || (rc = dmal(&b->dx32_dev, sizeof(float*) * n)))
    return fail(rc);
  if (cudaMallocHost(&b->host_out, sizeof(double) * 2 * n) != cudaSuccess ||
      cudaMallocHost(&b->host_live, sizeof(int) * n) != cudaSuccess)
    return fail(set_error(FSI_ECUDA, "fsi_batch_create: pinned host buffers"));
  if (cudaMemcpy(b->items_dev, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->item_first_dev, b->item_first.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(b->vbase_dev, vbase.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->off_dev, b->off.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->nloc_dev, nloc.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(set_error(FSI_ECUDA, "fsi_batch_create: copying the work lists"));
  int tm = 4, gm = 2;
  cache_lookup(tune_key(b, FSI_FP32), &tm, &gm);
  if ((rc = build_tiles(b, tm, gm)) || (rc = ensure_dx32(b))) return fail(rc);
  *out = b;
  return FSI_OK;
}

int fsi_batch_layout(const fsi_batch* b, int64_t* offsets, int32_t* target_mult, int32_t* grid_mult,
                     int64_t* launches) {
  if (!b) return set_error(FSI_EINVAL, "fsi_batch_layout: null handle");
  if (offsets)
    for (int i = 0; i <= b->n; ++i) offsets[i] = b->off[i];
  if (target_mult) *target_mult = b->target_mult;
  if (grid_mult) *grid_mult = b->grid_mult;
  if (launches) *launches = b->launches;
  return FSI_OK;
}

int fsi_batch_jvp(fsi_batch* b, const fsi_state* states, const double* dx, double* y, uint32_t flags) {
  if (!b || !states || !dx || !y) return set_error(FSI_EINVAL, "fsi_batch_jvp: null argument");
  const bool f32 = flags & FSI_FP32;
  int rc;
  if ((rc = stage_all(b, states, f32))) return rc;
  if (f32)
    BK_LAUNCH(b, P_KRY_CONV, bk_tofloat<<<b->nitems, BVB, 0, b->stream>>>(b->items_dev, nullptr, b->off_dev,
                                                                          b->nloc_dev, dx, b->dx32_dev, 0));
  if ((rc = record_set(b, &b->jvp_user, flags, dx, y))) return rc;
  for (fsi_mesh* m : b->meshes) m->applies++, m->dof_applied += b->off[1] - b->off[0];
  return run_set(b, b->jvp_user, 0);
}

int fsi_batch_gmres(fsi_batch* b, const fsi_state* states, const double* rhs, double* x, const fsi_solve_opts* o,
                    fsi_solve_info* infos) {
  if (!b || !states || !rhs || !x || !o) return set_error(FSI_EINVAL, "fsi_batch_gmres: null argument");
  if (o->m != b->mm) return set_error(FSI_EINVAL, "fsi_batch_gmres: opts.m must equal the batch's restart length");
  if (o->precond != FSI_PC_JACOBI && o->precond != FSI_PC_NONE && o->precond != FSI_PC_LEARNED)
    return set_error(FSI_EINVAL, "fsi_batch_gmres: unknown preconditioner");
  const bool learned = o->precond == FSI_PC_LEARNED;
  if (learned) {
    // flexible GMRES: every entry an NS block with a network attached, on the batch's stream
    for (int i = 0; i < b->n; ++i) {
      fsi_mesh* m = b->meshes[i];
      if (b->blocks[i] != FSI_BLOCK_NS || !m->pc)
        return set_error(FSI_EINVAL, "fsi_batch_gmres: FSI_PC_LEARNED needs NS entries with a network (fsi_set_pc)");
      if (m->stream != b->stream)
        return set_error(FSI_EINVAL, "fsi_batch_gmres: FSI_PC_LEARNED needs every instance on the batch's stream");
    }
    const int64_t zl = (int64_t)b->mm * b->ntot;
    if (b->zb_len < zl) {
      cudaFree(b->Zb);
      b->Zb = nullptr;
      b->zb_len = 0;
      FSI_CUDA(cudaMalloc(&b->Zb, sizeof(double) * (size_t)zl));
      b->zb_len = zl;
    }
    if (!b->zt) FSI_CUDA(cudaMalloc(&b->zt, sizeof(double) * (size_t)std::max<int64_t>(b->ntot, 1)));
    // the networks read this solve's staged states: capture their step again
    if (b->net_graph) cudaGraphExecDestroy(b->net_graph);
    b->net_graph = nullptr;
  }
  b->use_pc = learned ? 1 : 0;
  b->pc_alternate = (learned && (o->flags & FSI_PC_ALTERNATE)) ? 1 : 0;
  const bool f32 = o->precision == FSI_PREC_FP32_IR;
  const unsigned base = o->flags & ~(FSI_FP32 | FSI_HARVEST | FSI_PC_ALTERNATE | FSI_NO_STALL_STOP);
  const unsigned inner = f32 ? (base | FSI_FP32) : base;
  const int nb = b->n, NI = b->nitems;
  cudaStream_t s = b->stream;
  int rc;
  if ((rc = stage_all(b, states, f32))) return rc;
  // Jacobi diagonal of the inner operator, one launch per instance (once per solve)
  for (int i = 0; i < nb; ++i) {
    BlockInfo bi;
    if ((rc = block_info(b->meshes[i], b->blocks[i], &bi))) return rc;
    if (o->precond != FSI_PC_NONE) {  // Jacobi, or the network's input scaling and alternate directions
      if ((rc = op_diag(b->meshes[i], bi, b->dinv + b->off[i], f32 ? (base | FSI_FP32) : base))) return rc;
    } else {
      std::vector<double> ones(bi.n, 1.0);
      FSI_CUDA(cudaMemcpy(b->dinv + b->off[i], ones.data(), sizeof(double) * bi.n, cudaMemcpyHostToDevice));
    }
  }
  if (o->precond != FSI_PC_NONE)
    BK_LAUNCH(b, P_KRYLOV, bk_recip<<<608, 256, 0, s>>>(b->dinv, b->ntot));
  if ((rc = record_set(b, &b->jvp_inner, inner, b->z, b->w)) || (rc = record_set(b, &b->jvp_d, inner, b->d, b->t)))
    return rc;
  std::vector<int> iters(nb, 0), restarts(nb, 0), stalled(nb, 0), refin(nb, 0), fallback(nb, 0);
  std::vector<double> rel(nb, 0.0), inner_rel(nb, 0.0);
  std::vector<int> live(nb, 1);
  if (!f32) {
    FSI_CUDA(cudaMemcpyAsync(b->rin, rhs, sizeof(double) * b->ntot, cudaMemcpyDeviceToDevice, s));
    if ((rc = inner_solve(b, live, o->rtol, o->max_iter, false, iters, restarts, rel, stalled))) return rc;
    FSI_CUDA(cudaMemcpyAsync(x, b->d, sizeof(double) * b->ntot, cudaMemcpyDeviceToDevice, s));
    if (b->use_pc) {
      // instances the flexible solve left above rtol (a stalled network): Jacobi GMRES on
      // their remaining residual (the last cycle's r = rhs - A x), x += d
      std::vector<int> fb(nb, 0);
      double worst = 0.0;
      int nfb = 0;
      for (int i = 0; i < nb; ++i)
        if (rel[i] > o->rtol && iters[i] < o->max_iter) fb[i] = 1, ++nfb, worst = std::max(worst, rel[i]);
      if (nfb) {
        b->use_pc = 0;
        FSI_CUDA(cudaMemcpyAsync(b->rin, b->r, sizeof(double) * b->ntot, cudaMemcpyDeviceToDevice, s));
        std::vector<double> rel2(nb, 0.0);
        std::vector<int> st2(nb, 0);
        if ((rc = inner_solve(b, fb, o->rtol / worst, o->max_iter, false, iters, restarts, rel2, st2))) return rc;
        if ((rc = upload_live(b, fb))) return rc;
        BK_LAUNCH(b, P_KRYLOV, bk_axpy<<<NI, BVB, 0, s>>>(b->items_dev, b->live, b->off_dev, b->nloc_dev, 1.0, b->d,
                                                           x));
        for (int i = 0; i < nb; ++i)
          if (fb[i]) rel[i] *= rel2[i], stalled[i] = st2[i], fallback[i] = 1;
      }
    }
  } else {
    // float32 operator inside float64 refinement: x = 0, r = rhs; repeat: A32 d = r,
    // x += d, r = rhs - A64 x
    if ((rc = record_set(b, &b->jvp_outer, base, x, b->t))) return rc;
    FSI_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * b->ntot, s));
    if ((rc = upload_live(b, live))) return rc;
    BK_LAUNCH(b, P_KRYLOV, bk_copy_norm<<<NI, BVB, 0, s>>>(b->items_dev, nullptr, b->off_dev, b->nloc_dev, rhs,
                                                            b->rout, b->part));
    BK_LAUNCH(b, P_KRYLOV, bk_rn2<<<gx1(nb), 128, 0, s>>>(b->item_first_dev, b->part, b->K, nullptr, nb, b->out_dev));
    if ((rc = read_out(b))) return rc;
    std::vector<double> bn(nb), prev(nb, 1.0);
    for (int i = 0; i < nb; ++i) {
      bn[i] = std::sqrt(b->host_out[i]);
      if (!std::isfinite(bn[i])) return set_error(FSI_ENAN, "batch IR: right-hand side is not finite");
      rel[i] = bn[i] > 0.0 ? 1.0 : 0.0;
      live[i] = bn[i] > 0.0;
    }
    for (int k = 0; k < std::max(1, o->ir_max); ++k) {
      int nlive = 0;
      for (int i = 0; i < nb; ++i) {
        if (live[i] && (rel[i] <= o->rtol || iters[i] >= o->max_iter)) live[i] = 0;
        nlive += live[i];
      }
      if (!nlive) break;
      FSI_CUDA(cudaMemcpyAsync(b->rin, b->rout, sizeof(double) * b->ntot, cudaMemcpyDeviceToDevice, s));
      std::vector<int> st_in(nb, 0);
      if ((rc = inner_solve(b, live, o->ir_inner_rtol, o->max_iter, true, iters, restarts, inner_rel, st_in)))
        return rc;
      if ((rc = upload_live(b, live))) return rc;
      BK_LAUNCH(b, P_KRYLOV, bk_axpy<<<NI, BVB, 0, s>>>(b->items_dev, b->live, b->off_dev, b->nloc_dev, 1.0, b->d, x));
      if ((rc = run_set(b, b->jvp_outer, 2))) return rc;
      BK_LAUNCH(b, P_KRYLOV, bk_resid<<<NI, BVB, 0, s>>>(b->items_dev, b->live, b->off_dev, b->nloc_dev, rhs, b->t,
                                                          b->rout, b->part));
      BK_LAUNCH(b, P_KRYLOV, bk_rn2<<<gx1(nb), 128, 0, s>>>(b->item_first_dev, b->part, b->K, b->live, nb,
                                                             b->out_dev));
      if ((rc = read_out(b))) return rc;
      bool pc_stalled = false;
      for (int i = 0; i < nb; ++i) {
        if (!live[i]) continue;
        const double r2 = b->host_out[i];
        if (!std::isfinite(r2)) return set_error(FSI_ENAN, "batch IR: residual is not finite");
        prev[i] = rel[i];
        rel[i] = std::sqrt(r2) / bn[i];
        refin[i] = k + 1;
        const bool no_gain = rel[i] > o->rtol && rel[i] > 0.9 * prev[i];
        if (b->use_pc && (st_in[i] || no_gain)) {
          pc_stalled = true;  // the network failed its inner solve: Jacobi from here on
          fallback[i] = 1;
          continue;
        }
        if (no_gain) live[i] = 0, stalled[i] = 1;
      }
      if (pc_stalled) b->use_pc = 0;
    }
  }
  bool all = true;
  for (int i = 0; i < nb; ++i) {
    if (infos) {
      infos[i] = fsi_solve_info{};
      infos[i].iterations = iters[i];
      infos[i].restarts = restarts[i];
      infos[i].refinements = refin[i];
      infos[i].applies = iters[i] + restarts[i] + refin[i];
      infos[i].rel_res = rel[i];
      infos[i].stalled = stalled[i];
      infos[i].fallback = fallback[i];
    }
    all = all && rel[i] <= o->rtol;
  }
  b->use_pc = 0;
  FSI_CUDA(cudaStreamSynchronize(s));
  if (!all) return set_error(FSI_ENOCONV, "batch GMRES: tolerance not reached by every instance");
  return FSI_OK;
}

int fsi_batch_autotune(fsi_batch* b, const fsi_state* states, uint32_t flags, int32_t* target_mult,
                       int32_t* grid_mult, double* best_us) {
  if (!b || !states) return set_error(FSI_EINVAL, "fsi_batch_autotune: null argument");
  cudaStream_t s = b->stream;
  int rc;
  const bool f32 = flags & FSI_FP32;
  if ((rc = stage_all(b, states, f32))) return rc;
  BK_LAUNCH(b, P_KRYLOV, bk_zero<<<b->nitems, BVB, 0, s>>>(b->items_dev, nullptr, b->off_dev, b->nloc_dev, b->z));
  if (f32)
    BK_LAUNCH(b, P_KRY_CONV, bk_tofloat<<<b->nitems, BVB, 0, s>>>(b->items_dev, nullptr, b->off_dev, b->nloc_dev,
                                                                  b->z, b->dx32_dev, 0));
  // the two timing events, destroyed on every return
  struct Events {
    cudaEvent_t e[2] = {nullptr, nullptr};
    ~Events() {
      for (cudaEvent_t x : e)
        if (x) cudaEventDestroy(x);
    }
  } ev;
  FSI_CUDA(cudaEventCreate(&ev.e[0]));
  FSI_CUDA(cudaEventCreate(&ev.e[1]));
  cudaEvent_t e0 = ev.e[0], e1 = ev.e[1];
  double best = 1e300;
  int btm = b->target_mult, bgm = b->grid_mult;
  for (int tm : {1, 2, 4, 8})
    for (int gm : {1, 2, 4}) {
      if ((rc = build_tiles(b, tm, gm)) || (rc = record_set(b, &b->jvp_user, flags, b->z, b->w))) return rc;
      for (int w = 0; w < 2; ++w)
        if ((rc = run_set(b, b->jvp_user, 0))) return rc;
      FSI_CUDA(cudaEventRecord(e0, s));
      for (int r = 0; r < 5; ++r)
        if ((rc = run_set(b, b->jvp_user, 0))) return rc;
      FSI_CUDA(cudaEventRecord(e1, s));
      FSI_CUDA(cudaEventSynchronize(e1));
      float ms = 0.0f;
      FSI_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      const double us = 1e3 * ms / 5.0;
      if (us < best) best = us, btm = tm, bgm = gm;
    }
  if ((rc = build_tiles(b, btm, bgm))) return rc;
  cache_store(tune_key(b, flags), btm, bgm, best);
  if (target_mult) *target_mult = btm;
  if (grid_mult) *grid_mult = bgm;
  if (best_us) *best_us = best;
  return FSI_OK;
}

int fsi_batch_set_graph(fsi_batch* b, int32_t use_graph) {
  if (!b) return set_error(FSI_EINVAL, "fsi_batch_set_graph: null handle");
  b->use_graph = use_graph ? 1 : 0;
  return FSI_OK;
}

}  // extern "C"

// ================================================================ batched time steps
// Partitioned time steps (Section 2.5) of many independent instances at once: every
// block solve of a nonlinear iteration is one batched solve over all instances (NS),
// over all (instance, phase) pairs (the Allen-Cahn blocks of different phases do not
// depend on each other, so all N phases of all instances are one batch), and over all
// (instance, solid) pairs (B).  An instance whose blocks have all met the nonlinear
// tolerance gets a zero right-hand side from then on and drops out of the solves.
struct fsi_batch_stepper {
  std::vector<fsi_mesh*> meshes;
  int n = 0;
  fsi_batch* ns = nullptr;
  fsi_batch* ac = nullptr;
  fsi_batch* bb = nullptr;
  std::vector<int> ac_inst, b_inst;  // instance of each AC / B entry
  double* rhs = nullptr;             // largest concatenated block vector
  double* dx = nullptr;
};

namespace fsi {
namespace {

// rhs segment of every entry: -R_block of a live instance, zero otherwise
int batch_rhs(fsi_batch* b, const std::vector<int>& inst, const std::vector<int>& live, fsi_state* states, bool f32,
              double* rhs, bool ns_unpinned, unsigned flags) {
  int last = -1;
  for (int e = 0; e < b->n; ++e) {
    fsi_mesh* m = b->meshes[e];
    const int i = inst[e];
    BlockInfo bi;
    int rc = block_info(m, b->blocks[e], &bi);
    if (rc) return rc;
    double* r = rhs + b->off[e];
    if (!live[i]) {
      FSI_CUDA(cudaMemsetAsync(r, 0, sizeof(double) * bi.n, m->stream));
      continue;
    }
    if (i != last && (rc = stage(m, &states[i], f32))) return rc;
    last = i;
    if (bi.kind == 1) {
      double gb[2];
      if ((rc = op_coeffs(m, bi.index, gb))) return rc;
      m->gamma[bi.index] = m->fixed_gamma[bi.index] >= 0.0 ? m->fixed_gamma[bi.index] : gb[0];
      m->beta[bi.index] = gb[1];
    }
    PinGuard guard(m, (ns_unpinned && bi.kind == 0 && shifts_pressure(m, flags)) ? 0 : m->pin_active);
    if ((rc = op_residual(m, bi, r))) return rc;
    if ((rc = vec_scale_copy(m, -1.0, r, r, bi.n))) return rc;
  }
  return FSI_OK;
}

// x_block += dx of every live entry (NS: after the pressure shift), and the largest
// |dx_blk| / |x_blk| of each instance
int batch_update(fsi_batch* b, const std::vector<int>& inst, const std::vector<int>& live, fsi_state* states,
                 double* dx, std::vector<double>& ratio, unsigned flags) {
  for (int e = 0; e < b->n; ++e) {
    const int i = inst[e];
    if (!live[i]) continue;
    fsi_mesh* m = b->meshes[e];
    BlockInfo bi;
    int rc = block_info(m, b->blocks[e], &bi);
    if (rc) return rc;
    double* d = dx + b->off[e];
    if (bi.kind == 0 && shifts_pressure(m, flags) && (rc = pin_shift(m, states[i].x, d))) return rc;
    double* xb = states[i].x + (int64_t)bi.c0 * m->nn;
    if ((rc = vec_axpy(m, 1.0, d, xb, bi.n))) return rc;
    double d2, x2;
    if ((rc = vec_dot(m, d, d, bi.n, &d2)) || (rc = vec_dot(m, xb, xb, bi.n, &x2))) return rc;
    if (!std::isfinite(d2) || !std::isfinite(x2)) return set_error(FSI_ENAN, "fsi_batch_step: solution is not finite");
    ratio[i] = std::max(ratio[i], x2 > 0.0 ? std::sqrt(d2 / x2) : std::sqrt(d2));
  }
  return FSI_OK;
}

// one batched block solve of the live instances; per-instance statistics into infos
int batch_block(fsi_batch* b, const std::vector<int>& inst, const std::vector<int>& live, fsi_state* states,
                const fsi_solve_opts& o, double* rhs, double* dx, std::vector<double>& ratio, fsi_step_info* infos,
                int kind) {
  if (!b) return FSI_OK;
  const bool f32 = o.precision == FSI_PREC_FP32_IR;
  int rc;
  if ((rc = batch_rhs(b, inst, live, states, f32, rhs, kind == 0, o.flags))) return rc;
  std::vector<fsi_state> est(b->n);
  for (int e = 0; e < b->n; ++e) est[e] = states[inst[e]];
  std::vector<fsi_solve_info> si(b->n);
  {
    // the NS entries keep their pin node's continuity equation for the whole solve
    std::vector<PinGuard*> guards;
    for (int e = 0; e < b->n; ++e)
      if (kind == 0 && shifts_pressure(b->meshes[e], o.flags)) guards.push_back(new PinGuard(b->meshes[e], 0));
    rc = fsi_batch_gmres(b, est.data(), rhs, dx, &o, si.data());
    for (PinGuard* g : guards) delete g;
    if (rc && rc != FSI_ENOCONV) return rc;
  }
  for (int e = 0; e < b->n; ++e) {
    const int i = inst[e];
    if (!live[i]) continue;
    fsi_step_info& inf = infos[i];
    inf.worst_rel_res = std::max(inf.worst_rel_res, si[e].rel_res);
    if (si[e].stalled) inf.stalled_solves++;
    if (kind == 0) inf.gmres_iters_ns += si[e].iterations;
    else if (kind == 1) inf.gmres_iters_ac += si[e].iterations;
    else inf.gmres_iters_b += si[e].iterations;
    // the batched products of this entry, counted on its mesh like single-mesh applies
    b->meshes[e]->applies += si[e].applies;
    b->meshes[e]->dof_applied += (int64_t)si[e].applies * (b->off[e + 1] - b->off[e]);
  }
  return batch_update(b, inst, live, states, dx, ratio, o.flags);
}

}  // namespace
}  // namespace fsi

extern "C" {

int fsi_batch_stepper_destroy(fsi_batch_stepper* s) {
  if (!s) return FSI_OK;
  fsi_batch_destroy(s->ns);
  fsi_batch_destroy(s->ac);
  fsi_batch_destroy(s->bb);
  cudaFree(s->rhs);
  cudaFree(s->dx);
  delete s;
  return FSI_OK;
}

int fsi_batch_stepper_create(fsi_mesh* const* meshes, int32_t n, int32_t m, fsi_batch_stepper** out) {
  if (!meshes || !out || n < 1) return set_error(FSI_EINVAL, "fsi_batch_stepper_create: bad arguments");
  *out = nullptr;
  auto* s = new fsi_batch_stepper();
  s->meshes.assign(meshes, meshes + n);
  s->n = n;
  int rc = fsi_batch_create(meshes, n, FSI_BLOCK_NS, m, &s->ns);
  std::vector<fsi_mesh*> am, bm;
  std::vector<int32_t> ab, bbk;
  for (int i = 0; i < n && !rc; ++i) {
    if (!meshes[i]) rc = set_error(FSI_EINVAL, "fsi_batch_stepper_create: null mesh");
    else {
      for (int p = 0; p < meshes[i]->N; ++p) am.push_back(meshes[i]), ab.push_back(FSI_BLOCK_AC(p)), s->ac_inst.push_back(i);
      for (int q = 0; q < meshes[i]->ns; ++q) bm.push_back(meshes[i]), bbk.push_back(FSI_BLOCK_B(q)), s->b_inst.push_back(i);
    }
  }
  if (!rc && !am.empty()) rc = fsi_batch_create_blocks(am.data(), ab.data(), (int32_t)am.size(), m, &s->ac);
  if (!rc && !bm.empty()) rc = fsi_batch_create_blocks(bm.data(), bbk.data(), (int32_t)bm.size(), m, &s->bb);
  if (!rc) {
    int64_t cap = s->ns->ntot;
    if (s->ac) cap = std::max(cap, s->ac->ntot);
    if (s->bb) cap = std::max(cap, s->bb->ntot);
    if (cudaMalloc(&s->rhs, sizeof(double) * cap) != cudaSuccess || cudaMalloc(&s->dx, sizeof(double) * cap) != cudaSuccess)
      rc = set_error(FSI_ECUDA, "fsi_batch_stepper_create: work vectors");
  }
  if (rc) {
    fsi_batch_stepper_destroy(s);
    return rc;
  }
  *out = s;
  return FSI_OK;
}

int fsi_batch_step(fsi_batch_stepper* s, fsi_state* states, const fsi_step_opts* o, fsi_step_info* infos) {
  if (!s || !states || !o || !infos) return set_error(FSI_EINVAL, "fsi_batch_step: null argument");
  if (o->k_max < 1) return set_error(FSI_EINVAL, "fsi_batch_step: k_max must be >= 1");
  if (o->solve.precond != FSI_PC_JACOBI && o->solve.precond != FSI_PC_NONE && o->solve.precond != FSI_PC_LEARNED)
    return set_error(FSI_EINVAL, "fsi_batch_step: unknown preconditioner");
  // the network preconditions the NS blocks; the Allen-Cahn and B blocks use Jacobi
  fsi_solve_opts other = o->solve;
  if (other.precond == FSI_PC_LEARNED) other.precond = FSI_PC_JACOBI;
  const int n = s->n;
  std::vector<int64_t> a0(n), d0(n);
  int rc;
  for (int i = 0; i < n; ++i) {
    infos[i] = fsi_step_info{};
    a0[i] = s->meshes[i]->applies;
    d0[i] = s->meshes[i]->dof_applied;
    if (!states[i].x || !states[i].xn || !states[i].xdn) return set_error(FSI_EINVAL, "fsi_batch_step: null state");
    if ((rc = step_predict(s->meshes[i], &states[i]))) return rc;
  }
  std::vector<int> live(n, 1), ns_inst(n);
  for (int i = 0; i < n; ++i) ns_inst[i] = i;
  for (int k = 0; k < o->k_max; ++k) {
    std::vector<double> ratio(n, 0.0);
    if ((rc = batch_block(s->ns, ns_inst, live, states, o->solve, s->rhs, s->dx, ratio, infos, 0)) ||
        (rc = batch_block(s->ac, s->ac_inst, live, states, other, s->rhs, s->dx, ratio, infos, 1)) ||
        (rc = batch_block(s->bb, s->b_inst, live, states, other, s->rhs, s->dx, ratio, infos, 2)))
      return rc;
    int nlive = 0;
    for (int i = 0; i < n; ++i) {
      if (!live[i]) continue;
      infos[i].nl_iters = k + 1;
      infos[i].max_ratio = ratio[i];
      if (!o->fixed_iters && ratio[i] < o->nl_tol) live[i] = 0;
      nlive += live[i];
    }
    if (!nlive) break;
  }
  for (int i = 0; i < n; ++i)
    if ((rc = step_correct(s->meshes[i], &states[i]))) return rc;
  FSI_CUDA(cudaStreamSynchronize(s->ns->stream));
  for (int i = 0; i < n; ++i) {
    infos[i].applies = (int)(s->meshes[i]->applies - a0[i]);
    infos[i].dof_applied = s->meshes[i]->dof_applied - d0[i];
  }
  return FSI_OK;
}

}  // extern "C"
