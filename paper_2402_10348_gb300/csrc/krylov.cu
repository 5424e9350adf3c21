// Krylov solver of libfsi: restarted right-preconditioned GMRES(m) (the paper's
// linear solver, Section 2.5) on float64 vectors, optionally with a float32 operator
// inside float64 iterative refinement; the inner solves of the refinement keep their
// Arnoldi basis in float32 (Hessenberg, Givens and every residual stay float64).
//
// Basis layout: the vectors V_0..V_m are stored chunk-interleaved, CH = 256
// elements per chunk, all m+1 vectors of a chunk contiguous:
//     V_i[j] = V[(j / CH) * (M1 * CH) + i * CH + j % CH],   M1 = slots per chunk.
// A CTA of the projection kernels walks whole chunks, so it streams one contiguous
// block of k x 2 KiB per chunk instead of k separate streams 8.8 MB apart (measured
// 3.9 vs 2.7 TB/s read on GB300 for 33 vectors of the 64^3 NS block).
//
// Arnoldi step j (D = diag(dinv)):
//   w = J z, z = D V_j    (z written together with V_j; w: a contiguous work vector
//                          written by the operator)
//   h = V^T w and |w|^2 in one pass over V_0..V_j      (mdot_kernel)
//   w -= V h, |w|^2 and h2 = V^T w (the second pass's projections of the updated w)
//   in one pass                                           (upd_dot_kernel)
//   if |w_new| < |w_old| / sqrt(2): w -= V h2 (classical Gram-Schmidt with the DGKS
//   re-orthogonalization test; that update is launched always and exits at once when
//   the device-side flag says it is not needed)
//   Givens rotation of the new Hessenberg column and the residual estimate on the
//   device; V_{j+1} = w / |w| stored into its slot, and z = D V_{j+1} beside it.
// The host enqueues step j and only then waits for step j-1's residual estimate
// (copied to pinned memory), so it never stalls the GPU between steps; at most one
// step beyond convergence is computed and ignored.  The least-squares solution and
// x += D V y are device kernels.  One host synchronisation per restart recomputes
// the true residual b - A x.  All reductions use a fixed partition and a fixed
// summation order (bit-reproducible).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "pcnet.h"

namespace fsi {

constexpr int VB = 256;   // threads per CTA of the vector kernels
constexpr int CH = 256;   // elements per basis chunk (one per thread)
constexpr int DCH = 16;   // dot products per CTA pass
constexpr int MMAX = 64;  // largest restart length

static int vgrid(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + VB * 4 - 1) / (VB * 4), 152 * 4));
}
// two CTAs per SM: each streams enough chunks to amortise its end-of-kernel
// reduction of up to 16 sums (the reduction dominated at four CTAs per SM)
static int cgrid(int64_t nch) { return (int)std::max<int64_t>(1, std::min<int64_t>(nch, 152 * 2)); }
// the float32-basis kernels reduce in float32 up to the CTA (cheap): four CTAs per SM
// keep more loads in flight
template <typename VT>
static int cgrid_t(int64_t nch) {
  return sizeof(VT) == 4 ? (int)std::max<int64_t>(1, std::min<int64_t>(nch, 152 * 4)) : cgrid(nch);
}
// the basis store: a few chunks of 256 elements per CTA, eight CTAs per SM
static int chunk_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + CH - 1) / CH, 152 * 8)); }

// device-resident Arnoldi/Givens state (inside fsi_mesh::kry_dev)
struct KryDev {
  double h[MMAX + 2];      // current column (pass 1), then the accumulated column
  double h2[MMAX + 2];     // second pass
  double H[(MMAX + 1) * MMAX];
  double cs[MMAX], sn[MMAX], g[MMAX + 1], y[MMAX];
  double nrm_old, nrm_new, nrm_fin;
  double bnorm;
  double est;              // |g_{j+1}| / |b|
  int reorth;              // est, reorth, breakdown: one 16-byte copy to the host per step
  int breakdown;
  unsigned counter;        // CTAs done in sum_partials_decide (back to 0 after each use)
};

template <int K>
__device__ __forceinline__ void block_reduce_store(double (&acc)[K], int kc, double* out, int stride) {
  __shared__ double sm[K][VB / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    double v = acc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sm[i][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < kc) {
    double s = 0.0;
    for (int wi = 0; wi < VB / 32; ++wi) s += sm[threadIdx.x][wi];
    out[threadIdx.x * stride] = s;
  }
}

// The same for many float64 values with fewer float64 adds (this GPU issues them at a
// small fraction of the float32 rate; a plain shuffle tree costs 5 adds a lane per value).
// Inside a warp a transposing butterfly takes the first P values (P the largest power of
// two <= K, at most 32): at shuffle distance 16 a lane keeps half of its values and adds
// its partner's copy of that half, at distance 8 half of that half, and so on; after
// log2 P levels the lane holds value number lane >> (5 - log2 P) summed over the lanes
// that differ from it in the top log2 P bits, and plain shuffles over the remaining bits
// finish the warp's sum (P - 1 + 5 - log2 P adds a lane).  Values past P take plain trees.
template <int K>
__device__ __forceinline__ void block_reduce_store_bf(double (&acc)[K], int kc, double* out, int stride) {
  constexpr int P = K >= 32 ? 32 : K >= 16 ? 16 : K >= 8 ? 8 : K >= 4 ? 4 : K >= 2 ? 2 : 1;
  constexpr int L = P == 32 ? 5 : P == 16 ? 4 : P == 8 ? 3 : P == 4 ? 2 : P == 2 ? 1 : 0;
  __shared__ double smb[K][VB / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double a[P];
#pragma unroll
  for (int q = 0; q < P; ++q) a[q] = acc[q];
#pragma unroll
  for (int l = 0; l < L; ++l) {
    const int o = 16 >> l;
    const int half = P >> (l + 1);
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int q = 0; q < half; ++q) {
      const double send = up ? a[q] : a[q + half];  // the half the partner keeps
      const double keep = up ? a[q + half] : a[q];
      a[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  double s = a[0];
#pragma unroll
  for (int o = 16 >> L; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((lane & ((32 >> L) - 1)) == 0) smb[lane >> (5 - L)][warp] = s;
#pragma unroll
  for (int i = P; i < K; ++i) {
    double v = acc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) smb[i][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < kc) {
    double t = 0.0;
    for (int wi = 0; wi < VB / 32; ++wi) t += smb[threadIdx.x][wi];
    out[threadIdx.x * stride] = t;
  }
}

// The same in float32 up to the CTA's sums, which are stored as float64: this GPU
// issues float64 adds at 1/64 of the float32 rate, so a float64 tree over every
// thread's sums costs more than the float32 basis kernel's streaming.
template <int K>
__device__ __forceinline__ void block_reduce_store_f(float (&acc)[K], int kc, double* out, int stride) {
  __shared__ float smf[K][VB / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    float v = acc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) smf[i][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < kc) {
    float s = 0.f;
    for (int wi = 0; wi < VB / 32; ++wi) s += smf[threadIdx.x][wi];
    out[threadIdx.x * stride] = (double)s;
  }
}

// --------------------------------------------------------- basis (chunked) kernels
// The basis type VT is double for float64 solves and float for the inner solves of
// iterative refinement (a float32 operator inside float64 refinement: the inner solve
// only has to reduce its residual by ir_inner_rtol, far above float32 rounding, and the
// refinement's float64 residual removes what the inner solve leaves).  Products and
// per-thread sums are taken in VT, the sums across threads and CTAs in float64.  The work
// vector w, the preconditioner diagonal and every vector outside the basis stay float64.

// part[(ib + i) * G + cta] = sum over the CTA's chunks of V_{ib+i} . w, i < KC,
// ib = i0 + KC * blockIdx.y; with SELF the KC+1-th row is w . w (row i0 + KC).
template <int KC, bool SELF, typename VT>
__global__ void __launch_bounds__(VB) mdot_kernel(const VT* __restrict__ V, int M1, int i0,
                                                  const double* __restrict__ w, int64_t n, double* part,
                                                  const int* skip) {
  if (skip && !*skip) return;
  constexpr int NA = KC + (SELF ? 1 : 0);
  constexpr int NR = NA > 0 ? NA : 1;
  const int G = gridDim.x;
  const int ib = i0 + blockIdx.y * KC;
  const int64_t nch = (n + CH - 1) / CH;
  const int64_t per = (nch + G - 1) / G;
  const int64_t c0 = blockIdx.x * per, c1 = min(nch, c0 + per);
  VT acc[NR];
#pragma unroll
  for (int i = 0; i < NR; ++i) acc[i] = VT(0);
  for (int64_t c = c0; c < c1; ++c) {
    const int64_t j = c * CH + threadIdx.x;
    if (j >= n) break;
    const VT wj = (VT)w[j];
    const VT* blk = V + c * (int64_t)M1 * CH + (int64_t)ib * CH + threadIdx.x;
#pragma unroll
    for (int i = 0; i < KC; ++i) acc[i] += blk[i * CH] * wj;
    if (SELF) acc[NA - 1] += wj * wj;
  }
  double accd[NR];
#pragma unroll
  for (int i = 0; i < NR; ++i) accd[i] = (double)acc[i];
  block_reduce_store_bf<NR>(accd, NA, part + (int64_t)ib * G + blockIdx.x, G);
}

// The float32 basis: the same projections with 16-byte loads.  A CTA works on four
// chunks at a time, a thread on four adjacent elements of one chunk (one float4 per
// basis vector), so a warp moves as many bytes per load as with a float64 basis and
// keeps as many in flight.  Elements at or past n (the ragged end of the last chunk,
// whose basis slots hold stale bytes) are never read.
template <int KC, bool SELF>
__global__ void __launch_bounds__(VB) mdot4_kernel(const float* __restrict__ V, int M1, int i0,
                                                   const double* __restrict__ w, int64_t n, double* part,
                                                   const int* skip) {
  if (skip && !*skip) return;
  constexpr int NA = KC + (SELF ? 1 : 0);
  constexpr int NR = NA > 0 ? NA : 1;
  const int G = gridDim.x;
  const int ib = i0 + blockIdx.y * KC;
  const int64_t nch = (n + CH - 1) / CH;
  const int64_t per = (nch + G - 1) / G;
  const int64_t c0 = blockIdx.x * per, c1 = min(nch, c0 + per);
  const int sub = threadIdx.x >> 6;       // which of the CTA's four chunks
  const int e0 = (threadIdx.x & 63) * 4;  // first of the thread's four elements
  float acc[NR];
#pragma unroll
  for (int i = 0; i < NR; ++i) acc[i] = 0.f;
  for (int64_t c = c0 + sub; c < c1; c += 4) {
    const int64_t j = c * CH + e0;
    if (j >= n) break;
    const float* blk = V + c * (int64_t)M1 * CH + (int64_t)ib * CH + e0;
    float w0, w1, w2, w3;
    if (j + 4 <= n) {
      const double2 a = *reinterpret_cast<const double2*>(w + j);
      const double2 b = *reinterpret_cast<const double2*>(w + j + 2);
      w0 = (float)a.x, w1 = (float)a.y, w2 = (float)b.x, w3 = (float)b.y;
#pragma unroll
      for (int i = 0; i < KC; ++i) {
        const float4 v = *reinterpret_cast<const float4*>(blk + i * CH);
        acc[i] += (v.x * w0 + v.y * w1) + (v.z * w2 + v.w * w3);
      }
    } else {
      w0 = (float)w[j];
      w1 = j + 1 < n ? (float)w[j + 1] : 0.f;
      w2 = j + 2 < n ? (float)w[j + 2] : 0.f;
      w3 = 0.f;
#pragma unroll
      for (int i = 0; i < KC; ++i) {
        const float* p = blk + i * CH;
        float t = p[0] * w0;
        if (j + 1 < n) t += p[1] * w1;
        if (j + 2 < n) t += p[2] * w2;
        acc[i] += t;
      }
    }
    if (SELF) acc[NA - 1] += (w0 * w0 + w1 * w1) + (w2 * w2 + w3 * w3);
  }
  block_reduce_store_f<NR>(acc, NA, part + (int64_t)ib * G + blockIdx.x, G);
}

// out[i] = sum_c part[i*G + c] (fixed order), i = blockIdx.x
__global__ void sum_partials(const double* __restrict__ part, int G, double* out, const int* skip) {
  if (skip && !*skip) return;
  const int i = blockIdx.x;
  double s = 0.0;
  for (int c = threadIdx.x; c < G; c += VB) s += part[(int64_t)i * G + c];
  double acc[1] = {s};
  __shared__ double res;
  block_reduce_store<1>(acc, 1, &res, 1);
  __syncthreads();
  if (threadIdx.x == 0) out[i] = res;
}

// sum_{i<k} hs_i V_i[j] for the element of this thread in chunk blk (8 loads in flight)
template <typename VT>
__device__ __forceinline__ VT lin_comb_chunk(const VT* __restrict__ hs, const VT* __restrict__ blk, int k) {
  VT p[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int i = 0;
  for (; i + 8 <= k; i += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) p[u] += hs[i + u] * blk[(i + u) * CH];
  }
  for (; i < k; ++i) p[0] += hs[i] * blk[i * CH];
  return ((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7]));
}

// w -= sum_{i<k} h_i V_i ; part[cta] = partial of |w|^2   (w contiguous).  One fused
// multiply-add per basis element, chained on the element's value of w (no partial sums
// to add up afterwards: float64 adds are scarce on this GPU); the element's values of up
// to UPB basis vectors are loaded ahead of the chain.
constexpr int UPB = 32;
template <typename VT>
__global__ void __launch_bounds__(VB, 2) upd_kernel(double* __restrict__ w, const VT* __restrict__ V, int M1, int k,
                                                    const double* __restrict__ h, int64_t n, double* part,
                                                    const int* skip) {
  if (skip && !*skip) return;
  __shared__ VT nh[MMAX + 2];
  for (int i = threadIdx.x; i < k; i += VB) nh[i] = -(VT)h[i];
  __syncthreads();
  const int G = gridDim.x;
  const int64_t nch = (n + CH - 1) / CH;
  const int64_t per = (nch + G - 1) / G;
  const int64_t c0 = blockIdx.x * per, c1 = min(nch, c0 + per);
  VT nrm = VT(0);
  for (int64_t c = c0; c < c1; ++c) {
    const int64_t j = c * CH + threadIdx.x;
    if (j >= n) break;
    const VT* blk = V + c * (int64_t)M1 * CH + threadIdx.x;
    VT s = (VT)w[j];
    for (int i0 = 0; i0 < k; i0 += UPB) {
      const int cnt = min(UPB, k - i0);
      VT v[UPB];
#pragma unroll
      for (int u = 0; u < UPB; ++u) v[u] = u < cnt ? blk[(int64_t)(i0 + u) * CH] : VT(0);
#pragma unroll
      for (int u = 0; u < UPB; ++u) {
        if (u >= cnt) break;
        s = fma(nh[i0 + u], v[u], s);
      }
    }
    w[j] = (double)s;
    nrm = fma(s, s, nrm);
  }
  double nd[1] = {(double)nrm};
  block_reduce_store<1>(nd, 1, part + blockIdx.x, 1);
}

// The second-pass update for the float32 basis, laid out as mdot4_kernel: a CTA works on
// four chunks at a time, a thread on four adjacent elements (one float4 per basis vector,
// two double2 of w).  part[cta] = partial of |w|^2 (float32 up to the CTA's sum).
__global__ void __launch_bounds__(VB) upd4_kernel(double* __restrict__ w, const float* __restrict__ V, int M1, int k,
                                                  const double* __restrict__ h, int64_t n, double* part,
                                                  const int* skip) {
  if (skip && !*skip) return;
  __shared__ float hs[MMAX + 2];
  for (int i = threadIdx.x; i < k; i += VB) hs[i] = (float)h[i];
  __syncthreads();
  const int G = gridDim.x;
  const int64_t nch = (n + CH - 1) / CH;
  const int64_t per = (nch + G - 1) / G;
  const int64_t c0 = blockIdx.x * per, c1 = min(nch, c0 + per);
  const int sub = threadIdx.x >> 6;
  const int e0 = (threadIdx.x & 63) * 4;
  float nrm = 0.f;
  for (int64_t c = c0 + sub; c < c1; c += 4) {
    const int64_t j = c * CH + e0;
    if (j >= n) break;
    const float* blk = V + c * (int64_t)M1 * CH + e0;
    if (j + 4 <= n) {
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
      int i = 0;
      for (; i + 2 <= k; i += 2) {
        const float4 v0 = *reinterpret_cast<const float4*>(blk + i * CH);
        const float4 v1 = *reinterpret_cast<const float4*>(blk + (i + 1) * CH);
        a.x += hs[i] * v0.x; a.y += hs[i] * v0.y; a.z += hs[i] * v0.z; a.w += hs[i] * v0.w;
        b.x += hs[i + 1] * v1.x; b.y += hs[i + 1] * v1.y; b.z += hs[i + 1] * v1.z; b.w += hs[i + 1] * v1.w;
      }
      if (i < k) {
        const float4 v0 = *reinterpret_cast<const float4*>(blk + i * CH);
        a.x += hs[i] * v0.x; a.y += hs[i] * v0.y; a.z += hs[i] * v0.z; a.w += hs[i] * v0.w;
      }
      const double2 w01 = *reinterpret_cast<const double2*>(w + j);
      const double2 w23 = *reinterpret_cast<const double2*>(w + j + 2);
      const float s0 = (float)w01.x - (a.x + b.x), s1 = (float)w01.y - (a.y + b.y);
      const float s2 = (float)w23.x - (a.z + b.z), s3 = (float)w23.y - (a.w + b.w);
      *reinterpret_cast<double2*>(w + j) = make_double2((double)s0, (double)s1);
      *reinterpret_cast<double2*>(w + j + 2) = make_double2((double)s2, (double)s3);
      nrm += (s0 * s0 + s1 * s1) + (s2 * s2 + s3 * s3);
    } else {
      for (int e = 0; e < 4 && j + e < n; ++e) {
        float acc = 0.f;
        for (int i = 0; i < k; ++i) acc += hs[i] * blk[i * CH + e];
        const float se = (float)w[j + e] - acc;
        w[j + e] = (double)se;
        nrm += se * se;
      }
    }
  }
  float acc[1] = {nrm};
  block_reduce_store_f<1>(acc, 1, part + blockIdx.x, 1);
}

// Pass-1 update fused with the pass-2 projections: w' = w - sum_{i<k} h_i V_i, the
// partial |w'|^2 and the partial V_i . w' (i < k) of the updated vector, from one read
// of the basis: a thread keeps the k basis values of its element in registers, uses
// them for the update and then for the projections, and accumulates the projections
// in its own shared-memory column; the columns are added once at the end (float64).
// KMAX: k rounded up to a multiple of 8.  Rows of part: i < k the projections, row k
// the norm; part[row * G + cta].
constexpr int UDB = 128;  // threads per CTA (two elements of each 256-element chunk)
static_assert(UDB == 128, "the row sums take four columns per lane");
template <int KMAX, typename VT>
__global__ void __launch_bounds__(UDB) upd_dot_kernel(double* __restrict__ w, const VT* __restrict__ V, int M1,
                                                      int k, const double* __restrict__ h, int64_t n, double* part) {
  extern __shared__ __align__(16) unsigned char upd_smem[];
  VT* sacc = reinterpret_cast<VT*>(upd_smem);  // [KMAX + 1][UDB]
  __shared__ VT nhs[KMAX];
  const int t = threadIdx.x;
  for (int i = t; i < KMAX; i += UDB) nhs[i] = i < k ? -(VT)h[i] : VT(0);
  for (int i = 0; i <= KMAX; ++i) sacc[i * UDB + t] = VT(0);
  __syncthreads();
  const int G = gridDim.x;
  const int64_t nch = (n + CH - 1) / CH;
  const int64_t per = (nch + G - 1) / G;
  const int64_t c0 = blockIdx.x * per, c1 = min(nch, c0 + per);
  VT nrm = VT(0);
  for (int64_t c = c0; c < c1; ++c) {
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
      const int64_t j = c * CH + half * UDB + t;
      if (j >= n) continue;
      const VT* blk = V + c * (int64_t)M1 * CH + half * UDB + t;
      VT v[KMAX];
#pragma unroll
      for (int i = 0; i < KMAX; ++i) v[i] = i < k ? blk[i * CH] : VT(0);
      // one fused multiply-add per basis value, chained on w's value, and none for the
      // padding past k (float64 operations are what this kernel is bound by)
      VT ww = (VT)w[j];
#pragma unroll
      for (int i = 0; i < KMAX; ++i) {
        if (i >= k) break;
        ww = fma(nhs[i], v[i], ww);
      }
      w[j] = (double)ww;
      nrm = fma(ww, ww, nrm);
#pragma unroll
      for (int i = 0; i < KMAX; ++i) {
        if (i >= k) break;
        sacc[i * UDB + t] = fma(v[i], ww, sacc[i * UDB + t]);
      }
    }
  }
  sacc[KMAX * UDB + t] = nrm;
  __syncthreads();
  // one warp per row, lanes on consecutive columns, then a shuffle tree
  const int lane = t & 31;
  for (int i = t >> 5; i <= k; i += UDB / 32) {
    const VT* rp = sacc + (i < k ? i : KMAX) * UDB;
    double s = ((double)rp[lane] + (double)rp[lane + 32]) + ((double)rp[lane + 64] + (double)rp[lane + 96]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) part[(int64_t)i * G + blockIdx.x] = s;
  }
}

// The fused update for the float32 basis: a thread takes two adjacent elements of each
// chunk (one float2 per basis vector, one double2 of w), so a warp moves as many bytes
// per load as with a float64 basis.  Elements at or past n are never read.
template <int KMAX>
__global__ void __launch_bounds__(UDB) upd_dot2_kernel(double* __restrict__ w, const float* __restrict__ V, int M1,
                                                       int k, const double* __restrict__ h, int64_t n, double* part) {
  extern __shared__ __align__(16) unsigned char upd_smem[];
  float* sacc = reinterpret_cast<float*>(upd_smem);  // [KMAX + 1][UDB]
  __shared__ float hs[KMAX];
  const int t = threadIdx.x;
  for (int i = t; i < KMAX; i += UDB) hs[i] = i < k ? (float)h[i] : 0.f;
  for (int i = 0; i <= KMAX; ++i) sacc[i * UDB + t] = 0.f;
  __syncthreads();
  const int G = gridDim.x;
  const int64_t nch = (n + CH - 1) / CH;
  const int64_t per = (nch + G - 1) / G;
  const int64_t c0 = blockIdx.x * per, c1 = min(nch, c0 + per);
  const int e0 = 2 * t;
  float nrm = 0.f;
  for (int64_t c = c0; c < c1; ++c) {
    const int64_t j = c * CH + e0;
    if (j >= n) break;
    const bool pair = j + 2 <= n;
    const float* blk = V + c * (int64_t)M1 * CH + e0;
    float2 v[KMAX];
    if (pair) {
#pragma unroll
      for (int i = 0; i < KMAX; ++i) v[i] = i < k ? *reinterpret_cast<const float2*>(blk + i * CH) : make_float2(0.f, 0.f);
    } else {
#pragma unroll
      for (int i = 0; i < KMAX; ++i) v[i] = make_float2(i < k ? blk[i * CH] : 0.f, 0.f);
    }
    float sx0 = 0.f, sx1 = 0.f, sy0 = 0.f, sy1 = 0.f;
#pragma unroll
    for (int i = 0; i < KMAX; i += 2) {
      sx0 += hs[i] * v[i].x;
      sx1 += hs[i + 1] * v[i + 1].x;
      sy0 += hs[i] * v[i].y;
      sy1 += hs[i + 1] * v[i + 1].y;
    }
    float wx, wy;
    if (pair) {
      const double2 wd = *reinterpret_cast<const double2*>(w + j);
      wx = (float)wd.x - (sx0 + sx1);
      wy = (float)wd.y - (sy0 + sy1);
      *reinterpret_cast<double2*>(w + j) = make_double2((double)wx, (double)wy);
    } else {
      wx = (float)w[j] - (sx0 + sx1);
      wy = 0.f;
      w[j] = (double)wx;
    }
    nrm += wx * wx + wy * wy;
#pragma unroll
    for (int i = 0; i < KMAX; ++i) sacc[i * UDB + t] += v[i].x * wx + v[i].y * wy;
  }
  sacc[KMAX * UDB + t] = nrm;
  __syncthreads();
  // one warp per row, lanes on consecutive columns (no bank conflicts), float32 sums
  const int lane = t & 31;
  for (int i = t >> 5; i <= k; i += UDB / 32) {
    const float* rp = sacc + (i < k ? i : KMAX) * UDB;
    float s = (rp[lane] + rp[lane + 32]) + (rp[lane + 64] + rp[lane + 96]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) part[(int64_t)i * G + blockIdx.x] = (double)s;
  }
}

template <int KMAX, typename VT>
static int launch_upd_dot(fsi_mesh* m, int G, double* w, const VT* V, int M1, int k, const double* h, int64_t n) {
  const size_t smem = sizeof(VT) * (size_t)(KMAX + 1) * UDB;
  if constexpr (sizeof(VT) == 4) {
    if (int rc = ensure_smem_attr(reinterpret_cast<const void*>(&upd_dot2_kernel<KMAX>), smem)) return rc;
    upd_dot2_kernel<KMAX><<<G, UDB, smem, m->stream>>>(w, V, M1, k, h, n, m->partials_dot);
  } else {
    if (int rc = ensure_smem_attr(reinterpret_cast<const void*>(&upd_dot_kernel<KMAX, VT>), smem)) return rc;
    upd_dot_kernel<KMAX, VT><<<G, UDB, smem, m->stream>>>(w, V, M1, k, h, n, m->partials_dot);
  }
  return FSI_OK;
}

template <typename VT>
static int upd_dot(fsi_mesh* m, int G, double* w, const VT* V, int M1, int k, const double* h, int64_t n) {
  switch ((k + 7) / 8) {
    case 1: return launch_upd_dot<8>(m, G, w, V, M1, k, h, n);
    case 2: return launch_upd_dot<16>(m, G, w, V, M1, k, h, n);
    case 3: return launch_upd_dot<24>(m, G, w, V, M1, k, h, n);
    case 4: return launch_upd_dot<32>(m, G, w, V, M1, k, h, n);
    case 5: return launch_upd_dot<40>(m, G, w, V, M1, k, h, n);
    case 6: return launch_upd_dot<48>(m, G, w, V, M1, k, h, n);
    case 7: return launch_upd_dot<56>(m, G, w, V, M1, k, h, n);
    default: return launch_upd_dot<64>(m, G, w, V, M1, k, h, n);
  }
}

// V_slot[j] = src[j] * scale, scale = 1/sqrt(*n2) (n2 != null) or 1/K->nrm_fin; with z,
// also the next operator input z[j] = dinv[j] * V_slot[j] from the stored value (the
// float32 operator's increment when VT is float)
template <typename VT>
__global__ void store_slot(VT* __restrict__ V, int M1, int slot, const double* __restrict__ src, const double* n2,
                           const KryDev* K, int64_t n, const double* __restrict__ dinv, VT* __restrict__ z) {
  // the scale once per CTA: float64 division and square root are slow on this GPU
  __shared__ double s_sh;
  if (threadIdx.x == 0) {
    if (n2) {
      s_sh = 1.0 / sqrt(*n2);
    } else {
      const double nf = K->nrm_fin;
      s_sh = nf > 0.0 ? 1.0 / nf : 0.0;
    }
  }
  __syncthreads();
  const double s = s_sh;
  // one chunk of CH = VB elements per CTA pass
  const int64_t nch = (n + CH - 1) / CH;
  for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
    const int64_t j = c * CH + threadIdx.x;
    if (j >= n) continue;
    const VT v = (VT)(src[j] * s);
    V[c * (int64_t)M1 * CH + (int64_t)slot * CH + threadIdx.x] = v;
    if (z) {
      if constexpr (sizeof(VT) == 4) z[j] = (float)dinv[j] * v;  // the float32 operator's increment
      else z[j] = dinv[j] * v;
    }
  }
}

// z = dinv * V_slot (ZT float: the float32 operator's increment, written directly)
template <typename VT, typename ZT>
__global__ void precond_kernel(const VT* __restrict__ V, int M1, int slot, const double* __restrict__ dinv,
                               ZT* __restrict__ z, int64_t n) {
  const int64_t nch = (n + CH - 1) / CH;
  for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
    const int64_t j = c * CH + threadIdx.x;
    if (j < n) z[j] = (ZT)(dinv[j] * (double)V[c * (int64_t)M1 * CH + (int64_t)slot * CH + threadIdx.x]);
  }
}

// x += dinv * sum_i y_i V_i
template <typename VT>
__global__ void __launch_bounds__(VB) combine_kernel(double* __restrict__ x, const double* __restrict__ dinv,
                                                     const VT* __restrict__ V, int M1, int k, const KryDev* K,
                                                     int64_t n) {
  __shared__ VT ys[MMAX];
  for (int i = threadIdx.x; i < k; i += VB) ys[i] = (VT)K->y[i];
  __syncthreads();
  const int64_t nch = (n + CH - 1) / CH;
  for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
    const int64_t j = c * CH + threadIdx.x;
    if (j >= n) continue;
    x[j] += dinv[j] * (double)lin_comb_chunk<VT>(ys, V + c * (int64_t)M1 * CH + threadIdx.x, k);
  }
}

// z = V_slot (contiguous float64 copy of one basis vector)
template <typename VT>
__global__ void extract_kernel(const VT* __restrict__ V, int M1, int slot, double* __restrict__ z, int64_t n) {
  const int64_t nch = (n + CH - 1) / CH;
  for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
    const int64_t j = c * CH + threadIdx.x;
    if (j < n) z[j] = (double)V[c * (int64_t)M1 * CH + (int64_t)slot * CH + threadIdx.x];
  }
}

// x += sum_i y_i Z_i (flexible GMRES: the stored preconditioned directions)
__global__ void __launch_bounds__(VB) zcombine_kernel(double* __restrict__ x, const double* __restrict__ Z, int k,
                                                      const KryDev* K, int64_t n) {
  __shared__ double ys[MMAX];
  for (int i = threadIdx.x; i < k; i += VB) ys[i] = K->y[i];
  __syncthreads();
  for (int64_t j = blockIdx.x * (int64_t)VB + threadIdx.x; j < n; j += (int64_t)gridDim.x * VB) {
    double s = 0.0;
    for (int i = 0; i < k; ++i) s += ys[i] * Z[(int64_t)i * n + j];
    x[j] += s;
  }
}

// --------------------------------------------------------- small device kernels
// After pass 1: the column h[0..j], |w_old|^2 = h[j+1]; |w_new|^2 in h2[j+1] (the fused
// update's row of norms; h2[0..j] hold the pass-2 projections).  Read through a volatile
// pointer: other CTAs wrote h2 just before.
__device__ void orth_decide_body(KryDev* K, int j) {
  volatile double* h2 = K->h2;
  K->nrm_old = sqrt(K->h[j + 1]);
  K->nrm_new = h2[j + 1];
  const double nn = sqrt(K->nrm_new);
  K->reorth = (nn < K->nrm_old * 0.70710678118654752) ? 1 : 0;
  K->nrm_fin = nn;
}

// Rows of the fused update's partials into K->h2 (one CTA per row, fixed order); the last
// CTA to finish takes the DGKS decision, so no single-thread launch follows.
__global__ void sum_partials_decide(const double* __restrict__ part, int G, KryDev* K, int j) {
  const int i = blockIdx.x;
  double s = 0.0;
  for (int c = threadIdx.x; c < G; c += VB) s += part[(int64_t)i * G + c];
  double acc[1] = {s};
  __shared__ double res;
  __shared__ bool last;
  block_reduce_store<1>(acc, 1, &res, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    K->h2[i] = res;
    __threadfence();
    last = atomicAdd(&K->counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    K->counter = 0;
    orth_decide_body(K, j);
  }
}

// The second pass's |w|^2 (only when it ran) and the Givens step, in one CTA: the column,
// the rotations and the right-hand side are read into shared memory by all threads, one
// thread applies the rotations there (a chain of shared-memory operations, not of global
// loads), and the column goes back in parallel.  Column j of the Hessenberg matrix (h,
// plus h2 when the second pass ran, and the new norm below it) is rotated by the previous
// rotations, the new rotation zeroes its subdiagonal entry, and g and the residual
// estimate |g_{j+1}| / |b| follow.
__global__ void sum_partials_givens(const double* __restrict__ part, int G, KryDev* K, int j, int mm) {
  __shared__ double col[MMAX + 2], cs[MMAX], sn[MMAX];
  __shared__ double res;
  const int reorth = K->reorth;
  if (reorth) {
    double s = 0.0;
    for (int c = threadIdx.x; c < G; c += VB) s += part[c];
    double acc[1] = {s};
    block_reduce_store<1>(acc, 1, &res, 1);
  }
  for (int i = threadIdx.x; i <= j; i += VB) {
    double h = K->h[i];
    if (reorth) {
      h += K->h2[i];
      K->h[i] = h;
    }
    col[i] = h;
    if (i < j) {
      cs[i] = K->cs[i];
      sn[i] = K->sn[i];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (reorth) {
      K->nrm_new = res;
      K->nrm_fin = sqrt(res);
    }
    const double hn = K->nrm_fin;
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
      const double a = cs[i] * col[i] + sn[i] * col[i + 1];
      col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
      col[i] = a;
    }
    const double den = hypot(col[j], col[j + 1]);
    const double c = den > 0.0 ? col[j] / den : 1.0;
    const double sj = den > 0.0 ? col[j + 1] / den : 0.0;
    K->cs[j] = c;
    K->sn[j] = sj;
    col[j] = den;
    col[j + 1] = 0.0;
    const double gj = K->g[j];
    K->g[j + 1] = -sj * gj;
    K->g[j] = c * gj;
    K->est = fabs(K->g[j + 1]) / K->bnorm;
    K->breakdown = (hn == 0.0 || den == 0.0 || !isfinite(hn)) ? 1 : 0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= j + 1; i += VB) K->H[i * mm + j] = col[i];
}

// y = R^{-1} g for the first jend columns (back substitution).
__global__ void lsq_kernel(KryDev* K, int jend, int mm) {
  for (int i = jend - 1; i >= 0; --i) {
    double s = K->g[i];
    for (int k = i + 1; k < jend; ++k) s -= K->H[i * mm + k] * K->y[k];
    const double d = K->H[i * mm + i];
    K->y[i] = d != 0.0 ? s / d : 0.0;
  }
}

// start of a cycle: g = (|r|, 0, ...)
__global__ void cycle_start(KryDev* K, const double* rn2, int mm) {
  const double b = sqrt(*rn2);
  for (int i = 0; i <= mm; ++i) K->g[i] = 0.0;
  K->g[0] = b;
  K->nrm_fin = b;
}

// --------------------------------------------------------- contiguous vectors
// part[cta] = partial of a . b over a contiguous range
__global__ void __launch_bounds__(VB) dot_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                                                 double* part) {
  const int G = gridDim.x;
  const int64_t per = (n + G - 1) / G;
  const int64_t lo = blockIdx.x * per, hi = min(n, lo + per);
  double acc[1] = {0.0};
  for (int64_t j = lo + threadIdx.x; j < hi; j += VB) acc[0] += a[j] * b[j];
  block_reduce_store<1>(acc, 1, part + blockIdx.x, 1);
}
__global__ void axpby_kernel(double a, const double* __restrict__ x, double b, double* __restrict__ y, int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)VB + threadIdx.x; j < n; j += (int64_t)gridDim.x * VB) y[j] = a * x[j] + b * y[j];
}
__global__ void mul_kernel(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ y, int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)VB + threadIdx.x; j < n; j += (int64_t)gridDim.x * VB) y[j] = a[j] * b[j];
}
__global__ void recip_kernel(const double* __restrict__ a, double* __restrict__ y, int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)VB + threadIdx.x; j < n; j += (int64_t)gridDim.x * VB) {
    const double v = a[j];
    y[j] = v != 0.0 ? 1.0 / v : 1.0;
  }
}
__global__ void fill_kernel(double* y, double v, int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)VB + threadIdx.x; j < n; j += (int64_t)gridDim.x * VB) y[j] = v;
}

// ---------------------------------------------------------------- host helpers
template <int R, bool SELF, typename VT>
static void launch_mdot(fsi_mesh* m, dim3 grid, const VT* V, int M1, int i0, const double* w, int64_t n,
                        const int* skip) {
  if constexpr (sizeof(VT) == 4)
    mdot4_kernel<R, SELF><<<grid, VB, 0, m->stream>>>(V, M1, i0, w, n, m->partials_dot, skip);
  else
    mdot_kernel<R, SELF, VT><<<grid, VB, 0, m->stream>>>(V, M1, i0, w, n, m->partials_dot, skip);
}

template <bool SELF, typename VT>
static void launch_mdot_rem(fsi_mesh* m, int rem, dim3 g1, const VT* V, int M1, int i0, const double* w,
                            int64_t n, const int* skip) {
  switch (rem) {
    case 0: launch_mdot<0, SELF>(m, g1, V, M1, i0, w, n, skip); break;
    case 1: launch_mdot<1, SELF>(m, g1, V, M1, i0, w, n, skip); break;
    case 2: launch_mdot<2, SELF>(m, g1, V, M1, i0, w, n, skip); break;
    case 3: launch_mdot<3, SELF>(m, g1, V, M1, i0, w, n, skip); break;
    case 4: launch_mdot<4, SELF>(m, g1, V, M1, i0, w, n, skip); break;
    case 5: launch_mdot<5, SELF>(m, g1, V, M1, i0, w, n, skip); break;
    case 6: launch_mdot<6, SELF>(m, g1, V, M1, i0, w, n, skip); break;
    case 7: launch_mdot<7, SELF>(m, g1, V, M1, i0, w, n, skip); break;
    case 8: launch_mdot<8, SELF>(m, g1, V, M1, i0, w, n, skip); break;
    case 9: launch_mdot<9, SELF>(m, g1, V, M1, i0, w, n, skip); break;
    case 10: launch_mdot<10, SELF>(m, g1, V, M1, i0, w, n, skip); break;
    case 11: launch_mdot<11, SELF>(m, g1, V, M1, i0, w, n, skip); break;
    case 12: launch_mdot<12, SELF>(m, g1, V, M1, i0, w, n, skip); break;
    case 13: launch_mdot<13, SELF>(m, g1, V, M1, i0, w, n, skip); break;
    case 14: launch_mdot<14, SELF>(m, g1, V, M1, i0, w, n, skip); break;
    default: launch_mdot<15, SELF>(m, g1, V, M1, i0, w, n, skip); break;
  }
}

// out[0..k) = V_i . w for the basis slots i < k; with self, out[k] = w . w.
template <typename VT>
static int basis_dots(fsi_mesh* m, const VT* V, int M1, int k, const double* w, int64_t n, double* out, bool self,
                      const int* skip = nullptr) {
  const int G = cgrid_t<VT>((n + CH - 1) / CH);
  const int nfull = k / DCH, rem = k % DCH;
  if (nfull)
    FSI_LAUNCH(m, P_KRY_DOT, (launch_mdot<DCH, false>(m, dim3(G, nfull), V, M1, 0, w, n, skip)));
  if (rem || self) {
    if (self)
      FSI_LAUNCH(m, P_KRY_DOT, (launch_mdot_rem<true>(m, rem, dim3(G, 1), V, M1, nfull * DCH, w, n, skip)));
    else
      FSI_LAUNCH(m, P_KRY_DOT, (launch_mdot_rem<false>(m, rem, dim3(G, 1), V, M1, nfull * DCH, w, n, skip)));
  }
  const int rows = k + (self ? 1 : 0);
  FSI_LAUNCH(m, P_KRY_DOT, sum_partials<<<rows, VB, 0, m->stream>>>(m->partials_dot, G, out, skip));
  return FSI_OK;
}

// per-CTA partial sums of the reductions (fixed size, allocated on first use)
static int ensure_partials(fsi_mesh* m) {
  if (m->partials_dot) return FSI_OK;
  FSI_CUDA(cudaMalloc(&m->partials_dot, sizeof(double) * (size_t)(MMAX + 2 + DCH) * 152 * 4));
  return FSI_OK;
}

static int dot_dev(fsi_mesh* m, const double* a, const double* b, int64_t n, double* out) {
  int rc = ensure_partials(m);
  if (rc) return rc;
  const int G = vgrid(n);
  FSI_LAUNCH(m, P_KRY_DOT, dot_kernel<<<G, VB, 0, m->stream>>>(a, b, n, m->partials_dot));
  FSI_LAUNCH(m, P_KRY_DOT, sum_partials<<<1, VB, 0, m->stream>>>(m->partials_dot, G, out, nullptr));
  return FSI_OK;
}

int vec_dot(fsi_mesh* m, const double* a, const double* b, int64_t n, double* out_host) {
  int rc = dot_dev(m, a, b, n, m->red);
  if (rc) return rc;
  FSI_CUDA(cudaMemcpyAsync(m->red_host, m->red, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  FSI_CUDA(cudaStreamSynchronize(m->stream));
  *out_host = m->red_host[0];
  return FSI_OK;
}

int vec_axpy(fsi_mesh* m, double a, const double* x, double* y, int64_t n) {
  FSI_LAUNCH(m, P_KRYLOV, axpby_kernel<<<vgrid(n), VB, 0, m->stream>>>(a, x, 1.0, y, n));
  return FSI_OK;
}
int vec_scale_copy(fsi_mesh* m, double a, const double* x, double* y, int64_t n) {
  FSI_LAUNCH(m, P_KRYLOV, axpby_kernel<<<vgrid(n), VB, 0, m->stream>>>(a, x, 0.0, y, n));
  return FSI_OK;
}
int vec_mul(fsi_mesh* m, const double* a, const double* b, double* y, int64_t n) {
  FSI_LAUNCH(m, P_KRYLOV, mul_kernel<<<vgrid(n), VB, 0, m->stream>>>(a, b, y, n));
  return FSI_OK;
}
int vec_recip(fsi_mesh* m, const double* a, double* y, int64_t n) {
  FSI_LAUNCH(m, P_KRYLOV, recip_kernel<<<vgrid(n), VB, 0, m->stream>>>(a, y, n));
  return FSI_OK;
}

// basis: nch chunks x (mx + 1) slots x CH; wk: 7 contiguous work vectors
static int ensure_krylov(fsi_mesh* m, int64_t n, int mm) {
  if (m->kry_n >= n && m->kry_m >= mm && m->kry_dev) return FSI_OK;
  const int64_t nn = std::max(n, m->kry_n);
  const int mx = std::max(mm, m->kry_m);
  cudaFree(m->V);
  cudaFree(m->wk);
  cudaFree(m->dinv);
  m->V = m->wk = m->dinv = nullptr;
  const int64_t nch = (nn + CH - 1) / CH;
  FSI_CUDA(cudaMalloc(&m->V, sizeof(double) * (size_t)nch * (mx + 1) * CH));
  FSI_CUDA(cudaMalloc(&m->wk, sizeof(double) * (size_t)7 * nn));
  FSI_CUDA(cudaMalloc(&m->dinv, sizeof(double) * (size_t)nn));
  if (int rc = ensure_partials(m)) return rc;
  if (!m->kry_dev) {
    FSI_CUDA(cudaMalloc(&m->kry_dev, sizeof(KryDev)));
    FSI_CUDA(cudaMemset(m->kry_dev, 0, sizeof(KryDev)));
    FSI_CUDA(cudaMallocHost(&m->kry_est, sizeof(double) * 3 * (MMAX + 1)));
    m->kry_ev.resize(MMAX + 1);
    for (auto& e : m->kry_ev) FSI_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  m->kry_n = nn;
  m->kry_m = mx;
  return FSI_OK;
}

// One GMRES(m) solve A x = b from x = 0 with A = the block operator (flags) and the
// right preconditioner diag(dinv).  VT: the basis type (float exactly when the operator
// is the float32 one, i.e. the inner solves of iterative refinement).
template <typename VT>
static int gmres_core_t(fsi_mesh* m, const BlockInfo& blk, const double* b, double* x, int mm, double rtol,
                        int max_iter, unsigned flags, int* iters, int* restarts, double* rel_out, int* stalled,
                        fsi_pc* pc, fsi_pc* harvest) {
  constexpr bool F32 = sizeof(VT) == 4;
  const bool alternate = (flags & FSI_PC_ALTERNATE) != 0;
  const bool stall_stop = (flags & FSI_NO_STALL_STOP) == 0;
  flags &= ~(FSI_PC_ALTERNATE | FSI_NO_STALL_STOP);
  const int64_t n = blk.n;
  const int M1 = m->kry_m + 1;
  const int G = vgrid(n);
  VT* V = reinterpret_cast<VT*>(m->V);  // the float basis reuses the float64 allocation
  double* r = m->wk;
  double* z = m->wk + n;
  double* t = m->wk + 2 * n;
  double* w = m->wk + 6 * n;
  KryDev* K = static_cast<KryDev*>(m->kry_dev);
  double* est = m->kry_est;  // pinned, 3 slots per step: the estimate, then the reorth and breakdown ints
  FSI_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, m->stream));
  double bnorm2;
  int rc = vec_dot(m, b, b, n, &bnorm2);
  if (rc) return rc;
  if (!std::isfinite(bnorm2)) return set_error(FSI_ENAN, "GMRES: right-hand side is not finite");
  const double bnorm = std::sqrt(bnorm2);
  *rel_out = 0.0;
  *stalled = 0;
  if (bnorm == 0.0) return FSI_OK;
  FSI_CUDA(cudaMemcpyAsync(&K->bnorm, &bnorm, sizeof(double), cudaMemcpyHostToDevice, m->stream));
  FSI_CUDA(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->stream));
  double rel = 1.0, cycle_rel = 1.0;
  bool first_cycle = true;
  int n_arnoldi_pairs = 0;
  while (true) {
    // |r| on the device; the host needs it for the stopping and stall tests
    if ((rc = dot_dev(m, r, r, n, m->red))) return rc;
    FSI_CUDA(cudaMemcpyAsync(m->red_host, m->red, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    FSI_CUDA(cudaStreamSynchronize(m->stream));
    const double beta2 = m->red_host[0];
    if (!std::isfinite(beta2)) return set_error(FSI_ENAN, "GMRES: residual is not finite");
    rel = std::sqrt(beta2) / bnorm;
    if (rel <= rtol || *iters >= max_iter) break;
    if (stall_stop && !first_cycle && rel > 0.99 * cycle_rel) {
      *stalled = 1;
      break;
    }
    first_cycle = false;
    cycle_rel = rel;
    FSI_LAUNCH(m, P_KRY_SMALL, cycle_start<<<1, 1, 0, m->stream>>>(K, m->red, mm));
    // the operator input of the plain (Jacobi) steps: z = dinv V_j, written with V_j
    VT* zn = pc ? nullptr : (F32 ? reinterpret_cast<VT*>(m->dx32) : reinterpret_cast<VT*>(z));
    FSI_LAUNCH(m, P_KRYLOV, store_slot<VT><<<chunk_grid(n), VB, 0, m->stream>>>(V, M1, 0, r, m->red, K, n, m->dinv, zn));
    int jend = 0, enq = 0;
    bool done = false;
    const int jmax = std::min(mm, max_iter - *iters);
    const double vb = (double)sizeof(VT) * (double)n;  // bytes of one basis vector
    const double wb = 8.0 * (double)n;                 // bytes of the float64 work vector
    for (int j = 0; j < jmax && !done; ++j) {
      if (pc) {  // flexible GMRES: z_j = M(v_j), |v_j| = 1
        double* zj = m->Z + (int64_t)j * n;
        if (alternate && (j & 1)) {
          // every other direction is the plain Jacobi one: the least-squares step then
          // weights network and Jacobi directions separately
          FSI_LAUNCH(m, P_KRYLOV, (precond_kernel<VT, double><<<G, VB, 0, m->stream>>>(V, M1, j, m->dinv, zj, n)));
        } else {
          FSI_LAUNCH(m, P_KRYLOV, extract_kernel<VT><<<G, VB, 0, m->stream>>>(V, M1, j, t, n));
          if ((rc = pcn::apply(pc, t, 1.0, m->dinv, zj))) return rc;
        }
        if ((rc = op_jvp(m, blk, zj, w, flags))) return rc;
      } else {
        // z = dinv V_j was written with V_j (the float32 increment straight into the
        // operator's input buffer)
        if (F32) {
          if ((rc = op_jvp(m, blk, nullptr, w, flags | OP_DX32_READY))) return rc;
        } else {
          if ((rc = op_jvp(m, blk, z, w, flags))) return rc;
        }
        // broadband training pairs: A z_j = w exactly for the operator just applied
        // (harvesting solves run with the float64 basis)
        if (!F32 && harvest && j % 8 == 4 && n_arnoldi_pairs < 8) {
          if ((rc = pcn::add_pair(harvest, w, nullptr, z, nullptr, m->dinv))) return rc;
          ++n_arnoldi_pairs;
        }
      }
      // pass 1: h = V^T w and |w|^2 (slot j+1 of h)
      if ((rc = basis_dots(m, V, M1, j + 1, w, n, K->h, true))) return rc;
      // pass-1 update fused with the pass-2 projections of the updated vector
      {
        const int Gc = cgrid_t<VT>((n + CH - 1) / CH);
        FSI_LAUNCH(m, P_KRY_UPD, rc = upd_dot<VT>(m, Gc, w, V, M1, j + 1, K->h, n));
        if (rc) return rc;
        FSI_LAUNCH(m, P_KRY_UPD, sum_partials_decide<<<j + 2, VB, 0, m->stream>>>(m->partials_dot, Gc, K, j));
        prof_bytes(m, P_KRY_DOT, (j + 1) * vb + wb);      // j+1 basis vectors and w read once
        prof_bytes(m, P_KRY_UPD, (j + 1) * vb + 2 * wb);  // j+1 basis vectors and w read, w written
        // the pass-2 update only when the DGKS test asked for it (exits at once otherwise),
        // then its norm and the Givens step
        if constexpr (F32) {
          FSI_LAUNCH(m, P_KRY_UPD, upd4_kernel<<<Gc, VB, 0, m->stream>>>(w, reinterpret_cast<const float*>(V), M1,
                                                                        j + 1, K->h2, n, m->partials_dot, &K->reorth));
        } else {
          FSI_LAUNCH(m, P_KRY_UPD, upd_kernel<VT><<<Gc, VB, 0, m->stream>>>(w, V, M1, j + 1, K->h2, n,
                                                                             m->partials_dot, &K->reorth));
        }
        FSI_LAUNCH(m, P_KRY_SMALL, sum_partials_givens<<<1, VB, 0, m->stream>>>(m->partials_dot, Gc, K, j, mm));
      }
      FSI_LAUNCH(m, P_KRYLOV, store_slot<VT><<<chunk_grid(n), VB, 0, m->stream>>>(V, M1, j + 1, w, nullptr, K, n, m->dinv, zn));
      // estimate, reorth and breakdown flags: one copy (the fields are adjacent)
      FSI_CUDA(cudaMemcpyAsync(est + 3 * j, &K->est, sizeof(double) + 2 * sizeof(int), cudaMemcpyDeviceToHost,
                               m->stream));
      FSI_CUDA(cudaEventRecord(m->kry_ev[j], m->stream));
      ++*iters;
      jend = j + 1;
      enq = j + 1;
      // look at the previous step while this one runs
      if (j >= 1) {
        FSI_CUDA(cudaEventSynchronize(m->kry_ev[j - 1]));
        int bd = 0;
        memcpy(&bd, reinterpret_cast<const char*>(est + 3 * (j - 1)) + sizeof(double) + sizeof(int), sizeof(int));
        const double e = est[3 * (j - 1)];
        if (!std::isfinite(e)) return set_error(FSI_ENAN, "GMRES: Arnoldi vector is not finite");
        if (e <= rtol || bd) {
          jend = j;  // step j was computed for nothing
          done = true;
        }
      }
    }
    FSI_CUDA(cudaEventSynchronize(m->kry_ev[enq - 1]));
    if (!done && !std::isfinite(est[3 * (jend - 1)])) return set_error(FSI_ENAN, "GMRES: Arnoldi vector is not finite");
    for (int j = 0; j < enq; ++j) {  // the second passes that ran
      int ro = 0;
      memcpy(&ro, reinterpret_cast<const char*>(est + 3 * j) + sizeof(double), sizeof(int));
      if (ro) prof_bytes(m, P_KRY_UPD, (j + 1) * vb + 2 * wb);
    }
    FSI_LAUNCH(m, P_KRY_SMALL, lsq_kernel<<<1, 1, 0, m->stream>>>(K, jend, mm));
    if (pc) {
      FSI_LAUNCH(m, P_KRYLOV, zcombine_kernel<<<G, VB, 0, m->stream>>>(x, m->Z, jend, K, n));
    } else {
      FSI_LAUNCH(m, P_KRYLOV, combine_kernel<VT><<<cgrid((n + CH - 1) / CH), VB, 0, m->stream>>>(x, m->dinv, V, M1,
                                                                                                jend, K, n));
    }
    // true residual r = b - A x
    if ((rc = op_jvp(m, blk, x, t, flags))) return rc;
    FSI_CUDA(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->stream));
    if ((rc = vec_axpy(m, -1.0, t, r, n))) return rc;
    ++*restarts;
  }
  *rel_out = rel;
  return FSI_OK;
}

static int gmres_core(fsi_mesh* m, const BlockInfo& blk, const double* b, double* x, int mm, double rtol,
                      int max_iter, unsigned flags, int* iters, int* restarts, double* rel_out, int* stalled,
                      fsi_pc* pc = nullptr, fsi_pc* harvest = nullptr) {
  // harvesting solves keep the float64 basis: their Arnoldi pairs and refinement
  // checkpoints are the training data of the learned preconditioner
  if ((flags & FSI_FP32) && !harvest) {
    if (int rc = ensure_dx32(m)) return rc;
    return gmres_core_t<float>(m, blk, b, x, mm, rtol, max_iter, flags, iters, restarts, rel_out, stalled, pc,
                               harvest);
  }
  return gmres_core_t<double>(m, blk, b, x, mm, rtol, max_iter, flags, iters, restarts, rel_out, stalled, pc, harvest);
}

int gmres_solve(fsi_mesh* m, const BlockInfo& blk, const double* rhs, double* x, const fsi_solve_opts& o,
                fsi_solve_info* info) {
  const int mm = o.m;
  if (mm < 1 || mm > MMAX) return set_error(FSI_EINVAL, "GMRES: restart length must be in 1..64");
  const int64_t n = blk.n;
  int rc = ensure_krylov(m, n, mm);
  if (rc) return rc;
  const int64_t a0 = m->applies;
  // the learned preconditioner acts on the NS block only; other blocks use Jacobi
  fsi_pc* pc = (o.precond == FSI_PC_LEARNED && blk.kind == 0) ? m->pc : nullptr;
  if (o.precond == FSI_PC_LEARNED && blk.kind == 0 && !pc)
    return set_error(FSI_EINVAL, "GMRES: FSI_PC_LEARNED without an attached preconditioner (fsi_set_pc)");
  fsi_pc* harvest = ((o.flags & FSI_HARVEST) && blk.kind == 0 && m->pc && m->pc->cap > 0) ? m->pc : nullptr;
  const unsigned opflags =
      o.flags & ~(FSI_HARVEST | FSI_PC_ALTERNATE | FSI_NO_STALL_STOP | FSI_PINNED_SOLVE | OP_DX32_READY);
  // read by the solver loop only: network/Jacobi alternation, and no stop on stagnation
  const unsigned alt = o.flags & (FSI_PC_ALTERNATE | FSI_NO_STALL_STOP);
  const bool stall_stop = (o.flags & FSI_NO_STALL_STOP) == 0;
  if (pc && (m->Z_n < n * mm || !m->Z)) {
    cudaFree(m->Z);
    m->Z = nullptr;
    FSI_CUDA(cudaMalloc(&m->Z, sizeof(double) * (size_t)(n * mm)));
    m->Z_n = n * mm;
  }
  if (harvest && (rc = pcn::ensure_checkpoints(harvest))) return rc;
  // Jacobi diagonal (also the learned preconditioner's scale), from the operator the
  // inner solves apply: a preconditioner's rounding does not reach the refined solution,
  // and the float64 diagonal costs as much as 20 float32 ones on this GPU
  if (o.precond == FSI_PC_JACOBI || o.precond == FSI_PC_LEARNED || harvest) {
    const unsigned dflags = o.precision == FSI_PREC_FP32_IR ? (opflags | FSI_FP32) : (opflags & ~FSI_FP32);
    if ((rc = op_diag(m, blk, m->wk + 3 * n, dflags))) return rc;
    if ((rc = vec_recip(m, m->wk + 3 * n, m->dinv, n))) return rc;
  }
  if (o.precond == FSI_PC_NONE) {
    FSI_LAUNCH(m, P_KRYLOV, fill_kernel<<<vgrid(n), VB, 0, m->stream>>>(m->dinv, 1.0, n));
  }
  fsi_solve_info inf{};
  double rel = 0.0;
  int nck = 0;  // harvest checkpoints recorded
  auto checkpoint = [&](const double* xk, const double* rk) -> int {
    if (!harvest || nck >= pcn::CKMAX) return FSI_OK;
    FSI_CUDA(cudaMemcpyAsync(harvest->ck + (int64_t)nck * n, xk, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                             m->stream));
    FSI_CUDA(cudaMemcpyAsync(harvest->ck + (int64_t)(pcn::CKMAX + nck) * n, rk, sizeof(double) * n,
                             cudaMemcpyDeviceToDevice, m->stream));
    ++nck;
    return FSI_OK;
  };
  double* rfin = nullptr;  // final true residual (harvest)
  if (o.precision == FSI_PREC_FP64) {
    rc = gmres_core(m, blk, rhs, x, mm, o.rtol, o.max_iter, (opflags & ~FSI_FP32) | alt, &inf.iterations, &inf.restarts,
                    &rel, &inf.stalled, pc, pc ? nullptr : harvest);
    if (rc == FSI_ENAN && pc) {
      // the network produced non-finite directions (corrupted weights, overflow):
      // Jacobi GMRES solves from scratch
      inf.fallback = 1;
      pc = nullptr;
      rc = gmres_core(m, blk, rhs, x, mm, o.rtol, o.max_iter - inf.iterations,
                      (opflags & ~FSI_FP32) | (alt & FSI_NO_STALL_STOP),
                      &inf.iterations, &inf.restarts, &rel, &inf.stalled, nullptr, harvest);
    }
    if (rc) return rc;
    if (pc && rel > o.rtol && inf.iterations < o.max_iter) {
      // fallback: Jacobi GMRES on the remaining residual r = rhs - A x (in wk[0..n))
      double* d = m->wk + 4 * n;
      double* r = m->wk + 5 * n;
      FSI_CUDA(cudaMemcpyAsync(r, m->wk, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->stream));
      double rel2;
      int st2 = 0;
      rc = gmres_core(m, blk, r, d, mm, o.rtol / std::max(rel, 1e-300), o.max_iter - inf.iterations,
                      (opflags & ~FSI_FP32) | (alt & FSI_NO_STALL_STOP), &inf.iterations, &inf.restarts, &rel2, &st2, nullptr);
      if (rc) return rc;
      if ((rc = vec_axpy(m, 1.0, d, x, n))) return rc;
      rel *= rel2;
      inf.stalled = st2;
      inf.fallback = 1;
    }
    rfin = m->wk;  // rhs - A x (the fallback's final residual is the same vector)
    if (harvest) {  // the one checkpoint x_0 = 0, r_0 = rhs
      FSI_CUDA(cudaMemsetAsync(harvest->ck, 0, sizeof(double) * n, m->stream));
      FSI_CUDA(cudaMemcpyAsync(harvest->ck + (int64_t)pcn::CKMAX * n, rhs, sizeof(double) * n,
                               cudaMemcpyDeviceToDevice, m->stream));
      nck = 1;
    }
  } else {
    // x = 0; r = rhs; repeat: solve A32 d = r; x += d; r = rhs - A64 x
    double* d = m->wk + 4 * n;
    double* r = m->wk + 5 * n;
    FSI_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, m->stream));
    FSI_CUDA(cudaMemcpyAsync(r, rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->stream));
    double b2;
    if ((rc = vec_dot(m, rhs, rhs, n, &b2))) return rc;
    if (!std::isfinite(b2)) return set_error(FSI_ENAN, "IR: right-hand side is not finite");
    const double bnorm = std::sqrt(b2);
    rel = bnorm == 0.0 ? 0.0 : 1.0;
    fsi_pc* inner_pc = pc;
    for (int k = 0; k < std::max(1, o.ir_max) && rel > o.rtol; ++k) {
      if ((rc = checkpoint(x, r))) return rc;
      double inner_rel;
      int inner_stalled;
      rc = gmres_core(m, blk, r, d, mm, o.ir_inner_rtol, o.max_iter - inf.iterations, (opflags | FSI_FP32 | alt),
                      &inf.iterations, &inf.restarts, &inner_rel, &inner_stalled, inner_pc,
                      inner_pc ? nullptr : harvest);
      if (rc == FSI_ENAN && inner_pc) {
        // non-finite network directions: this refinement again, with Jacobi inner solves
        inner_pc = nullptr;
        inf.fallback = 1;
        --k;
        continue;
      }
      if (rc) return rc;
      if ((rc = vec_axpy(m, 1.0, d, x, n))) return rc;
      if ((rc = op_jvp(m, blk, x, d, opflags & ~FSI_FP32))) return rc;
      FSI_CUDA(cudaMemcpyAsync(r, rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->stream));
      if ((rc = vec_axpy(m, -1.0, d, r, n))) return rc;
      double r2;
      if ((rc = vec_dot(m, r, r, n, &r2))) return rc;
      if (!std::isfinite(r2)) return set_error(FSI_ENAN, "IR: residual is not finite");
      const double prev = rel;
      rel = bnorm > 0.0 ? std::sqrt(r2) / bnorm : 0.0;
      inf.refinements = k + 1;
      if (inf.iterations >= o.max_iter) break;
      const bool no_gain = rel > o.rtol && rel > 0.9 * prev;
      if (inner_pc && inner_stalled) {
        // the network failed its job (the inner solve): Jacobi GMRES finishes the
        // solve, retrying this refinement if it did not pay
        inner_pc = nullptr;
        inf.fallback = 1;
        if (no_gain) continue;
      }
      if (no_gain && stall_stop) {
        // the inner solve reached its tolerance but the float64 residual did not
        // follow: the refinement has stopped contracting
        inf.stalled = 1;
        break;
      }
    }
    rfin = r;
    if ((rc = check_tma(m))) return rc;
  }
  if (harvest) {
    // pairs (r_k - r*, x* - x_k): A (x* - x_k) = r_k - r* holds exactly for the
    // float64 operator that computed the residuals
    for (int k = 0; k < nck; ++k)
      if ((rc = pcn::add_pair(harvest, harvest->ck + (int64_t)(pcn::CKMAX + k) * n, rfin, x,
                              harvest->ck + (int64_t)k * n, m->dinv)))
        return rc;
  }
  if (pc && (rc = pcn::check_err(pc))) return rc;
  inf.rel_res = rel;
  inf.applies = (int)(m->applies - a0);
  if (info) *info = inf;
  if (!(rel <= o.rtol)) return set_error(FSI_ENOCONV, "GMRES: tolerance not reached");
  return FSI_OK;
}

}  // namespace fsi
