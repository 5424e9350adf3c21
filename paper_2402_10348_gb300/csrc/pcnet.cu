// Learned right preconditioner of the NS block (no counterpart in the paper, which
// solves every block with GMRES, Section 2.5): a 4-level, 16-channel 3D convolutional
// U-Net on the mesh's node grid, trained on the GPU by the kernels below and applied
// inside flexible GMRES.
//
// Network (3x3x3 zero-padded cross-correlations without bias, ReLU):
//   a_l = relu(conv x_l), e_l = relu(conv a_l), x_{l+1} = R e_l          l = 0, 1, 2
//   a_3 = relu(conv x_3), d_3 = relu(conv a_3)
//   b_l = relu(conv [e_l, P d_{l+1}]), d_l = relu(conv b_l)               l = 2, 1, 0
//   y   = conv d_0
// P is Q1 interpolation between node grids (a coarse grid keeps every other node),
// R = P^T / 8.
//
// Activations are bfloat16 in "octet planes": a C-channel tensor over an nx*ny*nz
// grid is C/8 planes of nz*ny*nx voxels, each voxel 8 channels = 16 bytes.
// Convolutions (forward and data gradient) run on the 5th-generation tensor cores:
// implicit GEMM with M = 128 output voxels (an 8 x 16 x-y tile of one z layer),
// N = output channels (16 or 32) and K = 27 taps x input channels, one
// tcgen05.mma (M128 N16|32 K16, bf16 x bf16 -> f32 in TMEM) per (tap, 16 input
// channels).  The A operand of tap (dx, dy, dz) is a shifted window of an input plane
// staged in shared memory without swizzle: 8 consecutive x voxels of one octet form a
// 128-byte core matrix, the next 8 rows (next y) sit 160 bytes further, the next 8
// channels one octet plane (2880 bytes) further.  Planes stream through a 4-slot ring
// (cp.async with zero fill at the grid boundary); the accumulator is double-buffered
// in TMEM so that one layer's epilogue overlaps the next layer's MMAs.
// Weight gradients are implicit GEMMs over voxels on the same tensor cores (per-CTA
// partials from TMEM, summed in a fixed order).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "pcnet.h"

namespace fsi {
namespace pcn {

constexpr int TILE_X = 8, TILE_Y = 16;               // output tile of one CTA layer: M = 128
constexpr int SX = TILE_X + 2, SY = TILE_Y + 2;      // staged input plane with a 1-voxel halo
constexpr int OCT_BYTES = SX * SY * 16;      // one channel octet of one staged plane
constexpr int NSLOT = 4;
constexpr int CONV_THREADS = 128;
// four per-component scales passed by value
struct D4 {
  double c[4];
};
// indicator planes fed to the network (by value)
struct Planes {
  const double* p[12];
  int n;
};

constexpr long long WAIT_LIMIT = 1LL << 22;  // bounded mbarrier polls (far above any MMA batch)

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  const int sz = valid ? 16 : 0;  // 0: zero-fill, nothing is read
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < WAIT_LIMIT; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void tmem_alloc(uint32_t holder, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(holder), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
// shared-memory matrix descriptor, no swizzle: start, leading (K-direction) and
// stride (M/N-direction) byte offsets between 8x16-byte core matrices; bit 46 is the
// descriptor version of this architecture
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: f32 accumulator, bf16 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int n, int m) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ float bf2f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }
__device__ __forceinline__ uint16_t f2bf(float f) { return __bfloat16_as_ushort(__float2bfloat16_rn(f)); }

__device__ __forceinline__ int64_t vox_addr(const TView& t, int oct, int x, int y, int z) {
  return ((((int64_t)(t.oct0 + oct) * t.nz + z) * t.ny + y) * t.nx + x) * 8;
}

// ------------------------------------------------------------------ convolution
template <int CIN, int N>
struct ConvCfg {
  static constexpr int KC = CIN / 16;                       // K chunks per tap
  static constexpr int SLOT = (CIN / 8) * OCT_BYTES;
  static constexpr int WBYTES = 27 * KC * N * 32;           // packed B operand
  static constexpr int NCOLS = 2 * N;                       // two f32 accumulators
  static constexpr int HEAD = 128;                          // barriers, TMEM address
  // the largest A address a descriptor forms is the last slot's last octet plane
  // (row group 15 of tap (2, 2) ends exactly at the plane's end), so the ring and
  // the weights are the whole footprint
  static constexpr int SMEM = HEAD + WBYTES + NSLOT * SLOT;
};

struct ConvArgs {
  TView in, out, mask;  // mask.p == nullptr: none
  float* out32;         // non-null: f32 planar [c][V] output of channels < nreal
  int nreal;
  const uint16_t* wpk;  // packed B operand: [27][KC][kgrp 2][ngrp N/8][8 n][8 k] bf16
  int zc, relu;
  int* err;
};

template <int CIN>
__device__ __forceinline__ void load_plane(const ConvArgs& a, uint32_t slot, int z, int x0, int y0) {
  constexpr int NCH = (CIN / 8) * SY * SX;
  const bool zin = z >= 0 && z < a.in.nz;
  for (int i = threadIdx.x; i < NCH; i += CONV_THREADS) {
    const int o = i / (SY * SX), rem = i - o * (SY * SX), yy = rem / SX, xx = rem - yy * SX;
    const int gx = x0 - 1 + xx, gy = y0 - 1 + yy;
    const bool v = zin && gx >= 0 && gx < a.in.nx && gy >= 0 && gy < a.in.ny;
    const uint16_t* src = v ? a.in.p + vox_addr(a.in, o, gx, gy, z) : a.in.p;
    cp_async16(slot + (uint32_t)(o * OCT_BYTES + (yy * SX + xx) * 16), src, v);
  }
}

template <int N>
__device__ __forceinline__ void conv_epilogue(const ConvArgs& a, uint32_t tmem, int buf, int z, int x0, int y0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = warp * 32 + lane;
  const int x = x0 + (m & 7), y = y0 + (m >> 3);
  const bool in = x < a.out.nx && y < a.out.ny;
  const int64_t V = (int64_t)a.out.nx * a.out.ny * a.out.nz;
  const int64_t vox = ((int64_t)z * a.out.ny + y) * a.out.nx + x;
#pragma unroll
  for (int h = 0; h < N / 16; ++h) {
    uint32_t r[16];
    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((buf & 1) * N + 16 * h), r);
    if (!in) continue;
    float v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
    if (a.mask.p) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const uint4 mv = *reinterpret_cast<const uint4*>(a.mask.p + vox_addr(a.mask, 2 * h + q, x, y, z));
        const uint32_t w[4] = {mv.x, mv.y, mv.z, mv.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const uint16_t hb = (uint16_t)(w[k >> 1] >> (16 * (k & 1)));
          if (!(bf2f(hb) > 0.0f)) v[8 * q + k] = 0.0f;
        }
      }
    }
    if (a.relu) {
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = fmaxf(v[k], 0.0f);
    }
    if (a.out32) {
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (16 * h + k < a.nreal) a.out32[(int64_t)(16 * h + k) * V + vox] = v[k];
    } else {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        uint4 o;
        o.x = (uint32_t)f2bf(v[8 * q + 0]) | ((uint32_t)f2bf(v[8 * q + 1]) << 16);
        o.y = (uint32_t)f2bf(v[8 * q + 2]) | ((uint32_t)f2bf(v[8 * q + 3]) << 16);
        o.z = (uint32_t)f2bf(v[8 * q + 4]) | ((uint32_t)f2bf(v[8 * q + 5]) << 16);
        o.w = (uint32_t)f2bf(v[8 * q + 6]) | ((uint32_t)f2bf(v[8 * q + 7]) << 16);
        *reinterpret_cast<uint4*>(a.out.p + vox_addr(a.out, 2 * h + q, x, y, z)) = o;
      }
    }
  }
}

template <int CIN, int N>
__global__ void __launch_bounds__(CONV_THREADS) conv_mma_kernel(ConvArgs a) {
  using C = ConvCfg<CIN, N>;
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm);
  uint32_t* holder = reinterpret_cast<uint32_t*>(sm + 16);
  const uint32_t wbase = smem_u32(sm + C::HEAD);
  const uint32_t sbase = wbase + C::WBYTES;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int x0 = blockIdx.x * TILE_X, y0 = blockIdx.y * TILE_Y;
  const int z0 = blockIdx.z * a.zc;
  const int z1 = min(z0 + a.zc, a.out.nz);
  if (z0 >= z1) return;  // uniform over the CTA, before any barrier or allocation

  if (tid == 0) {
    mbar_init(smem_u32(&bars[0]), 1);
    mbar_init(smem_u32(&bars[1]), 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(holder), C::NCOLS);
  for (int i = tid; i < C::WBYTES / 16; i += CONV_THREADS) cp_async16(wbase + 16 * i, a.wpk + 8 * i, true);
  for (int p = 0; p < 3; ++p) load_plane<CIN>(a, sbase + p * C::SLOT, z0 - 1 + p, x0, y0);
  cp_async_commit();
  cp_async_wait_all();
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *holder;
  constexpr uint32_t IDESC = idesc_bf16(N, 128);
  const int nl = z1 - z0;
  bool bad = false;
  for (int it = 0; it <= nl; ++it) {
    if (it >= 1) {  // layer it-1's MMAs: its accumulator is ready, the slot of plane z-2 is free
      const int pv = it - 1;
      const bool ok = mbar_wait(smem_u32(&bars[pv & 1]), (uint32_t)((pv >> 1) & 1));
      if (__syncthreads_or(!ok)) {
        bad = true;
        break;
      }
      tc_fence_after();
    }
    if (it < nl) {
      const int p = z0 + it + 2;
      if (p <= z1) load_plane<CIN>(a, sbase + ((it + 3) & 3) * C::SLOT, p, x0, y0);
      cp_async_commit();
      if (tid == 0) {
        const uint32_t d = tmem + (uint32_t)((it & 1) * N);
        uint32_t acc = 0;
#pragma unroll 1
        for (int dz = 0; dz < 3; ++dz) {
          const uint32_t sl = sbase + (uint32_t)(((it + dz) & 3) * C::SLOT);
#pragma unroll
          for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx)
#pragma unroll
              for (int c = 0; c < C::KC; ++c) {
                const int t = dz * 9 + dy * 3 + dx;
                const uint32_t aa = sl + (uint32_t)(2 * c * OCT_BYTES + (dy * SX + dx) * 16);
                const uint32_t ba = wbase + (uint32_t)((t * C::KC + c) * (N * 32));
                mma_bf16(d, sdesc(aa, OCT_BYTES, SX * 16), sdesc(ba, (N / 8) * 128, 128), IDESC, acc);
                acc = 1;
              }
        }
        mma_commit(smem_u32(&bars[it & 1]));
      }
      __syncwarp();
    }
    if (it >= 1) conv_epilogue<N>(a, tmem, it - 1, z0 + it - 1, x0, y0);
    cp_async_wait_all();
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
  }
  if (bad) {
    cp_async_wait_all();
    if (tid == 0) atomicExch(a.err, 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, C::NCOLS);
}

// ------------------------------------------------------------------ weight packing
// forward: B[t][c][kg][ng][n8][k8] = W[co = 8 ng + n8][ci = 16 c + 8 kg + k8][t]
// data gradient: the adjoint is a convolution with flipped taps and swapped
// channels: B[t][0][kg][ng][n8][k8] = W[co = 8 kg + k8][ci = 8 ng + n8][26 - t]
__global__ void pack_weights_kernel(const float* __restrict__ W, int cout, int cin, int npad, int bwd,
                                    uint16_t* __restrict__ out) {
  const int kdim = bwd ? 16 : cin;  // K channels per tap (forward: cin; adjoint: cout padded)
  const int ndim = bwd ? cin : npad;
  const int total = 27 * kdim * ndim;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int k8 = e & 7, n8 = (e >> 3) & 7;
    int r = e >> 6;
    const int ng = r % (ndim / 8);
    r /= ndim / 8;
    const int kg = r & 1;
    r >>= 1;
    const int kc = kdim / 16;
    const int c = r % kc;
    const int t = r / kc;
    const int n = 8 * ng + n8, k = 16 * c + 8 * kg + k8;
    float v = 0.0f;
    if (!bwd) {
      if (n < cout) v = W[((int64_t)n * cin + k) * 27 + t];
    } else {
      if (k < cout) v = W[((int64_t)k * cin + n) * 27 + (26 - t)];
    }
    out[e] = f2bf(v);
  }
}

// ------------------------------------------------------------------ transfer operators
// coarse[X] = s * sum_{d in {-1,0,1}^3} 2^-(|dx|+|dy|+|dz|) fine[2X + d]  (then * [mask > 0])
__global__ void restrict_kernel(TView f, TView c, float s, TView mask) {
  const int64_t Vc = (int64_t)c.nx * c.ny * c.nz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 2 * Vc; i += (int64_t)gridDim.x * blockDim.x) {
    const int o = (int)(i / Vc);
    const int64_t v = i - o * Vc;
    const int X = (int)(v % c.nx), Y = (int)((v / c.nx) % c.ny), Z = (int)(v / ((int64_t)c.nx * c.ny));
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int dz = -1; dz <= 1; ++dz) {
      const int z = 2 * Z + dz;
      if (z < 0 || z >= f.nz) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        const int y = 2 * Y + dy;
        if (y < 0 || y >= f.ny) continue;
        for (int dx = -1; dx <= 1; ++dx) {
          const int x = 2 * X + dx;
          if (x < 0 || x >= f.nx) continue;
          const float w = 1.0f / (float)(1 << (abs(dx) + abs(dy) + abs(dz)));
          const uint4 q = *reinterpret_cast<const uint4*>(f.p + vox_addr(f, o, x, y, z));
          const uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
          for (int k = 0; k < 8; ++k) acc[k] += w * bf2f((uint16_t)(u[k >> 1] >> (16 * (k & 1))));
        }
      }
    }
    uint4 mk = make_uint4(0, 0, 0, 0);
    if (mask.p) mk = *reinterpret_cast<const uint4*>(mask.p + vox_addr(mask, o, X, Y, Z));
    const uint32_t mu[4] = {mk.x, mk.y, mk.z, mk.w};
    uint32_t outw[4];
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
      float a0 = s * acc[k], a1 = s * acc[k + 1];
      if (mask.p) {
        if (!(bf2f((uint16_t)(mu[k >> 1])) > 0.0f)) a0 = 0.0f;
        if (!(bf2f((uint16_t)(mu[k >> 1] >> 16)) > 0.0f)) a1 = 0.0f;
      }
      outw[k >> 1] = (uint32_t)f2bf(a0) | ((uint32_t)f2bf(a1) << 16);
    }
    *reinterpret_cast<uint4*>(c.p + vox_addr(c, o, X, Y, Z)) = make_uint4(outw[0], outw[1], outw[2], outw[3]);
  }
}

// fine[x] = (s * sum_X P[x, X] coarse[X] + add[x]) * [mask[x] > 0]   (add, mask optional)
__global__ void prolong_kernel(TView c, TView f, float s, TView add, TView mask) {
  const int64_t Vf = (int64_t)f.nx * f.ny * f.nz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 2 * Vf; i += (int64_t)gridDim.x * blockDim.x) {
    const int o = (int)(i / Vf);
    const int64_t v = i - o * Vf;
    const int x = (int)(v % f.nx), y = (int)((v / f.nx) % f.ny), z = (int)(v / ((int64_t)f.nx * f.ny));
    const int xs[2] = {x >> 1, (x + 1) >> 1}, ys[2] = {y >> 1, (y + 1) >> 1}, zs[2] = {z >> 1, (z + 1) >> 1};
    const int nxs = (x & 1) ? 2 : 1, nys = (y & 1) ? 2 : 1, nzs = (z & 1) ? 2 : 1;
    const float w = 1.0f / (float)(nxs * nys * nzs);
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int a2 = 0; a2 < nzs; ++a2)
      for (int a1 = 0; a1 < nys; ++a1)
        for (int a0 = 0; a0 < nxs; ++a0) {
          const uint4 q = *reinterpret_cast<const uint4*>(c.p + vox_addr(c, o, xs[a0], ys[a1], zs[a2]));
          const uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
          for (int k = 0; k < 8; ++k) acc[k] += w * bf2f((uint16_t)(u[k >> 1] >> (16 * (k & 1))));
        }
    uint32_t ad[4] = {0, 0, 0, 0}, mu[4] = {0, 0, 0, 0};
    if (add.p) {
      const uint4 q = *reinterpret_cast<const uint4*>(add.p + vox_addr(add, o, x, y, z));
      ad[0] = q.x, ad[1] = q.y, ad[2] = q.z, ad[3] = q.w;
    }
    if (mask.p) {
      const uint4 q = *reinterpret_cast<const uint4*>(mask.p + vox_addr(mask, o, x, y, z));
      mu[0] = q.x, mu[1] = q.y, mu[2] = q.z, mu[3] = q.w;
    }
    uint32_t outw[4];
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
      float r0 = s * acc[k], r1 = s * acc[k + 1];
      if (add.p) {
        r0 += bf2f((uint16_t)ad[k >> 1]);
        r1 += bf2f((uint16_t)(ad[k >> 1] >> 16));
      }
      if (mask.p) {
        if (!(bf2f((uint16_t)mu[k >> 1]) > 0.0f)) r0 = 0.0f;
        if (!(bf2f((uint16_t)(mu[k >> 1] >> 16)) > 0.0f)) r1 = 0.0f;
      }
      outw[k >> 1] = (uint32_t)f2bf(r0) | ((uint32_t)f2bf(r1) << 16);
    }
    *reinterpret_cast<uint4*>(f.p + vox_addr(f, o, x, y, z)) = make_uint4(outw[0], outw[1], outw[2], outw[3]);
  }
}

// float32 planar versions for the network output (nc channels [c][voxel]):
// coarse = (1/8) P^T fine, fine = P coarse
__global__ void restrict_f32_kernel(const float* __restrict__ f, Grid3 gf, float* __restrict__ c, Grid3 gc, int nc) {
  const int64_t Vc = gc.nv(), Vf = gf.nv();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc * Vc; i += (int64_t)gridDim.x * blockDim.x) {
    const int ch = (int)(i / Vc);
    const int64_t v = i - ch * Vc;
    const int X = (int)(v % gc.nx), Y = (int)((v / gc.nx) % gc.ny), Z = (int)(v / ((int64_t)gc.nx * gc.ny));
    float acc = 0.0f;
    for (int dz = -1; dz <= 1; ++dz) {
      const int z = 2 * Z + dz;
      if (z < 0 || z >= gf.nz) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        const int y = 2 * Y + dy;
        if (y < 0 || y >= gf.ny) continue;
        for (int dx = -1; dx <= 1; ++dx) {
          const int x = 2 * X + dx;
          if (x < 0 || x >= gf.nx) continue;
          acc += f[ch * Vf + ((int64_t)z * gf.ny + y) * gf.nx + x] / (float)(1 << (abs(dx) + abs(dy) + abs(dz)));
        }
      }
    }
    c[i] = 0.125f * acc;
  }
}
__global__ void prolong_f32_kernel(const float* __restrict__ c, Grid3 gc, float* __restrict__ f, Grid3 gf, int nc) {
  const int64_t Vc = gc.nv(), Vf = gf.nv();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc * Vf; i += (int64_t)gridDim.x * blockDim.x) {
    const int ch = (int)(i / Vf);
    const int64_t v = i - ch * Vf;
    const int x = (int)(v % gf.nx), y = (int)((v / gf.nx) % gf.ny), z = (int)(v / ((int64_t)gf.nx * gf.ny));
    const int xs[2] = {x >> 1, (x + 1) >> 1}, ys[2] = {y >> 1, (y + 1) >> 1}, zs[2] = {z >> 1, (z + 1) >> 1};
    const int nxs = (x & 1) ? 2 : 1, nys = (y & 1) ? 2 : 1, nzs = (z & 1) ? 2 : 1;
    float acc = 0.0f;
    for (int a2 = 0; a2 < nzs; ++a2)
      for (int a1 = 0; a1 < nys; ++a1)
        for (int a0 = 0; a0 < nxs; ++a0) acc += c[ch * Vc + ((int64_t)zs[a2] * gc.ny + ys[a1]) * gc.nx + xs[a0]];
    f[i] = acc / (float)(nxs * nys * nzs);
  }
}

// ------------------------------------------------------------------ weight gradient
// g[(co cin + ci) 27 + t] = sum_b part[b][co][ci][t] for co < cout, in block order
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, int nblk, int cin, int cout,
                                    float* __restrict__ g) {
  const int n = cout * cin * 27;
  const int stride = 16 * cin * 27;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * stride + e];
    g[e] = s;
  }
}

// ------------------------------------------------------------------ weight gradient on tensor cores
// dW[co][ci][t] = sum_v dY[v][co] X[v + delta_t][ci] as implicit GEMMs, one per group of
// MT = 128 / CIN taps: D[(t_local, ci)][co] (M = 128, N = 16) accumulates over K = voxels,
// 16 voxels per tcgen05.mma.  Both operands are staged K-major without swizzle (core
// matrix = 8 rows x 8 voxels, the layout the convolution's B operand uses):
// A[m][k] = X[v_k + delta_t(m)][ci(m)], B[co][k] = dY[v_k][co].  Each CTA walks a
// contiguous range of voxels with double-buffered staging; its TMEM accumulators (16
// columns per tap group) become per-CTA partials in the [co][ci][27] layout that
// wgrad_reduce_kernel sums in a fixed order.
constexpr int WGM_THREADS = 128;
constexpr int WGM_KS = 16;  // voxels per stage: one MMA K-step

template <int CIN>
struct WgmCfg {
  static constexpr int MT = 128 / CIN;             // taps per group
  static constexpr int NG = (27 + MT - 1) / MT;    // tap groups
  static constexpr int ABYTES = 128 * WGM_KS * 2;  // one group's A tile
  static constexpr int BBYTES = 16 * WGM_KS * 2;
  static constexpr int STAGE = NG * ABYTES + BBYTES;
  static constexpr int HEAD = 128;
  static constexpr int SMEM = HEAD + 2 * STAGE;
  static constexpr int NCOLS = NG * 16 <= 32 ? 32 : (NG * 16 <= 64 ? 64 : 128);
};

template <int CIN>
__global__ void __launch_bounds__(WGM_THREADS) wgrad_mma_kernel(TView x, TView g, int spc, int64_t nstages,
                                                              float* __restrict__ part, int* err) {
  using C = WgmCfg<CIN>;
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm);
  uint32_t* holder = reinterpret_cast<uint32_t*>(sm + 16);
  uint8_t* stage_base = sm + C::HEAD;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t V = (int64_t)g.nx * g.ny * g.nz;
  const int64_t s0 = (int64_t)blockIdx.x * spc, s1 = min(nstages, s0 + spc);
  if (tid == 0) {
    mbar_init(smem_u32(&bars[0]), 1);
    mbar_init(smem_u32(&bars[1]), 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(holder), C::NCOLS);
  // both buffers start at zero: the rows of the taps past 26 stay zero
  for (int i = tid; i < 2 * C::STAGE / 16; i += WGM_THREADS)
    reinterpret_cast<uint4*>(stage_base)[i] = make_uint4(0, 0, 0, 0);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *holder;
  constexpr uint32_t IDESC = idesc_bf16(16, 128);
  bool bad = false;
  for (int64_t st = s0; st < s1; ++st) {
    const int it = (int)(st - s0), b = it & 1;
    if (it >= 2) {  // the MMAs that read this buffer two stages ago are done
      const bool ok = mbar_wait(smem_u32(&bars[b]), (uint32_t)(((it - 2) >> 1) & 1));
      if (__syncthreads_or(!ok)) {
        bad = true;
        break;
      }
    }
    uint16_t* A = reinterpret_cast<uint16_t*>(stage_base + b * C::STAGE);
    uint16_t* B = reinterpret_cast<uint16_t*>(stage_base + b * C::STAGE + C::NG * C::ABYTES);
    const int64_t vbase = st * WGM_KS;
    // A: items (voxel k, tap t, input octet o)
    for (int i = tid; i < WGM_KS * 27 * (CIN / 8); i += WGM_THREADS) {
      const int k = i % WGM_KS, rest = i / WGM_KS, t = rest % 27, o = rest / 27;
      const int64_t v = vbase + k;
      uint4 q = make_uint4(0, 0, 0, 0);
      if (v < V) {
        const int vx = (int)(v % g.nx), vy = (int)((v / g.nx) % g.ny), vz = (int)(v / ((int64_t)g.nx * g.ny));
        const int xx = vx + t % 3 - 1, yy = vy + (t / 3) % 3 - 1, zz = vz + t / 9 - 1;
        if (xx >= 0 && xx < x.nx && yy >= 0 && yy < x.ny && zz >= 0 && zz < x.nz)
          q = *reinterpret_cast<const uint4*>(x.p + vox_addr(x, o, xx, yy, zz));
      }
      const uint32_t u[4] = {q.x, q.y, q.z, q.w};
      uint16_t* At = A + (t / C::MT) * (C::ABYTES / 2);
      const int m0 = (t % C::MT) * CIN + o * 8;  // rows m0 .. m0+7 (one core-matrix row group)
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int m = m0 + e;
        At[((k >> 3) * 16 + (m >> 3)) * 64 + (m & 7) * 8 + (k & 7)] = (uint16_t)(u[e >> 1] >> (16 * (e & 1)));
      }
    }
    // B: items (voxel k, gradient octet q)
    for (int i = tid; i < WGM_KS * 2; i += WGM_THREADS) {
      const int k = i % WGM_KS, qo = i / WGM_KS;
      const int64_t v = vbase + k;
      uint4 q = make_uint4(0, 0, 0, 0);
      if (v < V) {
        const int vx = (int)(v % g.nx), vy = (int)((v / g.nx) % g.ny), vz = (int)(v / ((int64_t)g.nx * g.ny));
        q = *reinterpret_cast<const uint4*>(g.p + vox_addr(g, qo, vx, vy, vz));
      }
      const uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int co = qo * 8 + e;
        B[((k >> 3) * 2 + (co >> 3)) * 64 + (co & 7) * 8 + (k & 7)] = (uint16_t)(u[e >> 1] >> (16 * (e & 1)));
      }
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t abase = smem_u32(A), bbase = smem_u32(B);
#pragma unroll 1
      for (int gi = 0; gi < C::NG; ++gi)
        mma_bf16(tmem + (uint32_t)(gi * 16), sdesc(abase + gi * C::ABYTES, 16 * 128, 128), sdesc(bbase, 2 * 128, 128),
                 IDESC, it > 0 ? 1u : 0u);
      mma_commit(smem_u32(&bars[b]));
    }
    __syncwarp();
  }
  const int nst = (int)(s1 - s0);
  if (!bad && nst > 0) {
    const int last = nst - 1;
    const bool ok = mbar_wait(smem_u32(&bars[last & 1]), (uint32_t)((last >> 1) & 1));
    if (__syncthreads_or(!ok)) bad = true;
  }
  if (!bad) {
    tc_fence_after();
    const int m = warp * 32 + lane;
    const int t_local = m / CIN, ci = m % CIN;
    float* dst = part + (int64_t)blockIdx.x * (16 * CIN * 27);
#pragma unroll 1
    for (int gi = 0; gi < C::NG; ++gi) {
      uint32_t r[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(gi * 16), r);
      const int t = gi * C::MT + t_local;
      if (t < 27) {
#pragma unroll
        for (int co = 0; co < 16; ++co)
          dst[((int64_t)co * CIN + ci) * 27 + t] = nst > 0 ? __uint_as_float(r[co]) : 0.0f;
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, C::NCOLS);
}

// ------------------------------------------------------------------ loss
// valid(c, v) = !(dmask[v] bit c); d = valid ? y[c][v] - t[c][v] / kc_c : 0;
// loss partial += w d^2; dy[v][c] = 2 w d / cnt (channels >= cout: 0); w: the pair's weight
__global__ void loss_kernel(const float* __restrict__ y, const uint16_t* __restrict__ t,
                            const uint8_t* __restrict__ dmask, int cout, int64_t V, float inv_cnt, float4 kinv,
                            float wgt, TView dy, double* __restrict__ part) {
  double s = 0.0;
  const float ki[4] = {kinv.x, kinv.y, kinv.z, kinv.w};
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(v % dy.nx), yy = (int)((v / dy.nx) % dy.ny), z = (int)(v / ((int64_t)dy.nx * dy.ny));
    float gch[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) gch[c] = 0.0f;
    const uint8_t mk = dmask ? dmask[v] : 0;
    for (int c = 0; c < cout; ++c) {
      const bool valid = !((mk >> c) & 1);
      const float d = valid ? y[(int64_t)c * V + v] - bf2f(t[(int64_t)c * V + v]) * ki[c] : 0.0f;
      s += (double)wgt * d * d;
      gch[c] = 2.0f * wgt * d * inv_cnt;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      uint4 o;
      o.x = (uint32_t)f2bf(gch[8 * q + 0]) | ((uint32_t)f2bf(gch[8 * q + 1]) << 16);
      o.y = (uint32_t)f2bf(gch[8 * q + 2]) | ((uint32_t)f2bf(gch[8 * q + 3]) << 16);
      o.z = (uint32_t)f2bf(gch[8 * q + 4]) | ((uint32_t)f2bf(gch[8 * q + 5]) << 16);
      o.w = (uint32_t)f2bf(gch[8 * q + 6]) | ((uint32_t)f2bf(gch[8 * q + 7]) << 16);
      *reinterpret_cast<uint4*>(dy.p + vox_addr(dy, q, x, yy, z)) = o;
    }
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// out[slot] = scale * sum of part[0..n)  (one CTA, fixed order)
__global__ void sum_kernel(const double* __restrict__ part, int n, double scale, double* __restrict__ out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = scale * sh[0];
}

// ------------------------------------------------------------------ Adam
__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int64_t n, float lr, float b1, float b2, float eps,
                            float bc1, float bc2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

// ------------------------------------------------------------------ preconditioner I/O
// network input: ch c < ncomp: s_c = (D^{-1} r)_c * g / dbar_c (0 on Dirichlet rows);
// then either the indicator planes ph (ch ncomp + i = phi_i) or, modulated, the
// products ch ncomp + ncomp i + c = s_c (1 + phi_i) / 2; other channels 0.  Rows are
// mesh nodes (level-0 voxels).
__global__ void pc_pack_kernel(const double* __restrict__ r, const double* __restrict__ dinv, Planes ph,
                               int modulate, const uint8_t* __restrict__ dmask, int ncomp, double g, D4 dbinv,
                               int64_t nn, TView xin) {
  const double* db = dbinv.c;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nn; v += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(v % xin.nx), y = (int)((v / xin.nx) % xin.ny), z = (int)(v / ((int64_t)xin.nx * xin.ny));
    const uint8_t mk = dmask ? dmask[v] : 0;
    float ch[16];
    double sv[4] = {0, 0, 0, 0};
#pragma unroll
    for (int c = 0; c < 16; ++c) ch[c] = 0.0f;
    for (int c = 0; c < ncomp; ++c) {
      const int64_t i = (int64_t)c * nn + v;
      sv[c] = ((mk >> c) & 1) ? 0.0 : dinv[i] * r[i] * g * db[c];
      ch[c] = (float)sv[c];
    }
    if (modulate) {
      for (int i = 0; i < ph.n; ++i) {
        const double a = 0.5 * (1.0 + ph.p[i][v]);
        for (int c = 0; c < ncomp; ++c) ch[ncomp + ncomp * i + c] = (float)(sv[c] * a);
      }
    } else {
      for (int i = 0; i < ph.n; ++i) ch[ncomp + i] = (float)ph.p[i][v];
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      uint4 o;
      o.x = (uint32_t)f2bf(ch[8 * q + 0]) | ((uint32_t)f2bf(ch[8 * q + 1]) << 16);
      o.y = (uint32_t)f2bf(ch[8 * q + 2]) | ((uint32_t)f2bf(ch[8 * q + 3]) << 16);
      o.z = (uint32_t)f2bf(ch[8 * q + 4]) | ((uint32_t)f2bf(ch[8 * q + 5]) << 16);
      o.w = (uint32_t)f2bf(ch[8 * q + 6]) | ((uint32_t)f2bf(ch[8 * q + 7]) << 16);
      *reinterpret_cast<uint4*>(xin.p + vox_addr(xin, q, x, y, z)) = o;
    }
  }
}

// z_c = (D^{-1} r)_c + h dk_c y_c, z_c = r_c on Dirichlet rows
__global__ void pc_unpack_kernel(const double* __restrict__ r, const double* __restrict__ dinv,
                                 const float* __restrict__ y, const uint8_t* __restrict__ dmask, int ncomp,
                                 double h, D4 dk, int64_t nn, double* __restrict__ z) {
  const double* d = dk.c;
  const int64_t n = (int64_t)ncomp * nn;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / nn);
    const int64_t v = i - (int64_t)c * nn;
    const bool dir = dmask && ((dmask[v] >> c) & 1);
    z[i] = dir ? r[i] : dinv[i] * r[i] + h * d[c] * (double)y[i];
  }
}

// training target t_c = (e_c - (D^{-1} r)_c) g / dbar_c (0 on Dirichlet rows), with
// r = ra - rb and e = ea - eb
__global__ void pc_target_kernel(const double* __restrict__ ra, const double* __restrict__ rb,
                                 const double* __restrict__ ea, const double* __restrict__ eb,
                                 const double* __restrict__ dinv, const uint8_t* __restrict__ dmask, int ncomp,
                                 double g, D4 dbinv, int64_t nn, uint16_t* __restrict__ t) {
  const double* db = dbinv.c;
  const int64_t n = (int64_t)ncomp * nn;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / nn);
    const int64_t v = i - (int64_t)c * nn;
    const bool dir = dmask && ((dmask[v] >> c) & 1);
    const double r = ra[i] - (rb ? rb[i] : 0.0);
    const double e = ea[i] - (eb ? eb[i] : 0.0);
    t[i] = f2bf(dir ? 0.0f : (float)((e - dinv[i] * r) * g * db[c]));
  }
}

// r = a - b
__global__ void sub_kernel(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ r,
                           int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = a[i] - b[i];
}

// per component: sum of dinv and count over non-Dirichlet rows (sums[2c], sums[2c+1])
__global__ void dinv_mean_kernel(const double* __restrict__ dinv, const uint8_t* __restrict__ dmask, int ncomp,
                                 int64_t nn, double* __restrict__ part) {
  double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nn; v += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t mk = dmask ? dmask[v] : 0;
    for (int c = 0; c < ncomp; ++c)
      if (!((mk >> c) & 1)) {
        s[2 * c] += dinv[(int64_t)c * nn + v];
        s[2 * c + 1] += 1.0;
      }
  }
  __shared__ double sh[8][256];
  for (int k = 0; k < 8; ++k) sh[k][threadIdx.x] = s[k];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < 8; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 8) part[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = sh[threadIdx.x][0];
}

// per component: sum of t^2 over valid rows of pairs [0, npairs) (kc normalisation)
__global__ void target_rms_kernel(const uint16_t* __restrict__ t, int64_t pair_stride, int npairs,
                                  const uint8_t* __restrict__ dmask, int ncomp, int64_t nn, double* __restrict__ part) {
  double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int p = 0; p < npairs; ++p)
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nn; v += (int64_t)gridDim.x * blockDim.x) {
      const uint8_t mk = dmask ? dmask[v] : 0;
      for (int c = 0; c < ncomp; ++c)
        if (!((mk >> c) & 1)) {
          const float q = bf2f(t[p * pair_stride + (int64_t)c * nn + v]);
          s[2 * c] += (double)q * q;
          s[2 * c + 1] += 1.0;
        }
    }
  __shared__ double sh[8][256];
  for (int k = 0; k < 8; ++k) sh[k][threadIdx.x] = s[k];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < 8; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 8) part[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = sh[threadIdx.x][0];
}

}  // namespace pcn
}  // namespace fsi

// ====================================================================== host side
using namespace fsi;
using namespace fsi::pcn;

namespace {

int vgrid1(int64_t n, int tb = 256) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + tb - 1) / tb, 152 * 8)); }

TView view(uint16_t* p, int noct, int oct0, const Grid3& g) { return TView{p, noct, oct0, g.nx, g.ny, g.nz}; }
TView none() { return TView{nullptr, 0, 0, 0, 0, 0}; }

template <int CIN, int N>
int launch_conv(fsi_pc* pc, const TView& in, const TView& out, const TView& mask, float* out32, int nreal,
                const uint16_t* wpk, int relu) {
  using C = ConvCfg<CIN, N>;
  fsi_mesh* m = pc->m;
  if (int rc = ensure_smem_attr(reinterpret_cast<const void*>(&conv_mma_kernel<CIN, N>), C::SMEM)) return rc;
  const int gx = (out.nx + TILE_X - 1) / TILE_X, gy = (out.ny + TILE_Y - 1) / TILE_Y;
  const int cols = gx * gy;
  // CTAs resident per SM (shared memory bound) x 152 SMs: enough z-chunks to fill them
  const int per_sm = std::max(1, std::min(8, (227 * 1024) / (C::SMEM + 1024)));
  const int zc = std::max(1, (int)((int64_t)out.nz * cols / (per_sm * 152)));
  const int gz = (out.nz + zc - 1) / zc;
  ConvArgs a{in, out, mask, out32, nreal, wpk, zc, relu, pc->err};
  FSI_LAUNCH(m, P_PC_CONV, (conv_mma_kernel<CIN, N><<<dim3(gx, gy, gz), CONV_THREADS, C::SMEM, m->stream>>>(a)));
  // algorithmic bytes: input and output channels once per voxel, plus the mask
  const double V = (double)out.nx * out.ny * out.nz;
  prof_bytes(m, P_PC_CONV, V * (2.0 * CIN + (out32 ? 4.0 * nreal : 2.0 * N) + (mask.p ? 2.0 * N : 0.0)));
  pc->flops += 2.0 * V * 27.0 * CIN * N;
  return FSI_OK;
}

int conv(fsi_pc* pc, int cin, int n, const TView& in, const TView& out, const TView& mask, float* out32, int nreal,
         const uint16_t* wpk, int relu) {
  if (cin == 16 && n == 16) return launch_conv<16, 16>(pc, in, out, mask, out32, nreal, wpk, relu);
  if (cin == 32 && n == 16) return launch_conv<32, 16>(pc, in, out, mask, out32, nreal, wpk, relu);
  if (cin == 16 && n == 32) return launch_conv<16, 32>(pc, in, out, mask, out32, nreal, wpk, relu);
  return set_error(FSI_EINVAL, "pc: unsupported convolution shape");
}

template <int CIN>
int launch_wgrad_mma(fsi_pc* pc, const TView& x, const TView& g, int* nblk_out) {
  using C = WgmCfg<CIN>;
  fsi_mesh* m = pc->m;
  if (int rc = ensure_smem_attr(reinterpret_cast<const void*>(&wgrad_mma_kernel<CIN>), C::SMEM)) return rc;
  const int64_t V = (int64_t)g.nx * g.ny * g.nz;
  const int64_t nst = (V + WGM_KS - 1) / WGM_KS;
  const int per_sm = std::max(1, std::min(std::min(8, 512 / C::NCOLS), (227 * 1024) / (C::SMEM + 1024)));
  const int64_t target = (int64_t)per_sm * 152;
  const int spc = (int)std::max<int64_t>(1, (nst + target - 1) / target);
  const int nblk = (int)((nst + spc - 1) / spc);
  if ((int64_t)nblk * 16 * CIN * 27 > pc->wpart_n) return set_error(FSI_EINVAL, "pc: weight-gradient scratch too small");
  FSI_LAUNCH(m, P_PC_WGRAD, (wgrad_mma_kernel<CIN><<<nblk, WGM_THREADS, C::SMEM, m->stream>>>(x, g, spc, nst,
                                                                                              pc->wpart, pc->err)));
  *nblk_out = nblk;
  return FSI_OK;
}

int wgrad(fsi_pc* pc, int layer, const TView& x, const TView& g) {
  fsi_mesh* m = pc->m;
  const int cin = pc->lcin[layer], cout = pc->lcout[layer];
  int nblk = 0, rc;
  if (cin == 16) rc = launch_wgrad_mma<16>(pc, x, g, &nblk);
  else rc = launch_wgrad_mma<32>(pc, x, g, &nblk);
  if (rc) return rc;
  const int n = cout * cin * 27;
  FSI_LAUNCH(m, P_PC_WGRAD, (wgrad_reduce_kernel<<<(n + 255) / 256, 256, 0, m->stream>>>(pc->wpart, nblk, cin, cout,
                                                                                          pc->grad + pc->woff[layer])));
  pc->flops += 2.0 * (double)g.nx * g.ny * g.nz * 27.0 * cin * 16;
  return FSI_OK;
}

int restrict_(fsi_pc* pc, const TView& f, const TView& c, float s, const TView& mask) {
  const int64_t n = 2LL * c.nx * c.ny * c.nz;
  FSI_LAUNCH(pc->m, P_PC_AUX, (restrict_kernel<<<vgrid1(n), 256, 0, pc->m->stream>>>(f, c, s, mask)));
  return FSI_OK;
}
int prolong_(fsi_pc* pc, const TView& c, const TView& f, float s, const TView& add, const TView& mask) {
  const int64_t n = 2LL * f.nx * f.ny * f.nz;
  FSI_LAUNCH(pc->m, P_PC_AUX, (prolong_kernel<<<vgrid1(n), 256, 0, pc->m->stream>>>(c, f, s, add, mask)));
  return FSI_OK;
}

}  // namespace

namespace fsi {
namespace pcn {

// layer indices in storage order
enum { ENC0A, ENC0B, ENC1A, ENC1B, ENC2A, ENC2B, BOTA, BOTB, DEC2A, DEC2B, DEC1A, DEC1B, DEC0A, DEC0B, OUT };
static int enc_a(int l) { return 2 * l; }
static int enc_b(int l) { return 2 * l + 1; }
static int dec_a(int l) { return DEC2A + 2 * (2 - l); }
static int dec_b(int l) { return DEC2A + 2 * (2 - l) + 1; }

int pack_weights(fsi_pc* pc) {
  fsi_mesh* m = pc->m;
  for (int l = 0; l < NLAYER; ++l) {
    const int cin = pc->lcin[l], cout = pc->lcout[l];
    const int npad = 16;
    const float* W = pc->w + pc->woff[l];
    const int nf = 27 * cin * npad;
    FSI_LAUNCH(m, P_PC_AUX, (pack_weights_kernel<<<(nf + 255) / 256, 256, 0, m->stream>>>(W, cout, cin, npad, 0,
                                                                                          pc->wf[l])));
    if (l != ENC0A) {
      const int nb = 27 * 16 * cin;
      FSI_LAUNCH(m, P_PC_AUX, (pack_weights_kernel<<<(nb + 255) / 256, 256, 0, m->stream>>>(W, cout, cin, npad, 1,
                                                                                            pc->wb[l])));
    }
  }
  return FSI_OK;
}

// y32 = network(x0)
int forward(fsi_pc* pc, const uint16_t* x0) {
  int rc;
  const Grid3* G = pc->lv;
  TView X0 = view(const_cast<uint16_t*>(x0), 2, 0, G[0]);
  TView nm = none();
  for (int l = 0; l < 3; ++l) {
    TView xin = l == 0 ? X0 : view(pc->x[l], 2, 0, G[l]);
    TView a = view(pc->a[l], 2, 0, G[l]);
    TView e = view(pc->cat[l], 4, 0, G[l]);
    if ((rc = conv(pc, pc->lcin[enc_a(l)], 16, xin, a, nm, nullptr, 0, pc->wf[enc_a(l)], !pc->linear))) return rc;
    if ((rc = conv(pc, 16, 16, a, e, nm, nullptr, 0, pc->wf[enc_b(l)], !pc->linear))) return rc;
    if ((rc = restrict_(pc, e, view(pc->x[l + 1], 2, 0, G[l + 1]), 0.125f, nm))) return rc;
  }
  {
    TView a3 = view(pc->a[3], 2, 0, G[3]), d3 = view(pc->d[3], 2, 0, G[3]);
    if ((rc = conv(pc, 16, 16, view(pc->x[3], 2, 0, G[3]), a3, nm, nullptr, 0, pc->wf[BOTA], !pc->linear))) return rc;
    if ((rc = conv(pc, 16, 16, a3, d3, nm, nullptr, 0, pc->wf[BOTB], !pc->linear))) return rc;
  }
  for (int l = 2; l >= 0; --l) {
    TView cat = view(pc->cat[l], 4, 0, G[l]);
    if ((rc = prolong_(pc, view(pc->d[l + 1], 2, 0, G[l + 1]), view(pc->cat[l], 4, 2, G[l]), 1.0f, nm, nm))) return rc;
    TView b = view(pc->b[l], 2, 0, G[l]), d = view(pc->d[l], 2, 0, G[l]);
    if ((rc = conv(pc, 32, 16, cat, b, nm, nullptr, 0, pc->wf[dec_a(l)], !pc->linear))) return rc;
    if ((rc = conv(pc, 16, 16, b, d, nm, nullptr, 0, pc->wf[dec_b(l)], !pc->linear))) return rc;
  }
  return conv(pc, 16, 16, view(pc->d[0], 2, 0, G[0]), view(pc->a[0], 2, 0, G[0]) /* unused */, nm, pc->y32,
              pc->cout, pc->wf[OUT], 0);
}

// gradient of the loss of target t (planar bf16 [cout][V0]) w.r.t. the weights into
// pc->grad; the loss (mean over valid rows times wgt, float64) into the device slot `loss`
int backward(fsi_pc* pc, const uint16_t* x0, const uint16_t* t, double* loss, double wgt = 1.0) {
  fsi_mesh* m = pc->m;
  int rc;
  const Grid3* G = pc->lv;
  const int64_t V0 = G[0].nv();
  TView nm = none();
  // ReLU derivative: mask by the stored activation (none for the linear network)
  auto mk = [&](const TView& t) { return pc->linear ? nm : t; };
  TView gy = view(pc->gd[0] /* reused as dL/dy */, 2, 0, G[0]);
  {
    const int nb = vgrid1(V0);
    const float4 kinv = make_float4((float)(1.0 / pc->kc[0]), (float)(1.0 / pc->kc[1]), (float)(1.0 / pc->kc[2]),
                                    (float)(1.0 / pc->kc[3]));
    FSI_LAUNCH(m, P_PC_AUX, (loss_kernel<<<nb, 256, 0, m->stream>>>(pc->y32, t, pc->dmask, pc->cout, V0,
                                                                   (float)(1.0 / pc->valid_rows), kinv,
                                                                   (float)wgt, gy, pc->lpart)));
    FSI_LAUNCH(m, P_PC_AUX, (sum_kernel<<<1, 256, 0, m->stream>>>(pc->lpart, nb, 1.0 / pc->valid_rows, loss)));
  }
  // output layer
  if ((rc = wgrad(pc, OUT, view(pc->d[0], 2, 0, G[0]), gy))) return rc;
  TView gd0 = view(pc->gb[0], 2, 0, G[0]);  // dL/d(d_0) pre-activation, kept in gb[0] until used
  if ((rc = conv(pc, 16, 16, gy, gd0, mk(view(pc->d[0], 2, 0, G[0])), nullptr, 0, pc->wb[OUT], 0))) return rc;
  TView gd = gd0;
  for (int l = 0; l < 3; ++l) {
    TView b = view(pc->b[l], 2, 0, G[l]);
    TView gb = view(pc->ga[l], 2, 0, G[l]);  // dL/d(b_l) pre-activation
    if ((rc = wgrad(pc, dec_b(l), b, gd))) return rc;
    if ((rc = conv(pc, 16, 16, gd, gb, mk(b), nullptr, 0, pc->wb[dec_b(l)], 0))) return rc;
    TView cat = view(pc->cat[l], 4, 0, G[l]);
    TView gcat = view(pc->gcat[l], 4, 0, G[l]);
    if ((rc = wgrad(pc, dec_a(l), cat, gb))) return rc;
    if ((rc = conv(pc, 16, 32, gb, gcat, nm, nullptr, 0, pc->wb[dec_a(l)], 0))) return rc;
    TView gdn = view(pc->gd[l + 1], 2, 0, G[l + 1]);
    // the adjoint of P is P^T (the restriction kernel with scale 1)
    if ((rc = restrict_(pc, view(pc->gcat[l], 4, 2, G[l]), gdn, 1.0f, mk(view(pc->d[l + 1], 2, 0, G[l + 1]))))) return rc;
    gd = gdn;
  }
  TView a3 = view(pc->a[3], 2, 0, G[3]);
  TView ga3 = view(pc->ga[3], 2, 0, G[3]);
  if ((rc = wgrad(pc, BOTB, a3, gd))) return rc;
  if ((rc = conv(pc, 16, 16, gd, ga3, mk(a3), nullptr, 0, pc->wb[BOTB], 0))) return rc;
  TView x3 = view(pc->x[3], 2, 0, G[3]);
  TView gx = view(pc->gx[3], 2, 0, G[3]);
  if ((rc = wgrad(pc, BOTA, x3, ga3))) return rc;
  if ((rc = conv(pc, 16, 16, ga3, gx, nm, nullptr, 0, pc->wb[BOTA], 0))) return rc;
  for (int l = 2; l >= 0; --l) {
    TView e = view(pc->cat[l], 4, 0, G[l]);
    TView ge = view(pc->ge[l], 2, 0, G[l]);
    if ((rc = prolong_(pc, gx, ge, 0.125f, view(pc->gcat[l], 4, 0, G[l]), mk(e)))) return rc;
    TView a = view(pc->a[l], 2, 0, G[l]);
    TView ga = view(pc->ga[l], 2, 0, G[l]);
    if ((rc = wgrad(pc, enc_b(l), a, ge))) return rc;
    if ((rc = conv(pc, 16, 16, ge, ga, mk(a), nullptr, 0, pc->wb[enc_b(l)], 0))) return rc;
    TView xin = l == 0 ? view(const_cast<uint16_t*>(x0), 2, 0, G[0]) : view(pc->x[l], 2, 0, G[l]);
    if ((rc = wgrad(pc, enc_a(l), xin, ga))) return rc;
    if (l > 0) {
      gx = view(pc->gx[l], 2, 0, G[l]);
      if ((rc = conv(pc, 16, 16, ga, gx, nm, nullptr, 0, pc->wb[enc_a(l)], 0))) return rc;
    }
  }
  return FSI_OK;
}

int adam(fsi_pc* pc, float lr) {
  fsi_mesh* m = pc->m;
  ++pc->adam_t;
  const double b1 = 0.9, b2 = 0.999;
  const float bc1 = (float)(1.0 - std::pow(b1, (double)pc->adam_t));
  const float bc2 = (float)(1.0 - std::pow(b2, (double)pc->adam_t));
  FSI_LAUNCH(m, P_PC_AUX, (adam_kernel<<<vgrid1(pc->nw), 256, 0, m->stream>>>(pc->w, pc->mo, pc->vo, pc->grad, pc->nw,
                                                                             lr, (float)b1, (float)b2, 1e-8f, bc1,
                                                                             bc2)));
  return FSI_OK;
}

// the indicator planes the input uses: all phases, or the solids when modulated
static Planes input_planes(const fsi_pc* pc) {
  const fsi_mesh* m = pc->m;
  Planes p{};
  const double* base = m->staged_xa + 4 * m->nn;
  if (pc->modulate) {
    for (int i = 0; i < m->N && p.n < 3; ++i)
      if (m->phases[i].is_solid) p.p[p.n++] = base + (int64_t)i * m->nn;
  } else {
    for (int i = 0; i < m->N && i < 12; ++i) p.p[p.n++] = base + (int64_t)i * m->nn;
  }
  return p;
}

// z = M(r) for a block vector r (device [ncomp][nn]) with known norm rnorm, using the
// Jacobi inverse diagonal dinv and the staged phases
int apply(fsi_pc* pc, const double* r, double rnorm, const double* dinv, double* z) {
  fsi_mesh* m = pc->m;
  const int64_t nn = m->nn;
  if (!(rnorm > 0.0) || !std::isfinite(rnorm)) {
    FSI_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * pc->ncomp * nn, m->stream));
    return FSI_OK;
  }
  int rc;
  const double nrows = (double)pc->ncomp * nn;
  const double g = std::sqrt(nrows) / rnorm;
  const D4 dbinv = {{1.0 / pc->dbar[0], 1.0 / pc->dbar[1], 1.0 / pc->dbar[2], 1.0 / pc->dbar[3]}};
  TView xin = view(pc->xin, 2, 0, pc->lv[0]);
  FSI_LAUNCH(m, P_PC_AUX, (pc_pack_kernel<<<vgrid1(nn), 256, 0, m->stream>>>(
                              r, dinv, input_planes(pc), pc->modulate, pc->dmask, pc->ncomp, g, dbinv, nn, xin)));
  if ((rc = forward(pc, pc->xin))) return rc;
  if (pc->smooth) {  // y <- P R y: keep the smooth part of the correction
    const Grid3 g0 = pc->lv[0], g1 = pc->lv[1];
    FSI_LAUNCH(m, P_PC_AUX, (restrict_f32_kernel<<<vgrid1(pc->cout * g1.nv()), 256, 0, m->stream>>>(
                                pc->y32, g0, pc->ys1, g1, pc->cout)));
    FSI_LAUNCH(m, P_PC_AUX, (prolong_f32_kernel<<<vgrid1(pc->cout * g0.nv()), 256, 0, m->stream>>>(
                                pc->ys1, g1, pc->y32, g0, pc->cout)));
  }
  const double h = rnorm / std::sqrt(nrows);
  const D4 dk = {{pc->dbar[0] * pc->kc[0], pc->dbar[1] * pc->kc[1], pc->dbar[2] * pc->kc[2],
                   pc->dbar[3] * pc->kc[3]}};
  FSI_LAUNCH(m, P_PC_AUX, (pc_unpack_kernel<<<vgrid1(pc->ncomp * nn), 256, 0, m->stream>>>(
                              r, dinv, pc->y32, pc->dmask, pc->ncomp, h, dk, nn, z)));
  return FSI_OK;
}

// one training pair from r = ra - rb, e = ea - eb (rb, eb nullable) at the staged
// state; dbar is fixed from dinv by the first pair
int add_pair(fsi_pc* pc, const double* ra, const double* rb, const double* ea, const double* eb, const double* dinv) {
  fsi_mesh* m = pc->m;
  const int64_t nn = m->nn;
  const int64_t n = pc->ncomp * nn;
  int rc;
  if (!pc->have_dbar) {
    const int nb = 152;
    FSI_LAUNCH(m, P_PC_AUX, (dinv_mean_kernel<<<nb, 256, 0, m->stream>>>(dinv, pc->dmask, pc->ncomp, nn, pc->lpart)));
    std::vector<double> h(8 * nb);
    FSI_CUDA(cudaMemcpyAsync(h.data(), pc->lpart, sizeof(double) * 8 * nb, cudaMemcpyDeviceToHost, m->stream));
    FSI_CUDA(cudaStreamSynchronize(m->stream));
    for (int c = 0; c < pc->ncomp; ++c) {
      double s = 0, k = 0;
      for (int b = 0; b < nb; ++b) s += h[(2 * c) * nb + b], k += h[(2 * c + 1) * nb + b];
      pc->dbar[c] = (k > 0 && s > 0) ? s / k : 1.0;
    }
    pc->have_dbar = true;
  }
  const double* r = ra;
  if (rb) {
    FSI_LAUNCH(m, P_PC_AUX, (sub_kernel<<<vgrid1(n), 256, 0, m->stream>>>(ra, rb, pc->tmp, n)));
    r = pc->tmp;
  }
  double r2;
  if ((rc = vec_dot(m, r, r, n, &r2))) return rc;
  if (!(r2 > 0.0) || !std::isfinite(r2)) return FSI_OK;  // nothing to learn from
  const double rnorm = std::sqrt(r2);
  const int slot = pc->head;
  pc->head = (pc->head + 1) % pc->cap;
  pc->count = std::min(pc->count + 1, pc->cap);
  const double g = std::sqrt((double)n) / rnorm;
  const D4 dbinv = {{1.0 / pc->dbar[0], 1.0 / pc->dbar[1], 1.0 / pc->dbar[2], 1.0 / pc->dbar[3]}};
  TView xin = view(pc->ds_in + (int64_t)slot * pc->in_stride, 2, 0, pc->lv[0]);
  FSI_LAUNCH(m, P_PC_AUX, (pc_pack_kernel<<<vgrid1(nn), 256, 0, m->stream>>>(
                              r, dinv, input_planes(pc), pc->modulate, pc->dmask, pc->ncomp, g, dbinv, nn, xin)));
  FSI_LAUNCH(m, P_PC_AUX, (pc_target_kernel<<<vgrid1(n), 256, 0, m->stream>>>(
                              r, nullptr, ea, eb, dinv, pc->dmask, pc->ncomp, g, dbinv, nn,
                              pc->ds_t + (int64_t)slot * pc->t_stride)));
  // the target's sum of squares per component (the pair's loss weight at training)
  const int nb = 152;
  FSI_LAUNCH(m, P_PC_AUX, (target_rms_kernel<<<nb, 256, 0, m->stream>>>(pc->ds_t + (int64_t)slot * pc->t_stride,
                                                                       pc->t_stride, 1, pc->dmask, pc->ncomp, nn,
                                                                       pc->lpart)));
  std::vector<double> h(8 * nb);
  FSI_CUDA(cudaMemcpyAsync(h.data(), pc->lpart, sizeof(double) * 8 * nb, cudaMemcpyDeviceToHost, m->stream));
  FSI_CUDA(cudaStreamSynchronize(m->stream));
  for (int c = 0; c < 4; ++c) {
    double ss = 0.0;
    if (c < pc->ncomp)
      for (int b = 0; b < nb; ++b) ss += h[(2 * c) * nb + b];
    pc->pair_ss[(size_t)slot * 4 + c] = ss;
  }
  return FSI_OK;
}

int fit_norm(fsi_pc* pc) {
  fsi_mesh* m = pc->m;
  if (pc->count == 0) return set_error(FSI_EINVAL, "pc: no training pairs");
  const int nb = 152;
  FSI_LAUNCH(m, P_PC_AUX, (target_rms_kernel<<<nb, 256, 0, m->stream>>>(pc->ds_t, pc->t_stride, pc->count, pc->dmask,
                                                                       pc->ncomp, m->nn, pc->lpart)));
  std::vector<double> h(8 * nb);
  FSI_CUDA(cudaMemcpyAsync(h.data(), pc->lpart, sizeof(double) * 8 * nb, cudaMemcpyDeviceToHost, m->stream));
  FSI_CUDA(cudaStreamSynchronize(m->stream));
  for (int c = 0; c < pc->ncomp; ++c) {
    double s = 0, k = 0;
    for (int b = 0; b < nb; ++b) s += h[(2 * c) * nb + b], k += h[(2 * c + 1) * nb + b];
    pc->kc[c] = (k > 0 && s > 0) ? std::sqrt(s / k) : 1.0;
  }
  return FSI_OK;
}

int check_err(fsi_pc* pc) {
  int e = 0;
  FSI_CUDA(cudaMemcpyAsync(&e, pc->err, sizeof(int), cudaMemcpyDeviceToHost, pc->m->stream));
  FSI_CUDA(cudaStreamSynchronize(pc->m->stream));
  if (e) return set_error(FSI_ETIMEOUT, "pc: a tensor-core completion wait gave up");
  return FSI_OK;
}

}  // namespace pcn
}  // namespace fsi

// ====================================================================== C ABI
namespace {
template <typename T>
int dalloc(T** p, int64_t n) {
  FSI_CUDA(cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)std::max<int64_t>(n, 1)));
  FSI_CUDA(cudaMemset(*p, 0, sizeof(T) * (size_t)std::max<int64_t>(n, 1)));
  return FSI_OK;
}
}  // namespace

extern "C" {

int fsi_pc_create(fsi_mesh* m, const fsi_pc_desc* d, fsi_pc** out) {
  if (!m || !d || !out) return set_error(FSI_EINVAL, "fsi_pc_create: null argument");
  *out = nullptr;
  if (d->block != FSI_BLOCK_NS) return set_error(FSI_EINVAL, "fsi_pc_create: only the NS block is supported");
  if (!d->modulate && 4 + m->N > 16)
    return set_error(FSI_EINVAL, "fsi_pc_create: more than 12 phases do not fit 16 input channels");
  if (d->n_pairs_cap < 0) return set_error(FSI_EINVAL, "fsi_pc_create: negative pair capacity");
  FSI_CUDA(cudaSetDevice(m->dev));
  auto* pc = new fsi_pc();
  pc->m = m;
  pc->ncomp = 4;
  pc->cout = 4;
  pc->nph = m->N;
  pc->linear = d->linear != 0;
  pc->modulate = d->modulate != 0;
  pc->smooth = d->smooth != 0;
  if (pc->modulate) {
    int ns = 0;
    for (int i = 0; i < m->N; ++i) ns += m->phases[i].is_solid ? 1 : 0;
    if (ns > 3) {
      delete pc;
      return set_error(FSI_EINVAL, "fsi_pc_create: modulated input takes at most 3 solid phases");
    }
  }
  pc->lv[0] = Grid3{m->g.nx + 1, m->g.ny + 1, m->g.nz + 1};
  for (int l = 1; l < NLEVEL; ++l)
    pc->lv[l] = Grid3{pc->lv[l - 1].nx / 2 + 1, pc->lv[l - 1].ny / 2 + 1, pc->lv[l - 1].nz / 2 + 1};
  // layer table (storage order of the weights)
  const int cins[NLAYER] = {16, 16, 16, 16, 16, 16, 16, 16, 32, 16, 32, 16, 32, 16, 16};
  int64_t off = 0;
  for (int l = 0; l < NLAYER; ++l) {
    pc->lcin[l] = cins[l];
    pc->lcout[l] = l == OUT ? pc->cout : 16;
    pc->woff[l] = off;
    off += (int64_t)pc->lcout[l] * pc->lcin[l] * 27;
  }
  pc->nw = off;
  int rc = FSI_OK;
  auto fail = [&](int code) {
    fsi_pc_destroy(pc);
    return code;
  };
  if ((rc = dalloc(&pc->w, pc->nw)) || (rc = dalloc(&pc->mo, pc->nw)) || (rc = dalloc(&pc->vo, pc->nw)) ||
      (rc = dalloc(&pc->grad, pc->nw)))
    return fail(rc);
  int64_t pk = 0;
  for (int l = 0; l < NLAYER; ++l) pk += 2 * 27 * 16 * (int64_t)pc->lcin[l];
  if ((rc = dalloc(&pc->wpk, pk))) return fail(rc);
  pk = 0;
  for (int l = 0; l < NLAYER; ++l) {
    pc->wf[l] = pc->wpk + pk;
    pk += 27 * 16 * (int64_t)pc->lcin[l];
    pc->wb[l] = pc->wpk + pk;
    pk += 27 * 16 * (int64_t)pc->lcin[l];
  }
  for (int l = 0; l < NLEVEL; ++l) {
    const int64_t v8 = pc->lv[l].nv() * 8;
    if ((rc = dalloc(&pc->x[l], 2 * v8)) || (rc = dalloc(&pc->a[l], 2 * v8)) || (rc = dalloc(&pc->b[l], 2 * v8)) ||
        (rc = dalloc(&pc->d[l], 2 * v8)) || (rc = dalloc(&pc->cat[l], 4 * v8)) || (rc = dalloc(&pc->gd[l], 2 * v8)) ||
        (rc = dalloc(&pc->ga[l], 2 * v8)) || (rc = dalloc(&pc->gb[l], 2 * v8)) ||
        (rc = dalloc(&pc->gcat[l], 4 * v8)) || (rc = dalloc(&pc->ge[l], 2 * v8)) || (rc = dalloc(&pc->gx[l], 2 * v8)))
      return fail(rc);
  }
  const int64_t V0 = pc->lv[0].nv();
  if ((rc = dalloc(&pc->xin, 2 * V0 * 8)) || (rc = dalloc(&pc->y32, (int64_t)pc->cout * V0)) ||
      (rc = dalloc(&pc->tmp, (int64_t)pc->ncomp * m->nn)) || (rc = dalloc(&pc->lpart, 8 * 1216)) ||
      (rc = dalloc(&pc->ys1, (int64_t)pc->cout * pc->lv[1].nv())) ||
      (rc = dalloc(&pc->loss_dev, 1 << 16)) || (rc = dalloc(&pc->err, 1)))
    return fail(rc);
  // weight-gradient partials: room for the launch with the most CTAs over all levels
  {
    int64_t nblk = 0;
    for (int l = 0; l < NLEVEL; ++l) {
      const Grid3& g = pc->lv[l];
      const int gx = (g.nx + TILE_X - 1) / TILE_X, gy = (g.ny + TILE_Y - 1) / TILE_Y;
      const int zc = std::max(1, (int)((int64_t)g.nz * gx * gy / (2 * 152)));
      nblk = std::max(nblk, (int64_t)gx * gy * ((g.nz + zc - 1) / zc));
    }
    pc->wpart_n = std::max<int64_t>(nblk, 8 * 152) * 16 * 32 * 27;
    if ((rc = dalloc(&pc->wpart, pc->wpart_n))) return fail(rc);
  }
  pc->dmask = m->mask;
  // valid rows for the loss: rows without a Dirichlet condition
  {
    std::vector<uint8_t> hm(m->nn);
    FSI_CUDA(cudaMemcpy(hm.data(), m->mask, m->nn, cudaMemcpyDeviceToHost));
    int64_t cnt = 0;
    for (int64_t v = 0; v < m->nn; ++v)
      for (int c = 0; c < pc->ncomp; ++c) cnt += !((hm[v] >> c) & 1);
    pc->valid_rows = (double)std::max<int64_t>(cnt, 1);
  }
  pc->cap = d->n_pairs_cap;
  pc->pair_ss.assign((size_t)std::max(pc->cap, 1) * 4, 0.0);
  pc->in_stride = 2 * V0 * 8;
  pc->t_stride = (int64_t)pc->ncomp * m->nn;
  if (pc->cap > 0) {
    if ((rc = dalloc(&pc->ds_in, pc->cap * pc->in_stride)) || (rc = dalloc(&pc->ds_t, pc->cap * pc->t_stride)))
      return fail(rc);
  }
  for (int c = 0; c < 4; ++c) pc->dbar[c] = pc->kc[c] = 1.0;
  *out = pc;
  return FSI_OK;
}

int fsi_pc_destroy(fsi_pc* pc) {
  if (!pc) return FSI_OK;
  if (pc->m && pc->m->pc == pc) pc->m->pc = nullptr;
  cudaFree(pc->w), cudaFree(pc->mo), cudaFree(pc->vo), cudaFree(pc->grad), cudaFree(pc->wpk);
  for (int l = 0; l < NLEVEL; ++l) {
    cudaFree(pc->x[l]), cudaFree(pc->a[l]), cudaFree(pc->b[l]), cudaFree(pc->d[l]), cudaFree(pc->cat[l]);
    cudaFree(pc->gd[l]), cudaFree(pc->ga[l]), cudaFree(pc->gb[l]), cudaFree(pc->gcat[l]), cudaFree(pc->ge[l]);
    cudaFree(pc->gx[l]);
  }
  cudaFree(pc->xin), cudaFree(pc->y32), cudaFree(pc->ys1), cudaFree(pc->tmp), cudaFree(pc->lpart), cudaFree(pc->loss_dev);
  cudaFree(pc->err), cudaFree(pc->wpart), cudaFree(pc->ds_in), cudaFree(pc->ds_t), cudaFree(pc->ck);
  delete pc;
  return FSI_OK;
}

int fsi_pc_layout(const fsi_pc* pc, int32_t* n_layers, int64_t* n_weights, int32_t* fan, int32_t* grids) {
  if (!pc) return set_error(FSI_EINVAL, "fsi_pc_layout: null handle");
  if (n_layers) *n_layers = NLAYER;
  if (n_weights) *n_weights = pc->nw;
  if (fan)
    for (int l = 0; l < NLAYER; ++l) fan[2 * l] = pc->lcout[l], fan[2 * l + 1] = pc->lcin[l];
  if (grids)
    for (int l = 0; l < NLEVEL; ++l) grids[3 * l] = pc->lv[l].nx, grids[3 * l + 1] = pc->lv[l].ny, grids[3 * l + 2] = pc->lv[l].nz;
  return FSI_OK;
}

int fsi_pc_set_weights(fsi_pc* pc, const float* w, int64_t n) {
  if (!pc || !w || n != pc->nw) return set_error(FSI_EINVAL, "fsi_pc_set_weights: bad arguments");
  fsi_mesh* m = pc->m;
  FSI_CUDA(cudaMemcpyAsync(pc->w, w, sizeof(float) * n, cudaMemcpyHostToDevice, m->stream));
  FSI_CUDA(cudaMemsetAsync(pc->mo, 0, sizeof(float) * n, m->stream));
  FSI_CUDA(cudaMemsetAsync(pc->vo, 0, sizeof(float) * n, m->stream));
  pc->adam_t = 0;
  int rc = pack_weights(pc);
  if (rc) return rc;
  FSI_CUDA(cudaStreamSynchronize(m->stream));
  return FSI_OK;
}

int fsi_pc_get_weights(const fsi_pc* pc, float* w, int64_t n) {
  if (!pc || !w || n != pc->nw) return set_error(FSI_EINVAL, "fsi_pc_get_weights: bad arguments");
  FSI_CUDA(cudaMemcpyAsync(w, pc->w, sizeof(float) * n, cudaMemcpyDeviceToHost, pc->m->stream));
  FSI_CUDA(cudaStreamSynchronize(pc->m->stream));
  return FSI_OK;
}

int fsi_pc_set_norm(fsi_pc* pc, const double* dbar, const double* kc) {
  if (!pc || !dbar || !kc) return set_error(FSI_EINVAL, "fsi_pc_set_norm: null argument");
  for (int c = 0; c < pc->ncomp; ++c) {
    if (!(dbar[c] > 0.0) || !(kc[c] > 0.0)) return set_error(FSI_EINVAL, "fsi_pc_set_norm: scales must be > 0");
    pc->dbar[c] = dbar[c];
    pc->kc[c] = kc[c];
  }
  pc->have_dbar = true;
  return FSI_OK;
}

int fsi_pc_get_norm(const fsi_pc* pc, double* dbar, double* kc) {
  if (!pc || !dbar || !kc) return set_error(FSI_EINVAL, "fsi_pc_get_norm: null argument");
  for (int c = 0; c < pc->ncomp; ++c) dbar[c] = pc->dbar[c], kc[c] = pc->kc[c];
  return FSI_OK;
}

int fsi_pc_forward(fsi_pc* pc, const uint16_t* x_in, float* y) {
  if (!pc || !x_in || !y) return set_error(FSI_EINVAL, "fsi_pc_forward: null argument");
  int rc = forward(pc, x_in);
  if (rc) return rc;
  const int64_t V0 = pc->lv[0].nv();
  FSI_CUDA(cudaMemcpyAsync(y, pc->y32, sizeof(float) * pc->cout * V0, cudaMemcpyDeviceToDevice, pc->m->stream));
  return check_err(pc);
}

int fsi_pc_grad(fsi_pc* pc, const uint16_t* x_in, const uint16_t* target, float* grad, double* loss) {
  if (!pc || !x_in || !target || !grad || !loss) return set_error(FSI_EINVAL, "fsi_pc_grad: null argument");
  int rc;
  if ((rc = forward(pc, x_in)) || (rc = backward(pc, x_in, target, pc->loss_dev))) return rc;
  FSI_CUDA(cudaMemcpyAsync(grad, pc->grad, sizeof(float) * pc->nw, cudaMemcpyDeviceToDevice, pc->m->stream));
  FSI_CUDA(cudaMemcpyAsync(loss, pc->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, pc->m->stream));
  return check_err(pc);
}

int fsi_pc_apply(fsi_pc* pc, const fsi_state* st, const double* r, double* z) {
  if (!pc || !st || !r || !z) return set_error(FSI_EINVAL, "fsi_pc_apply: null argument");
  fsi_mesh* m = pc->m;
  int rc;
  if ((rc = stage(m, st, false))) return rc;
  BlockInfo b;
  if ((rc = block_info(m, FSI_BLOCK_NS, &b))) return rc;
  if ((rc = op_diag(m, b, pc->tmp, FSI_ELASTIC_AUG))) return rc;
  if ((rc = vec_recip(m, pc->tmp, pc->tmp, b.n))) return rc;
  double r2;
  if ((rc = vec_dot(m, r, r, b.n, &r2))) return rc;
  if ((rc = apply(pc, r, std::sqrt(r2), pc->tmp, z))) return rc;
  return check_err(pc);
}

namespace fsi {
namespace pcn {
// --------------------------------------------------- synthetic smooth training pairs
// A counter-based standard normal per (key, field, coarse node): the splitmix64 finaliser
// of the counter gives two uniforms, Box-Muller gives the normal.
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__device__ __forceinline__ double normal_at(uint64_t key) {
  const uint64_t a = mix64(key), b = mix64(key ^ 0xD1B54A32D192ED03ull);
  const double u1 = ((double)(a >> 11) + 0.5) * 0x1.0p-53, u2 = ((double)(b >> 11) + 0.5) * 0x1.0p-53;
  return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// z_f(node) = trilinear interpolation of normals on a coarse grid of L[axis] intervals
// spanning the box (L = the mesh's own intervals: a normal per node); velocity rows with a
// Dirichlet condition are 0.  Per CTA partial sums of the pressure into part[cta].
__global__ void smooth_field_kernel(double* __restrict__ z, int nx, int ny, int nz, int lx, int ly, int lz,
                                    uint64_t key, const uint8_t* __restrict__ mask, int64_t nn,
                                    double* __restrict__ part) {
  double psum = 0.0;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < nn; n += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(n % (nx + 1));
    const int j = (int)((n / (nx + 1)) % (ny + 1));
    const int k = (int)(n / ((int64_t)(nx + 1) * (ny + 1)));
    const double ux = (double)i * lx / nx, uy = (double)j * ly / ny, uz = (double)k * lz / nz;
    const int cx = min((int)ux, lx - 1), cy = min((int)uy, ly - 1), cz = min((int)uz, lz - 1);
    const double tx = ux - cx, ty = uy - cy, tz = uz - cz;
    const uint8_t mk = mask[n];
    for (int f = 0; f < 4; ++f) {
      double v = 0.0;
      for (int c = 0; c < 8; ++c) {
        const int ax = c & 1, ay = (c >> 1) & 1, az = (c >> 2) & 1;
        const double w = (ax ? tx : 1.0 - tx) * (ay ? ty : 1.0 - ty) * (az ? tz : 1.0 - tz);
        const uint64_t id = (((uint64_t)(cz + az) * (ly + 1) + (cy + ay)) * (lx + 1) + (cx + ax)) * 4 + f;
        v += w * normal_at(key ^ mix64(id));
      }
      if (f < 3 && ((mk >> f) & 1)) v = 0.0;
      z[f * nn + n] = v;
      if (f == 3) psum += v;
    }
  }
  __shared__ double red[256];
  red[threadIdx.x] = psum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += red[i];
    part[blockIdx.x] = t;
  }
}

// p -= mean(p), the mean summed from the CTA partials in a fixed order
__global__ void sub_mean_kernel(double* __restrict__ p, const double* __restrict__ part, int nparts, int64_t nn) {
  double t = 0.0;
  for (int i = 0; i < nparts; ++i) t += part[i];
  const double mean = t / (double)nn;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < nn; n += (int64_t)gridDim.x * blockDim.x)
    p[n] -= mean;
}
}  // namespace pcn
}  // namespace fsi

int fsi_pc_add_smooth_pairs(fsi_pc* pc, const fsi_state* st, int32_t count, uint64_t seed) {
  if (!pc || !st || count < 0) return set_error(FSI_EINVAL, "fsi_pc_add_smooth_pairs: bad argument");
  if (pc->cap <= 0) return set_error(FSI_EINVAL, "fsi_pc_add_smooth_pairs: the preconditioner holds no pair storage");
  if (pc->ncomp != 4) return set_error(FSI_EINVAL, "fsi_pc_add_smooth_pairs: the preconditioner is not the NS block's");
  fsi_mesh* m = pc->m;
  if (m->tet) return set_error(FSI_EINVAL, "fsi_pc_add_smooth_pairs: structured meshes only");
  int rc;
  if ((rc = stage(m, st, false))) return rc;
  BlockInfo b;
  if ((rc = block_info(m, FSI_BLOCK_NS, &b))) return rc;
  // the system of the step's NS solves: unpinned where the step shifts the pressure
  PinGuard guard(m, shifts_pressure(m, FSI_ELASTIC_AUG) ? 0 : m->pin_active);
  if (sizeof(double) * b.n > sizeof(uint16_t) * 4 * pc->lv[0].nv() * 8)
    return set_error(FSI_EINVAL, "fsi_pc_add_smooth_pairs: scratch too small");
  double* dinv = reinterpret_cast<double*>(pc->gcat[0]);
  if ((rc = op_diag(m, b, dinv, FSI_ELASTIC_AUG))) return rc;
  if ((rc = vec_recip(m, dinv, dinv, b.n))) return rc;
  constexpr int NB = 152;
  // the field, its product and the mean's partial sums; freed on every return (an early
  // return from a failed launch included), after the stream has finished with them
  struct Scratch {
    double* p = nullptr;
    cudaStream_t s = nullptr;
    ~Scratch() {
      if (p) {
        cudaStreamSynchronize(s);
        cudaFree(p);
      }
    }
  } buf;
  buf.s = m->stream;
  FSI_CUDA(cudaMalloc(&buf.p, sizeof(double) * 2 * b.n + sizeof(double) * NB));
  double* z = buf.p;
  double* y = z + b.n;
  double* part = y + b.n;
  const Geom& g = m->g;
  const int nmax = std::max(g.nx, std::max(g.ny, g.nz));
  for (int32_t k = 0; k < count && rc == FSI_OK; ++k) {
    // coarse spacing 2, 4, 8, 16, 32 intervals along the longest axis, then every node
    const int level = k % 6;
    auto coarse = [&](int n) {
      if (level == 5) return n;
      const int l = (int)std::lround((double)(2 << level) * n / nmax);
      return std::max(1, std::min(n, l));
    };
    const uint64_t key = seed * 0x2545F4914F6CDD1Dull + (uint64_t)k;
    FSI_LAUNCH(m, P_PC_AUX, (fsi::pcn::smooth_field_kernel<<<NB, 256, 0, m->stream>>>(
                                z, g.nx, g.ny, g.nz, coarse(g.nx), coarse(g.ny), coarse(g.nz), key, m->mask, m->nn,
                                part)));
    FSI_LAUNCH(m, P_PC_AUX, (fsi::pcn::sub_mean_kernel<<<vgrid1(m->nn), 256, 0, m->stream>>>(z + 3 * m->nn, part,
                                                                                             NB, m->nn)));
    if ((rc = op_jvp(m, b, z, y, FSI_ELASTIC_AUG))) break;
    rc = fsi::pcn::add_pair(pc, y, nullptr, z, nullptr, dinv);
  }
  const cudaError_t se = cudaStreamSynchronize(m->stream);
  if (rc) return rc;
  if (se != cudaSuccess) return set_error(FSI_ECUDA, cudaGetErrorString(se));
  return FSI_OK;
}

int fsi_pc_add_pair(fsi_pc* pc, const fsi_state* st, const double* r, const double* e) {
  if (!pc || !st || !r || !e) return set_error(FSI_EINVAL, "fsi_pc_add_pair: null argument");
  if (pc->cap <= 0) return set_error(FSI_EINVAL, "fsi_pc_add_pair: the preconditioner holds no pair storage");
  fsi_mesh* m = pc->m;
  int rc;
  if ((rc = stage(m, st, false))) return rc;
  BlockInfo b;
  if ((rc = block_info(m, FSI_BLOCK_NS, &b))) return rc;
  double* dinv = pc->tmp;
  // dinv is needed next to r - rb in tmp: use the gradient scratch of level 0 as a second vector
  if (sizeof(double) * b.n > sizeof(uint16_t) * 4 * pc->lv[0].nv() * 8)
    return set_error(FSI_EINVAL, "fsi_pc_add_pair: scratch too small");
  dinv = reinterpret_cast<double*>(pc->gcat[0]);
  if ((rc = op_diag(m, b, dinv, FSI_ELASTIC_AUG))) return rc;
  if ((rc = vec_recip(m, dinv, dinv, b.n))) return rc;
  if ((rc = add_pair(pc, r, nullptr, e, nullptr, dinv))) return rc;
  FSI_CUDA(cudaStreamSynchronize(m->stream));
  return FSI_OK;
}

int fsi_pc_pairs(const fsi_pc* pc, int32_t* n) {
  if (!pc || !n) return set_error(FSI_EINVAL, "fsi_pc_pairs: null argument");
  *n = pc->count;
  return FSI_OK;
}

int fsi_pc_fit_norm(fsi_pc* pc) {
  if (!pc) return set_error(FSI_EINVAL, "fsi_pc_fit_norm: null handle");
  return fit_norm(pc);
}

int fsi_pc_train(fsi_pc* pc, int32_t iters, float lr, const int32_t* order, float* loss_out) {
  if (!pc || iters < 0 || (iters > 0 && !order)) return set_error(FSI_EINVAL, "fsi_pc_train: bad arguments");
  if (pc->count == 0) return set_error(FSI_EINVAL, "fsi_pc_train: no training pairs");
  if (iters > (1 << 16)) return set_error(FSI_EINVAL, "fsi_pc_train: at most 65536 iterations per call");
  fsi_mesh* m = pc->m;
  int rc;
  for (int it = 0; it < iters; ++it) {
    const int p = order[it];
    if (p < 0 || p >= pc->count) return set_error(FSI_EINVAL, "fsi_pc_train: pair index out of range");
    const uint16_t* xin = pc->ds_in + (int64_t)p * pc->in_stride;
    const uint16_t* t = pc->ds_t + (int64_t)p * pc->t_stride;
    // relative error: the pair's loss is divided by the mean square of its scaled target
    double ms = 0.0;
    for (int c = 0; c < pc->ncomp; ++c) ms += pc->pair_ss[(size_t)p * 4 + c] / (pc->kc[c] * pc->kc[c]);
    ms /= pc->valid_rows;
    const double wgt = ms > 0.0 ? 1.0 / ms : 1.0;
    if ((rc = pack_weights(pc)) || (rc = forward(pc, xin)) || (rc = backward(pc, xin, t, pc->loss_dev + it, wgt)) ||
        (rc = adam(pc, lr)))
      return rc;
  }
  if ((rc = pack_weights(pc))) return rc;
  if (loss_out && iters > 0) {
    std::vector<double> h(iters);
    FSI_CUDA(cudaMemcpyAsync(h.data(), pc->loss_dev, sizeof(double) * iters, cudaMemcpyDeviceToHost, m->stream));
    FSI_CUDA(cudaStreamSynchronize(m->stream));
    for (int i = 0; i < iters; ++i) loss_out[i] = (float)h[i];
  }
  return check_err(pc);
}

int fsi_set_pc(fsi_mesh* m, fsi_pc* pc) {
  if (!m) return set_error(FSI_EINVAL, "fsi_set_pc: null mesh");
  if (pc && pc->m != m) return set_error(FSI_EINVAL, "fsi_set_pc: preconditioner belongs to another mesh");
  m->pc = pc;
  return FSI_OK;
}

}  // extern "C"

namespace fsi {
namespace pcn {
int ensure_checkpoints(fsi_pc* pc) {
  if (pc->ck) return FSI_OK;
  const int64_t n = (int64_t)pc->ncomp * pc->m->nn;
  FSI_CUDA(cudaMalloc(&pc->ck, sizeof(double) * (size_t)(2 * CKMAX * n)));
  pc->ck_n = CKMAX;
  return FSI_OK;
}
}  // namespace pcn
}  // namespace fsi
