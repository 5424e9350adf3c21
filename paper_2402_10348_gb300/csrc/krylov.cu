// Krylov solver of libfsi: restarted right-preconditioned GMRES with classical
// Gram-Schmidt applied twice (CGS2), Givens rotations on the host, float64 vectors;
// optional float32 operator inside float64 iterative refinement.  Every reduction
// is deterministic (fixed partition, fixed summation order).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace fsi {

constexpr int VB = 256;          // threads per CTA of the vector kernels
constexpr int DCH = 16;          // dot products per CTA pass

static int vgrid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + VB * 8 - 1) / (VB * 8), 152 * 4)); }

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

// part[i*G + cta] = sum over the CTA's range of V_i . w,  i in [16*blockIdx.y, ...)
__global__ void __launch_bounds__(VB) mdot_kernel(const double* __restrict__ V, int64_t ldv, int k,
                                                  const double* __restrict__ w, int64_t n, double* part) {
  const int G = gridDim.x;
  const int i0 = blockIdx.y * DCH;
  const int kc = min(DCH, k - i0);
  const int64_t per = (n + G - 1) / G;
  const int64_t lo = blockIdx.x * per, hi = min(n, lo + per);
  double acc[DCH];
#pragma unroll
  for (int i = 0; i < DCH; ++i) acc[i] = 0.0;
  for (int64_t j = lo + threadIdx.x; j < hi; j += VB) {
    const double wj = w[j];
#pragma unroll
    for (int i = 0; i < DCH; ++i)
      if (i < kc) acc[i] += V[(int64_t)(i0 + i) * ldv + j] * wj;
  }
  block_reduce_store<DCH>(acc, kc, part + (int64_t)i0 * G + blockIdx.x, G);
}

// out[i] = (accumulate ? out[i] : 0) + sum_c part[i*G + c]  (fixed order)
__global__ void sum_partials(const double* __restrict__ part, int G, double* out, int accumulate) {
  const int i = blockIdx.x;
  double s = 0.0;
  for (int c = threadIdx.x; c < G; c += VB) s += part[(int64_t)i * G + c];
  double acc[1] = {s};
  __shared__ double res;
  double* dst = &res;
  block_reduce_store<1>(acc, 1, dst, 1);
  __syncthreads();
  if (threadIdx.x == 0) out[i] = accumulate ? out[i] + res : res;
}

// w -= sum_i h_i V_i ; optionally part[cta] = partial of |w|^2
__global__ void __launch_bounds__(VB) upd_kernel(double* __restrict__ w, const double* __restrict__ V, int64_t ldv,
                                                 int k, const double* __restrict__ h, int64_t n, double* part) {
  __shared__ double hs[128];
  for (int i = threadIdx.x; i < k; i += VB) hs[i] = h[i];
  __syncthreads();
  const int G = gridDim.x;
  const int64_t per = (n + G - 1) / G;
  const int64_t lo = blockIdx.x * per, hi = min(n, lo + per);
  double nrm[1] = {0.0};
  for (int64_t j = lo + threadIdx.x; j < hi; j += VB) {
    double s = w[j];
    for (int i = 0; i < k; ++i) s -= hs[i] * V[(int64_t)i * ldv + j];
    w[j] = s;
    nrm[0] += s * s;
  }
  if (part) block_reduce_store<1>(nrm, 1, part + blockIdx.x, 1);
}

__global__ void scale_by_norm(double* w, const double* nrm2, int64_t n) {
  const double s = 1.0 / sqrt(*nrm2);
  for (int64_t j = blockIdx.x * (int64_t)VB + threadIdx.x; j < n; j += (int64_t)gridDim.x * VB) w[j] *= s;
}

// x += dinv * sum_i y_i V_i
__global__ void combine_kernel(double* __restrict__ x, const double* __restrict__ dinv, const double* __restrict__ V,
                               int64_t ldv, int k, const double* __restrict__ y, int64_t n) {
  __shared__ double ys[128];
  for (int i = threadIdx.x; i < k; i += VB) ys[i] = y[i];
  __syncthreads();
  for (int64_t j = blockIdx.x * (int64_t)VB + threadIdx.x; j < n; j += (int64_t)gridDim.x * VB) {
    double s = 0.0;
    for (int i = 0; i < k; ++i) s += ys[i] * V[(int64_t)i * ldv + j];
    x[j] += dinv[j] * s;
  }
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
static int dot_to_device(fsi_mesh* m, const double* V, int64_t ldv, int k, const double* w, int64_t n, double* out,
                         int accumulate) {
  const int G = vgrid(n);
  dim3 grid(G, (k + DCH - 1) / DCH);
  FSI_LAUNCH(m, P_KRYLOV, mdot_kernel<<<grid, VB, 0, m->stream>>>(V, ldv, k, w, n, m->partials_dot));
  FSI_LAUNCH(m, P_KRYLOV, sum_partials<<<k, VB, 0, m->stream>>>(m->partials_dot, G, out, accumulate));
  return FSI_OK;
}

int vec_dot(fsi_mesh* m, const double* a, const double* b, int64_t n, double* out_host) {
  int rc = dot_to_device(m, a, 0, 1, b, n, m->red, 0);
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

static int ensure_krylov(fsi_mesh* m, int64_t n, int mm) {
  if (m->kry_n >= n && m->kry_m >= mm) return FSI_OK;
  const int64_t nn = std::max(n, m->kry_n);
  const int mx = std::max(mm, m->kry_m);
  cudaFree(m->V);
  cudaFree(m->wk);
  cudaFree(m->dinv);
  cudaFree(m->yvec);
  cudaFree(m->partials_dot);
  m->V = m->wk = m->dinv = m->yvec = m->partials_dot = nullptr;
  FSI_CUDA(cudaMalloc(&m->V, sizeof(double) * (size_t)(mx + 1) * nn));
  FSI_CUDA(cudaMalloc(&m->wk, sizeof(double) * (size_t)6 * nn));
  FSI_CUDA(cudaMalloc(&m->dinv, sizeof(double) * (size_t)nn));
  FSI_CUDA(cudaMalloc(&m->yvec, sizeof(double) * 256));
  FSI_CUDA(cudaMalloc(&m->partials_dot, sizeof(double) * (size_t)(mx + 1 + DCH) * 152 * 4));
  m->kry_n = nn;
  m->kry_m = mx;
  return FSI_OK;
}

// One GMRES(m) solve A x = b from x = 0 with A = the block operator (flags) and the
// right preconditioner diag(dinv).  Host-side Hessenberg least squares.
static int gmres_core(fsi_mesh* m, const BlockInfo& blk, const double* b, double* x, int mm, double rtol,
                      int max_iter, unsigned flags, int* iters, int* restarts, double* rel_out) {
  const int64_t n = blk.n;
  double* V = m->V;
  double* r = m->wk;
  double* z = m->wk + n;
  double* t = m->wk + 2 * n;
  double* dev = m->red;  // [0..127] h1, [128..255] h2, [256] nrm2
  FSI_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, m->stream));
  double bnorm2;
  int rc = vec_dot(m, b, b, n, &bnorm2);
  if (rc) return rc;
  if (!std::isfinite(bnorm2)) return set_error(FSI_ENAN, "GMRES: right-hand side is not finite");
  const double bnorm = std::sqrt(bnorm2);
  *rel_out = 0.0;
  if (bnorm == 0.0) return FSI_OK;
  FSI_CUDA(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->stream));
  std::vector<double> H((mm + 1) * mm), cs(mm), sn(mm), g(mm + 1), y(mm);
  auto Hij = [&](int i, int j) -> double& { return H[i * mm + j]; };
  double rel = 1.0;
  while (true) {
    double beta2;
    if ((rc = vec_dot(m, r, r, n, &beta2))) return rc;
    if (!std::isfinite(beta2)) return set_error(FSI_ENAN, "GMRES: residual is not finite");
    const double beta = std::sqrt(beta2);
    rel = beta / bnorm;
    if (rel <= rtol || *iters >= max_iter) break;
    if ((rc = vec_scale_copy(m, 1.0 / beta, r, V, n))) return rc;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jend = 0;
    for (int j = 0; j < mm; ++j) {
      double* w = V + (int64_t)(j + 1) * n;
      if ((rc = vec_mul(m, m->dinv, V + (int64_t)j * n, z, n))) return rc;
      if ((rc = op_jvp(m, blk, z, w, flags))) return rc;
      // CGS2
      if ((rc = dot_to_device(m, V, n, j + 1, w, n, dev, 0))) return rc;
      FSI_LAUNCH(m, P_KRYLOV, upd_kernel<<<vgrid(n), VB, 0, m->stream>>>(w, V, n, j + 1, dev, n, nullptr));
      if ((rc = dot_to_device(m, V, n, j + 1, w, n, dev + 128, 0))) return rc;
      const int G = vgrid(n);
      FSI_LAUNCH(m, P_KRYLOV, upd_kernel<<<G, VB, 0, m->stream>>>(w, V, n, j + 1, dev + 128, n, m->partials_dot));
      FSI_LAUNCH(m, P_KRYLOV, sum_partials<<<1, VB, 0, m->stream>>>(m->partials_dot, G, dev + 256, 0));
      FSI_CUDA(cudaMemcpyAsync(m->red_host, dev, sizeof(double) * 257, cudaMemcpyDeviceToHost, m->stream));
      FSI_CUDA(cudaStreamSynchronize(m->stream));
      const double* hh = m->red_host;
      for (int i = 0; i <= j; ++i) Hij(i, j) = hh[i] + hh[128 + i];
      const double hn2 = hh[256];
      if (!std::isfinite(hn2)) return set_error(FSI_ENAN, "GMRES: Arnoldi vector is not finite");
      const double hn = std::sqrt(hn2);
      Hij(j + 1, j) = hn;
      if (hn > 0.0) {
        FSI_LAUNCH(m, P_KRYLOV, scale_by_norm<<<vgrid(n), VB, 0, m->stream>>>(w, dev + 256, n));
      }
      for (int i = 0; i < j; ++i) {
        const double a = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
        Hij(i + 1, j) = -sn[i] * Hij(i, j) + cs[i] * Hij(i + 1, j);
        Hij(i, j) = a;
      }
      const double den = std::hypot(Hij(j, j), Hij(j + 1, j));
      cs[j] = den > 0.0 ? Hij(j, j) / den : 1.0;
      sn[j] = den > 0.0 ? Hij(j + 1, j) / den : 0.0;
      Hij(j, j) = den;
      Hij(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++*iters;
      jend = j + 1;
      if (std::fabs(g[j + 1]) / bnorm <= rtol || *iters >= max_iter || hn == 0.0 || den == 0.0) break;
    }
    for (int i = jend - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < jend; ++k) s -= Hij(i, k) * y[k];
      y[i] = Hij(i, i) != 0.0 ? s / Hij(i, i) : 0.0;
    }
    FSI_CUDA(cudaMemcpyAsync(m->yvec, y.data(), sizeof(double) * jend, cudaMemcpyHostToDevice, m->stream));
    FSI_LAUNCH(m, P_KRYLOV, combine_kernel<<<vgrid(n), VB, 0, m->stream>>>(x, m->dinv, V, n, jend, m->yvec, n));
    // true residual r = b - A x
    if ((rc = op_jvp(m, blk, x, t, flags))) return rc;
    FSI_CUDA(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->stream));
    if ((rc = vec_axpy(m, -1.0, t, r, n))) return rc;
    ++*restarts;
    // make sure the host vector y is no longer needed before it is reused
    FSI_CUDA(cudaStreamSynchronize(m->stream));
  }
  *rel_out = rel;
  return FSI_OK;
}

int gmres_solve(fsi_mesh* m, const BlockInfo& blk, const double* rhs, double* x, const fsi_solve_opts& o,
                fsi_solve_info* info) {
  const int mm = o.m;
  if (mm < 1 || mm > 64) return set_error(FSI_EINVAL, "GMRES: restart length must be in 1..64");
  const int64_t n = blk.n;
  int rc = ensure_krylov(m, n, mm);
  if (rc) return rc;
  const int64_t a0 = m->applies;
  // Jacobi diagonal of the float64 operator
  if (o.precond == FSI_PC_JACOBI) {
    if ((rc = op_diag(m, blk, m->wk + 3 * n, o.flags & ~FSI_FP32))) return rc;
    if ((rc = vec_recip(m, m->wk + 3 * n, m->dinv, n))) return rc;
  } else {
    FSI_LAUNCH(m, P_KRYLOV, fill_kernel<<<vgrid(n), VB, 0, m->stream>>>(m->dinv, 1.0, n));
  }
  fsi_solve_info inf{};
  double rel = 0.0;
  if (o.precision == FSI_PREC_FP64) {
    rc = gmres_core(m, blk, rhs, x, mm, o.rtol, o.max_iter, o.flags & ~FSI_FP32, &inf.iterations, &inf.restarts, &rel);
    if (rc) return rc;
  } else {
    // x = 0; r = rhs; repeat: solve A32 d = r; x += d; r = rhs - A64 x
    double* d = m->wk + 4 * n;
    double* r = m->wk + 5 * n;
    FSI_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, m->stream));
    FSI_CUDA(cudaMemcpyAsync(r, rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->stream));
    double b2;
    if ((rc = vec_dot(m, rhs, rhs, n, &b2))) return rc;
    const double bnorm = std::sqrt(b2);
    rel = bnorm == 0.0 ? 0.0 : 1.0;
    for (int k = 0; k < std::max(1, o.ir_max) && rel > o.rtol; ++k) {
      double inner_rel;
      // the inner solve needs its own right-hand side copy: gmres_core uses wk[0..3n)
      rc = gmres_core(m, blk, r, d, mm, o.ir_inner_rtol, o.max_iter - inf.iterations,
                      (o.flags | FSI_FP32), &inf.iterations, &inf.restarts, &inner_rel);
      if (rc) return rc;
      if ((rc = vec_axpy(m, 1.0, d, x, n))) return rc;
      if ((rc = op_jvp(m, blk, x, d, o.flags & ~FSI_FP32))) return rc;
      FSI_CUDA(cudaMemcpyAsync(r, rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->stream));
      if ((rc = vec_axpy(m, -1.0, d, r, n))) return rc;
      double r2;
      if ((rc = vec_dot(m, r, r, n, &r2))) return rc;
      if (!std::isfinite(r2)) return set_error(FSI_ENAN, "IR: residual is not finite");
      rel = bnorm > 0.0 ? std::sqrt(r2) / bnorm : 0.0;
      inf.refinements = k + 1;
      if (inf.iterations >= o.max_iter) break;
    }
  }
  inf.rel_res = rel;
  inf.applies = (int)(m->applies - a0);
  if (info) *info = inf;
  if (!(rel <= o.rtol)) return set_error(FSI_ENOCONV, "GMRES: tolerance not reached");
  return FSI_OK;
}

}  // namespace fsi
