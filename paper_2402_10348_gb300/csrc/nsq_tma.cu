// Float32 NS product from the quadrature-point coefficients, staged by the Tensor
// Memory Accelerator (the FSI_FP32 product of the NS block inside mixed-precision
// iterative refinement).
//
// The product is bound by streaming the coefficient planes (8 points x 44 or 20 float32
// values per element, Section 2.4's linearization frozen per solve): one thread per
// element reading 352 scattered planes keeps too few loads in flight.  Here a CTA owns a
// tile of 64 x 2 elements of one element layer and receives, per quadrature point, one
// four-dimensional TMA box (x 64, y 2, coefficient 44 or 20, layer-point 1) of the
// coefficient array C[((ez * 8 + q) * 44 + c) * nxyp + ey * nxp + ex] into shared memory
// (22.5 KB), double-buffered on two mbarriers: the copy of point q + 2 runs while point
// q is evaluated.  Thread (tx, ty) evaluates element (x0 + tx, y0 + ty) exactly as the
// element-centric kernel (nsq_point on the interpolated increment) and writes its 32
// corner contributions into E[8 * field + corner][element]; ns_node_kernel sums them.
//
// Every mbarrier wait is bounded; a wait that gives up sets *err, the CTA stops issuing
// copies, waits (bounded) for the copies it has in flight and writes NaN contributions.
#include <cuda.h>

#include "ops_impl.cuh"

namespace fsi {
namespace {

constexpr int TBX = NSQ_TBX, TBY = NSQ_TBY;  // CTA tile of elements (x, y), one thread each
constexpr int TSTAGES = 2;
constexpr long long TWAIT = 1LL << 22;

__device__ __forceinline__ uint32_t sptr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < TWAIT; ++i) {
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

// one box of coefficients of layer-point zq into dst; completion counted on bar
__device__ __forceinline__ void load_box(uint32_t dst, const CUtensorMap* map, uint32_t bar, uint32_t bytes, int x0,
                                         int y0, int zq) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x0), "r"(y0), "r"(0), "r"(zq), "r"(bar)
      : "memory");
}

// coefficient accessor over one element's column of a staged box
struct SmemCoef {
  const float* p;
  __device__ __forceinline__ float operator()(int i) const { return p[i * (TBX * TBY)]; }
};

// One CTA's tile: elements (x0 .. x0 + 63, y0 .. y0 + 1) of layer ez, ncoef coefficients per
// point staged from the tensor map `map` (in kernel parameter or global memory) into
// `stage` ([TSTAGES][ncoef][TBY][TBX]); contributions into E (element plane pitch nxyp).
__device__ __forceinline__ void nsq_tma_tile(float* stage, const CUtensorMap* map, int ncoef,
                                             const float* __restrict__ dx, float* __restrict__ E, int nx, int ny,
                                             int nz, int nxp, int64_t nxyp, int64_t nn, float al, float cmass,
                                             float rhx, float rhy, float rhz, int x0, int y0, int ez, int* err) {
  __shared__ __align__(8) uint64_t bar[TSTAGES];
  __shared__ int failed;
  const int SF = ncoef * TBX * TBY;  // floats per stage
  const uint32_t SBYTES = (uint32_t)SF * sizeof(float);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TBX + tx;
  if (tid == 0) {
    failed = 0;
    for (int s = 0; s < TSTAGES; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sptr(&bar[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (int s = 0; s < TSTAGES; ++s) load_box(sptr(stage + s * SF), map, sptr(&bar[s]), SBYTES, x0, y0, ez * 8 + s);
  // the increment at the element's corners (while the first boxes arrive)
  const int ex = x0 + tx, ey = y0 + ty;
  const bool valid = ex < nx && ey < ny;
  float x[4][8], c[4][8];
  const int64_t sy = nx + 1, sz = (int64_t)(nx + 1) * (ny + 1);
  const int64_t n0 = ex + sy * ey + sz * ez;
  const int64_t off[8] = {0, 1, sy, sy + 1, sz, sz + 1, sz + sy, sz + sy + 1};
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      x[f][a] = valid ? __ldg(dx + f * nn + n0 + off[a]) : 0.0f;
      c[f][a] = 0.0f;
    }
  int q = 0;
  for (; q < 8; ++q) {
    const int s = q % TSTAGES;
    if (!bar_wait(sptr(&bar[s]), (uint32_t)((q / TSTAGES) & 1))) atomicExch(&failed, 1);
    __syncthreads();
    if (failed) break;
    if (valid) {
      QW<float> w;
      w.set(q);
      float dv[3], gd[3][3];
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) {
        const VG<float> r = interp_vg(x[kk], w, rhx, rhy, rhz);
        dv[kk] = r.v; gd[kk][0] = r.gx; gd[kk][1] = r.gy; gd[kk][2] = r.gz;
      }
      const VG<float> dpr = interp_vg(x[3], w, rhx, rhy, rhz);
      const float dgp[3] = {dpr.gx, dpr.gy, dpr.gz};
      nsq_point<float>(SmemCoef{stage + s * SF + tid}, ncoef == NCQ, dv, gd, dpr.v, dgp, al, cmass, w, rhx, rhy, rhz,
                       c);
    }
    __syncthreads();  // every thread is done with stage s
    if (tid == 0 && q + TSTAGES < 8) load_box(sptr(stage + s * SF), map, sptr(&bar[s]), SBYTES, x0, y0, ez * 8 + q + TSTAGES);
  }
  if (failed) {
    // copies issued for points q .. min(q + TSTAGES, 8) - 1 may still be in flight; the
    // product of this tile is NaN, so the solve that uses it stops on a non-finite vector
    if (tid == 0) {
      if (err) *err = 1;
      for (int p = q; p < 8 && p < q + TSTAGES; ++p) bar_wait(sptr(&bar[p % TSTAGES]), (uint32_t)((p / TSTAGES) & 1));
    }
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int a = 0; a < 8; ++a) c[f][a] = __int_as_float(0x7fc00000);
  }
  if (!valid) return;
  const int64_t e = (int64_t)ez * nxyp + (int64_t)ey * nxp + ex;
  const int64_t es = (int64_t)nz * nxyp;
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int a = 0; a < 8; ++a) E[(8 * f + a) * es + e] = c[f][a];
}

__global__ void __launch_bounds__(TBX * TBY) nsq_tma_kernel(const __grid_constant__ CUtensorMap map, int ncoef,
                                                            const float* __restrict__ dx, float* __restrict__ E, int nx,
                                                            int ny, int nz, int nxp, int64_t nxyp, int64_t nn, float al,
                                                            float cmass, float rhx, float rhy, float rhz, int* err) {
  extern __shared__ __align__(128) float stage[];
  const int nbx = (nx + TBX - 1) / TBX, nby = (ny + TBY - 1) / TBY;
  int64_t b = blockIdx.x;
  const int bx = (int)(b % nbx);
  b /= nbx;
  const int by = (int)(b % nby);
  const int ez = (int)(b / nby);
  nsq_tma_tile(stage, &map, ncoef, dx, E, nx, ny, nz, nxp, nxyp, nn, al, cmass, rhx, rhy, rhz, bx * TBX, by * TBY, ez,
               err);
}

// Batched: one CTA per work item (instance, x block, y block, layer); the instance's
// parameters and tensor map come from its record in global memory.
__global__ void __launch_bounds__(TBX * TBY) nsq_tma_batch_kernel(const NSQBatchRec* __restrict__ recs,
                                                                  const int4* __restrict__ items, const int* active) {
  extern __shared__ __align__(128) float stage[];
  const int4 it = items[blockIdx.x];
  if (active && !active[it.x]) return;
  const NSQBatchRec& R = recs[it.x];
  nsq_tma_tile(stage, reinterpret_cast<const CUtensorMap*>(R.map), R.elastic ? NCQ : NCQ_FLUID, R.dx32, R.E, R.nx,
               R.ny, R.nz, R.nxp, R.nxyp, R.nn, R.al, R.cm, R.rhx, R.rhy, R.rhz, it.y * TBX, it.z * TBY, it.w, R.err);
}

// Batched float64 product from the coefficients (nsq_elem_body): one CTA of 64 x 2
// threads per (instance, x block, y block, layer) work item
__global__ void __launch_bounds__(TBX * TBY) nsq_elem_batch_kernel(const NSQBatchRec* __restrict__ recs,
                                                                   const int4* __restrict__ items, const int* active) {
  const int4 it = items[blockIdx.x];
  if (active && !active[it.x]) return;
  const NSQBatchRec& R = recs[it.x];
  const int ex = it.y * TBX + threadIdx.x, ey = it.z * TBY + threadIdx.y;
  if (ex >= R.nx || ey >= R.ny) return;
  nsq_elem_body<double>(R.cq64, R.dx, R.E64, R.nx, R.ny, R.nz, R.nxp, R.nxyp, R.nn, R.elastic, R.al64, R.cm64,
                        R.rh64[0], R.rh64[1], R.rh64[2], ex, ey, it.w);
}

// Batched node sums: one CTA per (instance, 128 consecutive nodes)
template <typename T>
__global__ void __launch_bounds__(128) ns_node_batch_kernel(const NSQBatchRec* __restrict__ recs,
                                                            const int4* __restrict__ items, const int* active) {
  const int4 it = items[blockIdx.x];
  if (active && !active[it.x]) return;
  const NSQBatchRec& R = recs[it.x];
  const int64_t n = (int64_t)it.y * 128 + threadIdx.x;
  if (n >= R.nn) return;
  const int nx = R.nx, ny = R.ny, nz = R.nz;
  const int i = (int)(n % (nx + 1));
  const int64_t jk = n / (nx + 1);
  const int j = (int)(jk % (ny + 1)), k = (int)(jk / (ny + 1));
  const int64_t es = (int64_t)nz * R.nxyp;
  const T* E = sizeof(T) == 8 ? reinterpret_cast<const T*>(R.E64) : reinterpret_cast<const T*>(R.E);
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
        const int64_t e = (int64_t)ez * R.nxyp + (int64_t)ey * R.nxp + ex;
        const int a = ax + 2 * ay + 4 * az;
#pragma unroll
        for (int f = 0; f < 4; ++f) s[f] += E[(8 * f + a) * es + e];
      }
    }
  }
  const uint8_t mk = R.mask[n];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const bool dir = ((mk >> f) & 1) && (f < 3 || R.pin);
    R.y[f * R.nn + n] = dir ? (R.dx ? R.dx[f * R.nn + n] : (double)R.dx32[f * R.nn + n]) : R.W * (double)s[f];
  }
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled lookup_encode() {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return reinterpret_cast<EncodeTiled>(fn);
}

int encode_maps(fsi_mesh* m, int nxp, int64_t nxyp) {
  static const EncodeTiled enc = lookup_encode();  // thread-safe one-time lookup
  if (!enc) return set_error(FSI_ECUDA, "NS float32 product: cuTensorMapEncodeTiled not available");
  const Geom& g = m->g;
  const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)NCQ, (cuuint64_t)g.nz * 8};
  const cuuint64_t strides[3] = {(cuuint64_t)nxp * 4, (cuuint64_t)nxyp * 4, (cuuint64_t)NCQ * nxyp * 4};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  for (int k = 0; k < 2; ++k) {
    const cuuint32_t box[4] = {TBX, TBY, (cuuint32_t)(k == 0 ? NCQ : NCQ_FLUID), 1};
    CUtensorMap* map = reinterpret_cast<CUtensorMap*>(m->cq_tmap + 128 * k);
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, m->cq32, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(FSI_ECUDA, "NS float32 product: tensor map encoding failed");
  }
  m->cq_tmap_base = m->cq32;
  return FSI_OK;
}

}  // namespace

static_assert(sizeof(CUtensorMap) == 128, "tensor map storage");

int check_tma(fsi_mesh* m) {
  if (!m->tma_err) return FSI_OK;
  int e = 0;
  FSI_CUDA(cudaMemcpyAsync(&e, m->tma_err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  FSI_CUDA(cudaStreamSynchronize(m->stream));
  if (e) return set_error(FSI_ECUDA, "NS float32 product: a coefficient copy did not complete within its bounded wait");
  return FSI_OK;
}

int nsq_batch_record(fsi_mesh* m, unsigned flags, bool f64, const double* dx, double* y, float* dx32,
                     NSQBatchRec* rec) {
  const unsigned eflags = flags & FSI_ELASTIC_AUG;
  if (m->cq_gen != m->stage_gen || m->cq_flags != eflags || !m->cq64)
    if (int rc = ns_build(m, flags)) return rc;
  const Geom& g = m->g;
  const int nxp = cq_pitch(m);
  const int64_t nxyp = (int64_t)nxp * g.ny;
  if (int rc = ensure_elem_scratch(m, 32, nxyp)) return rc;
  if (!f64 && m->cq_tmap_base != m->cq32)
    if (int rc = encode_maps(m, nxp, nxyp)) return rc;
  if (!m->tma_err) {
    FSI_CUDA(cudaMalloc(&m->tma_err, sizeof(int)));
    FSI_CUDA(cudaMemsetAsync(m->tma_err, 0, sizeof(int), m->stream));
  }
  const int elastic = (eflags && m->ns > 0) ? 1 : 0;
  memset(rec, 0, sizeof(*rec));
  if (f64) {
    rec->cq64 = m->cq64;
    rec->E64 = m->ke_e;
  } else {
    memcpy(rec->map, m->cq_tmap + (elastic ? 0 : 128), 128);
  }
  rec->al64 = m->P.alpha;
  rec->cm64 = m->P.c_mass;
  rec->rh64[0] = 1.0 / g.hx;
  rec->rh64[1] = 1.0 / g.hy;
  rec->rh64[2] = 1.0 / g.hz;
  rec->dx32 = dx32;
  rec->dx = dx;
  rec->E = reinterpret_cast<float*>(m->ke_e);
  rec->y = y;
  rec->mask = m->mask;
  rec->err = m->tma_err;
  rec->nxyp = nxyp;
  rec->nn = m->nn;
  rec->W = g.hx * g.hy * g.hz / 8.0;
  rec->nx = g.nx;
  rec->ny = g.ny;
  rec->nz = g.nz;
  rec->nxp = nxp;
  rec->pin = m->pin_active;
  rec->elastic = elastic;
  rec->al = (float)m->P.alpha;
  rec->cm = (float)m->P.c_mass;
  rec->rhx = (float)(1.0 / g.hx);
  rec->rhy = (float)(1.0 / g.hy);
  rec->rhz = (float)(1.0 / g.hz);
  return FSI_OK;
}

int nsq_batch_launch(bool f64, const NSQBatchRec* recs, const int4* eitems, int neitems, const int4* nitems,
                     int nnitems, const int* active, cudaStream_t s) {
  if (f64) {
    if (neitems > 0) nsq_elem_batch_kernel<<<neitems, dim3(TBX, TBY), 0, s>>>(recs, eitems, active);
    if (nnitems > 0) ns_node_batch_kernel<double><<<nnitems, 128, 0, s>>>(recs, nitems, active);
    FSI_CUDA(cudaGetLastError());
    return FSI_OK;
  }
  const size_t smem = sizeof(float) * (size_t)TSTAGES * NCQ * TBX * TBY;
  if (neitems > 0) nsq_tma_batch_kernel<<<neitems, dim3(TBX, TBY), smem, s>>>(recs, eitems, active);
  if (nnitems > 0) ns_node_batch_kernel<float><<<nnitems, 128, 0, s>>>(recs, nitems, active);
  FSI_CUDA(cudaGetLastError());
  return FSI_OK;
}

int launch_nsq_tma(fsi_mesh* m, int elastic, float* E, const double* dx, double* y) {
  const Geom& g = m->g;
  const int nxp = cq_pitch(m);
  const int64_t nxyp = (int64_t)nxp * g.ny;
  if (m->cq_tmap_base != m->cq32)
    if (int rc = encode_maps(m, nxp, nxyp)) return rc;
  if (!m->tma_err) {
    FSI_CUDA(cudaMalloc(&m->tma_err, sizeof(int)));
    FSI_CUDA(cudaMemsetAsync(m->tma_err, 0, sizeof(int), m->stream));
  }
  const int64_t nblk = (int64_t)((g.nx + TBX - 1) / TBX) * ((g.ny + TBY - 1) / TBY) * g.nz;
  if (nblk > INT32_MAX) return set_error(FSI_EINVAL, "NS float32 product: mesh too large for one launch");
  const CUtensorMap* map = reinterpret_cast<const CUtensorMap*>(m->cq_tmap + (elastic ? 0 : 128));
  const int ncoef = elastic ? NCQ : NCQ_FLUID;
  const size_t smem = sizeof(float) * (size_t)TSTAGES * ncoef * TBX * TBY;
  const dim3 blk(TBX, TBY);
  const float al = (float)m->P.alpha, cm = (float)m->P.c_mass;
  const float rx = (float)(1.0 / g.hx), ry = (float)(1.0 / g.hy), rz = (float)(1.0 / g.hz);
  FSI_LAUNCH(m, P_NS_JVP32,
             (nsq_tma_kernel<<<(unsigned)nblk, blk, smem, m->stream>>>(*map, ncoef, m->dx32, E, g.nx, g.ny, g.nz, nxp,
                                                                      nxyp, m->nn, al, cm, rx, ry, rz, m->tma_err)));
  (void)dx;
  (void)y;
  return FSI_OK;
}

}  // namespace fsi
