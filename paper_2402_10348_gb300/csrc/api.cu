// C ABI of libfsi: mesh handle, staging, operator dispatch, time step.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "internal.h"

namespace fsi {

static thread_local std::string g_err;

int set_error(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_check(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? FSI_ENOMEM : FSI_ECUDA;
}

int ensure_smem_attr(const void* func, size_t bytes) {
  int dev = 0;
  FSI_CUDA(cudaGetDevice(&dev));
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = done[std::make_pair(func, dev)];
  if (have >= bytes) return FSI_OK;
  FSI_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  have = bytes;
  return FSI_OK;
}

static const char* kProfNames[P_NCLS] = {
    "stage", "ns_residual", "ns_jvp_f64", "ns_jvp_f32", "ns_diag", "ac_residual", "ac_jvp_f64", "ac_jvp_f32",
    "ac_diag", "b_residual", "b_jvp_f64", "b_jvp_f32", "b_diag", "gamma_beta", "krylov_vector", "init",
    "krylov_dot", "krylov_update", "krylov_scalar", "to_float", "pc_conv", "pc_wgrad", "pc_aux", "op_builds", "ns_jvp_f64_em", "node_sums"};
constexpr int PROF_PAIRS = 4096;

int prof_harvest(fsi_mesh* m) {
  Profiler& p = m->prof;
  if (p.used == 0) return FSI_OK;
  FSI_CUDA(cudaEventSynchronize(p.ev[2 * (p.used - 1) + 1]));
  for (int i = 0; i < p.used; ++i) {
    float ms = 0.f;
    FSI_CUDA(cudaEventElapsedTime(&ms, p.ev[2 * i], p.ev[2 * i + 1]));
    p.ms[p.cls[i]] += ms;
  }
  p.used = 0;
  return FSI_OK;
}

int prof_begin(fsi_mesh* m, int cls) {
  Profiler& p = m->prof;
  p.launches[cls]++;
  if (!p.on) return FSI_OK;
  if (p.used == PROF_PAIRS) {
    int rc = prof_harvest(m);
    if (rc) return rc;
  }
  p.cls[p.used] = cls;
  FSI_CUDA(cudaEventRecord(p.ev[2 * p.used], m->stream));
  return FSI_OK;
}

int prof_end(fsi_mesh* m, int cls) {
  Profiler& p = m->prof;
  if (!p.on) return FSI_OK;
  FSI_CUDA(cudaEventRecord(p.ev[2 * p.used + 1], m->stream));
  p.used++;
  return FSI_OK;
}

void tile_grid(const fsi_mesh* m, dim3* grid) {
  const int ncx = (m->g.nx + 1 + OX - 1) / OX;
  const int ncy = (m->g.ny + 1 + OY - 1) / OY;
  const int planes = m->g.nz + 1;
  const int chunks = (planes + m->g.zc - 1) / m->g.zc;
  *grid = dim3(ncx, ncy, chunks);
}

// --------------------------------------------------------------- staging
// x^{n+alpha} = x^n + alpha (x^{n+1} - x^n) (pressure plane: p^{n+1}),
// dx/dt^{n+alpha_m} = dx^n + alpha_m (dx^{n+1} - dx^n),
// dx^{n+1} = dx^n + (x^{n+1} - x^n - dt dx^n) / (varsigma dt)      (Section 2.1.2),
// rho = sum_i alpha^i rho^i, mu = sum_i alpha^i mu^i, alpha^s = (1 + phi^s)/2.
__global__ void stage_kernel(const double* __restrict__ x, const double* __restrict__ xn,
                             const double* __restrict__ xdn, double* xa, double* xd, double* mat,
                             float* xa32, float* xd32, float* mat32, int ncomp, int64_t nn, Phys P,
                             int write_xa) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < nn; n += stride) {
    double rho = 0.0, mu = 0.0;
    for (int c = 0; c < ncomp; ++c) {
      const int64_t o = (int64_t)c * nn + n;
      const double x1 = x[o], x0 = xn[o], d0 = xdn[o];
      const double a = (c == 3) ? x1 : x0 + P.alpha * (x1 - x0);
      const double d1 = d0 + (x1 - x0 - P.dt * d0) / (P.vs * P.dt);
      const double dam = d0 + P.alpha_m * (d1 - d0);
      if (write_xa) xa[o] = a;
      xd[o] = dam;
      if (xa32) { xa32[o] = (float)a; xd32[o] = (float)dam; }
      if (c >= 4 && c < 4 + P.N) {
        const double al = (1.0 + a) / 2.0;
        rho += al * P.rho[c - 4];
        mu += al * P.mu[c - 4];
      }
    }
    mat[n] = rho;
    mat[nn + n] = mu;
    if (mat32) { mat32[n] = (float)rho; mat32[nn + n] = (float)mu; }
    for (int s = 0; s < P.ns; ++s) {
      const int64_t o = (int64_t)(4 + P.solid_phase[s]) * nn + n;
      const double a = write_xa ? xa[o] : x[o];
      const double al = (1.0 + a) / 2.0;
      mat[(2 + s) * nn + n] = al;
      if (mat32) mat32[(2 + s) * nn + n] = (float)al;
    }
  }
}

static int vec_grid(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)std::min<int64_t>(b, 152 * 8);
}

int stage(fsi_mesh* m, const fsi_state* st, bool fp32) {
  if (!st || !st->x || !st->xn || !st->xdn) return set_error(FSI_EINVAL, "state: null pointer");
  const bool alpha1 = m->P.alpha == 1.0;
  const size_t bytes = sizeof(double) * (size_t)m->ncomp * m->nn;
  if (!alpha1 && !m->xa) FSI_CUDA(cudaMalloc(&m->xa, bytes));
  if (fp32 && !m->xa32) {
    FSI_CUDA(cudaMalloc(&m->xa32, bytes / 2));
    FSI_CUDA(cudaMalloc(&m->xd32, bytes / 2));
    FSI_CUDA(cudaMalloc(&m->mat32, sizeof(float) * (2 + m->ns) * m->nn));
  }
  FSI_LAUNCH(m, P_STAGE,
             stage_kernel<<<vec_grid(m->nn), 256, 0, m->stream>>>(
                 st->x, st->xn, st->xdn, alpha1 ? nullptr : m->xa, m->xd, m->mat, fp32 ? m->xa32 : nullptr,
                 fp32 ? m->xd32 : nullptr, fp32 ? m->mat32 : nullptr, m->ncomp, m->nn, m->P, alpha1 ? 0 : 1));
  m->staged_x = st->x;
  m->staged_xa = alpha1 ? st->x : m->xa;
  ++m->stage_gen;
  return FSI_OK;
}

int block_info(const fsi_mesh* m, int32_t block, BlockInfo* bi) {
  const int kind = (block >> 16) & 0xff, idx = block & 0xffff;
  if (block == FSI_BLOCK_NS) {
    *bi = BlockInfo{0, 0, 0, 4, 4 * m->nn};
    return FSI_OK;
  }
  if (kind == 1 && idx < m->N) {
    *bi = BlockInfo{1, idx, 4 + idx, 1, m->nn};
    return FSI_OK;
  }
  if (kind == 2 && idx < m->ns) {
    *bi = BlockInfo{2, idx, 4 + m->N + 6 * idx, 6, 6 * m->nn};
    return FSI_OK;
  }
  return set_error(FSI_EINVAL, "invalid block id");
}

// the tetrahedral kernels of a block (tet.cu)
static int tet_op(fsi_mesh* m, const BlockInfo& b, int mode, const double* dx, double* y, unsigned flags) {
  if (b.kind == 0) return tet_ns(m, mode, dx, y, flags);
  if (b.kind == 1) return tet_ac(m, mode, b.index, dx, y, flags);
  return tet_b(m, mode, b.index, dx, y, flags);
}

int op_residual(fsi_mesh* m, const BlockInfo& b, double* r) {
  m->applies++;
  m->dof_applied += b.n;
  if (m->tet) return tet_op(m, b, 0, nullptr, r, 0);
  if (b.kind == 0) return launch_ns<double>(m, 0, nullptr, r, 0);
  if (b.kind == 1) return launch_ac<double>(m, 0, b.index, nullptr, r);
  return launch_b<double>(m, 0, b.index, nullptr, r);
}

__global__ void to_float_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) b[i] = (float)a[i];
}

int ensure_dx32(fsi_mesh* m) {
  if (!m->dx32) FSI_CUDA(cudaMalloc(&m->dx32, sizeof(float) * 6 * (size_t)m->nn));
  return FSI_OK;
}

int op_jvp(fsi_mesh* m, const BlockInfo& b, const double* dx, double* y, unsigned flags) {
  m->applies++;
  m->dof_applied += b.n;
  if (m->tet) return tet_op(m, b, 1, dx, y, flags & ~OP_DX32_READY);
  const bool f32 = flags & FSI_FP32;
  if (f32) {  // float copy of the increment for the float32 kernels (unless the caller wrote it)
    if (int rc = ensure_dx32(m)) return rc;
    if (!(flags & OP_DX32_READY))
      FSI_LAUNCH(m, P_KRY_CONV, to_float_kernel<<<vec_grid(b.n), 256, 0, m->stream>>>(dx, m->dx32, b.n));
  }
  flags &= ~OP_DX32_READY;
  if (b.kind == 0) {
    // recorded (batched) launches take the per-element kernel; single launches the
    // product from the quadrature-point coefficients
    if (m->rec) return f32 ? launch_ns<float>(m, 1, dx, y, flags) : launch_ns<double>(m, 1, dx, y, flags);
    return f32 ? launch_nsq<float>(m, dx, y, flags) : launch_nsq<double>(m, dx, y, flags);
  }
  if (b.kind == 1)
    return f32 ? launch_ac<float>(m, 1, b.index, dx, y) : launch_ac<double>(m, 1, b.index, dx, y);
  return f32 ? launch_b<float>(m, 1, b.index, dx, y) : launch_b<double>(m, 1, b.index, dx, y);
}

int op_diag(fsi_mesh* m, const BlockInfo& b, double* d, unsigned flags) {
  if (m->tet) return tet_op(m, b, 2, nullptr, d, flags);
  const bool f32 = flags & FSI_FP32;
  if (b.kind == 0)
    return f32 ? launch_ns<float>(m, 2, nullptr, d, flags) : launch_ns<double>(m, 2, nullptr, d, flags);
  if (b.kind == 1)
    return f32 ? launch_ac<float>(m, 2, b.index, nullptr, d) : launch_ac<double>(m, 2, b.index, nullptr, d);
  return f32 ? launch_b<float>(m, 2, b.index, nullptr, d) : launch_b<double>(m, 2, b.index, nullptr, d);
}

// Dirichlet data (velocity faces by priority, interior box, pressure pin).
static void build_bc(const fsi_mesh_desc* d, std::vector<uint8_t>& mask, std::vector<double>& vD) {
  const int nx = d->nx, ny = d->ny, nz = d->nz;
  const int64_t nn = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  mask.assign(nn, 0);
  vD.assign(3 * nn, 0.0);
  const double hx = d->lx / nx, hy = d->ly / ny, hz = d->lz / nz;
  for (int k = 0; k <= nz; ++k)
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i <= nx; ++i) {
        const int64_t n = i + (int64_t)(nx + 1) * (j + (int64_t)(ny + 1) * k);
        const bool on[6] = {i == 0, i == nx, j == 0, j == ny, k == 0, k == nz};
        int best = -1;
        for (int f = 0; f < 6; ++f) {
          if (!on[f] || d->faces[f].kind != FSI_BC_DIRICHLET) continue;
          if (best < 0 || d->faces[f].priority > d->faces[best].priority) best = f;
        }
        if (best >= 0) {
          mask[n] |= 7;
          for (int c = 0; c < 3; ++c) vD[c * nn + n] = d->faces[best].vel[c];
        }
        if (d->has_box) {
          const double x = i * hx, y = j * hy, z = k * hz;
          if (x >= d->box_lo[0] && x <= d->box_hi[0] && y >= d->box_lo[1] && y <= d->box_hi[1] &&
              z >= d->box_lo[2] && z <= d->box_hi[2]) {
            mask[n] |= 7;
            for (int c = 0; c < 3; ++c) vD[c * nn + n] = d->box_vel[c];
          }
        }
      }
  if (d->pin_node >= 0 && d->pin_node < nn) mask[d->pin_node] |= 8;
}

}  // namespace fsi

using namespace fsi;

extern "C" {

const char* fsi_last_error(void) { return g_err.c_str(); }

int fsi_create_mesh(const fsi_mesh_desc* d, fsi_mesh** out) {
  if (!d || !out) return set_error(FSI_EINVAL, "fsi_create_mesh: null argument");
  *out = nullptr;
  if (d->nx < 1 || d->ny < 1 || d->nz < 1) return set_error(FSI_EINVAL, "mesh: nx, ny, nz must be >= 1");
  if (!(d->lx > 0 && d->ly > 0 && d->lz > 0)) return set_error(FSI_EINVAL, "mesh: box lengths must be > 0");
  if (d->n_phase < 1 || d->n_phase > MAXP || !d->phases) return set_error(FSI_EINVAL, "mesh: need 1..16 phases");
  if (!(d->dt > 0) || !(d->eps > 0)) return set_error(FSI_EINVAL, "mesh: dt and eps must be > 0");
  if (!(d->rho_inf >= 0 && d->rho_inf <= 1)) return set_error(FSI_EINVAL, "mesh: rho_inf must be in [0,1]");
  const int64_t nn = (int64_t)(d->nx + 1) * (d->ny + 1) * (d->nz + 1);
  if (d->pin_node >= nn) return set_error(FSI_EINVAL, "mesh: pin_node out of range");
  int ns = 0;
  for (int i = 0; i < d->n_phase; ++i) {
    if (!(d->phases[i].rho > 0) || d->phases[i].mu < 0) return set_error(FSI_EINVAL, "phase: rho > 0, mu >= 0");
    if (d->phases[i].is_solid) ++ns;
  }
  if (ns > MAXS) return set_error(FSI_EINVAL, "mesh: at most 16 solids");
  fsi_mesh* m = new fsi_mesh();
  m->dev = d->device;
  if (cudaSetDevice(d->device) != cudaSuccess) {
    delete m;
    return set_error(FSI_ECUDA, "cudaSetDevice failed");
  }
  m->N = d->n_phase;
  m->ns = ns;
  m->ncomp = 4 + m->N + 6 * ns;
  m->nn = nn;
  m->lx = d->lx; m->ly = d->ly; m->lz = d->lz;
  m->phases.assign(d->phases, d->phases + d->n_phase);
  Geom& g = m->g;
  g.nx = d->nx; g.ny = d->ny; g.nz = d->nz;
  g.nn = nn;
  g.hx = d->lx / d->nx; g.hy = d->ly / d->ny; g.hz = d->lz / d->nz;
  {
    const int cols = ((g.nx + 1 + OX - 1) / OX) * ((g.ny + 1 + OY - 1) / OY);
    const int planes = g.nz + 1;
    int chunks = std::max(1, std::min(planes, (152 + cols / 2) / cols));
    g.zc = (planes + chunks - 1) / chunks;
    g.ncx = (g.nx + 1 + OX - 1) / OX;
    g.ncy = (g.ny + 1 + OY - 1) / OY;
  }
  Phys& P = m->P;
  P.dt = d->dt;
  P.alpha = 1.0 / (1.0 + d->rho_inf);
  P.alpha_m = 0.5 * (3.0 - d->rho_inf) / (1.0 + d->rho_inf);
  P.vs = 0.5 + P.alpha_m - P.alpha;
  P.c_mass = P.alpha_m / (P.vs * P.dt);
  P.c_el = P.alpha * P.vs * P.dt / P.alpha_m;
  P.c_i = d->c_i;
  P.eps = d->eps;
  P.eta = d->eta;
  P.Gd[0] = 4.0 / (g.hx * g.hx);
  P.Gd[1] = 4.0 / (g.hy * g.hy);
  P.Gd[2] = 4.0 / (g.hz * g.hz);
  P.GG = P.Gd[0] * P.Gd[0] + P.Gd[1] * P.Gd[1] + P.Gd[2] * P.Gd[2];
  P.trG = P.Gd[0] + P.Gd[1] + P.Gd[2];
  for (int c = 0; c < 3; ++c) P.grav[c] = d->gravity[c];
  P.N = m->N;
  P.ns = ns;
  int s = 0;
  for (int i = 0; i < m->N; ++i) {
    P.rho[i] = d->phases[i].rho;
    P.mu[i] = d->phases[i].mu;
    P.muL[i] = d->phases[i].mu_L;
    if (d->phases[i].is_solid) P.solid_phase[s++] = i;
  }
  for (int i = 0; i < MAXP; ++i) m->fixed_gamma[i] = -1.0;
  m->pin_node = d->pin_node >= 0 ? d->pin_node : -1;
  m->enclosed = 1;
  for (int f = 0; f < 6; ++f)
    if (d->faces[f].kind != FSI_BC_DIRICHLET) m->enclosed = 0;
  std::vector<uint8_t> mask;
  std::vector<double> vD;
  build_bc(d, mask, vD);
  int rc = FSI_OK;
  auto fail = [&](cudaError_t e, const char* w) {
    rc = cuda_check(e, w);
    fsi_destroy_mesh(m);
    return rc;
  };
  cudaError_t e;
  if ((e = cudaMalloc(&m->mask, nn)) != cudaSuccess) return fail(e, "cudaMalloc mask");
  if ((e = cudaMalloc(&m->vD, sizeof(double) * 3 * nn)) != cudaSuccess) return fail(e, "cudaMalloc vD");
  if ((e = cudaMalloc(&m->xd, sizeof(double) * m->ncomp * nn)) != cudaSuccess) return fail(e, "cudaMalloc xd");
  if ((e = cudaMalloc(&m->mat, sizeof(double) * (2 + ns) * nn)) != cudaSuccess) return fail(e, "cudaMalloc mat");
  if ((e = cudaMalloc(&m->red, sizeof(double) * 1024)) != cudaSuccess) return fail(e, "cudaMalloc red");
  if ((e = cudaMallocHost(&m->red_host, sizeof(double) * 1024)) != cudaSuccess) return fail(e, "cudaMallocHost");
  if ((e = cudaMemcpy(m->mask, mask.data(), nn, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e, "copy mask");
  if ((e = cudaMemcpy(m->vD, vD.data(), sizeof(double) * 3 * nn, cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail(e, "copy vD");
  *out = m;
  return FSI_OK;
}

int fsi_destroy_mesh(fsi_mesh* m) {
  if (!m) return FSI_OK;
  cudaFree(m->mask);
  cudaFree(m->vD);
  cudaFree(m->xa);
  cudaFree(m->xd);
  cudaFree(m->mat);
  cudaFree(m->xa32);
  cudaFree(m->xd32);
  cudaFree(m->mat32);
  cudaFree(m->partials);
  cudaFree(m->red);
  if (m->red_host) cudaFreeHost(m->red_host);
  cudaFree(m->V);
  cudaFree(m->wk);
  cudaFree(m->dinv);
  cudaFree(m->yvec);
  cudaFree(m->partials_dot);
  cudaFree(m->step_ws);
  cudaFree(m->kry_dev);
  cudaFree(m->dx32);
  cudaFree(m->Z);
  cudaFree(m->cq64);
  cudaFree(m->cq32);
  cudaFree(m->ke64);
  cudaFree(m->ke_e);
  cudaFree(m->tma_err);
  cudaFree(m->ake64);
  cudaFree(m->bke64);
  tet_free(m->tet);
  if (m->kry_est) cudaFreeHost(m->kry_est);
  for (cudaEvent_t e : m->kry_ev) cudaEventDestroy(e);
  for (cudaEvent_t e : m->prof.ev) cudaEventDestroy(e);
  delete m;
  return FSI_OK;
}

int fsi_profile(fsi_mesh* m, int32_t enable) {
  if (!m) return set_error(FSI_EINVAL, "null mesh");
  Profiler& p = m->prof;
  if (enable) {
    if (p.ev.empty()) {
      p.ev.resize(2 * PROF_PAIRS);
      p.cls.resize(PROF_PAIRS);
      for (auto& e : p.ev) FSI_CUDA(cudaEventCreate(&e));
    }
    int rc = prof_harvest(m);
    if (rc) return rc;
    for (int c = 0; c < P_NCLS; ++c) { p.launches[c] = 0; p.ms[c] = 0.0; p.bytes[c] = 0.0; }
    p.on = true;
  } else {
    int rc = prof_harvest(m);
    if (rc) return rc;
    p.on = false;
  }
  return FSI_OK;
}

int fsi_profile_read(fsi_mesh* m, fsi_profile_entry* out, int32_t* n_out) {
  if (!m || !out) return set_error(FSI_EINVAL, "null argument");
  FSI_CUDA(cudaStreamSynchronize(m->stream));
  int rc = prof_harvest(m);
  if (rc) return rc;
  for (int c = 0; c < P_NCLS; ++c) {
    memset(out[c].name, 0, sizeof(out[c].name));
    strncpy(out[c].name, kProfNames[c], sizeof(out[c].name) - 1);
    out[c].launches = m->prof.launches[c];
    out[c].ms = m->prof.ms[c];
    out[c].bytes = m->prof.bytes[c];
  }
  if (n_out) *n_out = P_NCLS;
  return FSI_OK;
}

int fsi_set_stream(fsi_mesh* m, void* stream) {
  if (!m) return set_error(FSI_EINVAL, "null mesh");
  m->stream = (cudaStream_t)stream;
  return FSI_OK;
}

int fsi_mesh_info(const fsi_mesh* m, int32_t* ncomp, int64_t* nn, int32_t* n_solid) {
  if (!m) return set_error(FSI_EINVAL, "null mesh");
  if (ncomp) *ncomp = m->ncomp;
  if (nn) *nn = m->nn;
  if (n_solid) *n_solid = m->ns;
  return FSI_OK;
}

int fsi_residual(fsi_mesh* m, int32_t block, const fsi_state* st, double* r) {
  if (!m || !r) return set_error(FSI_EINVAL, "fsi_residual: null argument");
  BlockInfo b;
  int rc = block_info(m, block, &b);
  if (rc) return rc;
  if ((rc = stage(m, st, false))) return rc;
  return op_residual(m, b, r);
}

int fsi_jvp(fsi_mesh* m, int32_t block, const fsi_state* st, const double* dx, double* y, uint32_t flags) {
  if (!m || !dx || !y) return set_error(FSI_EINVAL, "fsi_jvp: null argument");
  BlockInfo b;
  int rc = block_info(m, block, &b);
  if (rc) return rc;
  if ((rc = stage(m, st, flags & FSI_FP32))) return rc;
  return op_jvp(m, b, dx, y, flags & ~OP_DX32_READY);
}

int fsi_diag(fsi_mesh* m, int32_t block, const fsi_state* st, double* d, uint32_t flags) {
  if (!m || !d) return set_error(FSI_EINVAL, "fsi_diag: null argument");
  BlockInfo b;
  int rc = block_info(m, block, &b);
  if (rc) return rc;
  if ((rc = stage(m, st, flags & FSI_FP32))) return rc;
  return op_diag(m, b, d, flags);
}

int fsi_update_ac_coeffs(fsi_mesh* m, int32_t phase, const fsi_state* st, double* out) {
  if (!m || phase < 0 || phase >= (m ? m->N : 0)) return set_error(FSI_EINVAL, "fsi_update_ac_coeffs: bad phase");
  int rc = stage(m, st, false);
  if (rc) return rc;
  double gb[2];
  if ((rc = op_coeffs(m, phase, gb))) return rc;
  m->gamma[phase] = m->fixed_gamma[phase] >= 0.0 ? m->fixed_gamma[phase] : gb[0];
  m->beta[phase] = gb[1];
  if (out) {
    out[0] = m->gamma[phase];
    out[1] = m->beta[phase];
  }
  return FSI_OK;
}

int fsi_set_ac_coeffs(fsi_mesh* m, int32_t phase, double gamma, double beta) {
  if (!m || phase < 0 || phase >= m->N) return set_error(FSI_EINVAL, "fsi_set_ac_coeffs: bad phase");
  m->gamma[phase] = gamma;
  m->beta[phase] = beta;
  return FSI_OK;
}

int fsi_fix_gamma(fsi_mesh* m, int32_t phase, double gamma) {
  if (!m || phase < 0 || phase >= m->N) return set_error(FSI_EINVAL, "fsi_fix_gamma: bad phase");
  m->fixed_gamma[phase] = gamma;
  return FSI_OK;
}

int fsi_set_pressure_pin(fsi_mesh* m, int32_t active) {
  if (!m) return set_error(FSI_EINVAL, "fsi_set_pressure_pin: null mesh");
  if (active != 0 && active != 1) return set_error(FSI_EINVAL, "fsi_set_pressure_pin: active must be 0 or 1");
  m->pin_active = active;
  return FSI_OK;
}

}  // extern "C"
