// fsi_gmres and fsi_step: block solves and the partitioned time step.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace fsi {

// x^{n+1} = x^n, then the velocity Dirichlet values and the pressure pin.
__global__ void predictor_kernel(double* x, const double* xn, const uint8_t* mask, const double* vD, int ncomp,
                                 int64_t nn) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < nn; n += stride) {
    const uint8_t mk = mask[n];
    for (int c = 0; c < ncomp; ++c) {
      double v = xn[(int64_t)c * nn + n];
      if (c < 3 && ((mk >> c) & 1)) v = vD[(int64_t)c * nn + n];
      if (c == 3 && (mk & 8)) v = 0.0;
      x[(int64_t)c * nn + n] = v;
    }
  }
}

// dx^{n+1} = dx^n + (x^{n+1} - x^n - dt dx^n)/(varsigma dt); x^n <- x^{n+1}.
__global__ void corrector_kernel(const double* x, double* xn, double* xdn, double dt, double vs, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += stride) {
    const double x1 = x[j], x0 = xn[j], d0 = xdn[j];
    xdn[j] = d0 + (x1 - x0 - dt * d0) / (vs * dt);
    xn[j] = x1;
  }
}

static int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

// Pressure level after an NS solve with the pin node's continuity equation kept: the
// update of the pinned formulation is the computed one minus the constant that brings
// p^{n+1} at the pin node to zero, s = x_p[pin] + dx_p[pin] (constant pressure is a null
// mode of the enclosed domain's system, so the shifted update solves it as well).
__global__ void pin_shift_value(const double* xp, const double* dxp, int pin, double* s) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *s = xp[pin] + dxp[pin];
}
__global__ void pin_shift_apply(double* dxp, const double* s, int64_t nn) {
  const double v = *s;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < nn; n += stride) dxp[n] -= v;
}

int step_predict(fsi_mesh* m, fsi_state* st) {
  FSI_LAUNCH(m, P_STAGE, predictor_kernel<<<grid_for(m->nn), 256, 0, m->stream>>>(st->x, st->xn, m->mask, m->vD,
                                                                                   m->ncomp, m->nn));
  return FSI_OK;
}

int step_correct(fsi_mesh* m, fsi_state* st) {
  const int64_t n = m->nn * m->ncomp;
  FSI_LAUNCH(m, P_STAGE, corrector_kernel<<<grid_for(n), 256, 0, m->stream>>>(st->x, st->xn, st->xdn, m->P.dt,
                                                                                 m->P.vs, n));
  return FSI_OK;
}

bool shifts_pressure(const fsi_mesh* m, unsigned solve_flags) {
  return m->pin_node >= 0 && m->enclosed && m->pin_active && !(solve_flags & FSI_PINNED_SOLVE);
}

int pin_shift(fsi_mesh* m, const double* x, double* dx) {
  const int64_t nn = m->nn;
  FSI_LAUNCH(m, P_STAGE, pin_shift_value<<<1, 32, 0, m->stream>>>(x + 3 * nn, dx + 3 * nn, m->pin_node, m->red + 8));
  FSI_LAUNCH(m, P_STAGE, pin_shift_apply<<<grid_for(nn), 256, 0, m->stream>>>(dx + 3 * nn, m->red + 8, nn));
  return FSI_OK;
}

}  // namespace fsi

using namespace fsi;

extern "C" {

int fsi_gmres(fsi_mesh* m, int32_t block, const fsi_state* st, const double* rhs, double* x,
              const fsi_solve_opts* o, fsi_solve_info* info) {
  if (!m || !rhs || !x || !o) return set_error(FSI_EINVAL, "fsi_gmres: null argument");
  BlockInfo b;
  int rc = block_info(m, block, &b);
  if (rc) return rc;
  if ((rc = stage(m, st, o->precision == FSI_PREC_FP32_IR))) return rc;
  return gmres_solve(m, b, rhs, x, *o, info);
}

int fsi_step(fsi_mesh* m, fsi_state* st, const fsi_step_opts* o, fsi_step_info* info) {
  if (!m || !st || !o) return set_error(FSI_EINVAL, "fsi_step: null argument");
  if (o->k_max < 1) return set_error(FSI_EINVAL, "fsi_step: k_max must be >= 1");
  const int64_t nn = m->nn;
  const int64_t nmax = 6 * nn;
  if (m->step_ws_n < nmax) {
    cudaFree(m->step_ws);
    m->step_ws = nullptr;
    FSI_CUDA(cudaMalloc(&m->step_ws, sizeof(double) * 2 * nmax));
    m->step_ws_n = nmax;
  }
  double* rhs = m->step_ws;
  double* dx = m->step_ws + nmax;
  const bool fp32 = o->solve.precision == FSI_PREC_FP32_IR;
  fsi_step_info inf{};
  const int64_t a0 = m->applies, d0 = m->dof_applied;
  int rc;
  if ((rc = step_predict(m, st))) return rc;
  const int nblocks = 1 + m->N + m->ns;
  for (int k = 0; k < o->k_max; ++k) {
    double max_ratio = 0.0;
    for (int bi = 0; bi < nblocks; ++bi) {
      const int32_t id = bi == 0 ? FSI_BLOCK_NS : (bi <= m->N ? FSI_BLOCK_AC(bi - 1) : FSI_BLOCK_B(bi - 1 - m->N));
      BlockInfo b;
      if ((rc = block_info(m, id, &b))) return rc;
      if ((rc = stage(m, st, fp32))) return rc;
      if (b.kind == 1) {
        double gb[2];
        if ((rc = op_coeffs(m, b.index, gb))) return rc;
        m->gamma[b.index] = m->fixed_gamma[b.index] >= 0.0 ? m->fixed_gamma[b.index] : gb[0];
        m->beta[b.index] = gb[1];
      }
      // NS block of an enclosed domain: the pin node keeps its continuity equation in
      // the solve and the pressure level is set by the shift below
      const bool shift = b.kind == 0 && shifts_pressure(m, o->solve.flags);
      fsi_solve_info si{};
      {
        PinGuard guard(m, shift ? 0 : m->pin_active);
        if ((rc = op_residual(m, b, rhs))) return rc;
        if ((rc = vec_scale_copy(m, -1.0, rhs, rhs, b.n))) return rc;
        rc = gmres_solve(m, b, rhs, dx, o->solve, &si);
        if (rc && rc != FSI_ENOCONV) return rc;
      }
      if (shift && (rc = pin_shift(m, st->x, dx))) return rc;
      inf.worst_rel_res = std::max(inf.worst_rel_res, si.rel_res);
      if (si.stalled) inf.stalled_solves++;
      if (si.fallback) inf.fallback_solves++;
      if (b.kind == 0) inf.gmres_iters_ns += si.iterations;
      else if (b.kind == 1) inf.gmres_iters_ac += si.iterations;
      else inf.gmres_iters_b += si.iterations;
      double* xb = st->x + (int64_t)b.c0 * nn;
      if ((rc = vec_axpy(m, 1.0, dx, xb, b.n))) return rc;
      double d2, x2;
      if ((rc = vec_dot(m, dx, dx, b.n, &d2))) return rc;
      if ((rc = vec_dot(m, xb, xb, b.n, &x2))) return rc;
      if (!std::isfinite(d2) || !std::isfinite(x2)) return set_error(FSI_ENAN, "fsi_step: solution is not finite");
      const double ratio = x2 > 0.0 ? std::sqrt(d2 / x2) : std::sqrt(d2);
      max_ratio = std::max(max_ratio, ratio);
    }
    inf.nl_iters = k + 1;
    inf.max_ratio = max_ratio;
    if (!o->fixed_iters && max_ratio < o->nl_tol) break;
  }
  if ((rc = step_correct(m, st))) return rc;
  FSI_CUDA(cudaStreamSynchronize(m->stream));
  inf.applies = (int)(m->applies - a0);
  inf.dof_applied = m->dof_applied - d0;
  if (info) *info = inf;
  return FSI_OK;
}

}  // extern "C"
