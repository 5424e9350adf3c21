// Element physics of the four equation sets, evaluated by the tile engine.
//
// Notation at a quadrature point (velocities, phases and B at n+alpha, rates at
// n+alpha_m, p at n+1; rho, mu blended nodal fields, alpha^s = (1+phi^s)/2):
//   L_kj = d v_k / d x_j,  acc_k = dv_k + v_j L_kj,
//   R_m,k = rho acc_k + d_k p - rho g_k,  R_c = L_jj,
//   tau_m = ((2/dt)^2 + v.G v + C_I (mu/rho)^2 G:G)^(-1/2),  tau_c = 1/(tr G tau_m).
// Momentum (test N_a e_k): N_a rho (acc_k - g_k)
//   + d_j N_a [ -p d_kj + mu (L_kj + L_jk) + E_kj + tau_m v_j R_m,k + tau_c rho R_c d_kj ]
//   E = sum_s alpha^s mu_L^s (B^s - I)
// Continuity (test N_a): N_a R_c + d_j N_a (tau_m/rho) R_m,j            (Eq. PG_NS)
// Allen-Cahn (Eq. PPV_AC, plain Galerkin coefficients):
//   N_a R_phi + d_j N_a (gamma eps^2 d_j phi + tau_phi v_j R_phi),
//   R_phi = dphi + v.grad phi + gamma (F'(phi) - beta sqrt F(phi)),
//   tau_phi = ((2/dt)^2 + v.Gv + 9 (gamma eps^2)^2 G:G + (gamma (3phi^2-1))^2)^(-1/2)
// B transport (Eq. semiCGT), each stored component c = (k,l):
//   (N_a + tau_B v.grad N_a) Rb_kl,
//   Rb = alpha (dB + (v.grad)B - L B - B L^T) + (1 - alpha)(B - I),
//   tau_B = ((2/dt)^2 + v.G v)^(-1/2).
// Jacobian-vector products differentiate in x^{n+1} with every tau, gamma, beta,
// phi (NS) and B (NS) frozen: d(x^{n+alpha}) = alpha dx, d(dx^{n+alpha_m}) = c_m dx,
// c_m = alpha_m/(varsigma dt).  The NS product adds the solid-stress linearization
// of Section 2.4:  sum_s alpha^s mu_L^s c_el ( -(vt.grad)B^s + grad vt B^s + B^s grad vt^T ),
// vt = alpha dv, c_el = alpha varsigma dt / alpha_m.
#pragma once
#include "q1_tile.cuh"

namespace fsi {

constexpr int MAXP = 16;   // phases
constexpr int MAXS = 16;   // solids
constexpr int MAXF = 40;   // staged fields per kernel

// Resident 256-thread CTAs per SM the register budget is cut for (one: a cap of
// 128 registers spills and measured slower for the float32 NS product).
#ifndef FSI_MINB_F32
#define FSI_MINB_F32 1
#endif
template <typename T>
struct MinBlocks { static constexpr int value = sizeof(T) == 4 ? FSI_MINB_F32 : 1; };

struct Phys {
  double dt, alpha, alpha_m, vs, c_mass, c_el, c_i, eps, eta;
  double Gd[3], GG, trG;
  double grav[3];
  int N, ns;
  double rho[MAXP], mu[MAXP], muL[MAXP];
  int solid_phase[MAXS];
};

// Nodal field sources for staging: a float64 kernel reads d[], a float32 kernel f[]
// (every staged field of a kernel has the kernel's compute type).
struct Fields {
  const double* d[MAXF];
  const float* f[MAXF];
};

template <typename T>
__device__ __forceinline__ const T* field_ptr(const Fields& F, int i);
template <>
__device__ __forceinline__ const double* field_ptr<double>(const Fields& F, int i) { return F.d[i]; }
template <>
__device__ __forceinline__ const float* field_ptr<float>(const Fields& F, int i) { return F.f[i]; }

// symmetric storage order [11, 22, 33, 12, 23, 13]
__host__ __device__ constexpr int sym_k(int c) { return c < 3 ? c : (c == 3 ? 0 : (c == 4 ? 1 : 0)); }
__host__ __device__ constexpr int sym_l(int c) { return c < 3 ? c : (c == 3 ? 1 : (c == 4 ? 2 : 2)); }
__host__ __device__ constexpr int sym_idx(int k, int l) {
  return k == l ? k : ((k + l == 1) ? 3 : ((k + l == 3) ? 4 : 5));
}

struct OutDesc {
  double* y;            // output block [NC][nn]
  const double* dx;     // JVP input block (Dirichlet rows copy it), or null
  const float* dx32;    // its float copy: the rows copy this one when dx is null
  const double* x;      // state x^{n+1} (residual Dirichlet rows), or null
  const uint8_t* mask;  // Dirichlet mask (NS only): bits 0-2 velocity, bit 3 pressure
  const double* vD;     // Dirichlet velocity values [3][nn]
  int accumulate;       // add into y instead of writing (later solid passes)
  int dirichlet;        // apply Dirichlet rows
  int pin;              // NS: the pressure pin row is active (mask bit 3); 0: the node keeps
                        // its continuity equation (the pressure level is fixed by a shift)
};

// ----------------------------------------------------------------- NS block
// Field layout (NSField): state v(3), p, dv/dt(3), rho, mu, then per solid in the
// pass: alpha^s, B^s(6); JVP: the input dv(3), dp first.
template <typename TT, int MODE>  // MODE 0: residual, 1: JVP, 2: diagonal
struct NSOp {
  using T = TT;
  static constexpr int NC = 4;
  static constexpr int MINB = MinBlocks<TT>::value;
  Fields F;
  int nf;           // staged field count
  int s0, s1;       // solids in this pass
  int fluid;        // 1: include the fluid/pressure terms (first pass)
  int elastic_aug;  // JVP/diagonal: add the solid-stress linearization
  Phys P;
  double rh[3], W;
  OutDesc out;

  __device__ __forceinline__ const T* fptr(int f) const { return field_ptr<T>(F, f); }
  using Red = NoRed;
  __device__ __forceinline__ void begin_cta(Red&) const {}
  __device__ __forceinline__ void end_cta(Red&) const {}

  __device__ void element(const Corners<T>& cr, const ElemCtx&, T (&c)[NC][8], Red&) const {
    const T rhx = T(rh[0]), rhy = T(rh[1]), rhz = T(rh[2]);
    const int base = (MODE == 1) ? 4 : 0;  // JVP: fields 0..3 are dv, dp
    const int fv = base, fp = base + 3, fvd = base + 4, frho = base + 7, fmu = base + 8, fsol = base + 9;
    const T alpha = T(P.alpha), cm = T(P.c_mass), cel = T(P.c_el);
    T u[8];
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
      QW<T> w;
      w.set(q);
      cr.get(frho, u); const T rho = interp_v(u, w);
      cr.get(fmu, u);  const T mu = interp_v(u, w);
      T v[3], L[3][3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        cr.get(fv + k, u);
        const VG<T> r = interp_vg(u, w, rhx, rhy, rhz);
        v[k] = r.v; L[k][0] = r.gx; L[k][1] = r.gy; L[k][2] = r.gz;
      }
      cr.get(fp, u);
      const VG<T> pr = interp_vg(u, w, rhx, rhy, rhz);
      const T gp[3] = {pr.gx, pr.gy, pr.gz};
      T Rm[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        cr.get(fvd + k, u);
        const T acc = interp_v(u, w) + v[0] * L[k][0] + v[1] * L[k][1] + v[2] * L[k][2];
        Rm[k] = rho * acc + gp[k] - rho * T(P.grav[k]);
      }
      const T vGv = T(P.Gd[0]) * v[0] * v[0] + T(P.Gd[1]) * v[1] * v[1] + T(P.Gd[2]) * v[2] * v[2];
      const T nu = mu / rho;
      const T dt2 = T(4.0) / (T(P.dt) * T(P.dt));
      const T tau_m = T(1) / sqrt(dt2 + vGv + T(P.c_i) * nu * nu * T(P.GG));
      const T tau_c = T(1) / (T(P.trG) * tau_m);
      const T Rc = L[0][0] + L[1][1] + L[2][2];

      if (MODE == 0) {
        T E[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        for (int s = s0; s < s1; ++s) {
          const int fs = fsol + 7 * (s - s0);
          cr.get(fs, u);
          const T a = interp_v(u, w) * T(P.muL[P.solid_phase[s]]);
#pragma unroll
          for (int cc = 0; cc < 6; ++cc) {
            cr.get(fs + 1 + cc, u);
            E[cc] += a * (interp_v(u, w) - (cc < 3 ? T(1) : T(0)));
          }
        }
        const T W = T(this->W);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          T gk[3];
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            T s = E[sym_idx(k, j)];
            if (fluid) {
              s += mu * (L[k][j] + L[j][k]) + tau_m * v[j] * Rm[k];
              if (j == k) s += -pr.v + tau_c * rho * Rc;
            }
            gk[j] = W * s;
          }
          const T fk = fluid ? W * (Rm[k] - gp[k]) : T(0);  // rho (acc_k - g_k)
          scatter_vg(c[k], w, fk, gk[0], gk[1], gk[2], rhx, rhy, rhz);
        }
        if (fluid) {
          const T r = W * tau_m / rho;
          scatter_vg(c[3], w, W * Rc, r * Rm[0], r * Rm[1], r * Rm[2], rhx, rhy, rhz);
        }
      } else if (MODE == 1) {
        T dv[3], dL[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          cr.get(k, u);
          const VG<T> r = interp_vg(u, w, rhx, rhy, rhz);
          dv[k] = r.v; dL[k][0] = alpha * r.gx; dL[k][1] = alpha * r.gy; dL[k][2] = alpha * r.gz;
        }
        cr.get(3, u);
        const VG<T> dpr = interp_vg(u, w, rhx, rhy, rhz);
        T vt[3], dRm[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) vt[k] = alpha * dv[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const T dacc = cm * dv[k] + vt[0] * L[k][0] + vt[1] * L[k][1] + vt[2] * L[k][2] +
                         v[0] * dL[k][0] + v[1] * dL[k][1] + v[2] * dL[k][2];
          dRm[k] = rho * dacc;
        }
        const T dgp[3] = {dpr.gx, dpr.gy, dpr.gz};
        T dE[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        if (elastic_aug) {
          for (int s = s0; s < s1; ++s) {
            const int fs = fsol + 7 * (s - s0);
            cr.get(fs, u);
            const T a = interp_v(u, w) * T(P.muL[P.solid_phase[s]]) * cel;
            T B[6], dd[6];
#pragma unroll
            for (int cc = 0; cc < 6; ++cc) {
              cr.get(fs + 1 + cc, u);
              const VG<T> r = interp_vg(u, w, rhx, rhy, rhz);
              B[cc] = r.v;
              dd[cc] = vt[0] * r.gx + vt[1] * r.gy + vt[2] * r.gz;
            }
            // P = grad(vt) B ; dE += a ( -dd + P + P^T )
#pragma unroll
            for (int cc = 0; cc < 6; ++cc) {
              const int k = sym_k(cc), l = sym_l(cc);
              T pkl = T(0), plk = T(0);
#pragma unroll
              for (int m = 0; m < 3; ++m) {
                pkl += dL[k][m] * B[sym_idx(m, l)];
                plk += dL[l][m] * B[sym_idx(m, k)];
              }
              dE[cc] += a * (pkl + plk - dd[cc]);
            }
          }
        }
        const T W = T(this->W);
        if (fluid) {
          const T dRc = dL[0][0] + dL[1][1] + dL[2][2];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            T gk[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
              T s = dE[sym_idx(k, j)] + mu * (dL[k][j] + dL[j][k]) + tau_m * (vt[j] * Rm[k] + v[j] * (dRm[k] + dgp[k]));
              if (j == k) s += -dpr.v + tau_c * rho * dRc;
              gk[j] = W * s;
            }
            scatter_vg(c[k], w, W * dRm[k], gk[0], gk[1], gk[2], rhx, rhy, rhz);
          }
          const T r = W * tau_m / rho;
          scatter_vg(c[3], w, W * dRc, r * (dRm[0] + dgp[0]), r * (dRm[1] + dgp[1]), r * (dRm[2] + dgp[2]),
                     rhx, rhy, rhz);
        } else {
#pragma unroll
          for (int k = 0; k < 3; ++k)
            scatter_vg(c[k], w, T(0), W * dE[sym_idx(k, 0)], W * dE[sym_idx(k, 1)], W * dE[sym_idx(k, 2)],
                       rhx, rhy, rhz);
        }
      } else {  // MODE 2: diagonal, trial = test = N_a e_k
        // per-solid terms of the augmentation: a_s, B^s and its divergence-like row sums
        T aB[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};  // sum_s a_s B^s
        T aG[3][3];                                      // sum_s a_s d_k B^s_kj  (row k, j)
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int j = 0; j < 3; ++j) aG[k][j] = T(0);
        if (elastic_aug) {
          for (int s = s0; s < s1; ++s) {
            const int fs = fsol + 7 * (s - s0);
            cr.get(fs, u);
            const T a = interp_v(u, w) * T(P.muL[P.solid_phase[s]]) * cel * alpha;
#pragma unroll
            for (int cc = 0; cc < 6; ++cc) {
              cr.get(fs + 1 + cc, u);
              const VG<T> r = interp_vg(u, w, rhx, rhy, rhz);
              aB[cc] += a * r.v;
              const int k = sym_k(cc), l = sym_l(cc);
              const T gk[3] = {r.gx, r.gy, r.gz};
              aG[k][l] += a * gk[k];
              if (k != l) aG[l][k] += a * gk[l];
            }
          }
        }
        const T W = T(this->W);
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
          const T N = w.wx[ax] * w.wy[ay] * w.wz[az];
          const T gN[3] = {(ax ? T(1) : T(-1)) * rhx * w.wy[ay] * w.wz[az],
                           (ay ? T(1) : T(-1)) * rhy * w.wx[ax] * w.wz[az],
                           (az ? T(1) : T(-1)) * rhz * w.wx[ax] * w.wy[ay]};
          const T vgN = v[0] * gN[0] + v[1] * gN[1] + v[2] * gN[2];
          const T gN2 = gN[0] * gN[0] + gN[1] * gN[1] + gN[2] * gN[2];
          // grad N^T (sum a_s B) grad N
          T BNN = T(0);
#pragma unroll
          for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int j = 0; j < 3; ++j) BNN += gN[m] * aB[sym_idx(m, j)] * gN[j];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const T da = cm * N + alpha * N * L[k][k] + alpha * vgN;
            T d = T(0);
            if (fluid)
              d = N * rho * da + alpha * mu * (gN2 + gN[k] * gN[k]) + tau_m * alpha * N * Rm[k] * gN[k] +
                  tau_m * vgN * rho * da + tau_c * rho * alpha * gN[k] * gN[k];
            if (elastic_aug) {
              T divrow = T(0), Bk = T(0);
#pragma unroll
              for (int j = 0; j < 3; ++j) {
                divrow += aG[k][j] * gN[j];
                Bk += aB[sym_idx(k, j)] * gN[j];
              }
              d += -N * divrow + BNN + Bk * gN[k];
            }
            c[k][a] += W * d;
          }
          if (fluid) c[3][a] += W * tau_m / rho * gN2;
        }
      }
    }
  }

  __device__ __forceinline__ void finish(const NodeCtx& nc, const T (&acc)[NC], Red&) const {
    const int64_t nn = nn_;
    const uint8_t m = out.mask ? out.mask[nc.n] : 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double* y = out.y + (int64_t)k * nn + nc.n;
      const bool dir = ((m >> k) & 1) && (k < 3 || out.pin);
      if (dir) {
        if (!out.dirichlet) continue;
        if (MODE == 0) {
          *y = out.x[(int64_t)k * nn + nc.n] - (k < 3 ? out.vD[(int64_t)k * nn + nc.n] : 0.0);
        } else if (MODE == 1) {
          *y = out.dx ? out.dx[(int64_t)k * nn + nc.n] : (double)out.dx32[(int64_t)k * nn + nc.n];
        } else {
          *y = 1.0;
        }
      } else {
        *y = out.accumulate ? *y + (double)acc[k] : (double)acc[k];
      }
    }
  }
  int64_t nn_;
};

// ----------------------------------------------- NS product from frozen coefficients
// Within one NS block solve every coefficient of the product is fixed: the state the
// Jacobian is taken at does not move.  NSBuildOp evaluates them once per solve, in
// float64, at every quadrature point of every element; the product (nsq_elem_kernel)
// then interpolates only the increment (dv, dp).  Per quadrature point:
//   0 rho, 1 mu, 2-4 v, 5-13 L_kj = d_j v_k (k-major), 14-16 R_m,
//   17 tau_m, 18 tau_c rho, 19 tau_m / rho,
//   20-25 aB = sum_s a_s B^s, 26-43 aG[c][m] = sum_s a_s d_m B^s_c (c in [11,22,33,12,23,13]),
//   a_s = alpha^s mu_L^s c_el (the solid-stress linearization of Section 2.4: its
//   dependence on the solids is linear in these two sums, whatever their number).
// Layout (one plane of elements per coefficient and quadrature point, x fastest with a
// padded pitch):  C[((ez * 8 + q) * NCQ + c) * nxyp + ey * nxp + ex].
constexpr int NCQ = 44;
constexpr int NCQ_FLUID = 20;

struct CoefArrays {
  double* c64;   // float64 coefficients (the build writes them)
  float* c32;    // float32 copy (rounded from float64), or null
  int nxp;       // x pitch (elements, padded)
  int64_t nxyp;  // nxp * ny
};

// Coefficient build: fields as NSOp MODE 0 (v(3), p, dv/dt(3), rho, mu, then alpha^s,
// B^s(6) per solid of the pass).  Only the CTA that owns an element writes it.  Later
// solid passes (fluid == 0) add their solids' sums into aB and aG.
struct NSBuildOp {
  using T = double;
  static constexpr int NC = 1;
  static constexpr int MINB = 1;
  Fields F;
  int nf;
  int s0, s1;
  int fluid;
  int elastic_aug;
  Phys P;
  double rh[3], W;
  CoefArrays C;

  __device__ __forceinline__ const T* fptr(int f) const { return field_ptr<T>(F, f); }
  using Red = NoRed;
  __device__ __forceinline__ void begin_cta(Red&) const {}
  __device__ __forceinline__ void end_cta(Red&) const {}

  __device__ __forceinline__ void put(int64_t idx, double v, bool add) const {
    if (add) v += C.c64[idx];
    C.c64[idx] = v;
    if (C.c32) C.c32[idx] = (float)v;
  }

  __device__ void element(const Corners<T>& cr, const ElemCtx& ec, T (&)[NC][8], Red&) const {
    if (!ec.owned) return;  // halo copies of this element are built by its owner
    const T rhx = rh[0], rhy = rh[1], rhz = rh[2];
    const int fv = 0, fp = 3, fvd = 4, frho = 7, fmu = 8, fsol = 9;
    const int64_t e0 = (int64_t)ec.ez * 8 * NCQ * C.nxyp + (int64_t)ec.ey * C.nxp + ec.ex;
    T u[8];
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
      QW<T> w;
      w.set(q);
      const int64_t b = e0 + (int64_t)q * NCQ * C.nxyp;
      T v[3], L[3][3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        cr.get(fv + k, u);
        const VG<T> r = interp_vg(u, w, rhx, rhy, rhz);
        v[k] = r.v; L[k][0] = r.gx; L[k][1] = r.gy; L[k][2] = r.gz;
      }
      if (fluid) {
        cr.get(frho, u); const T rho = interp_v(u, w);
        cr.get(fmu, u);  const T mu = interp_v(u, w);
        cr.get(fp, u);
        const VG<T> pr = interp_vg(u, w, rhx, rhy, rhz);
        const T gp[3] = {pr.gx, pr.gy, pr.gz};
        T Rm[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          cr.get(fvd + k, u);
          const T acc = interp_v(u, w) + v[0] * L[k][0] + v[1] * L[k][1] + v[2] * L[k][2];
          Rm[k] = rho * acc + gp[k] - rho * P.grav[k];
        }
        const T vGv = P.Gd[0] * v[0] * v[0] + P.Gd[1] * v[1] * v[1] + P.Gd[2] * v[2] * v[2];
        const T nu = mu / rho;
        const T tau_m = 1.0 / sqrt(4.0 / (P.dt * P.dt) + vGv + P.c_i * nu * nu * P.GG);
        const T tau_c = 1.0 / (P.trG * tau_m);
        put(b + 0 * C.nxyp, rho, false);
        put(b + 1 * C.nxyp, mu, false);
#pragma unroll
        for (int k = 0; k < 3; ++k) put(b + (2 + k) * C.nxyp, v[k], false);
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int j = 0; j < 3; ++j) put(b + (5 + 3 * k + j) * C.nxyp, L[k][j], false);
#pragma unroll
        for (int k = 0; k < 3; ++k) put(b + (14 + k) * C.nxyp, Rm[k], false);
        put(b + 17 * C.nxyp, tau_m, false);
        put(b + 18 * C.nxyp, tau_c * rho, false);
        put(b + 19 * C.nxyp, tau_m / rho, false);
      }
      T aB[6], aG[6][3];
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) {
        aB[cc] = 0.0;
        aG[cc][0] = aG[cc][1] = aG[cc][2] = 0.0;
      }
      if (elastic_aug) {
        for (int s = s0; s < s1; ++s) {
          const int fs = fsol + 7 * (s - s0);
          cr.get(fs, u);
          const T a = interp_v(u, w) * P.muL[P.solid_phase[s]] * P.c_el;
#pragma unroll
          for (int cc = 0; cc < 6; ++cc) {
            cr.get(fs + 1 + cc, u);
            const VG<T> r = interp_vg(u, w, rhx, rhy, rhz);
            aB[cc] += a * r.v;
            aG[cc][0] += a * r.gx;
            aG[cc][1] += a * r.gy;
            aG[cc][2] += a * r.gz;
          }
        }
      }
      const bool add = !fluid;
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) {
        put(b + (20 + cc) * C.nxyp, aB[cc], add);
#pragma unroll
        for (int mm = 0; mm < 3; ++mm) put(b + (26 + 3 * cc + mm) * C.nxyp, aG[cc][mm], add);
      }
    }
  }
  __device__ __forceinline__ void finish(const NodeCtx&, const T (&)[NC], Red&) const {}
};

// The product's arithmetic at one quadrature point, from the interpolated increment
// (dv, its gradient gd[k][j] = d_j dv_k, dp and its gradient dgp) and the point's
// coefficients k (the 44 above): the coefficients of the test functions, f[eq] of N_a and
// g[eq][j] of d_j N_a, for the three momentum equations and continuity (unweighted).
template <typename T, class Coef>
__device__ __forceinline__ void nsq_point_fg(const Coef& k, bool elastic, const T (&dv)[3], const T (&gd)[3][3],
                                             T dp, const T (&dgp)[3], T al, T cmass, T (&f)[4], T (&g)[4][3]) {
  const T rho = k(0), mu = k(1);
  const T v[3] = {k(2), k(3), k(4)};
  const T Rm[3] = {k(14), k(15), k(16)};
  const T tau_m = k(17), tc_rho = k(18), tm_rho = k(19);
  T dL[3][3], vt[3], dRm[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    vt[a] = al * dv[a];
#pragma unroll
    for (int b = 0; b < 3; ++b) dL[a][b] = al * gd[a][b];
  }
#pragma unroll
  for (int kk = 0; kk < 3; ++kk) {
    const T dacc = cmass * dv[kk] + vt[0] * k(5 + 3 * kk) + vt[1] * k(6 + 3 * kk) + vt[2] * k(7 + 3 * kk) +
                   v[0] * dL[kk][0] + v[1] * dL[kk][1] + v[2] * dL[kk][2];
    dRm[kk] = rho * dacc;
  }
  T dE[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  if (elastic) {
    T aB[6];
#pragma unroll
    for (int cc = 0; cc < 6; ++cc) aB[cc] = k(20 + cc);
#pragma unroll
    for (int cc = 0; cc < 6; ++cc) {
      const int kk = sym_k(cc), l = sym_l(cc);
      T pkl = T(0), plk = T(0);
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        pkl += dL[kk][m] * aB[sym_idx(m, l)];
        plk += dL[l][m] * aB[sym_idx(m, kk)];
      }
      const T dd = vt[0] * k(26 + 3 * cc) + vt[1] * k(27 + 3 * cc) + vt[2] * k(28 + 3 * cc);
      dE[cc] = pkl + plk - dd;
    }
  }
  const T dRc = dL[0][0] + dL[1][1] + dL[2][2];
#pragma unroll
  for (int kk = 0; kk < 3; ++kk) {
    const T sk = tau_m * (dRm[kk] + dgp[kk]);
    const T rk = tau_m * Rm[kk];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      T sj = dE[sym_idx(kk, j)] + mu * (dL[kk][j] + dL[j][kk]) + vt[j] * rk + v[j] * sk;
      if (j == kk) sj += -dp + tc_rho * dRc;
      g[kk][j] = sj;
    }
    f[kk] = dRm[kk];
  }
  f[3] = dRc;
#pragma unroll
  for (int j = 0; j < 3; ++j) g[3][j] = tm_rho * (dRm[j] + dgp[j]);
}

// The same, scattered to the 8 corners of a hex quadrature point (sum-factorised).
template <typename T, class Coef>
__device__ __forceinline__ void nsq_point(const Coef& k, bool elastic, const T (&dv)[3], const T (&gd)[3][3], T dp,
                                          const T (&dgp)[3], T al, T cmass, const QW<T>& w, T rhx, T rhy, T rhz,
                                          T (&c)[4][8]) {
  T f[4], g[4][3];
  nsq_point_fg<T>(k, elastic, dv, gd, dp, dgp, al, cmass, f, g);
#pragma unroll
  for (int eq = 0; eq < 4; ++eq) scatter_vg(c[eq], w, f[eq], g[eq][0], g[eq][1], g[eq][2], rhx, rhy, rhz);
}

// Coefficient accessor over a strided plane layout (loads through the read-only path).
template <typename T>
struct CoefRef {
  const T* p;
  int64_t s;
  __device__ __forceinline__ T operator()(int i) const { return __ldg(p + i * s); }
};


// ------------------------------------------- float64 NS product from element matrices
// GB300 issues float64 FMAs at 1/64 of the float32 rate, so a float64 solve that
// applies the product hundreds of times on one state stores each element's 32 x 32
// matrix (rows and columns ordered field-major: 8 corners of dv_x, dv_y, dv_z, dp) once
// and applies it with 1024 FMAs per element, against about 2400 for the coefficient
// form.  Layout: K[((ez * 1024 + i * 32 + j) * nxyp + ey * nxp + ex], unweighted (W
// per node as above).  Column j is the coefficient product of the unit increment j, so
// both forms are the same operator up to summation order.
constexpr int NKE = 32 * 32;


// ----------------------------------------------------------------- AC block
// fields: [dphi (JVP)], v(3), phi, dphi/dt
template <typename TT, int MODE>
struct ACOp {
  using T = TT;
  static constexpr int NC = 1;
  static constexpr int MINB = MinBlocks<TT>::value;
  Fields F;
  int nf;
  Phys P;
  double rh[3], W;
  double gamma, beta;
  OutDesc out;
  int64_t nn_;

  __device__ __forceinline__ const T* fptr(int f) const { return field_ptr<T>(F, f); }
  using Red = NoRed;
  __device__ __forceinline__ void begin_cta(Red&) const {}
  __device__ __forceinline__ void end_cta(Red&) const {}

  __device__ void element(const Corners<T>& cr, const ElemCtx&, T (&c)[NC][8], Red&) const {
    const T rhx = T(rh[0]), rhy = T(rh[1]), rhz = T(rh[2]);
    const int base = MODE == 1 ? 1 : 0;
    const T alpha = T(P.alpha), cm = T(P.c_mass);
    const T gam = T(gamma), bet = T(beta);
    const T k_hat = gam * T(P.eps) * T(P.eps);
    const T dt2 = T(4.0) / (T(P.dt) * T(P.dt));
    T u[8];
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
      QW<T> w;
      w.set(q);
      T v[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) { cr.get(base + k, u); v[k] = interp_v(u, w); }
      cr.get(base + 3, u);
      const VG<T> ph = interp_vg(u, w, rhx, rhy, rhz);
      const T phi = ph.v;
      const T vGv = T(P.Gd[0]) * v[0] * v[0] + T(P.Gd[1]) * v[1] * v[1] + T(P.Gd[2]) * v[2] * v[2];
      const T s_hat = gam * (T(3) * phi * phi - T(1));
      const T tau = T(1) / sqrt(dt2 + vGv + T(9) * k_hat * k_hat * T(P.GG) + s_hat * s_hat);
      const T W = T(this->W);
      if (MODE == 0) {
        cr.get(base + 4, u);
        const T pdot = interp_v(u, w);
        const T Fp = phi * phi * phi - phi;
        const T sF = T(0.5) * fabs(phi * phi - T(1));
        const T R = pdot + v[0] * ph.gx + v[1] * ph.gy + v[2] * ph.gz + gam * (Fp - bet * sF);
        scatter_vg(c[0], w, W * R, W * (k_hat * ph.gx + tau * v[0] * R), W * (k_hat * ph.gy + tau * v[1] * R),
                   W * (k_hat * ph.gz + tau * v[2] * R), rhx, rhy, rhz);
      } else {
        const T p2 = phi * phi - T(1);
        const T dsF = p2 > T(0) ? phi : (p2 < T(0) ? -phi : T(0));
        const T rp = gam * (T(3) * phi * phi - T(1) - bet * dsF);
        if (MODE == 1) {
          cr.get(0, u);
          const VG<T> d = interp_vg(u, w, rhx, rhy, rhz);
          const T dR = cm * d.v + alpha * (v[0] * d.gx + v[1] * d.gy + v[2] * d.gz) + alpha * rp * d.v;
          const T ka = k_hat * alpha;
          scatter_vg(c[0], w, W * dR, W * (ka * d.gx + tau * v[0] * dR), W * (ka * d.gy + tau * v[1] * dR),
                     W * (ka * d.gz + tau * v[2] * dR), rhx, rhy, rhz);
        } else {
#pragma unroll
          for (int a = 0; a < 8; ++a) {
            const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
            const T N = w.wx[ax] * w.wy[ay] * w.wz[az];
            const T gN[3] = {(ax ? T(1) : T(-1)) * rhx * w.wy[ay] * w.wz[az],
                             (ay ? T(1) : T(-1)) * rhy * w.wx[ax] * w.wz[az],
                             (az ? T(1) : T(-1)) * rhz * w.wx[ax] * w.wy[ay]};
            const T vgN = v[0] * gN[0] + v[1] * gN[1] + v[2] * gN[2];
            const T dR = cm * N + alpha * vgN + alpha * rp * N;
            c[0][a] += W * (N * dR + k_hat * alpha * (gN[0] * gN[0] + gN[1] * gN[1] + gN[2] * gN[2]) + tau * vgN * dR);
          }
        }
      }
    }
  }

  __device__ __forceinline__ void finish(const NodeCtx& nc, const T (&acc)[NC], Red&) const {
    out.y[nc.n] = (double)acc[0];
  }
};

// Float64 Allen-Cahn products through element matrices: the 8 x 8 matrix of the product of
// Eq. PPV_AC's linearization (gamma, beta, tau_phi frozen) per element, weighted,
//   K[b][a] = sum_q W ( N_b dR_a + khat alpha grad N_b . grad N_a + tau (v . grad N_b) dR_a ),
//   dR_a = c_m N_a + alpha v . grad N_a + alpha gamma (3 phi^2 - 1 - beta dsqrtF) N_a,
// layout K[((ez * 64 + b * 8 + a) * nxyp + ey * nxp + ex], built once the solve has taken
// ACE_AFTER float64 products (64 FMAs per element and product against about 2000 flops).
// Build fields: v(3), phi.
struct ACEBuildOp {
  using T = double;
  static constexpr int NC = 1;
  static constexpr int MINB = 1;
  Fields F;
  int nf;
  Phys P;
  double rh[3], W;
  double gamma, beta;
  double* K;
  int nxp;
  int64_t nxyp;

  __device__ __forceinline__ const T* fptr(int f) const { return field_ptr<T>(F, f); }
  using Red = NoRed;
  __device__ __forceinline__ void begin_cta(Red&) const {}
  __device__ __forceinline__ void end_cta(Red&) const {}

  __device__ void element(const Corners<T>& cr, const ElemCtx& ec, T (&)[NC][8], Red&) const {
    if (!ec.owned) return;
    const double rhx = rh[0], rhy = rh[1], rhz = rh[2];
    const double alpha = P.alpha, cm = P.c_mass, gam = gamma, bet = beta;
    const double k_hat = gam * P.eps * P.eps, ka = k_hat * alpha;
    const double dt2 = 4.0 / (P.dt * P.dt);
    double Ke[8][8];
#pragma unroll
    for (int b = 0; b < 8; ++b)
#pragma unroll
      for (int a = 0; a < 8; ++a) Ke[b][a] = 0.0;
    double u[8];
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
      QW<double> w;
      w.set(q);
      double v[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) { cr.get(k, u); v[k] = interp_v(u, w); }
      cr.get(3, u);
      const double phi = interp_v(u, w);
      const double vGv = P.Gd[0] * v[0] * v[0] + P.Gd[1] * v[1] * v[1] + P.Gd[2] * v[2] * v[2];
      const double s_hat = gam * (3.0 * phi * phi - 1.0);
      const double tau = 1.0 / sqrt(dt2 + vGv + 9.0 * k_hat * k_hat * P.GG + s_hat * s_hat);
      const double p2 = phi * phi - 1.0;
      const double dsF = p2 > 0.0 ? phi : (p2 < 0.0 ? -phi : 0.0);
      const double rp = gam * (3.0 * phi * phi - 1.0 - bet * dsF);
      double N[8], gN[8][3], vgN[8], dR[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
        N[a] = w.wx[ax] * w.wy[ay] * w.wz[az];
        gN[a][0] = (ax ? 1.0 : -1.0) * rhx * w.wy[ay] * w.wz[az];
        gN[a][1] = (ay ? 1.0 : -1.0) * rhy * w.wx[ax] * w.wz[az];
        gN[a][2] = (az ? 1.0 : -1.0) * rhz * w.wx[ax] * w.wy[ay];
        vgN[a] = v[0] * gN[a][0] + v[1] * gN[a][1] + v[2] * gN[a][2];
        dR[a] = cm * N[a] + alpha * vgN[a] + alpha * rp * N[a];
      }
#pragma unroll
      for (int b = 0; b < 8; ++b)
#pragma unroll
        for (int a = 0; a < 8; ++a)
          Ke[b][a] += W * (N[b] * dR[a] + ka * (gN[b][0] * gN[a][0] + gN[b][1] * gN[a][1] + gN[b][2] * gN[a][2]) +
                           tau * vgN[b] * dR[a]);
    }
    double* out = K + (int64_t)ec.ez * 64 * nxyp + (int64_t)ec.ey * nxp + ec.ex;
#pragma unroll
    for (int b = 0; b < 8; ++b)
#pragma unroll
      for (int a = 0; a < 8; ++a) out[(int64_t)(b * 8 + a) * nxyp] = Ke[b][a];
  }
  __device__ __forceinline__ void finish(const NodeCtx&, const T (&)[NC], Red&) const {}
};


// ----------------------------------------------------------------- B block
// fields: [dB(6) (JVP)], v(3), alpha^s, B(6), dB/dt(6)
template <typename TT, int MODE>
struct BOp {
  using T = TT;
  static constexpr int NC = 6;
  static constexpr int MINB = MinBlocks<TT>::value;
  Fields F;
  int nf;
  Phys P;
  double rh[3], W;
  OutDesc out;
  int64_t nn_;

  __device__ __forceinline__ const T* fptr(int f) const { return field_ptr<T>(F, f); }
  using Red = NoRed;
  __device__ __forceinline__ void begin_cta(Red&) const {}
  __device__ __forceinline__ void end_cta(Red&) const {}

  __device__ void element(const Corners<T>& cr, const ElemCtx&, T (&c)[NC][8], Red&) const {
    const T rhx = T(rh[0]), rhy = T(rh[1]), rhz = T(rh[2]);
    const int base = MODE == 1 ? 6 : 0;
    const T alpha = T(P.alpha), cm = T(P.c_mass);
    const T dt2 = T(4.0) / (T(P.dt) * T(P.dt));
    T u[8];
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
      QW<T> w;
      w.set(q);
      T v[3], L[3][3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        cr.get(base + k, u);
        const VG<T> r = interp_vg(u, w, rhx, rhy, rhz);
        v[k] = r.v; L[k][0] = r.gx; L[k][1] = r.gy; L[k][2] = r.gz;
      }
      cr.get(base + 3, u);
      const T al = interp_v(u, w);
      const T vGv = T(P.Gd[0]) * v[0] * v[0] + T(P.Gd[1]) * v[1] * v[1] + T(P.Gd[2]) * v[2] * v[2];
      const T tau = T(1) / sqrt(dt2 + vGv);
      const T W = T(this->W);
      if (MODE == 2) {
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
          const T N = w.wx[ax] * w.wy[ay] * w.wz[az];
          const T gN[3] = {(ax ? T(1) : T(-1)) * rhx * w.wy[ay] * w.wz[az],
                           (ay ? T(1) : T(-1)) * rhy * w.wx[ax] * w.wz[az],
                           (az ? T(1) : T(-1)) * rhz * w.wx[ax] * w.wy[ay]};
          const T vgN = v[0] * gN[0] + v[1] * gN[1] + v[2] * gN[2];
#pragma unroll
          for (int cc = 0; cc < 6; ++cc) {
            const int k = sym_k(cc), l = sym_l(cc);
            const T dR = al * (cm * N + alpha * vgN - alpha * N * (L[k][k] + L[l][l])) + (T(1) - al) * alpha * N;
            c[cc][a] += W * (N + tau * vgN) * dR;
          }
        }
        continue;
      }
      // B (residual: state; JVP: alpha dB) with gradient, and its rate
      T B[6], cv[6];
      const int fb = MODE == 1 ? 0 : base + 4;
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) {
        cr.get(fb + cc, u);
        const VG<T> r = interp_vg(u, w, rhx, rhy, rhz);
        const T sc = MODE == 1 ? alpha : T(1);
        B[cc] = sc * r.v;
        cv[cc] = sc * (v[0] * r.gx + v[1] * r.gy + v[2] * r.gz);
        if (MODE == 1) cv[cc] += cm * r.v;  // rate of the increment
      }
      if (MODE == 0) {
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) {
          cr.get(base + 10 + cc, u);
          cv[cc] += interp_v(u, w);
        }
      }
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) {
        const int k = sym_k(cc), l = sym_l(cc);
        T st = T(0);
#pragma unroll
        for (int m = 0; m < 3; ++m) st += L[k][m] * B[sym_idx(m, l)] + B[sym_idx(k, m)] * L[l][m];
        const T rec = B[cc] - ((MODE == 0 && cc < 3) ? T(1) : T(0));
        const T R = al * (cv[cc] - st) + (T(1) - al) * rec;
        const T tr = W * tau * R;
        scatter_vg(c[cc], w, W * R, tr * v[0], tr * v[1], tr * v[2], rhx, rhy, rhz);
      }
    }
  }

  __device__ __forceinline__ void finish(const NodeCtx& nc, const T (&acc)[NC], Red&) const {
#pragma unroll
    for (int cc = 0; cc < 6; ++cc) out.y[(int64_t)cc * nn_ + nc.n] = (double)acc[cc];
  }
};

// Float64 B products split for reuse within a solve.  The linearized transport of Eq.
// semiCGT is, for every stored component c, one scalar operator (mass, convection and the
// recovery term, tested with N_a + tau_B v . grad N_a) plus a pointwise coupling of the
// components through the stretching terms L dB + dB L^T.  Per element the build stores
//   S[a][b] = sum_q W (N_a + tau v.grad N_a) (al (c_m N_b + alpha v.grad N_b) + (1 - al) alpha N_b),
//   per point q: T_a(q) = W (N_a + tau v.grad N_a) al alpha (8) and L(q) = grad v (9),
// 200 values (layout K[((ez * 200 + c) * nxyp + ey * nxp + ex], c < 64: S, then 17 per
// point); the product is then
//   y_c,a = sum_b S[a][b] dB_c,b - sum_q T_a(q) (L dB(q) + dB(q) L^T)_c,
// 1440 FMAs per element against about 3200 for BOp<double,1>.  Build fields: v(3), alpha^s.
constexpr int NBK = 64 + 8 * 17;

struct BEBuildOp {
  using T = double;
  static constexpr int NC = 1;
  static constexpr int MINB = 1;
  Fields F;
  int nf;
  Phys P;
  double rh[3], W;
  double* K;
  int nxp;
  int64_t nxyp;

  __device__ __forceinline__ const T* fptr(int f) const { return field_ptr<T>(F, f); }
  using Red = NoRed;
  __device__ __forceinline__ void begin_cta(Red&) const {}
  __device__ __forceinline__ void end_cta(Red&) const {}

  __device__ void element(const Corners<T>& cr, const ElemCtx& ec, T (&)[NC][8], Red&) const {
    if (!ec.owned) return;
    const double rhx = rh[0], rhy = rh[1], rhz = rh[2];
    const double alpha = P.alpha, cm = P.c_mass;
    const double dt2 = 4.0 / (P.dt * P.dt);
    double* out = K + (int64_t)ec.ez * NBK * nxyp + (int64_t)ec.ey * nxp + ec.ex;
    double S[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) S[a][b] = 0.0;
    double u[8];
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
      QW<double> w;
      w.set(q);
      double v[3], L[3][3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        cr.get(k, u);
        const VG<double> r = interp_vg(u, w, rhx, rhy, rhz);
        v[k] = r.v; L[k][0] = r.gx; L[k][1] = r.gy; L[k][2] = r.gz;
      }
      cr.get(3, u);
      const double al = interp_v(u, w);
      const double vGv = P.Gd[0] * v[0] * v[0] + P.Gd[1] * v[1] * v[1] + P.Gd[2] * v[2] * v[2];
      const double tau = 1.0 / sqrt(dt2 + vGv);
      double N[8], test[8], trial[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
        N[a] = w.wx[ax] * w.wy[ay] * w.wz[az];
        const double vgN = v[0] * (ax ? 1.0 : -1.0) * rhx * w.wy[ay] * w.wz[az] +
                           v[1] * (ay ? 1.0 : -1.0) * rhy * w.wx[ax] * w.wz[az] +
                           v[2] * (az ? 1.0 : -1.0) * rhz * w.wx[ax] * w.wy[ay];
        test[a] = W * (N[a] + tau * vgN);
        trial[a] = al * (cm * N[a] + alpha * vgN) + (1.0 - al) * alpha * N[a];
      }
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) S[a][b] += test[a] * trial[b];
      const int64_t qb = 64 + 17 * q;
#pragma unroll
      for (int a = 0; a < 8; ++a) out[(qb + a) * nxyp] = test[a] * al * alpha;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int m = 0; m < 3; ++m) out[(qb + 8 + 3 * k + m) * nxyp] = L[k][m];
    }
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) out[(int64_t)(a * 8 + b) * nxyp] = S[a][b];
  }
  __device__ __forceinline__ void finish(const NodeCtx&, const T (&)[NC], Red&) const {}
};


// ----------------------------------------------------------------- gamma, beta
// fields: v(3), phi.  Node output: int N_p q and int N_p; band RMS and beta
// integrals reduced per CTA into partials[cta][4] = {sum val^2, n_band, int F', int sqrtF}.
struct CoefOp {
  using T = double;
  static constexpr int NC = 2;
  static constexpr int MINB = 1;
  Fields F;
  int nf;
  double rh[3], W;
  double* partials;
  int ncta_xy[2];
  const double* phi_node;  // nodal phi^{n+alpha}
  struct Red { double sv2, nband, sFp, ssF; };

  __device__ __forceinline__ const double* fptr(int f) const { return F.d[f]; }
  __device__ __forceinline__ void begin_cta(Red& r) const { r.sv2 = r.nband = r.sFp = r.ssF = 0.0; }

  __device__ void element(const Corners<double>& cr, const ElemCtx& ec, double (&c)[NC][8], Red& red) const {
    const double rhx = rh[0], rhy = rh[1], rhz = rh[2];
    double u[8];
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
      QW<double> w;
      w.set(q);
      double L[3][3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        cr.get(k, u);
        const VG<double> r = interp_vg(u, w, rhx, rhy, rhz);
        L[k][0] = r.gx; L[k][1] = r.gy; L[k][2] = r.gz;
      }
      cr.get(3, u);
      const VG<double> ph = interp_vg(u, w, rhx, rhy, rhz);
      const double g[3] = {ph.gx, ph.gy, ph.gz};
      const double n2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
      double num = 0.0;
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) num += g[j] * L[j][k] * g[k];
      const double qv = n2 < 1e-30 ? 0.0 : num / n2;
      scatter_v(c[0], w, W * qv);
      scatter_v(c[1], w, W);
      if (ec.owned) {
        red.sFp += W * (ph.v * ph.v * ph.v - ph.v);
        red.ssF += W * 0.5 * fabs(ph.v * ph.v - 1.0);
      }
    }
  }
  __device__ __forceinline__ void finish(const NodeCtx& nc, const double (&acc)[NC], Red& red) const {
    if (fabs(phi_node[nc.n]) <= 0.9) {
      const double val = fabs(acc[0] / acc[1]);
      red.sv2 += val * val;
      red.nband += 1.0;
    }
  }
  __device__ void end_cta(Red& red) const {
    __shared__ double scratch[NTHREADS / 32];
    const double a = block_sum(red.sv2, scratch);
    const double b = block_sum(red.nband, scratch);
    const double cF = block_sum(red.sFp, scratch);
    const double d = block_sum(red.ssF, scratch);
    if (threadIdx.x == 0) {
      const int64_t cta = blockIdx.x + (int64_t)ncta_xy[0] * (blockIdx.y + (int64_t)ncta_xy[1] * blockIdx.z);
      partials[4 * cta + 0] = a;
      partials[4 * cta + 1] = b;
      partials[4 * cta + 2] = cF;
      partials[4 * cta + 3] = d;
    }
  }
};

}  // namespace fsi
