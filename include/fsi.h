/* fsi.h - C ABI of libfsi: matrix-free Q1-hexahedral residuals, Jacobian-vector
 * products and solvers of the fully Eulerian phase-field FSI method of Mao & Jaiman
 * (arXiv 2402.10348), on one NVIDIA GB300 (sm_103a).
 *
 * Conventions (all calls):
 *  - Every call returns an int status (fsi_status); no exception crosses the ABI.
 *    On failure fsi_last_error() returns a message (thread-local, valid until the
 *    next failing call of the same thread).
 *  - Field arrays are DEVICE pointers owned by the caller, float64 unless stated.
 *    A nodal state x has ncomp = 4 + N + 6 n_s component planes of nn nodes each,
 *    component-major ("structure of arrays"):
 *        x[c*nn + n],  c = 0..2 velocity v, 3 pressure p, 4..4+N-1 phase
 *        indicators phi^i, 4+N+6s+m component m of the left Cauchy-Green tensor B^s
 *        of solid s in the order [B11, B22, B33, B12, B23, B13] (Section 2.5,
 *        second remark), node n = i + (nx+1)*(j + (ny+1)*k).
 *  - A block vector is the contiguous slice of a state's planes that a block owns:
 *        NS     planes 0..3        (4 nn values)        Eq. LS_NS
 *        AC(i)  plane 4+i          (nn values)          Eq. LS_AC
 *        B(s)   planes 4+N+6s..+5  (6 nn values)        Eq. LS_MC
 *  - Work is issued on the mesh's stream (fsi_set_stream; default the legacy
 *    stream) and is asynchronous unless a call says it synchronises.
 *  - The library owns only the opaque mesh handle and its workspace (allocated
 *    with cudaMalloc at creation and on first use of a solver, freed by
 *    fsi_destroy_mesh).
 */
#ifndef FSI_H
#define FSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FSI_OK = 0,
  FSI_EINVAL = 1,   /* invalid argument (sizes, indices, null pointers)        */
  FSI_ECUDA = 2,    /* a CUDA runtime call failed                               */
  FSI_ENOCONV = 3,  /* a solver did not reach its tolerance                     */
  FSI_ENAN = 4,     /* a residual or solver norm is NaN or Inf                  */
  FSI_ETIMEOUT = 5, /* a bounded device-side wait gave up                       */
  FSI_ENOMEM = 6    /* device allocation failed                                 */
} fsi_status;

/* Block identifiers. */
#define FSI_BLOCK_NS 0
#define FSI_BLOCK_AC(i) (0x10000 | (i))
#define FSI_BLOCK_B(s) (0x20000 | (s))

/* Velocity boundary kinds of a box face. */
#define FSI_BC_NATURAL 0   /* no Dirichlet condition (traction-free outflow)      */
#define FSI_BC_DIRICHLET 1 /* prescribed velocity                                 */

/* Material phase (Section 2.1.1: rho = sum alpha^i rho^i etc.). */
typedef struct {
  double rho;      /* density                                                   */
  double mu;       /* dynamic viscosity                                         */
  double mu_L;     /* shear modulus of a Neo-Hookean solid (0 for a fluid)      */
  int32_t is_solid;/* 1: the phase carries a left Cauchy-Green tensor B^s       */
  int32_t pad;
} fsi_phase;

typedef struct {
  int32_t kind;     /* FSI_BC_NATURAL or FSI_BC_DIRICHLET                       */
  int32_t priority; /* where Dirichlet faces meet, the higher priority wins;
                       ties: lowest face index (x-, x+, y-, y+, z-, z+)          */
  double vel[3];
} fsi_face_bc;

/* Problem on the box [0,lx]x[0,ly]x[0,lz] with nx*ny*nz uniform Q1 hexahedra. */
typedef struct {
  int32_t nx, ny, nz;
  int32_t n_phase;          /* N <= 16, of which n_s <= 16 solids               */
  double lx, ly, lz;
  const fsi_phase* phases;  /* host array of n_phase, copied at creation         */
  double gravity[3];        /* body force per unit mass                          */
  double eps;               /* interface thickness (Eq. Allen-Cahn)              */
  double eta;               /* mobility regularisation (Eq. continuous mobility) */
  double dt;                /* time step                                         */
  double rho_inf;           /* generalized-alpha spectral radius (paper: 0)      */
  double c_i;               /* inverse-estimate constant of tau_m                */
  fsi_face_bc faces[6];     /* x-, x+, y-, y+, z-, z+                            */
  int32_t has_box;          /* interior box of prescribed velocity (overrides faces) */
  int32_t pin_node;         /* node with p = 0, or -1                            */
  double box_lo[3], box_hi[3], box_vel[3];
  int32_t device;           /* CUDA device ordinal                               */
  int32_t pad;
} fsi_mesh_desc;

typedef struct fsi_mesh fsi_mesh;

/* Generalized-alpha state (Section 2.1.2): device arrays of ncomp*nn doubles. */
typedef struct {
  double* x;    /* x^{n+1} (the Newton unknown)                                  */
  double* xn;   /* x^n                                                           */
  double* xdn;  /* dx/dt^n                                                       */
} fsi_state;

/* fsi_jvp / fsi_diag flags */
#define FSI_ELASTIC_AUG 0x1u /* NS: add the solid-stress linearization (Section 2.4) */
#define FSI_FP32 0x2u        /* evaluate in float32 (inputs/outputs stay float64)  */

/* --------------------------------------------------------------- mesh */

/* Creates a mesh handle (Section 2: the uniform Q1 discretisation of the box,
 * the phase table, boundary conditions and time-integration parameters).
 * Validates sizes (n >= 1, N in 1..16, n_s <= 16, eps > 0, dt > 0, ...):
 * FSI_EINVAL on bad input, FSI_ENOMEM/FSI_ECUDA on device failures. */
int fsi_create_mesh(const fsi_mesh_desc* desc, fsi_mesh** out);
int fsi_destroy_mesh(fsi_mesh* mesh);
/* stream: a cudaStream_t (NULL = legacy default stream). */
int fsi_set_stream(fsi_mesh* mesh, void* stream);
/* ncomp, nn, number of solids. */
int fsi_mesh_info(const fsi_mesh* mesh, int32_t* ncomp, int64_t* nn, int32_t* n_solid);

/* --------------------------------------------------------------- operators */

/* Residual of one block at state st (Eq. PG_NS, Eq. PPV_AC, Eq. semiCGT), written to
 * the device block vector r_out.  Velocity Dirichlet rows return x - x_D, the pinned
 * pressure row returns p.  AC blocks use the phase's frozen gamma, beta (see
 * fsi_update_ac_coeffs / fsi_set_ac_coeffs). */
int fsi_residual(fsi_mesh* mesh, int32_t block, const fsi_state* st, double* r_out);

/* Jacobian-vector product y = J(st) dx of one block in x^{n+1} with the stabilisation
 * parameters, gamma, beta and the other blocks' fields frozen at st (Section 2.5).
 * Dirichlet rows are the identity.  flags: FSI_ELASTIC_AUG, FSI_FP32. */
int fsi_jvp(fsi_mesh* mesh, int32_t block, const fsi_state* st, const double* dx, double* y,
            uint32_t flags);

/* Diagonal of the same linear operator (the Jacobi preconditioner). */
int fsi_diag(fsi_mesh* mesh, int32_t block, const fsi_state* st, double* d_out, uint32_t flags);

/* Time-dependent mobility gamma^i (Section 2.2.2: RMS over nodes with |phi| <= 0.9 of
 * the lumped L2-projection of |grad phi^T grad v grad phi| / |grad phi|^2, over eta)
 * and beta^i = int F'(phi)/int sqrt F(phi) (Section 2.2.1) at st; stores them as the
 * phase's frozen coefficients and, if out != NULL, writes {gamma, beta} to the HOST
 * array out (synchronises the stream). */
int fsi_update_ac_coeffs(fsi_mesh* mesh, int32_t phase, const fsi_state* st, double* out);
/* Sets the frozen coefficients explicitly. */
int fsi_set_ac_coeffs(fsi_mesh* mesh, int32_t phase, double gamma, double beta);
/* Fixes gamma^i for the time step (gamma >= 0), or restores the mobility model (< 0). */
int fsi_fix_gamma(fsi_mesh* mesh, int32_t phase, double gamma);
/* Linear (P1) tetrahedral mesh, the paper's element for its falling-sphere and ship-ice
 * runs (Sections 5.3, 6).  d describes the physics and a box grid whose nodes
 * (nn = (nx+1)(ny+1)(nz+1), numbered as for the hexahedral mesh) and face boundary
 * conditions the tetrahedral mesh keeps; coords: host [3][nn] node coordinates (the
 * box faces' nodes on their faces); conn: host [ne][4] node indices of each element,
 * positively oriented (det(x1-x0, x2-x0, x3-x0) > 0), forming a conforming mesh.
 * Geometry (barycentric gradients, volumes, the stabilisation metric G = sum_k
 * grad(xi_k) grad(xi_k)^T) and the node-to-element lists are built here; the caller's
 * arrays are not kept.  Such a mesh carries every block's float64 residual, product and
 * diagonal, gamma and beta, GMRES and fsi_step (float64; FSI_FP32 and FSI_PREC_FP32_IR
 * return FSI_EINVAL); fsi_init_phases, the diagnostics and batches refuse it.  Errors:
 * FSI_EINVAL for an index out of range or an element of non-positive volume. */
int fsi_create_tet_mesh(const fsi_mesh_desc* desc, const double* coords, const int32_t* conn, int64_t ne,
                        fsi_mesh** out);

/* Pressure level of an enclosed domain (every face with a Dirichlet velocity; the
 * pressure is then determined up to a constant, Section 2.1.2's momentum/continuity
 * system has constant pressure in its null space).  active = 1 (default): the NS
 * residual, product and diagonal replace the continuity row of pin_node by the row
 * p = 0.  active = 0: that node keeps its continuity equation, and the system is
 * singular but consistent for residuals of states that meet the velocity conditions;
 * a solve of it plus the shift p -= p[pin_node] gives the pinned solution.  fsi_step
 * solves the NS block this way on enclosed domains (far better conditioned: the pin
 * row makes the near-constant pressure mode converge about 30x slower under Jacobi
 * GMRES on the 16^3 cavity and stall it above 1e-8 from 24^3 up) unless the solve
 * flag FSI_PINNED_SOLVE is given. */
int fsi_set_pressure_pin(fsi_mesh* mesh, int32_t active);

/* --------------------------------------------------------------- solvers */

#define FSI_PC_NONE 0
#define FSI_PC_JACOBI 1
#define FSI_PC_LEARNED 2  /* NS block: the attached network in flexible GMRES (fsi_set_pc);
                             other blocks fall back to FSI_PC_JACOBI                */

/* solve flag: record training pairs of the NS block into the attached learned
 * preconditioner (fsi_set_pc): for every refinement checkpoint x_k (FP32_IR; x_0 = 0)
 * the pair (r_k - r*, x* - x_k) with r_k = rhs - A x_k and x* the final iterate, and
 * from Jacobi-preconditioned Arnoldi steps j = 4, 12, 20, ... (at most 8 per inner
 * solve) the pair (A z_j, z_j), z_j = D^{-1} v_j, with the operator the step used */
#define FSI_HARVEST 0x10u
/* solve flag with FSI_PC_LEARNED: flexible GMRES takes the network's direction at even
 * Arnoldi steps and the Jacobi direction D^{-1} v_j at odd ones, so that its
 * least-squares step weights the two kinds separately.  The recommended mode: a linear
 * network trained on smooth error pairs corrects the low-frequency part of the residual
 * and leaves the high-frequency part to the Jacobi directions (with the network at every
 * step a solve can stall and fall back to Jacobi) */
#define FSI_PC_ALTERNATE 0x20u
/* solve flag: never stop on stagnation.  Without it a solve stops ("stalled") when a
 * whole restart cycle reduces the true residual by less than 1 % (FP32_IR: when a
 * refinement reduces it by less than 10 %); with it the solve runs until rtol or
 * max_iter (and, for FP32_IR, ir_max refinements) */
#define FSI_NO_STALL_STOP 0x40u
/* step flag (solve options of fsi_step): solve the NS block of an enclosed domain with
 * the pressure pin row instead of the continuity equation plus the pressure shift */
#define FSI_PINNED_SOLVE 0x80u

#define FSI_PREC_FP64 0     /* operator applies in float64                         */
#define FSI_PREC_FP32_IR 1  /* float32 operator inside float64 iterative refinement: the
                               inner solves keep their Arnoldi basis in float32 (float64
                               Hessenberg, Givens and residuals); FSI_HARVEST solves keep
                               the float64 basis */

typedef struct {
  int32_t m;          /* restart length (GMRES(m)), <= 64                         */
  int32_t max_iter;   /* total inner iterations                                   */
  double rtol;        /* stop when ||b - A x|| / ||b|| <= rtol                    */
  int32_t precond;    /* FSI_PC_*                                                 */
  int32_t precision;  /* FSI_PREC_*                                               */
  uint32_t flags;     /* operator flags (FSI_ELASTIC_AUG), FSI_HARVEST            */
  int32_t ir_max;     /* FP32_IR: maximum refinement steps                        */
  double ir_inner_rtol; /* FP32_IR: relative tolerance of each inner solve         */
} fsi_solve_opts;

typedef struct {
  int32_t iterations;   /* inner iterations (all restarts and refinements)       */
  int32_t restarts;
  int32_t refinements;  /* FP32_IR outer steps                                   */
  int32_t applies;      /* operator applies (all precisions)                     */
  double rel_res;       /* final ||b - A x|| / ||b|| (float64 operator)           */
  int32_t stalled;      /* 1: stopped because a whole restart cycle reduced the
                           true residual by less than 1 % (or an FP32_IR
                           refinement by less than 10 %)                          */
  int32_t fallback;     /* 1: the learned preconditioner stalled and Jacobi GMRES
                           finished the solve                                     */
} fsi_solve_info;

/* Solves J(st) x = rhs for one block by right-preconditioned restarted GMRES from
 * x = 0 (Arnoldi with classical Gram-Schmidt and the DGKS second pass, Givens rotations; the
 * paper solves every block with GMRES, Section 2.5).  rhs and x are device block
 * vectors.  Returns FSI_ENOCONV (x holds the last iterate) if rtol is not met within
 * max_iter.  Synchronises the stream. */
int fsi_gmres(fsi_mesh* mesh, int32_t block, const fsi_state* st, const double* rhs, double* x,
              const fsi_solve_opts* opts, fsi_solve_info* info);

typedef struct {
  int32_t k_max;         /* nonlinear iterations (paper: 20)                    */
  int32_t fixed_iters;   /* 1: always run k_max iterations (parity mode)        */
  double nl_tol;         /* ||dx_blk|| / ||x_blk|| < nl_tol for all blocks (5e-4) */
  fsi_solve_opts solve;
} fsi_step_opts;

typedef struct {
  int32_t nl_iters;
  int32_t gmres_iters_ns, gmres_iters_ac, gmres_iters_b;
  int32_t applies;           /* operator applies (residuals and products)      */
  int32_t stalled_solves;    /* block solves that stopped on stagnation        */
  int64_t dof_applied;       /* sum over applies of the block's DoF count      */
  double max_ratio;          /* last iteration's max ||dx_blk|| / ||x_blk||     */
  double worst_rel_res;      /* largest final linear relative residual         */
  int32_t fallback_solves;   /* FSI_PC_LEARNED solves finished by Jacobi GMRES */
  int32_t pad;
} fsi_step_info;

/* One partitioned time step (Section 2.1.2 predictor-multicorrector, Section 2.5):
 * predictor x^{n+1} = x^n with the velocity Dirichlet values; k_max nonlinear
 * iterations of NS -> AC(0..N-1) (gamma, beta frozen per block) -> B(0..n_s-1), each
 * a Newton step solved by fsi_gmres; corrector dx/dt^{n+1} from the
 * generalized-alpha relation; then x^n <- x^{n+1}, dx/dt^n <- dx/dt^{n+1}.
 * Synchronises the stream. */
int fsi_step(fsi_mesh* mesh, fsi_state* st, const fsi_step_opts* opts, fsi_step_info* info);

/* --------------------------------------------------------------- initialisation */

/* Triangulated closed surface (host arrays, copied). */
typedef struct {
  const double* verts;  /* [n_verts][3]                                         */
  const int32_t* tris;  /* [n_tris][3] vertex indices                           */
  int32_t n_verts, n_tris;
} fsi_surface;

#define FSI_RULE_SURFACE 0     /* phi = signed-distance profile of one surface   */
#define FSI_RULE_COMPLEMENT 1  /* alpha = max(0, 1 - sum of surface alphas) x plane */

typedef struct {
  int32_t kind;
  int32_t surface;     /* FSI_RULE_SURFACE: surface index                         */
  double plane_z;      /* FSI_RULE_COMPLEMENT: plane z = plane_z                  */
  int32_t plane_side;  /* 0 none, +1 keep z < plane_z, -1 keep z > plane_z       */
  int32_t pad;
} fsi_phase_rule;

/* Phase-indicator initialisation (Section 3, Algorithms 1 and 2): for every surface
 * the grid-cell nearest-vertex distance (gx*gy*gz cells over the node bounding box,
 * triangles binned by their bounding boxes grown by 3 eps) and the +x ray-casting
 * sign with non-duplicated plane partitioning (chi = 1e-12 L^2, L the box diagonal),
 * phi = +-tanh(d/(sqrt2 eps)) (positive inside) or +-1 in cells without triangles;
 * then each phase by its rule.
 * phi_out: device [n_phase][nn].  tags_out: device int32 [n_surf][4][nn] or NULL:
 * {cell id, nearest vertex (-1 outside interface cells), crossing number, inside}.
 * Integer tags are bit-identical to a sequential evaluation of the same rules.
 * FSI_EINVAL if the number of distinct crossing keys of one ray exceeds 64.
 * Synchronises the stream. */
int fsi_init_phases(fsi_mesh* mesh, const fsi_surface* surfaces, int32_t n_surf,
                    const fsi_phase_rule* rules, int32_t gx, int32_t gy, int32_t gz,
                    double* phi_out, int32_t* tags_out);

/* --------------------------------------------------------------- diagnostics
 * Centre of mass of solid `solid` (Section 5.2): x_c = int x alpha^s / int alpha^s,
 * alpha^s = (1 + phi^s)/2, integrated exactly element by element (the operators'
 * 2x2x2 Gauss rule is exact for these integrands).  x: device state [ncomp][nn] (only
 * the solid's phase plane is read).  out: host double[3].  Deterministic (fixed-order
 * sums).  Synchronises the stream.  FSI_EINVAL for a bad solid index or an indicator
 * with no positive mass. */
int fsi_center_of_mass(fsi_mesh* mesh, const double* x, int32_t solid, double* out);

/* Point tracking (Appendix C): moves n points, device double [n][3] (x, y, z per point)
 * in place, by one forward-Euler step p <- p + dt v(p), v the trilinear interpolant of
 * the velocity planes of the device state x (pass x^{n+1}) in the element that holds
 * the point; a point outside the box is located at its position clamped onto the box.
 * n = 0 is a no-op; n < 0 is FSI_EINVAL.  Asynchronous. */
int fsi_track_points(fsi_mesh* mesh, const double* x, int64_t n, double* points);

/* --------------------------------------------------------------- allocation-free variant
 * (no counterpart in the paper.)  gamma and beta of one phase, as fsi_update_ac_coeffs
 * computes them, for callers that cannot call cudaMalloc: code that must not
 * synchronise the device (cudaMalloc and cudaFree may) and code inside a framework
 * whose allocator owns all device memory.  It needs no mesh handle and allocates
 * nothing: its per-CTA partial sums live in a file-scope __device__ array of the
 * library, 512 KiB per device, held by every GPU that loads the library until the
 * process exits.
 *   v          device float64 [3][nn]: v^{n+alpha} (x^{n+1} when rho_inf = 0)
 *   phi        device float64 [nn]:    phi^{n+alpha} of the phase
 *   gamma_beta device float64 [2]:     written {gamma, beta} (stream-ordered)
 *   stream     cudaStream_t (NULL = legacy default stream)
 * Meshes needing more than 16384 per-CTA partial sums (about 37 M nodes) are
 * rejected with FSI_EINVAL.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current: make that first call
 * before any stream capture.  All calls share the one array, which keeps the last
 * call's contents (every launch overwrites the slots it reads, so nothing has to
 * start at zero); calls that overlap on the GPU race on it. */
int fsi_gamma_beta_noalloc(int32_t nx, int32_t ny, int32_t nz, double lx, double ly, double lz, double eta,
                           const double* v, const double* phi, double* gamma_beta, void* stream);

/* --------------------------------------------------------------- learned preconditioner
 * (no counterpart in the paper, which prescribes GMRES but no preconditioner.)
 * A 3D convolutional U-Net on the mesh's node grid acts as a flexible right
 * preconditioner of the NS block: z = M(r) = D^{-1} r + (|r| / sqrt(n)) dbar_c kc_c y_c
 * on non-Dirichlet rows (z = r on Dirichlet rows), where D is the Jacobi diagonal,
 * n = 4 nn, and y = net(x) with input channels x_c = (D^{-1} r)_c sqrt(n) / (|r| dbar_c)
 * (0 on Dirichlet rows) for c < 4, then the N phase indicators phi^{n+alpha}, zero
 * padded to 16.  Network: 4 levels (node grids n -> n/2+1), 16 channels, 3x3x3
 * zero-padded convolutions without bias, ReLU:
 *   a_l = relu(conv x_l), e_l = relu(conv a_l), x_{l+1} = R e_l          (l = 0, 1, 2)
 *   a_3 = relu(conv x_3), d_3 = relu(conv a_3)
 *   b_l = relu(conv [e_l, P d_{l+1}]), d_l = relu(conv b_l)               (l = 2, 1, 0)
 *   y = conv d_0  (4 output channels)
 * with P the Q1 interpolation between node grids and R = P^T / 8.  Weights: 15
 * convolutions W[co][ci][kz][ky][kx] float32, concatenated in the order enc0a, enc0b,
 * enc1a, enc1b, enc2a, enc2b, bota, botb, dec2a, dec2b, dec1a, dec1b, dec0a, dec0b,
 * out; they compute in bfloat16 with float32 accumulation (5th-generation tensor
 * cores), activations are stored in bfloat16.
 * Tensors passed in/out (x_in, target) use the library's layout: x_in is 2 planes of
 * [nz+1][ny+1][nx+1] voxels x 8 bfloat16 (channels 0-7, then 8-15); target and y are
 * planar [4][nn] (bfloat16 resp. float32).  All pointers are device pointers unless
 * named _host.  Calls synchronise the mesh's stream. */
typedef struct fsi_pc fsi_pc;
typedef struct {
  int32_t block;        /* FSI_BLOCK_NS                                           */
  int32_t n_pairs_cap;  /* training pairs held on the device (ring buffer), >= 0   */
  int32_t linear;       /* 1: no ReLU, the network is a linear operator of its input */
  int32_t modulate;     /* 1: input channels 4.. are s_c (1 + phi_s) / 2 for each
                           solid s (at most 3) instead of the indicators, so that a
                           linear network keeps z = M(r) linear in r               */
  int32_t smooth;       /* 1: the output y is replaced by P R y before it is added
                           (its high-frequency part, where the bfloat16 rounding
                           noise sits, is dropped)                                  */
  int32_t pad;
} fsi_pc_desc;
int fsi_pc_create(fsi_mesh* mesh, const fsi_pc_desc* desc, fsi_pc** out);
int fsi_pc_destroy(fsi_pc* pc);
/* n_layers = 15; n_weights; fan[2*l] = out channels, fan[2*l+1] = in channels;
 * grids[3*l..] = node-grid size (x, y, z) of level l.  Outputs are nullable. */
int fsi_pc_layout(const fsi_pc* pc, int32_t* n_layers, int64_t* n_weights, int32_t* fan, int32_t* grids);
/* host float32 weights (n = n_weights); set_weights also resets Adam's state */
int fsi_pc_set_weights(fsi_pc* pc, const float* w_host, int64_t n);
int fsi_pc_get_weights(const fsi_pc* pc, float* w_host, int64_t n);
/* normalisation scales dbar_c, kc_c (host [4], > 0) */
int fsi_pc_set_norm(fsi_pc* pc, const double* dbar_host, const double* kc_host);
int fsi_pc_get_norm(const fsi_pc* pc, double* dbar_host, double* kc_host);
/* y = net(x_in) */
int fsi_pc_forward(fsi_pc* pc, const uint16_t* x_in, float* y);
/* gradient of L = mean over non-Dirichlet rows (c, v) of (y_c - target_c / kc_c)^2
 * w.r.t. the weights (grad: device float32 [n_weights]); loss_host: L */
int fsi_pc_grad(fsi_pc* pc, const uint16_t* x_in, const uint16_t* target, float* grad, double* loss_host);
/* z = M(r) at the state st (staged; D from the float64 NS diagonal with the
 * elastic augmentation); r, z: NS block vectors [4][nn] float64 */
int fsi_pc_apply(fsi_pc* pc, const fsi_state* st, const double* r, double* z);
/* stores the training pair (r, e) (A e = r) at the state st: input channels as in
 * an apply, target t_c = (e - D^{-1} r)_c sqrt(n) / (|r| dbar_c); the first pair
 * fixes dbar_c = mean of D^{-1}_c over non-Dirichlet rows */
int fsi_pc_add_pair(fsi_pc* pc, const fsi_state* st, const double* r, const double* e);
/* adds `count` synthetic training pairs (A z, z) of the NS block at the state st.  z: every
 * component (v, p) a trilinear interpolation of standard normals on a coarse grid of 2, 4,
 * 8, 16 or 32 intervals along the longest axis, or one normal per node (the six scales in
 * turn), 0 on velocity Dirichlet rows, the pressure's mean removed; A: the NS block's
 * Jacobian with the solid-stress linearization (Section 2.4), unpinned where fsi_step
 * shifts the pressure.  The normals come from a counter-based generator keyed by seed
 * (splitmix64 of the counter, Box-Muller).  The pairs enter the store as fsi_pc_add_pair's
 * do (the oldest are overwritten beyond the capacity).  Synchronises the mesh's stream.
 * Errors: FSI_EINVAL (null, count < 0, no pair storage, not the NS block's network, a
 * tetrahedral mesh). */
int fsi_pc_add_smooth_pairs(fsi_pc* pc, const fsi_state* st, int32_t count, uint64_t seed);
int fsi_pc_pairs(const fsi_pc* pc, int32_t* n_pairs);
/* kc_c = RMS of the stored targets' component c (non-Dirichlet rows) */
int fsi_pc_fit_norm(fsi_pc* pc);
/* iters Adam steps (lr; beta1 0.9, beta2 0.999, eps 1e-8), step i on the stored
 * pair p = order_host[i] with the relative loss L_p / mean over valid rows of
 * (target_p / kc)^2 (every pair weighs the same, whatever the scale of its error);
 * loss_host[i] (nullable) = that relative loss before step i */
int fsi_pc_train(fsi_pc* pc, int32_t iters, float lr, const int32_t* order_host, float* loss_host);
/* attaches pc to its mesh for FSI_PC_LEARNED and FSI_HARVEST (NULL detaches) */
int fsi_set_pc(fsi_mesh* mesh, fsi_pc* pc);

/* --------------------------------------------------------------- batched instances
 * (no counterpart in the paper, which treats one problem at a time.)  Many
 * independent meshes of uneven size solved together: one persistent launch applies
 * the block operator of every instance (its CTAs walk a list of (instance, tile)
 * items), and GMRES runs for all instances in lock-step with per-instance Arnoldi
 * state on the device; an instance that reaches its tolerance stops on the device
 * without a host round trip.  One restart cycle of the inner solve is captured as a
 * CUDA graph and replayed when the meshes' stream is not the legacy default stream.
 * Block vectors are concatenated: instance i owns [offsets[i], offsets[i+1]).
 * The meshes must share one device and one stream; they stay owned by the caller and
 * must outlive the batch. */
typedef struct fsi_batch fsi_batch;
/* block: the same block id for every instance (FSI_BLOCK_NS, FSI_BLOCK_AC(i),
 * FSI_BLOCK_B(s)); m: restart length (1..64) of fsi_batch_gmres.  The launch shape
 * comes from the autotuner cache if it holds this set of instances. */
int fsi_batch_create(fsi_mesh* const* meshes, int32_t n, int32_t block, int32_t m, fsi_batch** out);
int fsi_batch_destroy(fsi_batch* batch);
/* offsets: [n+1]; target_mult, grid_mult: the launch shape (tiles ~ target_mult x 152,
 * persistent CTAs = grid_mult x 152); launches: kernels launched by the batch so far
 * (a replayed graph counts its nodes).  Outputs are nullable. */
int fsi_batch_layout(const fsi_batch* batch, int64_t* offsets, int32_t* target_mult, int32_t* grid_mult,
                     int64_t* launches);
/* y = J_i(states[i]) dx for every instance (flags as in fsi_jvp).  NS batches: each
 * instance's quadrature-point coefficients are built at its state (Section 2.4's
 * linearization frozen), then one element launch over all instances' tiles (float32: the
 * coefficients TMA-staged) and one node launch; AC and B batches: one persistent launch of
 * the re-interpolating element operators. */
int fsi_batch_jvp(fsi_batch* batch, const fsi_state* states, const double* dx, double* y, uint32_t flags);
/* fsi_gmres for every instance (FSI_PREC_FP64 or FSI_PREC_FP32_IR; opts.m must be the
 * batch's m).  Preconditioners: Jacobi, none, or FSI_PC_LEARNED for NS batches whose
 * meshes all have a network attached (fsi_set_pc) and share the batch's stream: flexible
 * GMRES keeping each instance's directions, the network applied per instance (with
 * FSI_PC_ALTERNATE at even Arnoldi steps, Jacobi at odd ones), launched directly (no
 * captured cycle).  infos: [n], nullable.  Returns FSI_ENOCONV if some instance misses
 * rtol (its x holds the last iterate); FSI_EINVAL for a network on other blocks. */
int fsi_batch_gmres(fsi_batch* batch, const fsi_state* states, const double* rhs, double* x,
                    const fsi_solve_opts* opts, fsi_solve_info* infos);
/* the project's autotuner: times the batched operator apply over candidate launch
 * shapes (target_mult in {1,2,4,8} x grid_mult in {1,2,4}), keeps the fastest and
 * appends it to the cache file ($FSI_AUTOTUNE_CACHE, else
 * $HOME/.cache/fsi_gb300_autotune.txt) under a key of the instance shapes. */
int fsi_batch_autotune(fsi_batch* batch, const fsi_state* states, uint32_t flags, int32_t* target_mult,
                       int32_t* grid_mult, double* best_us);
/* 0: launch the restart cycles directly instead of through the captured graph */
int fsi_batch_set_graph(fsi_batch* batch, int32_t use_graph);
/* As fsi_batch_create with a block per entry: entry i solves block blocks[i] of
 * meshes[i]; a mesh may appear in several entries (e.g. every phase of it).  Entries
 * need one operator type: all NS, all AC or all B blocks. */
int fsi_batch_create_blocks(fsi_mesh* const* meshes, const int32_t* blocks, int32_t n, int32_t m,
                            fsi_batch** out);

/* Batched partitioned time steps (Section 2.5) of n independent instances (one device,
 * one stream): each nonlinear iteration solves the NS blocks of all live instances in
 * one batched GMRES, the Allen-Cahn blocks of all phases of all instances in one (the
 * phases' equations do not depend on each other), and the B blocks of all solids in
 * one; the pressure of enclosed domains is fixed as in fsi_step.  An instance stops
 * iterating once all its blocks meet nl_tol (unless fixed_iters).  states: n host
 * structs of device pointers, advanced in place; infos: n results.  opts.solve.m is the
 * stepper's restart length; Jacobi or no preconditioner.  Synchronises. */
typedef struct fsi_batch_stepper fsi_batch_stepper;
int fsi_batch_stepper_create(fsi_mesh* const* meshes, int32_t n, int32_t m, fsi_batch_stepper** out);
int fsi_batch_stepper_destroy(fsi_batch_stepper* stepper);
int fsi_batch_step(fsi_batch_stepper* stepper, fsi_state* states, const fsi_step_opts* opts, fsi_step_info* infos);

/* --------------------------------------------------------------- measurement
 * (no counterpart in the paper: timing support for the benchmark)
 * fsi_profile(mesh, 1) starts recording a CUDA event pair around every kernel the
 * mesh launches (counters reset); fsi_profile(mesh, 0) stops.  Launch counts are
 * kept whether or not events are recorded.  fsi_profile_read synchronises the
 * stream and returns, per kernel class, the launches and the summed event time. */
/* Measured ceilings of the current GPU, for rooflines: float32 and float64 FMA rates
 * (TFLOP/s, 8 independent FMA chains per thread on 8 x 256 threads per SM), read-only
 * and copy (read + write) bandwidth over 2 GiB buffers (GB/s), each the best of five
 * launches.  Allocates and frees 4 GiB of device memory; synchronises the device. */
int fsi_probe_peaks(double* fp32_tflops, double* fp64_tflops, double* read_gbs, double* copy_gbs);

#define FSI_PROF_CLASSES 26
typedef struct {
  char name[24];
  int64_t launches;
  double ms;            /* summed device time between the event pair (0 if off) */
  double bytes;         /* summed algorithmic DRAM bytes of the launches (vector
                           kernels: the vectors the algorithm reads and writes
                           once; 0 for classes that do not declare them)          */
} fsi_profile_entry;
int fsi_profile(fsi_mesh* mesh, int32_t enable);
int fsi_profile_read(fsi_mesh* mesh, fsi_profile_entry* out /* [FSI_PROF_CLASSES] */, int32_t* n_out);

/* --------------------------------------------------------------- errors */
const char* fsi_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FSI_H */
