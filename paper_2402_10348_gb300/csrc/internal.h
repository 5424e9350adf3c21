// Internal declarations shared by the translation units of libfsi.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fsi.h"
#include "ops.cuh"

struct fsi_batch;
namespace fsi {
struct TetData;  // tet.cu
}

namespace fsi {
// Kernel classes of the event profiler (fsi_profile).
enum ProfClass {
  P_STAGE, P_NS_RES, P_NS_JVP64, P_NS_JVP32, P_NS_DIAG, P_AC_RES, P_AC_JVP64, P_AC_JVP32,
  P_AC_DIAG, P_B_RES, P_B_JVP64, P_B_JVP32, P_B_DIAG, P_COEF, P_KRYLOV, P_INIT, P_KRY_DOT, P_KRY_UPD,
  P_KRY_SMALL, P_KRY_CONV, P_PC_CONV, P_PC_WGRAD, P_PC_AUX, P_NS_BUILD, P_NS_JVP64E, P_NODE_SUM, P_NCLS
};
struct Profiler {
  bool on = false;
  int64_t launches[P_NCLS] = {};
  double ms[P_NCLS] = {};
  double bytes[P_NCLS] = {};   // algorithmic HBM bytes declared by the launch sites
  std::vector<cudaEvent_t> ev;  // pool of event pairs
  std::vector<int> cls;         // class of each recorded pair
  int used = 0;                 // pairs recorded since the last harvest
};
// Records the operator structs that the launchers would launch, instead of
// launching them (batched launches, batch.cu): one struct per instance, all of one
// type, replayed by `launch` as a single persistent launch over every instance.
struct BatchRec {
  std::vector<unsigned char> bytes;  // concatenated operator structs
  size_t op_size = 0;
  int count = 0;
  int cls = 0;
  size_t smem = 0;                   // largest dynamic shared memory of the records
  int (*launch)(fsi_batch* b, const void* ops_dev, size_t smem, int cls, int use_active) = nullptr;
  void* (*upload)(const BatchRec& r) = nullptr;
};
}  // namespace fsi

struct fsi_mesh {
  int dev = 0;
  cudaStream_t stream = nullptr;
  fsi::Geom g{};
  fsi::Phys P{};
  int N = 0, ns = 0, ncomp = 0;
  int64_t nn = 0;
  std::vector<fsi_phase> phases;
  double lx = 0, ly = 0, lz = 0;
  // boundary data
  uint8_t* mask = nullptr;  // [nn]
  int pin_node = -1;        // node of the pressure pin (mask bit 3), or -1
  int pin_active = 1;       // 0: NS operators keep the pin node's continuity equation
  int enclosed = 0;         // every face has a Dirichlet velocity: constant p is a null mode
  double* vD = nullptr;     // [3][nn]
  // staged state (x^{n+alpha}, dx/dt^{n+alpha_m}, blended materials)
  double* xa = nullptr;     // only when alpha != 1
  double* xd = nullptr;     // [ncomp][nn]
  double* mat = nullptr;    // [2 + ns][nn]: rho, mu, alpha^s
  float* xa32 = nullptr;    // float copies for FSI_FP32
  float* xd32 = nullptr;
  float* mat32 = nullptr;
  float* dx32 = nullptr;     // float copy of a product's increment (FSI_FP32)
  const double* staged_x = nullptr;  // x^{n+1} of the last staging (p and Dirichlet rows)
  int64_t stage_gen = 0;             // staging count: coefficients built at another count are stale
  // quadrature-point coefficients of the NS product (NSBuildOp in ops.cuh, nsq_elem_kernel)
  double* cq64 = nullptr;
  float* cq32 = nullptr;
  int64_t cq_len = 0;                // allocated coefficients (each array)
  int64_t cq_gen = -1;               // stage_gen of the last build
  unsigned cq_flags = 0;             // FSI_ELASTIC_AUG of the last build
  // TMA descriptors of the float32 coefficients (boxes of 44 and of 20 values; nsq_tma.cu),
  // encoded for the allocation at cq_tmap_base; tma_err: a bounded wait gave up
  alignas(64) unsigned char cq_tmap[256] = {};
  const void* cq_tmap_base = nullptr;
  int* tma_err = nullptr;
  // float64 element matrices of the NS product (nse_elem_kernel), built from the coefficients once
  // a state has taken NSE_AFTER float64 products
  double* ke64 = nullptr;
  int64_t ke_len = 0;
  double* ke_e = nullptr;            // [slots][elements] corner contributions of the element-centric products
  int64_t ke_e_len = 0;
  int64_t ke_gen = -1;               // cq_gen they were built from
  int64_t f64_gen = -1, f64_count = 0;  // float64 NS products applied at coefficient build f64_gen
  int64_t cq_builds = 0;             // coefficient builds so far (a new build invalidates ke64)
  // float64 Allen-Cahn element matrices (ace_elem_kernel) of one phase at one staging
  double* ake64 = nullptr;
  int64_t ake_len = 0;
  int64_t ake_gen = -1, ake_count = 0;  // staging the products were counted at / built for
  int ake_phase = -1, ake_built = 0;
  double ake_gamma = 0.0, ake_beta = 0.0;
  // float64 B split operators (be_elem_kernel) of one solid at one staging
  double* bke64 = nullptr;
  int64_t bke_len = 0;
  int64_t bke_gen = -1, bke_count = 0;
  int bke_solid = -1, bke_built = 0;
  const double* staged_xa = nullptr; // the x^{n+alpha} array in use
  // coefficients
  double gamma[fsi::MAXP] = {0};
  double beta[fsi::MAXP] = {0};
  double fixed_gamma[fsi::MAXP];
  double* partials = nullptr;
  int64_t n_partials = 0;
  // reduction scratch
  double* red = nullptr;     // device scratch for vector reductions
  double* red_host = nullptr;// pinned host mirror
  // Krylov workspace
  int64_t kry_n = 0;
  int kry_m = 0;
  double* V = nullptr;       // [m+1][n]
  double* wk = nullptr;      // [4][n] work vectors
  double* dinv = nullptr;    // [n]
  double* yvec = nullptr;    // [m+1] device
  double* partials_dot = nullptr;  // per-CTA partial dot products
  void* kry_dev = nullptr;   // device Arnoldi/Givens state
  double* kry_est = nullptr; // pinned host copies of the residual estimates
  std::vector<cudaEvent_t> kry_ev;
  double* step_ws = nullptr; // [2][max block] time-step work vectors
  int64_t step_ws_n = 0;
  double* Z = nullptr;       // [m][n] FGMRES preconditioned directions
  int64_t Z_n = 0;
  fsi_pc* pc = nullptr;      // attached learned preconditioner (NS block), not owned
  fsi::TetData* tet = nullptr;  // linear tetrahedra (fsi_create_tet_mesh): NS operators by connectivity
  fsi::BatchRec* rec = nullptr;  // non-null: operator launches are recorded, not run
  // counters (step info)
  int64_t applies = 0;
  int64_t dof_applied = 0;
  fsi::Profiler prof;
};

namespace fsi {

int set_error(int code, const std::string& msg);
int cuda_check(cudaError_t e, const char* what);
#define FSI_CUDA(call)                                   \
  do {                                                   \
    cudaError_t _e = (call);                             \
    if (_e != cudaSuccess) return fsi::cuda_check(_e, #call); \
  } while (0)

// staging of x^{n+alpha}, dx/dt^{n+alpha_m} and materials (api.cu)
int stage(fsi_mesh* m, const fsi_state* st, bool fp32);

// block bookkeeping
struct BlockInfo {
  int kind;   // 0 NS, 1 AC, 2 B
  int index;
  int c0;     // first component plane
  int nc;     // component planes
  int64_t n;  // vector length
};
int block_info(const fsi_mesh* m, int32_t block, BlockInfo* bi);

// operator launches on staged state (ops_f64.cu / ops_f32.cu)
int op_residual(fsi_mesh* m, const BlockInfo& b, double* r);
int op_jvp(fsi_mesh* m, const BlockInfo& b, const double* dx, double* y, unsigned flags);
// op_jvp flag, internal only: with FSI_FP32, the float32 increment is already in m->dx32
// (the Krylov solver's preconditioner kernel wrote it) and dx is not read
constexpr unsigned OP_DX32_READY = 0x80000000u;
int ensure_dx32(fsi_mesh* m);  // allocates m->dx32 (6 x nn floats) on first use
int op_diag(fsi_mesh* m, const BlockInfo& b, double* d, unsigned flags);
int op_coeffs(fsi_mesh* m, int phase, double* gamma_beta);  // synchronises
// Final fixed-order sum of the gamma/beta per-CTA partials {sum val^2, n_band, int F',
// int sqrt F} into out[0] = gamma, out[1] = beta (ops_f64.cu; one CTA of NTHREADS).
// Shared by fsi_update_ac_coeffs and fsi_gamma_beta_noalloc.
__global__ void coef_finalize(const double* partials, int64_t n, double eta, double* out);

template <typename T>
int launch_ns(fsi_mesh* m, int mode, const double* dx, double* y, unsigned flags);
// NS product from the quadrature-point coefficients (built first when stale)
int ns_build(fsi_mesh* m, unsigned flags);  // ops_f64.cu
// float32 NS product from the coefficients with TMA-staged coefficient boxes: the element
// contributions into E (nsq_tma.cu)
int launch_nsq_tma(fsi_mesh* m, int elastic, float* E, const double* dx, double* y);
// FSI_ECUDA if a bounded wait of that kernel gave up since the flag was allocated (syncs)
int check_tma(fsi_mesh* m);
// One instance's float32 NS product in a batched launch (nsq_tma.cu): the TMA descriptor of
// its coefficients, its increment (float copy and float64 for the Dirichlet rows), its
// contribution scratch and output, its geometry.  64-byte aligned (the descriptor's rule).
struct alignas(64) NSQBatchRec {
  unsigned char map[128];
  const double* cq64;  // float64 products: the coefficients, read directly
  double* E64;         // float64 products: the contribution scratch
  const float* dx32;
  const double* dx;
  float* E;
  double* y;
  const uint8_t* mask;
  int* err;
  int64_t nxyp, nn;
  double W;
  double al64, cm64, rh64[3];  // the float64 product's constants
  int nx, ny, nz, nxp, pin, elastic;
  float al, cm, rhx, rhy, rhz;
};
// builds the instance's coefficients (if stale), scratch and descriptor and fills rec;
// f64: a float64 product (coefficients read directly, no descriptor)
int nsq_batch_record(fsi_mesh* m, unsigned flags, bool f64, const double* dx, double* y, float* dx32,
                     NSQBatchRec* rec);
// element and node launches of a batch (recs in device memory; items: (instance, x block,
// y block, layer) and (instance, 128-node block)); active gates instances (nullable)
int nsq_batch_launch(bool f64, const NSQBatchRec* recs, const int4* eitems, int neitems, const int4* nitems,
                     int nnitems, const int* active, cudaStream_t s);
constexpr int NSQ_TBX = 64, NSQ_TBY = 2;  // element tile of the TMA product
// [slots][elements] scratch of the element-centric products, grown on demand (ops_f64.cu)
int ensure_elem_scratch(fsi_mesh* m, int slots, int64_t nxyp);
// float64 NS product through element matrices (built first when stale), ops_f64.cu
int launch_nse(fsi_mesh* m, const double* dx, double* y, unsigned flags);
// float64 Allen-Cahn product of one phase through element matrices (ops_f64.cu)
int launch_ace(fsi_mesh* m, int phase, const double* dx, double* y);
// float64 B product of one solid through the split operator (ops_f64.cu)
int launch_be(fsi_mesh* m, int solid, const double* dx, double* y);
constexpr int NSE_AFTER = 8;  // float64 products on one coefficient build before the matrices pay
// Allen-Cahn element matrices: a build costs about three re-interpolating products and
// each matrix product a fifteenth of one; the B split operator's build costs less than one
// re-interpolating product, so it is built at the first product of a solve
constexpr int ACE_AFTER = 2;
constexpr int BE_AFTER = 0;
template <typename T>
int launch_nsq(fsi_mesh* m, const double* dx, double* y, unsigned flags);
template <typename T>
int launch_ac(fsi_mesh* m, int mode, int phase, const double* dx, double* y);
template <typename T>
int launch_b(fsi_mesh* m, int mode, int s, const double* dx, double* y);

// vector helpers (krylov.cu)
int vec_dot(fsi_mesh* m, const double* a, const double* b, int64_t n, double* out_host);  // synchronises
int vec_axpy(fsi_mesh* m, double alpha, const double* x, double* y, int64_t n);          // y += a x
int vec_scale_copy(fsi_mesh* m, double alpha, const double* x, double* y, int64_t n);    // y = a x
int vec_mul(fsi_mesh* m, const double* a, const double* b, double* y, int64_t n);        // y = a*b
int vec_recip(fsi_mesh* m, const double* a, double* y, int64_t n);                      // y = 1/a
int gmres_solve(fsi_mesh* m, const BlockInfo& b, const double* rhs, double* x, const fsi_solve_opts& o,
                fsi_solve_info* info);

// tile launch geometry
void tile_grid(const fsi_mesh* m, dim3* grid);

// linear tetrahedra (tet.cu): residual (mode 0), product (1), diagonal (2) of each block
int tet_ns(fsi_mesh* m, int mode, const double* dx, double* y, unsigned flags);
int tet_ac(fsi_mesh* m, int mode, int phase, const double* dx, double* y, unsigned flags);
int tet_b(fsi_mesh* m, int mode, int solid, const double* dx, double* y, unsigned flags);
int tet_coeffs(fsi_mesh* m, int phase, double* gamma_beta);  // synchronises
void tet_free(TetData* t);

// time-step pieces (step.cu): predictor and corrector launches, the pressure shift of
// enclosed domains after an NS solve that kept the pin node's continuity equation
int step_predict(fsi_mesh* m, fsi_state* st);
int step_correct(fsi_mesh* m, fsi_state* st);
bool shifts_pressure(const fsi_mesh* m, unsigned solve_flags);
int pin_shift(fsi_mesh* m, const double* x, double* dx);
// Sets the pressure pin of a mesh for a scope and restores it on leaving (also on errors).
struct PinGuard {
  fsi_mesh* m;
  int saved;
  PinGuard(fsi_mesh* mm, int active) : m(mm), saved(mm->pin_active) { m->pin_active = active; }
  ~PinGuard() { m->pin_active = saved; }
};

// Raises a kernel's cudaFuncAttributeMaxDynamicSharedMemorySize to at least `bytes` on
// the current device, once per (kernel, device, size); safe from several host threads.
int ensure_smem_attr(const void* func, size_t bytes);

// profiler: bracket every launch with prof_begin / prof_end (api.cu)
int prof_begin(fsi_mesh* m, int cls);
int prof_end(fsi_mesh* m, int cls);
inline void prof_bytes(fsi_mesh* m, int cls, double b) { m->prof.bytes[cls] += b; }
int prof_harvest(fsi_mesh* m);
#define FSI_LAUNCH(m, cls, ...)                      \
  do {                                               \
    int _rc = fsi::prof_begin((m), (cls));           \
    if (_rc) return _rc;                             \
    __VA_ARGS__;                                     \
    FSI_CUDA(cudaGetLastError());                    \
    if ((_rc = fsi::prof_end((m), (cls)))) return _rc; \
  } while (0)

}  // namespace fsi
