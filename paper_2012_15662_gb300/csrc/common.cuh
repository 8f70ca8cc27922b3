// Internal declarations shared by the engine's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/donof_ri.h"

namespace donof {

// Device-side status codes written into ctx->d_status by kernels.
enum DeviceStatus : int {
  DEV_OK = 0,
  DEV_METRIC_NOT_PD = 1,
  DEV_NONFINITE = 2,
  DEV_TIMEOUT = 3,
};

// Generic strided batched FP64 GEMM: C[b](m,n) = alpha * sum_k A[b](m,k) B[b](k,n) + beta * C[b](m,n)
// with element (m,k) of A at A[b*sAb + m*sAm + k*sAk] (likewise B, C).
struct Gemm64 {
  int M, N, K, batch;
  const double* A;
  long long sAb, sAm, sAk;
  const double* B;
  long long sBb, sBk, sBn;
  double* C;
  long long sCb, sCm, sCn;
  double alpha, beta;
};

// Mixed-precision (split TF32) buffers, allocated only for DONOF_RI_TF32X3.
struct MixedBuffers;
// Digit-plane buffers, allocated only for DONOF_RI_SLICE4.
struct S4Buffers;

}  // namespace donof

struct donof_ri_ctx {
  int nbf, naux, n_atoms, n_strong, n_weak_per, n_omega;
  int precision;
  cudaStream_t stream;
  long long launches;

  // problem statement (device copies)
  double* d_atom_xyz;
  double* d_atom_charge;
  int* d_bf_atom;
  double* d_bf_alpha;
  int* d_aux_atom;
  double* d_aux_alpha;
  int* d_subspace;
  int* d_weak_rank;

  // setup products (FP64)
  double* d_S;      // [nbf][nbf]
  double* d_H;      // [nbf][nbf]
  double* d_G;      // [naux][naux], lower triangle = L after init
  double* d_B;      // [naux][nbf][nbf] fitted tensor (FP64)
  double* d_enuc;   // [1]
  double* d_scratch_max;  // [1]

  // per-iteration FP64 state
  double* d_C;      // [nbf][nbf] column-major orbitals
  double* d_bh;     // [naux][n_omega][nbf]
  double* d_d;      // [naux][n_omega]
  double* d_bf;     // [naux][n_omega][n_omega]
  double* d_J;      // [n_omega][n_omega]
  double* d_K;      // [n_omega][n_omega]
  double* d_Jao;    // [n_omega][nbf][nbf]
  double* d_Kao;    // [n_omega][nbf][nbf]
  double* d_W;      // [n_omega][nbf][nbf]
  double* d_HC;     // [nbf][n_omega]
  double* d_Y;      // [nbf][n_omega]
  double* d_lambda; // [nbf][nbf] column-major
  double* d_gamma;  // [n_strong*n_weak_per]
  double* d_n;      // [n_omega]
  double* d_A;      // [n_omega][n_omega]
  double* d_Bc;     // [n_omega][n_omega]
  double* d_E;      // [1]
  double* d_Hd;     // [n_omega] C_p^T H C_p (occupation optimisation)
  double* d_on;     // [2*N_I*N_g + 1] occupation optimisation: gamma, gradient, energy
  int* d_on_info;   // [2]
  float* d_feat;    // [N_I][3 + 4 N_g] learned-guess features
  double* d_rot;    // [4 nbf^2 + 2] rotation-step scratch (allocated on first use)
  double* d_ctr;    // contracted-Lagrangian scratch (allocated on first use)
  double* d_fl;     // F^lambda step scratch (allocated on first use)
  int* d_status;    // [1] device-side status (DeviceStatus)
  // metric factorisation (DONOF_RI_METRIC_*) and, for the modified one, its
  // tolerance and counts: 2x2 pivots, raised eigenvalues, interchanges
  int metric_mode;
  double metric_tol;
  int metric_info[3];

  donof::MixedBuffers* mixed;
  donof::S4Buffers* s4;

  // profiling: event pairs per hot-path row (see donof_ri_profile)
  int prof_enabled;
  struct ProfRec { int row; cudaEvent_t a, b; }* prof;
  int prof_n, prof_cap;

  // call-order state
  int have_half, have_full, have_ao, have_lambda;

  // Side stream of donof_ri_iteration: the occupation-dependent and orbital-only
  // prologue of the energy row runs there, concurrently with the transforms.
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_join;
  // Second side stream: independent launch groups inside one call (e.g. J_pq
  // beside the full transform), forked and joined within that call.
  cudaStream_t side2;
  cudaEvent_t ev_fork2, ev_join2;

  // CUDA graph of donof_ri_iteration (see the header)
  int capturing;
  cudaGraphExec_t graph_exec;
  const void* graph_key[7];
  int graph_mode;
  long long graph_launches;
};

namespace donof {

// ---- fork / join of a launch group onto ctx->side2 (api.cu) ----
// fork_begin: when a second stream exists and per-row profiling is off, makes
// side2 wait for the work issued so far and points ctx->stream at it (returns
// true).  fork_end: points ctx->stream back and records side2's completion;
// fork_join makes the main stream wait for it.  Row events are recorded on the
// main stream, so nothing is forked while profiling.
bool fork_begin(donof_ri_ctx* ctx, cudaStream_t* main_stream);
void fork_end(donof_ri_ctx* ctx, cudaStream_t main_stream);
int fork_join(donof_ri_ctx* ctx);

// ---- profiling scope (api.cu): records an event pair around a launch group ----
void prof_begin(donof_ri_ctx* ctx, int row, int* slot);
void prof_end(donof_ri_ctx* ctx, int slot);
struct ProfScope {
  donof_ri_ctx* ctx;
  int slot;
  ProfScope(donof_ri_ctx* c, int row) : ctx(c), slot(-1) { prof_begin(c, row, &slot); }
  ~ProfScope() { prof_end(ctx, slot); }
};

// ---- launch helpers (defined in setup64.cu) ----
int launch_dgemm(donof_ri_ctx* ctx, const Gemm64& g);
int setup_integrals(donof_ri_ctx* ctx);
int setup_cholesky_and_fit(donof_ri_ctx* ctx);
int fit_forward(donof_ri_ctx* ctx);
// A = L L^T in place (row-major n x n, lower factor) and R <- L^-1 R (R n x ncol row-major)
int cholesky_lower(donof_ri_ctx* ctx, double* A, int n, double* maxdiag, double rel_min);
int forward_subst(donof_ri_ctx* ctx, const double* L, int n, double* R, long long ncol);
void max_diag_public(donof_ri_ctx* ctx, const double* G, double* out);
// modchol.cu: G = P L D L^T P^T with the Cheng-Higham correction, B from it
int setup_modified_and_fit(donof_ri_ctx* ctx, double tol);

// ---- FP64 hot path (path64.cu) ----
int path64_transform(donof_ri_ctx* ctx, int mode);
int path64_jk_ao(donof_ri_ctx* ctx);
// Parts of the energy row: PREP needs only C, H and gamma (occupations, couplings,
// Fock weights, H C); MAIN needs J^(q), K^(q) as well (F^(p) C_p, lambda, E).
enum EnergyPart { ENERGY_PREP = 1, ENERGY_MAIN = 2, ENERGY_ALL = 3 };
int path64_energy(donof_ri_ctx* ctx, int part);
// contracted Lagrangian (no J^(q), K^(q)); scratch w [N_Omega][naux], X [naux][N_Omega]^2, Yp [naux][nbf][N_Omega]
int path64_energy_contracted(donof_ri_ctx* ctx, double* w, double* X, double* Yp);
int launch_check_finite(donof_ri_ctx* ctx, const double* x, long long n);
int launch_hc_public(donof_ri_ctx* ctx);
int onopt_launch(donof_ri_ctx* ctx, double* d_gamma, double* d_E, double* d_grad, int* d_info, int mode,
                 int max_iter, double gtol, double etol);
int onopt_features(donof_ri_ctx* ctx, float* d_X);
int rotate_orbitals(donof_ri_ctx* ctx, double radius, double* scratch, double* gnorm);
// rotate.cu: ctx->d_C <- d_C expm(kappa), kappa row-major in the first nbf^2 doubles of scratch
int apply_rotation(donof_ri_ctx* ctx, double* scratch);
int s4_autotune(donof_ri_ctx* ctx, int reps, int* report, int* tried);
int s4_set_schedule(donof_ri_ctx* ctx, int kind, int stages, int option);
// exact.cu: exact four-centre J^(q), K^(q), J, K into an FP64 context's buffers
int exact_jk(donof_ri_ctx* ctx);
// flambda.cu: one F^lambda step on ctx->d_C (nbf <= 160); scratch flambda_scratch_doubles(nbf) doubles
constexpr int FLAMBDA_MAX_NBF = 2048;  // largest basis of the F^lambda step
size_t flambda_scratch_doubles(int n);
int flambda_step(donof_ri_ctx* ctx, const double* dprev, int first, double bound, double* scratch, double* gmax,
                 int* sweeps);
int onopt_unfold(donof_ri_ctx* ctx, const float* d_Y, double clip, double* d_gamma);
// flambda.cu: eigenvectors (row-major U, ascending eps) of a symmetric FP64 matrix, n <= FLAMBDA_MAX_NBF
int eigh_sym(donof_ri_ctx* ctx, const double* F, int n, double* scratch, double* U, double* eps, int* sweeps);
int mlp_forward_device(donof_mlp* n, const float* dX, int B, float** dY);
int mlp_shape(const donof_mlp* n, int* F, int* O);
int launch_occupations_coupling(donof_ri_ctx* ctx);
int launch_energy_reduce(donof_ri_ctx* ctx);

// ---- mixed path (tc.cu) ----
int mixed_init(donof_ri_ctx* ctx);
void mixed_free(donof_ri_ctx* ctx);
int mixed_transform(donof_ri_ctx* ctx, int mode);
int mixed_jk_ao(donof_ri_ctx* ctx);
int mixed_energy(donof_ri_ctx* ctx, int part);

// ---- digit-plane path (s4.cu) ----
int s4_init(donof_ri_ctx* ctx);
void s4_free(donof_ri_ctx* ctx);
int s4_transform(donof_ri_ctx* ctx, int mode);
int s4_jk_ao(donof_ri_ctx* ctx);
int s4_energy(donof_ri_ctx* ctx, int part);
int s4_energy_contracted(donof_ri_ctx* ctx);
int s4_fetch(donof_ri_ctx* ctx, int what, double* dst, size_t count);
int s4_copy_ao(donof_ri_ctx* ctx, double* Jao, double* Kao, bool jao_dev, bool kao_dev);

}  // namespace donof

namespace donof {
// ---- programmatic dependent launch (the kernels of the iteration chain) ----
// A kernel launched with launch_pdl may be scheduled while its predecessor in
// the stream is still running.  It calls pdl_entry() before it touches global
// memory: griddepcontrol.wait returns once the predecessor grid has completed
// and its writes are visible, and griddepcontrol.launch_dependents then lets the
// next grid be scheduled, so each launch's latency hides behind the running
// kernel, one grid ahead.  Launched the ordinary way, both return at once.
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
}  // namespace donof

#define DONOF_CUDA_TRY(expr)                         \
  do {                                               \
    cudaError_t _e = (expr);                         \
    if (_e != cudaSuccess) return DONOF_RI_E_CUDA;   \
  } while (0)

#define DONOF_LAUNCH_CHECK(ctx)                      \
  do {                                               \
    (ctx)->launches++;                               \
    cudaError_t _e = cudaGetLastError();             \
    if (_e != cudaSuccess) return DONOF_RI_E_CUDA;   \
  } while (0)

static inline unsigned ceil_div_u(long long a, long long b) { return (unsigned)((a + b - 1) / b); }
