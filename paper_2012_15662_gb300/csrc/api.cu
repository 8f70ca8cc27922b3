// C ABI of the engine: argument checks, context lifetime, host/device
// pointer handling, call-order state and status codes.  Every computation is
// dispatched to the FP64 path (path64.cu) or the split-precision tensor-core
// path (tc.cu); nothing here computes.
#include "common.cuh"
#include "tcgen05.cuh"

#include <stdlib.h>
#include <string.h>

namespace donof {
int launch_lambda(donof_ri_ctx* ctx);
int launch_hc_public(donof_ri_ctx* ctx);
int mixed_fetch(donof_ri_ctx* ctx, int what, double* dst_host, size_t count);
int mixed_copy_ao(donof_ri_ctx* ctx, double* Jao, double* Kao, bool jao_dev, bool kao_dev);
}  // namespace donof

using namespace donof;

namespace donof {
void prof_begin(donof_ri_ctx* ctx, int row, int* slot) {
  *slot = -1;
  if (!ctx->prof_enabled || ctx->capturing) return;
  if (ctx->prof_n == ctx->prof_cap) {
    int cap = ctx->prof_cap ? 2 * ctx->prof_cap : 256;
    void* p = realloc(ctx->prof, sizeof(*ctx->prof) * cap);
    if (!p) return;
    ctx->prof = (donof_ri_ctx::ProfRec*)p;
    for (int i = ctx->prof_cap; i < cap; ++i) {
      ctx->prof[i].a = ctx->prof[i].b = nullptr;
    }
    ctx->prof_cap = cap;
  }
  donof_ri_ctx::ProfRec& r = ctx->prof[ctx->prof_n];
  if (!r.a && cudaEventCreate(&r.a) != cudaSuccess) { cudaGetLastError(); r.a = nullptr; return; }
  if (!r.b && cudaEventCreate(&r.b) != cudaSuccess) { cudaGetLastError(); r.b = nullptr; return; }
  r.row = row;
  cudaEventRecord(r.a, ctx->stream);
  *slot = ctx->prof_n++;
}

void prof_end(donof_ri_ctx* ctx, int slot) {
  if (slot < 0) return;
  cudaEventRecord(ctx->prof[slot].b, ctx->stream);
}

bool fork_begin(donof_ri_ctx* ctx, cudaStream_t* main_stream) {
  *main_stream = ctx->stream;
  if (!ctx->side2 || ctx->prof_enabled) return false;
  if (cudaEventRecord(ctx->ev_fork2, ctx->stream) != cudaSuccess ||
      cudaStreamWaitEvent(ctx->side2, ctx->ev_fork2, 0) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  ctx->stream = ctx->side2;
  return true;
}

void fork_end(donof_ri_ctx* ctx, cudaStream_t main_stream) {
  ctx->stream = main_stream;
  cudaEventRecord(ctx->ev_join2, ctx->side2);
}

int fork_join(donof_ri_ctx* ctx) {
  DONOF_CUDA_TRY(cudaStreamWaitEvent(ctx->stream, ctx->ev_join2, 0));
  return DONOF_RI_OK;
}
}  // namespace donof

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
static int dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc((void**)p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return DONOF_RI_E_OOM;
  }
  return DONOF_RI_OK;
}

static void dfree(void* p) {
  if (p) cudaFree(p);
}

// Page-locked host memory (cudaHostAlloc / cudaHostRegister): copies from and to
// it can be captured into a CUDA graph.
static bool is_pinned_host_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

// Read and clear the device-side status word; maps it to an ABI status.  While a
// graph is being captured nothing can be waited for: the caller of the graph
// launch reads the status afterwards.
static int consume_status(donof_ri_ctx* ctx) {
  if (ctx->capturing) return DONOF_RI_OK;
  int h = 0;
  if (cudaMemcpyAsync(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
    return DONOF_RI_E_CUDA;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return DONOF_RI_E_CUDA;
  if (h == DEV_OK) return DONOF_RI_OK;
  if (cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream) != cudaSuccess) return DONOF_RI_E_CUDA;
  if (h == DEV_METRIC_NOT_PD) return DONOF_RI_E_METRIC_NOT_PD;
  if (h == DEV_NONFINITE) return DONOF_RI_E_NONFINITE;
  if (h == DEV_TIMEOUT) return DONOF_RI_E_TIMEOUT;
  return DONOF_RI_E_CUDA;
}

static int validate_system(const donof_ri_system* s) {
  if (!s) return DONOF_RI_E_ARG;
  if (s->nbf < 1 || s->naux < 1 || s->n_atoms < 1 || s->n_strong < 1 || s->n_weak_per < 1) return DONOF_RI_E_ARG;
  if (!s->atom_xyz || !s->atom_charge || !s->bf_atom || !s->bf_alpha || !s->aux_atom || !s->aux_alpha ||
      !s->subspace || !s->weak_rank)
    return DONOF_RI_E_ARG;
  long long m = (long long)s->n_strong * (1 + s->n_weak_per);
  if (m > s->nbf) return DONOF_RI_E_ARG;
  if ((long long)s->nbf * s->nbf > (1LL << 30) || s->naux > 65535) return DONOF_RI_E_ARG;
  for (int i = 0; i < s->nbf; ++i)
    if (s->bf_atom[i] < 0 || s->bf_atom[i] >= s->n_atoms || !(s->bf_alpha[i] > 0.0)) return DONOF_RI_E_ARG;
  for (int i = 0; i < s->naux; ++i)
    if (s->aux_atom[i] < 0 || s->aux_atom[i] >= s->n_atoms || !(s->aux_alpha[i] > 0.0)) return DONOF_RI_E_ARG;
  // Pairing map: every subspace has one strong orbital and weak ranks 0..N_g-1 once each.
  int* seen = (int*)calloc((size_t)s->n_strong * (s->n_weak_per + 1), sizeof(int));
  if (!seen) return DONOF_RI_E_ARG;
  int rc = DONOF_RI_OK;
  for (long long p = 0; p < m && rc == DONOF_RI_OK; ++p) {
    int g = s->subspace[p], r = s->weak_rank[p];
    if (g < 0 || g >= s->n_strong || r < -1 || r >= s->n_weak_per) rc = DONOF_RI_E_ARG;
    else if (seen[(size_t)g * (s->n_weak_per + 1) + (r + 1)]++) rc = DONOF_RI_E_ARG;
  }
  free(seen);
  return rc;
}

extern "C" {

const char* donof_ri_strerror(int status) {
  switch (status) {
    case DONOF_RI_OK: return "ok";
    case DONOF_RI_E_ARG: return "invalid argument";
    case DONOF_RI_E_OOM: return "device allocation failed";
    case DONOF_RI_E_CUDA: return "CUDA runtime or launch error";
    case DONOF_RI_E_METRIC_NOT_PD: return "Coulomb metric is not numerically positive definite";
    case DONOF_RI_E_NONFINITE: return "non-finite value in an input";
    case DONOF_RI_E_TIMEOUT: return "a bounded device-side wait timed out";
    case DONOF_RI_E_STATE: return "call order: a required earlier call has not run";
    case DONOF_RI_E_UNSUPPORTED: return "unsupported device or precision";
    default: return "unknown status";
  }
}

long long donof_ri_launch_count(const donof_ri_ctx* ctx) { return ctx ? ctx->launches : -1; }

namespace donof {
// One thread waits, through the engine's bounded mbarrier wait, for phase 0 of a
// barrier that nothing arrives on: the wait runs out after limit_ns and records
// DEV_TIMEOUT in the context's status word, exactly as a timed-out wait inside a
// GEMM kernel does.  No copy or MMA is in flight, so the CTA exits cleanly.
__global__ void wait_timeout_check_kernel(unsigned long long limit_ns, int* status) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait_for(&bar, 0, &abort_flag, status, limit_ns);
}
}  // namespace donof

int donof_ri_check_wait_timeout(donof_ri_ctx* ctx, long long limit_ns) {
  if (!ctx || limit_ns < 1000 || limit_ns > 5000000000LL) return DONOF_RI_E_ARG;
  donof::wait_timeout_check_kernel<<<1, 32, 0, ctx->stream>>>((unsigned long long)limit_ns, ctx->d_status);
  DONOF_LAUNCH_CHECK(ctx);
  return DONOF_RI_OK;
}

int donof_ri_destroy(donof_ri_ctx* ctx) {
  if (!ctx) return DONOF_RI_OK;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->mixed) mixed_free(ctx);
  if (ctx->s4) s4_free(ctx);
  for (int i = 0; i < ctx->prof_cap; ++i) {
    if (ctx->prof[i].a) cudaEventDestroy(ctx->prof[i].a);
    if (ctx->prof[i].b) cudaEventDestroy(ctx->prof[i].b);
  }
  free(ctx->prof);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->ev_fork2) cudaEventDestroy(ctx->ev_fork2);
  if (ctx->ev_join2) cudaEventDestroy(ctx->ev_join2);
  if (ctx->side2) cudaStreamDestroy(ctx->side2);
  void* bufs[] = {ctx->d_atom_xyz, ctx->d_atom_charge, ctx->d_bf_atom, ctx->d_bf_alpha, ctx->d_aux_atom,
                  ctx->d_aux_alpha, ctx->d_subspace, ctx->d_weak_rank, ctx->d_S, ctx->d_H, ctx->d_G, ctx->d_B,
                  ctx->d_enuc, ctx->d_scratch_max, ctx->d_C, ctx->d_bh, ctx->d_d, ctx->d_bf, ctx->d_J, ctx->d_K,
                  ctx->d_Jao, ctx->d_Kao, ctx->d_W, ctx->d_HC, ctx->d_Y, ctx->d_lambda, ctx->d_gamma, ctx->d_n,
                  ctx->d_A, ctx->d_Bc, ctx->d_E, ctx->d_Hd, ctx->d_on, ctx->d_on_info, ctx->d_feat, ctx->d_rot, ctx->d_ctr, ctx->d_fl,
                  ctx->d_status};
  for (void* b : bufs) dfree(b);
  free(ctx);
  return DONOF_RI_OK;
}

int donof_ri_init(const donof_ri_system* sys, int precision, void* stream, donof_ri_ctx** out) {
  return donof_ri_init_ex(sys, precision, stream, nullptr, out);
}

int donof_ri_metric_info(const donof_ri_ctx* ctx, int* n_pivots_2x2, int* n_raised, int* n_interchanges) {
  if (!ctx) return DONOF_RI_E_ARG;
  if (n_pivots_2x2) *n_pivots_2x2 = ctx->metric_info[0];
  if (n_raised) *n_raised = ctx->metric_info[1];
  if (n_interchanges) *n_interchanges = ctx->metric_info[2];
  return DONOF_RI_OK;
}

int donof_ri_init_ex(const donof_ri_system* sys, int precision, void* stream, const donof_ri_options* opt,
                     donof_ri_ctx** out) {
  if (!out) return DONOF_RI_E_ARG;
  *out = nullptr;
  int rc = validate_system(sys);
  if (rc) return rc;
  const int metric = opt ? opt->metric : DONOF_RI_METRIC_CHOLESKY;
  const double metric_tol = opt ? opt->metric_tol : 0.0;
  if (metric != DONOF_RI_METRIC_CHOLESKY && metric != DONOF_RI_METRIC_MODIFIED) return DONOF_RI_E_ARG;
  if (metric == DONOF_RI_METRIC_MODIFIED && !(metric_tol > 0.0 && metric_tol < 1.0)) return DONOF_RI_E_ARG;
  if (precision != DONOF_RI_FP64 && precision != DONOF_RI_TF32X3 && precision != DONOF_RI_SLICE4) return DONOF_RI_E_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return DONOF_RI_E_UNSUPPORTED; }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return DONOF_RI_E_CUDA;
  if (prop.major != 10 || prop.minor != 3) return DONOF_RI_E_UNSUPPORTED;

  donof_ri_ctx* ctx = (donof_ri_ctx*)calloc(1, sizeof(donof_ri_ctx));
  if (!ctx) return DONOF_RI_E_OOM;
  ctx->nbf = sys->nbf;
  ctx->naux = sys->naux;
  ctx->n_atoms = sys->n_atoms;
  ctx->n_strong = sys->n_strong;
  ctx->n_weak_per = sys->n_weak_per;
  ctx->n_omega = sys->n_strong * (1 + sys->n_weak_per);
  ctx->precision = precision;
  ctx->stream = (cudaStream_t)stream;
  ctx->metric_mode = metric;
  ctx->metric_tol = metric_tol;
  const size_t nb = ctx->nbf, nx = ctx->naux, m = ctx->n_omega, na = ctx->n_atoms;
  const size_t nb2 = nb * nb;

#define TRY(x) do { rc = (x); if (rc) { donof_ri_destroy(ctx); return rc; } } while (0)
  TRY(dalloc(&ctx->d_atom_xyz, 3 * na));
  TRY(dalloc(&ctx->d_atom_charge, na));
  TRY(dalloc(&ctx->d_bf_atom, nb));
  TRY(dalloc(&ctx->d_bf_alpha, nb));
  TRY(dalloc(&ctx->d_aux_atom, nx));
  TRY(dalloc(&ctx->d_aux_alpha, nx));
  TRY(dalloc(&ctx->d_subspace, m));
  TRY(dalloc(&ctx->d_weak_rank, m));
  TRY(dalloc(&ctx->d_S, nb2));
  TRY(dalloc(&ctx->d_H, nb2));
  TRY(dalloc(&ctx->d_G, nx * nx));
  TRY(dalloc(&ctx->d_B, nx * nb2));
  TRY(dalloc(&ctx->d_enuc, 1));
  TRY(dalloc(&ctx->d_scratch_max, 1));
  TRY(dalloc(&ctx->d_C, nb2));
  TRY(dalloc(&ctx->d_J, m * m));
  TRY(dalloc(&ctx->d_K, m * m));
  TRY(dalloc(&ctx->d_HC, nb * m));
  TRY(dalloc(&ctx->d_Y, nb * m));
  TRY(dalloc(&ctx->d_lambda, nb2));
  TRY(dalloc(&ctx->d_gamma, (size_t)sys->n_strong * sys->n_weak_per));
  TRY(dalloc(&ctx->d_Hd, m));
  TRY(dalloc(&ctx->d_on, 2 * (size_t)sys->n_strong * sys->n_weak_per + 1));
  TRY(dalloc(&ctx->d_on_info, 2));
  TRY(dalloc(&ctx->d_feat, (size_t)sys->n_strong * (3 + 4 * (size_t)sys->n_weak_per)));
  TRY(dalloc(&ctx->d_n, m));
  TRY(dalloc(&ctx->d_A, m * m));
  TRY(dalloc(&ctx->d_Bc, m * m));
  TRY(dalloc(&ctx->d_E, 1));
  TRY(dalloc(&ctx->d_status, 1));
  if (precision == DONOF_RI_FP64) {
    TRY(dalloc(&ctx->d_bh, nx * m * nb));
    TRY(dalloc(&ctx->d_d, nx * m));
    TRY(dalloc(&ctx->d_bf, nx * m * m));
    TRY(dalloc(&ctx->d_Jao, m * nb2));
    TRY(dalloc(&ctx->d_Kao, m * nb2));
    TRY(dalloc(&ctx->d_W, m * nb2));
  }
  cudaStream_t s = ctx->stream;
#define CPY(dst, src, n) \
  do { if (cudaMemcpyAsync(dst, src, (n) * sizeof(*(src)), cudaMemcpyHostToDevice, s) != cudaSuccess) TRY(DONOF_RI_E_CUDA); } while (0)
  CPY(ctx->d_atom_xyz, sys->atom_xyz, 3 * na);
  CPY(ctx->d_atom_charge, sys->atom_charge, na);
  CPY(ctx->d_bf_atom, sys->bf_atom, nb);
  CPY(ctx->d_bf_alpha, sys->bf_alpha, nb);
  CPY(ctx->d_aux_atom, sys->aux_atom, nx);
  CPY(ctx->d_aux_alpha, sys->aux_alpha, nx);
  CPY(ctx->d_subspace, sys->subspace, m);
  CPY(ctx->d_weak_rank, sys->weak_rank, m);
#undef CPY
  if (cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s) != cudaSuccess) TRY(DONOF_RI_E_CUDA);
  if (cudaMemsetAsync(ctx->d_lambda, 0, nb2 * sizeof(double), s) != cudaSuccess) TRY(DONOF_RI_E_CUDA);
  TRY(setup_integrals(ctx));
  TRY(metric == DONOF_RI_METRIC_MODIFIED ? setup_modified_and_fit(ctx, metric_tol) : setup_cholesky_and_fit(ctx));
  TRY(consume_status(ctx));
  if (precision == DONOF_RI_TF32X3) TRY(mixed_init(ctx));
  if (precision == DONOF_RI_SLICE4) TRY(s4_init(ctx));
  if (cudaStreamSynchronize(s) != cudaSuccess) TRY(DONOF_RI_E_CUDA);
  TRY(consume_status(ctx));  // the overlap's factorisation of the SLICE4 working basis
  if (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->side2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_fork2, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join2, cudaEventDisableTiming) != cudaSuccess)
    TRY(DONOF_RI_E_CUDA);
#undef TRY
  *out = ctx;
  return DONOF_RI_OK;
}

int donof_ri_profile(donof_ri_ctx* ctx, int enable) {
  if (!ctx) return DONOF_RI_E_ARG;
  ctx->prof_enabled = enable ? 1 : 0;
  if (!enable) ctx->prof_n = 0;
  return DONOF_RI_OK;
}

int donof_ri_profile_read(donof_ri_ctx* ctx, int row, double* total_ms, long long* count) {
  if (!ctx || row < 0 || row >= DONOF_RI_NUM_ROWS || !total_ms || !count) return DONOF_RI_E_ARG;
  DONOF_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  double t = 0.0;
  long long c = 0;
  int keep = 0;
  for (int i = 0; i < ctx->prof_n; ++i) {
    donof_ri_ctx::ProfRec r = ctx->prof[i];
    if (r.row == row) {
      float ms = 0.f;
      DONOF_CUDA_TRY(cudaEventElapsedTime(&ms, r.a, r.b));
      t += ms;
      ++c;
    } else {
      ctx->prof[i] = ctx->prof[keep];
      ctx->prof[keep++] = r;
    }
  }
  ctx->prof_n = keep;
  *total_ms = t;
  *count = c;
  return DONOF_RI_OK;
}

int donof_ri_sync(donof_ri_ctx* ctx) {
  if (!ctx) return DONOF_RI_E_ARG;
  return consume_status(ctx);
}

// Copy the orbitals in and check them (first part of donof_ri_transform).
static int transform_input(donof_ri_ctx* ctx, const double* C) {
  const size_t nb2 = (size_t)ctx->nbf * ctx->nbf;
  cudaMemcpyKind kind = is_device_ptr(C) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  ProfScope ps(ctx, DONOF_RI_ROW_OTHER);
  DONOF_CUDA_TRY(cudaMemcpyAsync(ctx->d_C, C, nb2 * sizeof(double), kind, ctx->stream));
  return launch_check_finite(ctx, ctx->d_C, (long long)nb2);
}

static int transform_compute(donof_ri_ctx* ctx, int mode) {
  ctx->have_half = ctx->have_full = ctx->have_ao = ctx->have_lambda = 0;
  int rc = ctx->precision == DONOF_RI_FP64     ? path64_transform(ctx, mode)
           : ctx->precision == DONOF_RI_TF32X3 ? mixed_transform(ctx, mode)
                                               : s4_transform(ctx, mode);
  if (rc) return rc;
  ctx->have_half = 1;
  ctx->have_full = (mode == DONOF_RI_FULL);
  return DONOF_RI_OK;
}

int donof_ri_transform(donof_ri_ctx* ctx, const double* C, int mode) {
  if (!ctx || !C || (mode != DONOF_RI_HALF && mode != DONOF_RI_FULL)) return DONOF_RI_E_ARG;
  int rc = transform_input(ctx, C);
  if (rc) return rc;
  return transform_compute(ctx, mode);
}

static int copy_out(donof_ri_ctx* ctx, double* dst, const double* src, size_t count, bool* host_written) {
  if (!dst) return DONOF_RI_OK;
  bool dev = is_device_ptr(dst);
  DONOF_CUDA_TRY(cudaMemcpyAsync(dst, src, count * sizeof(double),
                                 dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
  if (!dev) *host_written = true;
  return DONOF_RI_OK;
}

int donof_ri_jk_mo(donof_ri_ctx* ctx, double* J, double* K) {
  if (!ctx) return DONOF_RI_E_ARG;
  if (!ctx->have_full) return DONOF_RI_E_STATE;
  const size_t m2 = (size_t)ctx->n_omega * ctx->n_omega;
  bool host = false;
  int rc = copy_out(ctx, J, ctx->d_J, m2, &host);
  if (rc) return rc;
  rc = copy_out(ctx, K, ctx->d_K, m2, &host);
  if (rc) return rc;
  return host ? consume_status(ctx) : DONOF_RI_OK;
}

int donof_ri_jk_ao_batch(donof_ri_ctx* ctx, double* Jao, double* Kao) {
  if (!ctx) return DONOF_RI_E_ARG;
  if (!ctx->have_half) return DONOF_RI_E_STATE;
  int rc = ctx->precision == DONOF_RI_FP64     ? path64_jk_ao(ctx)
           : ctx->precision == DONOF_RI_TF32X3 ? mixed_jk_ao(ctx)
                                               : s4_jk_ao(ctx);
  if (rc) return rc;
  ctx->have_ao = 1;
  if (!Jao && !Kao) return DONOF_RI_OK;
  const size_t n = (size_t)ctx->n_omega * ctx->nbf * ctx->nbf;
  bool host = false;
  if (ctx->precision == DONOF_RI_FP64) {
    if ((rc = copy_out(ctx, Jao, ctx->d_Jao, n, &host))) return rc;
    if ((rc = copy_out(ctx, Kao, ctx->d_Kao, n, &host))) return rc;
  } else {
    bool jd = is_device_ptr(Jao), kd = is_device_ptr(Kao);
    rc = ctx->precision == DONOF_RI_TF32X3 ? mixed_copy_ao(ctx, Jao, Kao, jd, kd) : s4_copy_ao(ctx, Jao, Kao, jd, kd);
    if (rc) return rc;
    host = (Jao && !jd) || (Kao && !kd);
  }
  return host ? consume_status(ctx) : DONOF_RI_OK;
}

// Copy the angles in and check them.
static int gamma_input(donof_ri_ctx* ctx, const double* gamma) {
  const size_t ng = (size_t)ctx->n_strong * ctx->n_weak_per;
  cudaMemcpyKind kind = is_device_ptr(gamma) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  ProfScope ps(ctx, DONOF_RI_ROW_OTHER);
  DONOF_CUDA_TRY(cudaMemcpyAsync(ctx->d_gamma, gamma, ng * sizeof(double), kind, ctx->stream));
  return launch_check_finite(ctx, ctx->d_gamma, (long long)ng);
}

static int energy_part(donof_ri_ctx* ctx, int part) {
  return ctx->precision == DONOF_RI_FP64     ? path64_energy(ctx, part)
         : ctx->precision == DONOF_RI_TF32X3 ? mixed_energy(ctx, part)
                                             : s4_energy(ctx, part);
}

static int energy_outputs(donof_ri_ctx* ctx, double* E, double* lambda) {
  ctx->have_lambda = 1;
  bool host = false;
  int rc;
  if ((rc = copy_out(ctx, E, ctx->d_E, 1, &host))) return rc;
  if ((rc = copy_out(ctx, lambda, ctx->d_lambda, (size_t)ctx->nbf * ctx->nbf, &host))) return rc;
  return host ? consume_status(ctx) : DONOF_RI_OK;
}

int donof_ri_energy_lagrangian(donof_ri_ctx* ctx, const double* gamma, double* E, double* lambda) {
  if (!ctx || !gamma) return DONOF_RI_E_ARG;
  if (!ctx->have_ao) return DONOF_RI_E_STATE;
  int rc = gamma_input(ctx, gamma);
  if (rc) return rc;
  if ((rc = energy_part(ctx, ENERGY_ALL))) return rc;
  return energy_outputs(ctx, E, lambda);
}

int donof_ri_autotune(donof_ri_ctx* ctx, int reps, int* report, int* tried) {
  if (!ctx || reps < 1 || reps > 1000) return DONOF_RI_E_ARG;
  if (ctx->precision != DONOF_RI_SLICE4) return DONOF_RI_E_UNSUPPORTED;
  if (!ctx->have_full || !ctx->have_ao) return DONOF_RI_E_STATE;
  int n = 0;
  int rc = s4_autotune(ctx, reps, report, &n);
  if (tried) *tried = n;
  // the kernels ran alone and the captured graph holds the old launch parameters
  ctx->have_half = ctx->have_full = ctx->have_ao = ctx->have_lambda = 0;
  if (ctx->graph_exec) {
    cudaGraphExecDestroy(ctx->graph_exec);
    ctx->graph_exec = nullptr;
  }
  if (rc) return rc;
  return consume_status(ctx);
}

int donof_ri_energy_lagrangian_contracted(donof_ri_ctx* ctx, const double* gamma, double* E, double* lambda) {
  if (!ctx || !gamma) return DONOF_RI_E_ARG;
  if (ctx->precision == DONOF_RI_SLICE4) {
    if (!ctx->have_half) return DONOF_RI_E_STATE;
    int rc = gamma_input(ctx, gamma);
    if (rc) return rc;
    if ((rc = s4_energy_contracted(ctx))) return rc;
    return energy_outputs(ctx, E, lambda);
  }
  if (ctx->precision != DONOF_RI_FP64) return DONOF_RI_E_UNSUPPORTED;
  if (!ctx->have_full) return DONOF_RI_E_STATE;
  const size_t nb = ctx->nbf, nx = ctx->naux, m = ctx->n_omega;
  int rc;
  if (!ctx->d_ctr && (rc = dalloc(&ctx->d_ctr, m * nx + nx * m * m + nx * nb * m))) return rc;
  if ((rc = gamma_input(ctx, gamma))) return rc;
  double* w = ctx->d_ctr;
  double* X = w + m * nx;
  double* Yp = X + nx * m * m;
  if ((rc = path64_energy_contracted(ctx, w, X, Yp))) return rc;
  return energy_outputs(ctx, E, lambda);
}

int donof_ri_exact_jk(donof_ri_ctx* ctx, const double* C, double* J, double* K) {
  if (!ctx || !C) return DONOF_RI_E_ARG;
  if (ctx->precision != DONOF_RI_FP64 || ctx->nbf > 256) return DONOF_RI_E_UNSUPPORTED;
  int rc = transform_input(ctx, C);
  if (rc) return rc;
  ctx->have_half = ctx->have_full = ctx->have_ao = ctx->have_lambda = 0;
  {
    ProfScope ps(ctx, DONOF_RI_ROW_OTHER);
    if ((rc = exact_jk(ctx))) return rc;
  }
  ctx->have_half = ctx->have_full = ctx->have_ao = 1;
  const size_t m2 = (size_t)ctx->n_omega * ctx->n_omega;
  bool host = false;
  if ((rc = copy_out(ctx, J, ctx->d_J, m2, &host))) return rc;
  if ((rc = copy_out(ctx, K, ctx->d_K, m2, &host))) return rc;
  return consume_status(ctx);
}

int donof_ri_set_schedule(donof_ri_ctx* ctx, int kind, int stages, int option) {
  if (!ctx) return DONOF_RI_E_ARG;
  if (ctx->precision != DONOF_RI_SLICE4) return DONOF_RI_E_UNSUPPORTED;
  int rc = s4_set_schedule(ctx, kind, stages, option);
  if (rc) return rc;
  // the captured graph holds the old launch parameters
  if (ctx->graph_exec) {
    cudaGraphExecDestroy(ctx->graph_exec);
    ctx->graph_exec = nullptr;
  }
  return DONOF_RI_OK;
}

int donof_ri_rotate_orbitals(donof_ri_ctx* ctx, double radius, double* C, double* gmax) {
  if (!ctx || !(radius >= 0.0) || !(radius <= 3.2)) return DONOF_RI_E_ARG;
  if (!ctx->have_lambda) return DONOF_RI_E_STATE;
  const size_t nb2 = (size_t)ctx->nbf * ctx->nbf;
  int rc;
  if (!ctx->d_rot && (rc = dalloc(&ctx->d_rot, 4 * nb2 + 2))) return rc;
  double g = 0.0;
  {
    ProfScope ps(ctx, DONOF_RI_ROW_OTHER);
    if ((rc = rotate_orbitals(ctx, radius, ctx->d_rot, &g))) return rc;
  }
  if (radius > 0.0 && g > 0.0) ctx->have_half = ctx->have_full = ctx->have_ao = ctx->have_lambda = 0;
  if (gmax) *gmax = g;
  bool host = false;
  if ((rc = copy_out(ctx, C, ctx->d_C, nb2, &host))) return rc;
  return host ? consume_status(ctx) : DONOF_RI_OK;
}

int donof_ri_apply_rotation(donof_ri_ctx* ctx, const double* kappa, double* C) {
  if (!ctx || !kappa) return DONOF_RI_E_ARG;
  const size_t nb2 = (size_t)ctx->nbf * ctx->nbf;
  int rc;
  if (!ctx->d_rot && (rc = dalloc(&ctx->d_rot, 4 * nb2 + 2))) return rc;
  {
    ProfScope ps(ctx, DONOF_RI_ROW_OTHER);
    DONOF_CUDA_TRY(cudaMemcpyAsync(ctx->d_rot, kappa, nb2 * sizeof(double),
                                   is_device_ptr(kappa) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                   ctx->stream));
    if ((rc = apply_rotation(ctx, ctx->d_rot))) return rc;
  }
  ctx->have_half = ctx->have_full = ctx->have_ao = ctx->have_lambda = 0;
  bool host = false;
  if ((rc = copy_out(ctx, C, ctx->d_C, nb2, &host))) return rc;
  return host ? consume_status(ctx) : DONOF_RI_OK;
}

// One iteration with the energy row's prologue (occupations, couplings, Fock
// weights and H C, which need only C and gamma) forked onto the side stream, so
// that it runs concurrently with the transforms; joined before F^(p) C_p.  The
// buffers it writes are read by no kernel of the transforms.  Not used while
// per-row profiling is on (the row events are recorded on the main stream).
int donof_ri_flambda_step(donof_ri_ctx* ctx, double* diag, int first, double bound, double* C, double* gmax,
                          int* sweeps) {
  if (!ctx || !(bound > 0.0) || (!first && !diag)) return DONOF_RI_E_ARG;
  if (!ctx->have_lambda) return DONOF_RI_E_STATE;
  if (ctx->nbf > FLAMBDA_MAX_NBF) return DONOF_RI_E_UNSUPPORTED;
  const size_t nb = ctx->nbf, nb2 = nb * nb;
  int rc;
  const size_t fls = flambda_scratch_doubles(ctx->nbf);
  if (!ctx->d_fl && (rc = dalloc(&ctx->d_fl, fls + nb))) return rc;
  double* dprev = ctx->d_fl + fls;  // previous eigenvalues (device copy)
  if (!first) {
    DONOF_CUDA_TRY(cudaMemcpyAsync(dprev, diag, nb * sizeof(double),
                                   is_device_ptr(diag) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                   ctx->stream));
    if ((rc = launch_check_finite(ctx, dprev, (long long)nb))) return rc;
  }
  double g = 0.0;
  int sw = 0;
  {
    ProfScope ps(ctx, DONOF_RI_ROW_OTHER);
    if ((rc = flambda_step(ctx, dprev, first ? 1 : 0, bound, ctx->d_fl, &g, &sw))) return rc;
  }
  ctx->have_half = ctx->have_full = ctx->have_ao = ctx->have_lambda = 0;
  if (gmax) *gmax = g;
  if (sweeps) *sweeps = sw;
  bool host = false;
  const double* eps = ctx->d_fl + 6 * nb2;
  if (diag && (rc = copy_out(ctx, diag, eps, nb, &host))) return rc;
  if ((rc = copy_out(ctx, C, ctx->d_C, nb2, &host))) return rc;
  return consume_status(ctx);
}

static int iteration_forked(donof_ri_ctx* ctx, const double* C, const double* gamma, int mode, double* J, double* K,
                            double* E, double* lambda) {
  int rc = transform_input(ctx, C);
  if (rc) return rc;
  cudaStream_t main_stream = ctx->stream;
  DONOF_CUDA_TRY(cudaEventRecord(ctx->ev_fork, main_stream));
  DONOF_CUDA_TRY(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
  ctx->stream = ctx->side;
  rc = gamma_input(ctx, gamma);
  if (!rc) rc = energy_part(ctx, ENERGY_PREP);
  ctx->stream = main_stream;
  // joined even after an error so that a stream capture stays well formed
  DONOF_CUDA_TRY(cudaEventRecord(ctx->ev_join, ctx->side));
  if (!rc) rc = transform_compute(ctx, mode);
  if (!rc && mode == DONOF_RI_FULL && (J || K)) rc = donof_ri_jk_mo(ctx, J, K);
  if (!rc) rc = donof_ri_jk_ao_batch(ctx, nullptr, nullptr);
  DONOF_CUDA_TRY(cudaStreamWaitEvent(main_stream, ctx->ev_join, 0));
  if (rc) return rc;
  if ((rc = energy_part(ctx, ENERGY_MAIN))) return rc;
  return energy_outputs(ctx, E, lambda);
}

static int iteration_eager(donof_ri_ctx* ctx, const double* C, const double* gamma, int mode, double* J, double* K,
                           double* E, double* lambda) {
  if (ctx->side && !ctx->prof_enabled) return iteration_forked(ctx, C, gamma, mode, J, K, E, lambda);
  int rc = donof_ri_transform(ctx, C, mode);
  if (rc) return rc;
  if (mode == DONOF_RI_FULL && (J || K)) {
    if ((rc = donof_ri_jk_mo(ctx, J, K))) return rc;
  }
  if ((rc = donof_ri_jk_ao_batch(ctx, nullptr, nullptr))) return rc;
  return donof_ri_energy_lagrangian(ctx, gamma, E, lambda);
}

int donof_ri_iteration(donof_ri_ctx* ctx, const double* C, const double* gamma, int mode, double* J, double* K,
                       double* E, double* lambda, int use_graph) {
  if (!ctx || !C || !gamma || (mode != DONOF_RI_HALF && mode != DONOF_RI_FULL)) return DONOF_RI_E_ARG;
  const void* key[7] = {C, gamma, J, K, E, lambda, nullptr};
  bool graphable = use_graph && ctx->stream != nullptr;
  bool host_out = false;
  for (int i = 0; i < 6 && graphable; ++i) {
    if (!key[i] || is_device_ptr(key[i])) continue;
    if (is_pinned_host_ptr(key[i])) host_out = host_out || i >= 2;
    else graphable = false;
  }
  if (!graphable) return iteration_eager(ctx, C, gamma, mode, J, K, E, lambda);
  bool hit = ctx->graph_exec && ctx->graph_mode == mode;
  for (int i = 0; i < 7 && hit; ++i) hit = ctx->graph_key[i] == key[i];
  if (!hit) {
    if (ctx->graph_exec) {
      cudaGraphExecDestroy(ctx->graph_exec);
      ctx->graph_exec = nullptr;
    }
    DONOF_CUDA_TRY(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    ctx->capturing = 1;
    long long l0 = ctx->launches;
    int rc = iteration_eager(ctx, C, gamma, mode, J, K, E, lambda);
    ctx->capturing = 0;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (rc || e != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return rc ? rc : DONOF_RI_E_CUDA;
    }
    e = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      ctx->graph_exec = nullptr;
      cudaGetLastError();
      return DONOF_RI_E_CUDA;
    }
    ctx->graph_launches = ctx->launches - l0;
    ctx->launches = l0;
    for (int i = 0; i < 7; ++i) ctx->graph_key[i] = key[i];
    ctx->graph_mode = mode;
  }
  DONOF_CUDA_TRY(cudaGraphLaunch(ctx->graph_exec, ctx->stream));
  ctx->launches += ctx->graph_launches;
  ctx->have_half = 1;
  ctx->have_full = (mode == DONOF_RI_FULL);
  ctx->have_ao = 1;
  ctx->have_lambda = 1;
  // results in host memory are complete once the stream has reached them
  return host_out ? consume_status(ctx) : DONOF_RI_OK;
}

int donof_ri_optimize_occupations(donof_ri_ctx* ctx, double* gamma, int max_iter, double gtol, double etol, double* E,
                                  double* grad, int* info) {
  if (!ctx || !gamma || max_iter < 0 || max_iter > 1000000 || !(gtol >= 0.0) || !(etol >= 0.0)) return DONOF_RI_E_ARG;
  if (!ctx->have_full) return DONOF_RI_E_STATE;
  const size_t ng = (size_t)ctx->n_strong * ctx->n_weak_per;
  double* dg = ctx->d_on;
  double* dgrad = ctx->d_on + ng;
  double* dE = ctx->d_on + 2 * ng;
  const bool gdev = is_device_ptr(gamma);
  int rc;
  ProfScope ps(ctx, DONOF_RI_ROW_OTHER);
  DONOF_CUDA_TRY(cudaMemcpyAsync(dg, gamma, ng * sizeof(double), gdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                 ctx->stream));
  if ((rc = launch_check_finite(ctx, dg, (long long)ng))) return rc;
  if ((rc = onopt_launch(ctx, dg, dE, dgrad, ctx->d_on_info, max_iter > 0 ? 1 : 0, max_iter, gtol, etol))) return rc;
  bool host = false;
  if ((rc = copy_out(ctx, gamma, dg, ng, &host))) return rc;
  if ((rc = copy_out(ctx, E, dE, 1, &host))) return rc;
  if ((rc = copy_out(ctx, grad, dgrad, ng, &host))) return rc;
  if (info) {
    DONOF_CUDA_TRY(cudaMemcpyAsync(info, ctx->d_on_info, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    host = true;
  }
  return host ? consume_status(ctx) : DONOF_RI_OK;
}

int donof_ri_on_features(donof_ri_ctx* ctx, float* X) {
  if (!ctx || !X) return DONOF_RI_E_ARG;
  if (!ctx->have_full) return DONOF_RI_E_STATE;
  int rc;
  ProfScope ps(ctx, DONOF_RI_ROW_OTHER);
  if ((rc = onopt_features(ctx, ctx->d_feat))) return rc;
  const size_t n = (size_t)ctx->n_strong * (3 + 4 * (size_t)ctx->n_weak_per);
  const bool dev = is_device_ptr(X);
  DONOF_CUDA_TRY(cudaMemcpyAsync(X, ctx->d_feat, n * sizeof(float), dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 ctx->stream));
  return dev ? DONOF_RI_OK : consume_status(ctx);
}

int donof_ri_gamma_guess(donof_ri_ctx* ctx, donof_mlp* net, double clip, double* gamma) {
  if (!ctx || !net || !gamma || !(clip >= 0.0) || !(clip < 0.7853981633974483)) return DONOF_RI_E_ARG;
  if (!ctx->have_full) return DONOF_RI_E_STATE;
  int F = 0, O = 0;
  mlp_shape(net, &F, &O);
  if (F != 3 + 4 * ctx->n_weak_per || O != ctx->n_weak_per) return DONOF_RI_E_ARG;
  int rc;
  ProfScope ps(ctx, DONOF_RI_ROW_OTHER);
  if ((rc = onopt_features(ctx, ctx->d_feat))) return rc;
  // the network runs on its own stream: order it after the features
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return DONOF_RI_E_CUDA;
  float* dY = nullptr;
  if ((rc = mlp_forward_device(net, ctx->d_feat, ctx->n_strong, &dY))) return rc;
  if (cudaDeviceSynchronize() != cudaSuccess) return DONOF_RI_E_CUDA;
  const size_t ng = (size_t)ctx->n_strong * ctx->n_weak_per;
  if ((rc = onopt_unfold(ctx, dY, clip, ctx->d_on))) return rc;
  bool host = false;
  if ((rc = copy_out(ctx, gamma, ctx->d_on, ng, &host))) return rc;
  return host ? consume_status(ctx) : DONOF_RI_OK;
}

int donof_ri_fetch(donof_ri_ctx* ctx, int what, double* dst, size_t count) {
  if (!ctx || !dst) return DONOF_RI_E_ARG;
  const size_t nb = ctx->nbf, nx = ctx->naux, m = ctx->n_omega;
  const double* src = nullptr;
  size_t n = 0;
  switch (what) {
    case DONOF_RI_FETCH_B: src = ctx->d_B; n = nx * nb * nb; break;
    case DONOF_RI_FETCH_HCORE: src = ctx->d_H; n = nb * nb; break;
    case DONOF_RI_FETCH_OVERLAP: src = ctx->d_S; n = nb * nb; break;
    case DONOF_RI_FETCH_METRIC: src = ctx->d_G; n = nx * nx; break;
    case DONOF_RI_FETCH_ENUC: src = ctx->d_enuc; n = 1; break;
    case DONOF_RI_FETCH_OCC: src = ctx->d_n; n = m; break;
    case DONOF_RI_FETCH_BHALF: n = nx * m * nb; src = ctx->d_bh; break;
    case DONOF_RI_FETCH_DIAG: n = nx * m; src = ctx->d_d; break;
    default: return DONOF_RI_E_ARG;
  }
  if (count != n) return DONOF_RI_E_ARG;
  if ((what == DONOF_RI_FETCH_BHALF || what == DONOF_RI_FETCH_DIAG) && !ctx->have_half) return DONOF_RI_E_STATE;
  if (ctx->precision == DONOF_RI_TF32X3 && (what == DONOF_RI_FETCH_BHALF || what == DONOF_RI_FETCH_DIAG))
    return mixed_fetch(ctx, what, dst, count);
  if (ctx->precision == DONOF_RI_SLICE4 && (what == DONOF_RI_FETCH_BHALF || what == DONOF_RI_FETCH_DIAG))
    return s4_fetch(ctx, what, dst, count);
  DONOF_CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return consume_status(ctx);
}

}  // extern "C"
