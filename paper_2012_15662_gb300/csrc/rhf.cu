// Closed-shell RI Hartree-Fock orbitals: the starting natural orbitals of the
// paper's calculations (Sec. 4, Computational Details: the guess NOs come from a
// Hartree-Fock calculation).  Roothaan-Hall equations in the overlap metric,
//   F C = S C eps,  F = H + J[D] - K[D] / 2,  D = 2 C_occ C_occ^T,
// with the RI Coulomb and exchange matrices from the engine's fitted tensor,
//   J[D]_{mu nu} = sum_P B^P_{mu nu} c_P,  c_P = 2 sum_i b^P_ii,
//   K[D] / 2     = sum_i sum_P b^P_{i mu} b^P_{i nu}      (b^P_{i nu} = sum_mu C_{mu i} B^P_{mu nu}),
// i over the N_I lowest orbitals (the strong ones of the pairing scheme), iterated
// from the core-Hamiltonian guess with Pulay's DIIS (the Fock matrices of the last
// eight iterations combined with the coefficients that minimise the norm of the
// combined error F D S - S D F, subject to their sum being one).  The generalised
// eigenproblem is solved in the basis orthonormalised by the Cholesky factor of S
// (F' = L^-1 F L^-T, C = L^-T V) with the F^lambda step's symmetric eigensolver.
// Everything is FP64 on the device (the fitted tensor in FP64 exists in every
// context); the host keeps the loop, the convergence test and the DIIS system of
// at most nine unknowns.
#include "common.cuh"

#include <math.h>
#include <string.h>

#include <utility>
#include <vector>

namespace donof {

constexpr int RHF_NDIIS = 8;

// c_P = 2 sum_i sum_nu bocc[P][i][nu] Ct[i][nu]: one warp per P, a fixed reduction order.
__global__ void rhf_cp_kernel(const double* bocc, const double* Ct, int nx, int no, int nb, double* cP) {
  const int P = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
  if (P >= nx) return;
  const double* b = bocc + (size_t)P * no * nb;
  double s = 0.0;
  for (long long e = lane; e < (long long)no * nb; e += 32) s += b[e] * Ct[e];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) cP[P] = 2.0 * s;
}

// out = a X + b Y + c Z elementwise (Y, Z may be null)
__global__ void rhf_axpy3_kernel(long long n, double a, const double* X, double b, const double* Y, double c,
                                 const double* Z, double* out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = a * X[i];
  if (Y) v += b * Y[i];
  if (Z) v += c * Z[i];
  out[i] = v;
}

// err = X - X^T (X = F D S; S D F = X^T for symmetric F, D, S)
__global__ void rhf_comm_kernel(int n, const double* X, double* err) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)n * n) return;
  const int r = (int)(i / n), c = (int)(i % n);
  err[i] = X[i] - X[(size_t)c * n + r];
}

// out[k] = sum_i X_k[i] Y[i] for k < m (one block per k, fixed order), and out[m] =
// max |Y| when maxabs (one more block).
__global__ void rhf_dots_kernel(long long n, const double* const* X, int m, const double* Y, double* out,
                                int maxabs) {
  __shared__ double red[256];
  const int k = blockIdx.x;
  double s = 0.0;
  if (k < m) {
    const double* x = X[k];
    for (long long i = threadIdx.x; i < n; i += blockDim.x) s += x[i] * Y[i];
  } else if (maxabs) {
    for (long long i = threadIdx.x; i < n; i += blockDim.x) s = fmax(s, fabs(Y[i]));
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = k < m ? red[threadIdx.x] + red[threadIdx.x + o]
                                                  : fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[k] = red[0];
}

// E = e_nuc + sum_i sum_nu Y[i][nu] Ct[i][nu] (Y = C_occ^T (H + F)), one block, fixed order.
__global__ void rhf_energy_kernel(const double* Y, const double* Ct, long long n, const double* enuc, double* E) {
  __shared__ double red[256];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s += Y[i] * Ct[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *E = *enuc + red[0];
}

__global__ void rhf_identity_kernel(int n, double* X) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)n * n) return;
  X[i] = (i / n == i % n) ? 1.0 : 0.0;
}

// C = alpha op(A) op(B) for row-major matrices (A: M x K after op, B: K x N after op).
static int rhf_mm(donof_ri_ctx* ctx, int M, int N, int K, const double* A, bool at, const double* B, bool bt,
                  double* C, double alpha = 1.0) {
  Gemm64 g{};
  g.M = M; g.N = N; g.K = K; g.batch = 1;
  g.A = A; g.sAm = at ? 1 : K; g.sAk = at ? M : 1;
  g.B = B; g.sBk = bt ? 1 : N; g.sBn = bt ? K : 1;
  g.C = C; g.sCm = N; g.sCn = 1;
  g.alpha = alpha; g.beta = 0.0;
  return launch_dgemm(ctx, g);
}

// Solve the (m+1) x (m+1) DIIS system [B -1; -1 0] [c; l] = [0; -1] by Gaussian
// elimination with partial pivoting; false when it is singular to working precision.
static bool diis_solve(const std::vector<double>& Bm, int m, int ld, std::vector<double>& c) {
  const int n = m + 1;
  std::vector<double> A((size_t)n * (n + 1), 0.0);
  double scale = 0.0;
  for (int i = 0; i < m; ++i) scale = fmax(scale, fabs(Bm[(size_t)i * ld + i]));
  if (!(scale > 0.0)) scale = 1.0;
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) A[(size_t)i * (n + 1) + j] = Bm[(size_t)i * ld + j] / scale;
    A[(size_t)i * (n + 1) + m] = -1.0;
    A[(size_t)m * (n + 1) + i] = -1.0;
  }
  A[(size_t)m * (n + 1) + n] = -1.0;
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[(size_t)i * (n + 1) + k]) > fabs(A[(size_t)piv * (n + 1) + k])) piv = i;
    if (!(fabs(A[(size_t)piv * (n + 1) + k]) > 1e-14)) return false;
    if (piv != k)
      for (int j = 0; j <= n; ++j) std::swap(A[(size_t)k * (n + 1) + j], A[(size_t)piv * (n + 1) + j]);
    for (int i = k + 1; i < n; ++i) {
      const double f = A[(size_t)i * (n + 1) + k] / A[(size_t)k * (n + 1) + k];
      for (int j = k; j <= n; ++j) A[(size_t)i * (n + 1) + j] -= f * A[(size_t)k * (n + 1) + j];
    }
  }
  std::vector<double> x(n, 0.0);
  for (int i = n - 1; i >= 0; --i) {
    double s = A[(size_t)i * (n + 1) + n];
    for (int j = i + 1; j < n; ++j) s -= A[(size_t)i * (n + 1) + j] * x[j];
    x[i] = s / A[(size_t)i * (n + 1) + i];
  }
  c.assign(x.begin(), x.begin() + m);
  for (double v : c)
    if (!isfinite(v)) return false;
  return true;
}

static bool rhf_is_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct RhfBuffers {
  double *Ls, *Li, *F, *Fp, *V, *Ct, *eps, *bocc, *cP, *Jm, *Km, *X, *Y, *W1, *DS, *Fd, *Ed, *dots, *scr;
  double* Fs[RHF_NDIIS];
  double* Es[RHF_NDIIS];
  const double** ptrs;
};

// Ct (row-major C^T, rows the orbitals by ascending eigenvalue) and eps from the
// generalised eigenproblem F C = S C eps, through F' = Li F Li^T and C = Li^T V.
static int rhf_eigh(donof_ri_ctx* ctx, RhfBuffers& b, const double* F) {
  const int n = ctx->nbf;
  int rc;
  if ((rc = rhf_mm(ctx, n, n, n, b.Li, false, F, false, b.X))) return rc;      // X = Li F
  if ((rc = rhf_mm(ctx, n, n, n, b.X, false, b.Li, true, b.Fp))) return rc;     // F' = X Li^T
  if ((rc = eigh_sym(ctx, b.Fp, n, b.scr, b.V, b.eps, nullptr))) return rc;
  return rhf_mm(ctx, n, n, n, b.V, true, b.Li, false, b.Ct);                     // Ct = V^T Li
}

static int rhf_run(donof_ri_ctx* ctx, RhfBuffers& b, int max_iter, double tol, double* Eh, int* iters,
                   double* comh) {
  const int n = ctx->nbf, nx = ctx->naux, no = ctx->n_strong;
  const long long n2 = (long long)n * n;
  cudaStream_t s = ctx->stream;
  const unsigned nblk = ceil_div_u(n2, 256);
  int rc;
  // S = L L^T, Li = L^-1
  DONOF_CUDA_TRY(cudaMemcpyAsync(b.Ls, ctx->d_S, n2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if ((rc = cholesky_lower(ctx, b.Ls, n, ctx->d_scratch_max, 1e-14))) return rc;
  rhf_identity_kernel<<<nblk, 256, 0, s>>>(n, b.Li);
  DONOF_LAUNCH_CHECK(ctx);
  if ((rc = forward_subst(ctx, b.Ls, n, b.Li, n))) return rc;
  // core-Hamiltonian guess
  if ((rc = rhf_eigh(ctx, b, ctx->d_H))) return rc;
  std::vector<double> Bm((size_t)RHF_NDIIS * RHF_NDIIS, 0.0);
  int nst = 0, head = 0;  // stored DIIS vectors, ring position of the next
  double E = 0.0, com = INFINITY;
  int it = 0;
  for (it = 1; it <= max_iter; ++it) {
    // bocc[P][i][nu] = sum_mu C_{mu i} B^P_{mu nu} for the occupied i
    {
      Gemm64 g{};
      g.M = no; g.N = n; g.K = n; g.batch = nx;
      g.A = b.Ct; g.sAb = 0; g.sAm = n; g.sAk = 1;
      g.B = ctx->d_B; g.sBb = n2; g.sBk = n; g.sBn = 1;
      g.C = b.bocc; g.sCb = (long long)no * n; g.sCm = n; g.sCn = 1;
      g.alpha = 1.0; g.beta = 0.0;
      if ((rc = launch_dgemm(ctx, g))) return rc;
    }
    rhf_cp_kernel<<<ceil_div_u(nx, 8), 256, 0, s>>>(b.bocc, b.Ct, nx, no, n, b.cP);
    DONOF_LAUNCH_CHECK(ctx);
    {
      Gemm64 g{};  // J = sum_P c_P B^P
      g.M = 1; g.N = (int)n2; g.K = nx; g.batch = 1;
      g.A = b.cP; g.sAm = 0; g.sAk = 1;
      g.B = ctx->d_B; g.sBk = n2; g.sBn = 1;
      g.C = b.Jm; g.sCm = n2; g.sCn = 1;
      g.alpha = 1.0; g.beta = 0.0;
      if ((rc = launch_dgemm(ctx, g))) return rc;
      Gemm64 k{};  // K[D]/2 = sum_{P,i} bocc[(P,i)]^T bocc[(P,i)]
      k.M = n; k.N = n; k.K = nx * no; k.batch = 1;
      k.A = b.bocc; k.sAm = 1; k.sAk = n;
      k.B = b.bocc; k.sBk = n; k.sBn = 1;
      k.C = b.Km; k.sCm = n; k.sCn = 1;
      k.alpha = 1.0; k.beta = 0.0;
      if ((rc = launch_dgemm(ctx, k))) return rc;
    }
    rhf_axpy3_kernel<<<nblk, 256, 0, s>>>(n2, 1.0, ctx->d_H, 1.0, b.Jm, -1.0, b.Km, b.F);  // F = H + J - K/2
    DONOF_LAUNCH_CHECK(ctx);
    // E = E_nuc + sum_i C_i^T (H + F) C_i
    rhf_axpy3_kernel<<<nblk, 256, 0, s>>>(n2, 1.0, ctx->d_H, 1.0, b.F, 0.0, nullptr, b.X);
    DONOF_LAUNCH_CHECK(ctx);
    if ((rc = rhf_mm(ctx, no, n, n, b.Ct, false, b.X, false, b.Y))) return rc;
    rhf_energy_kernel<<<1, 256, 0, s>>>(b.Y, b.Ct, (long long)no * n, ctx->d_enuc, b.Ed);
    DONOF_LAUNCH_CHECK(ctx);
    // err = F D S - S D F with D S = 2 C_occ (C_occ^T S)
    if ((rc = rhf_mm(ctx, no, n, n, b.Ct, false, ctx->d_S, false, b.W1))) return rc;
    if ((rc = rhf_mm(ctx, n, n, no, b.Ct, true, b.W1, false, b.DS, 2.0))) return rc;
    if ((rc = rhf_mm(ctx, n, n, n, b.F, false, b.DS, false, b.X))) return rc;
    double* slot_e = b.Es[head];
    double* slot_f = b.Fs[head];
    rhf_comm_kernel<<<nblk, 256, 0, s>>>(n, b.X, slot_e);
    DONOF_LAUNCH_CHECK(ctx);
    DONOF_CUDA_TRY(cudaMemcpyAsync(slot_f, b.F, n2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    // dots of the new error with every stored one (itself included) and max |err|
    const int m = nst < RHF_NDIIS ? nst + 1 : RHF_NDIIS;
    std::vector<const double*> hp(RHF_NDIIS);
    std::vector<int> slot_of(m);  // stored vectors in ring order, the new one last
    for (int k = 0; k < m; ++k) {
      const int sl = (head - (m - 1) + k + RHF_NDIIS) % RHF_NDIIS;
      slot_of[k] = sl;
      hp[k] = b.Es[sl];
    }
    DONOF_CUDA_TRY(cudaMemcpyAsync(b.ptrs, hp.data(), m * sizeof(double*), cudaMemcpyHostToDevice, s));
    rhf_dots_kernel<<<m + 1, 256, 0, s>>>(n2, b.ptrs, m, slot_e, b.dots, 1);
    DONOF_LAUNCH_CHECK(ctx);
    double hd[RHF_NDIIS + 1];
    DONOF_CUDA_TRY(cudaMemcpyAsync(hd, b.dots, (m + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
    DONOF_CUDA_TRY(cudaMemcpyAsync(&E, b.Ed, sizeof(double), cudaMemcpyDeviceToHost, s));
    DONOF_CUDA_TRY(cudaStreamSynchronize(s));
    com = hd[m];
    if (!isfinite(com) || !isfinite(E)) return DONOF_RI_E_NONFINITE;
    if (com <= tol) {
      if ((rc = rhf_eigh(ctx, b, b.F))) return rc;
      break;
    }
    // DIIS matrix over ring slots: row/column of the new slot from the dots
    for (int k = 0; k < m; ++k) {
      Bm[(size_t)slot_of[k] * RHF_NDIIS + head] = hd[k];
      Bm[(size_t)head * RHF_NDIIS + slot_of[k]] = hd[k];
    }
    nst = m;
    head = (head + 1) % RHF_NDIIS;
    // coefficients over the stored vectors in ring order; drop the oldest while singular
    std::vector<double> c;
    int use = m;
    std::vector<double> sub;
    while (use > 0) {
      sub.assign((size_t)use * use, 0.0);
      for (int i = 0; i < use; ++i)
        for (int j = 0; j < use; ++j)
          sub[(size_t)i * use + j] = Bm[(size_t)slot_of[m - use + i] * RHF_NDIIS + slot_of[m - use + j]];
      if (diis_solve(sub, use, use, c)) break;
      --use;
    }
    if (use == 0) return DONOF_RI_E_NONFINITE;
    // F_diis = sum_k c_k F_k (pairs of terms per launch, in ring order)
    DONOF_CUDA_TRY(cudaMemsetAsync(b.Fd, 0, n2 * sizeof(double), s));
    for (int k = 0; k < use; ++k) {
      rhf_axpy3_kernel<<<nblk, 256, 0, s>>>(n2, 1.0, b.Fd, c[k], b.Fs[slot_of[m - use + k]], 0.0, nullptr, b.Fd);
      DONOF_LAUNCH_CHECK(ctx);
    }
    if ((rc = rhf_eigh(ctx, b, b.Fd))) return rc;
  }
  *Eh = E;
  *iters = it > max_iter ? max_iter : it;
  *comh = com;
  return DONOF_RI_OK;
}

}  // namespace donof

extern "C" int donof_ri_rhf(donof_ri_ctx* ctx, int max_iter, double tol, double* C, double* eps, double* E,
                            int* iterations, double* commutator) {
  using namespace donof;
  if (!ctx || !C || max_iter < 1 || !(tol > 0.0)) return DONOF_RI_E_ARG;
  const int n = ctx->nbf, nx = ctx->naux, no = ctx->n_strong;
  if (n > FLAMBDA_MAX_NBF || no < 1 || no > n) return DONOF_RI_E_UNSUPPORTED;
  const long long n2 = (long long)n * n;
  RhfBuffers b{};
  std::vector<void*> owned;
  auto dal = [&](double** p, size_t count) -> bool {
    if (cudaMalloc((void**)p, count * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    owned.push_back(*p);
    return true;
  };
  bool ok = dal(&b.Ls, n2) && dal(&b.Li, n2) && dal(&b.F, n2) && dal(&b.Fp, n2) && dal(&b.V, n2) && dal(&b.Ct, n2) &&
            dal(&b.eps, n) && dal(&b.bocc, (size_t)nx * no * n) && dal(&b.cP, nx) && dal(&b.Jm, n2) &&
            dal(&b.Km, n2) && dal(&b.X, n2) && dal(&b.Y, (size_t)no * n) && dal(&b.W1, (size_t)no * n) &&
            dal(&b.DS, n2) && dal(&b.Fd, n2) && dal(&b.Ed, 1) && dal(&b.dots, RHF_NDIIS + 1) &&
            dal(&b.scr, flambda_scratch_doubles(n));
  for (int k = 0; ok && k < RHF_NDIIS; ++k) ok = dal(&b.Fs[k], n2) && dal(&b.Es[k], n2);
  if (ok) {
    if (cudaMalloc((void**)&b.ptrs, RHF_NDIIS * sizeof(double*)) != cudaSuccess) {
      cudaGetLastError();
      ok = false;
    } else {
      owned.push_back((void*)b.ptrs);
    }
  }
  int rc = ok ? DONOF_RI_OK : DONOF_RI_E_OOM;
  double Eh = 0.0, com = 0.0;
  int its = 0;
  if (!rc) rc = rhf_run(ctx, b, max_iter, tol, &Eh, &its, &com);
  if (!rc) {
    // C column-major = row-major C^T
    cudaMemcpyKind kc = rhf_is_device(C) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (cudaMemcpyAsync(C, b.Ct, n2 * sizeof(double), kc, ctx->stream) != cudaSuccess) rc = DONOF_RI_E_CUDA;
    if (!rc && eps) {
      cudaMemcpyKind ke = rhf_is_device(eps) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
      if (cudaMemcpyAsync(eps, b.eps, n * sizeof(double), ke, ctx->stream) != cudaSuccess) rc = DONOF_RI_E_CUDA;
    }
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = DONOF_RI_E_CUDA;
  }
  cudaStreamSynchronize(ctx->stream);
  for (void* p : owned) cudaFree(p);
  if (!rc) {
    int h = 0;  // a device-side fault recorded on the way (the overlap's factorisation)
    if (cudaMemcpy(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DONOF_RI_E_CUDA;
    if (h) {
      cudaMemset(ctx->d_status, 0, sizeof(int));
      return h == DEV_METRIC_NOT_PD ? DONOF_RI_E_METRIC_NOT_PD
                                    : (h == DEV_TIMEOUT ? DONOF_RI_E_TIMEOUT : DONOF_RI_E_NONFINITE);
    }
  }
  if (rc) return rc;
  if (E) *E = Eh;
  if (iterations) *iterations = its;
  if (commutator) *commutator = com;
  return DONOF_RI_OK;
}
