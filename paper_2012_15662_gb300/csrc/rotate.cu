// Orbital rotation step for fixed occupations (Sec. 2, "Orbital Optimization with
// RI"): C -> C expm(kappa) with kappa = -r G / max|G|, G_qp = lambda_qp - lambda_pq
// the rotation gradient (dE/dkappa_qp = 4 G_qp) from the Lagrangian of the last
// donof_ri_energy_lagrangian, and r a trust radius chosen by the caller.  This is
// the plain rotation driver's step; the paper's own step (iterative
// diagonalisation of F^lambda) is a later addition.
//
// expm by scaling and squaring: X = kappa / 2^s with ||X||_1 <= 1/4, Taylor
// series to order 12 in Horner form (truncation below 1e-17), then s squarings;
// the rotated orbitals are re-orthonormalised in the overlap metric by one
// Newton-Schulz step C <- C (3 I - C^T S C) / 2, which removes the rounding drift
// of repeated steps (the orbitals are orthonormal functions, C^T S C = I; a
// rotation in orbital space keeps that exactly, so the step only corrects
// rounding and expects orbitals that are S-orthonormal on entry).
// All FP64, with the library's tiled DGEMM.
#include "common.cuh"

#include <math.h>

namespace donof {

// kappa[q][p] (row-major) = scale (lambda_qp - lambda_pq); lambda column-major.
__global__ void rot_kappa_kernel(const double* lam, int nb, double scale, double* kappa) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)nb * nb) return;
  const int q = (int)(i / nb), p = (int)(i % nb);
  kappa[i] = scale * (lam[(size_t)p * nb + q] - lam[(size_t)q * nb + p]);
}

// out[0] = max_qp |lambda_qp - lambda_pq|, out[1] = max_q sum_p |same| (the 1-norm of G).
__global__ void rot_norms_kernel(const double* lam, int nb, double* out) {
  __shared__ double rmax[256], rsum[256];
  double mx = 0.0, sm = 0.0;
  for (int q = threadIdx.x; q < nb; q += 256) {
    double row = 0.0;
    for (int p = 0; p < nb; ++p) {
      const double g = fabs(lam[(size_t)p * nb + q] - lam[(size_t)q * nb + p]);
      mx = fmax(mx, g);
      row += g;
    }
    sm = fmax(sm, row);
  }
  rmax[threadIdx.x] = mx;
  rsum[threadIdx.x] = sm;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      rmax[threadIdx.x] = fmax(rmax[threadIdx.x], rmax[threadIdx.x + s]);
      rsum[threadIdx.x] = fmax(rsum[threadIdx.x], rsum[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = rmax[0];
    out[1] = rsum[0];
  }
}

// M = a I + b X (row-major n x n)
__global__ void rot_axpy_identity_kernel(int n, double a, double b, const double* X, double* M) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)n * n) return;
  const int r = (int)(i / n), c = (int)(i % n);
  M[i] = (r == c ? a : 0.0) + (X ? b * X[i] : 0.0);
}

static int gemm_rr(donof_ri_ctx* ctx, int n, const double* A, bool At, const double* B, double* C, double alpha,
                   double beta) {
  // C = alpha op(A) B + beta C, all row-major n x n; op(A) = A or A^T
  Gemm64 g{};
  g.M = n; g.N = n; g.K = n; g.batch = 1;
  g.A = A;
  g.sAm = At ? 1 : n;
  g.sAk = At ? n : 1;
  g.B = B; g.sBk = n; g.sBn = 1;
  g.C = C; g.sCm = n; g.sCn = 1;
  g.alpha = alpha; g.beta = beta;
  return launch_dgemm(ctx, g);
}

// 1-norm of a row-major n x n matrix (max over columns of the column sums of |X|) into out[0].
__global__ void rot_norm1_kernel(const double* X, int n, double* out) {
  __shared__ double red[256];
  double m = 0.0;
  for (int c = threadIdx.x; c < n; c += 256) {
    double col = 0.0;
    for (int r = 0; r < n; ++r) col += fabs(X[(size_t)r * n + c]);
    m = fmax(m, col);
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

// X <- a X (row-major n x n)
__global__ void rot_scale_kernel(int n, double a, double* X) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < (long long)n * n) X[i] *= a;
}

// C <- C expm(2^s X) for X = K (row-major, already scaled so that ||X||_1 <= 1/4),
// then one Newton-Schulz step in the overlap metric.  K, U, T, W: n x n scratch.
static int apply_scaled_rotation(donof_ri_ctx* ctx, int s, double* K, double* U, double* T, double* W) {
  const int n = ctx->nbf;
  const long long n2 = (long long)n * n;
  const unsigned int nblk = ceil_div_u(n2, 256);
  // Horner: U = I + X (I + X/2 (I + ... (I + X/12)))
  rot_axpy_identity_kernel<<<nblk, 256, 0, ctx->stream>>>(n, 1.0, 1.0 / 12.0, K, U);
  DONOF_LAUNCH_CHECK(ctx);
  int rc;
  for (int k = 11; k >= 1; --k) {
    rot_axpy_identity_kernel<<<nblk, 256, 0, ctx->stream>>>(n, 1.0, 0.0, nullptr, T);
    DONOF_LAUNCH_CHECK(ctx);
    if ((rc = gemm_rr(ctx, n, K, false, U, T, 1.0 / k, 1.0))) return rc;  // T = I + X U / k
    double* t = U;
    U = T;
    T = t;
  }
  for (int k = 0; k < s; ++k) {  // U <- U U
    if ((rc = gemm_rr(ctx, n, U, false, U, T, 1.0, 0.0))) return rc;
    double* t = U;
    U = T;
    T = t;
  }
  // d_C is column-major, i.e. row-major C^T: (C U)^T = U^T C^T
  if ((rc = gemm_rr(ctx, n, U, true, ctx->d_C, T, 1.0, 0.0))) return rc;
  // Newton-Schulz in the overlap metric: C <- C (3 I - C^T S C) / 2.  With Ct = C^T
  // (row-major, in T): X = S C = S Ct^T (into K, free after the exponential), then
  // W = Ct X = C^T S C; Ct <- Z Ct with Z = (3 I - W) / 2 (symmetric).
  {
    Gemm64 g{};
    g.M = n; g.N = n; g.K = n; g.batch = 1;
    g.A = ctx->d_S; g.sAm = n; g.sAk = 1;
    g.B = T; g.sBk = 1; g.sBn = n;
    g.C = K; g.sCm = n; g.sCn = 1;
    g.alpha = 1.0; g.beta = 0.0;
    if ((rc = launch_dgemm(ctx, g))) return rc;  // K = S C
    if ((rc = gemm_rr(ctx, n, T, false, K, W, 1.0, 0.0))) return rc;  // W = C^T S C
  }
  rot_axpy_identity_kernel<<<nblk, 256, 0, ctx->stream>>>(n, 1.5, -0.5, W, U);  // Z = (3 I - W) / 2
  DONOF_LAUNCH_CHECK(ctx);
  if ((rc = gemm_rr(ctx, n, U, false, T, ctx->d_C, 1.0, 0.0))) return rc;
  return DONOF_RI_OK;
}

// Rotates ctx->d_C in place; gnorm[0] = max|G| (host).  Scratch: 4 n^2 + 2 doubles.
int rotate_orbitals(donof_ri_ctx* ctx, double radius, double* scratch, double* gnorm) {
  const int n = ctx->nbf;
  const long long n2 = (long long)n * n;
  double *K = scratch, *U = scratch + n2, *T = scratch + 2 * n2, *W = scratch + 3 * n2, *nrm = scratch + 4 * n2;
  rot_norms_kernel<<<1, 256, 0, ctx->stream>>>(ctx->d_lambda, n, nrm);
  DONOF_LAUNCH_CHECK(ctx);
  double norms[2];
  DONOF_CUDA_TRY(cudaMemcpyAsync(norms, nrm, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  DONOF_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  *gnorm = norms[0];
  if (!(norms[0] > 0.0) || !(radius > 0.0)) return DONOF_RI_OK;
  // ||kappa||_1 = radius * ||G||_1 / max|G|; scale by 2^-s so that ||X||_1 <= 1/4
  const double k1 = radius * norms[1] / norms[0];
  int s = 0;
  while (k1 / ldexp(1.0, s) > 0.25 && s < 60) ++s;
  const double scale = -radius / norms[0] / ldexp(1.0, s);
  const unsigned int nblk = ceil_div_u(n2, 256);
  rot_kappa_kernel<<<nblk, 256, 0, ctx->stream>>>(ctx->d_lambda, n, scale, K);
  DONOF_LAUNCH_CHECK(ctx);
  return apply_scaled_rotation(ctx, s, K, U, T, W);
}

// Rotates ctx->d_C in place by expm(kappa), kappa a device copy (row-major n x n).
// Scratch: 4 n^2 + 2 doubles (kappa may already sit in its first n^2).
int apply_rotation(donof_ri_ctx* ctx, double* scratch) {
  const int n = ctx->nbf;
  const long long n2 = (long long)n * n;
  double *K = scratch, *U = scratch + n2, *T = scratch + 2 * n2, *W = scratch + 3 * n2, *nrm = scratch + 4 * n2;
  rot_norm1_kernel<<<1, 256, 0, ctx->stream>>>(K, n, nrm);
  DONOF_LAUNCH_CHECK(ctx);
  double k1 = 0.0;
  DONOF_CUDA_TRY(cudaMemcpyAsync(&k1, nrm, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  DONOF_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (!isfinite(k1)) return DONOF_RI_E_NONFINITE;
  int s = 0;
  while (k1 / ldexp(1.0, s) > 0.25 && s < 60) ++s;
  if (s > 0) {
    rot_scale_kernel<<<ceil_div_u(n2, 256), 256, 0, ctx->stream>>>(n, ldexp(1.0, -s), K);
    DONOF_LAUNCH_CHECK(ctx);
  }
  return apply_scaled_rotation(ctx, s, K, U, T, W);
}

}  // namespace donof
