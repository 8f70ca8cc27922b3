// The paper's orbital step (Sec. 2, "Orbital Optimization with RI"): the natural
// orbitals follow from iterative diagonalisations of a symmetric matrix F^lambda
// built from the orthonormality Lagrangian,
//   F_qp = lambda_qp - lambda_pq (q > p, mirrored), F_pp from an aufbau ordering
// (the previous step's eigenvalues; lambda_pp at the first step),
// and the orbitals are rotated onto its eigenvectors taken in increasing order of
// eigenvalue.  Off-diagonal elements larger than a bound are scaled by powers of
// 1/10 (damping; the paper gives no rule).  At a stationary point lambda is
// symmetric, F^lambda is diagonal and the step leaves the orbitals unchanged.
//
// Device plan (nbf <= 160): one CTA holds F^lambda and the accumulated rotation
// in shared memory (FP32) and diagonalises by cyclic Jacobi with round-robin pair
// ordering (every round rotates nbf/2 disjoint pairs: columns, then rows); the
// rotation is kept as X = V - I so that small rotations keep their relative
// precision.  The eigenvectors, sorted by eigenvalue, are then refined in FP64
// (orthonormalisation and two first-order corrections against F^lambda in FP64),
// C U is formed in FP64 and one Newton-Schulz step restores orthonormality to
// FP64 rounding.
#include "common.cuh"

#include <math.h>

namespace donof {

constexpr int FL_MAXN = 160;

__global__ void __launch_bounds__(1024, 1) flambda_jacobi_kernel(int n, const double* lam, const double* dprev,
                                                                 int first, double bound, double* U, double* eps,
                                                                 double* gmax, int* sweeps_out) {
  extern __shared__ float fl_smem[];
  const int ld = n + 1;
  float* A = fl_smem;              // [n][n + 1]
  float* X = A + (size_t)n * ld;   // [n][n + 1], V - I
  __shared__ float cs[FL_MAXN / 2], sn[FL_MAXN / 2], cm1[FL_MAXN / 2];
  __shared__ int pp[FL_MAXN / 2], qq[FL_MAXN / 2];
  __shared__ float red[32], redg[32];
  __shared__ double redd[32];
  __shared__ int s_done;
  __shared__ float s_md;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid % 32, wid = tid / 32;
  // F^lambda (lambda column-major: lambda_qp at p * n + q) and the gradient norm
  double gm = 0.0;
  for (int e = tid; e < n * n; e += nt) {
    const int q = e / n, p = e % n;
    float v;
    X[q * ld + p] = 0.f;
    if (q == p) {
      v = (float)(first ? lam[(size_t)p * n + p] : dprev[p]);
    } else {
      const int hi = q > p ? q : p, lo = q > p ? p : q;
      double g = lam[(size_t)lo * n + hi] - lam[(size_t)hi * n + lo];  // lambda_{hi lo} - lambda_{lo hi}
      gm = fmax(gm, fabs(g));
      double a = fabs(g);
      for (int k = 0; k < 700 && a > bound; ++k) {  // bounded: at most 700 decades
        g *= 0.1;
        a *= 0.1;
      }
      v = isfinite(g) ? (float)g : 0.f;
    }
    A[q * ld + p] = v;
  }
  for (int o = 16; o > 0; o >>= 1) gm = fmax(gm, __shfl_xor_sync(0xffffffffu, gm, o));
  if (lane == 0) redd[wid] = gm;
  __syncthreads();
  if (tid == 0 && gmax) {
    double m = 0.0;
    for (int w = 0; w < nt / 32; ++w) m = fmax(m, redd[w]);
    *gmax = m;
  }
  const int nn = n + (n & 1);  // players of the round-robin (a dummy when n is odd)
  const int npair = nn / 2;
  int sweep = 0;
  for (; sweep < 30; ++sweep) {
    // convergence: largest off-diagonal element against the largest diagonal one
    float off = 0.f, dia = 0.f;
    for (int e = tid; e < n * n; e += nt) {
      const int i = e / n, j = e % n;
      const float a = fabsf(A[i * ld + j]);
      if (i == j) dia = fmaxf(dia, a);
      else off = fmaxf(off, a);
    }
    for (int o = 16; o > 0; o >>= 1) {
      off = fmaxf(off, __shfl_xor_sync(0xffffffffu, off, o));
      dia = fmaxf(dia, __shfl_xor_sync(0xffffffffu, dia, o));
    }
    if (lane == 0) {
      red[wid] = off;
      redg[wid] = dia;
    }
    __syncthreads();
    if (tid == 0) {
      float mo = 0.f, md = 0.f;
      for (int w = 0; w < nt / 32; ++w) {
        mo = fmaxf(mo, red[w]);
        md = fmaxf(md, redg[w]);
      }
      // FP32 rounding leaves off-diagonal noise of a few 1e-7 of the largest element
      s_done = !(mo > 1e-6f * fmaxf(md, 1e-30f)) ? 1 : 0;
      s_md = md;
    }
    __syncthreads();
    if (s_done) break;
    for (int r = 0; r < nn - 1; ++r) {
      // pairs of this round and their rotations
      if (tid < npair) {
        const int k = tid;
        const int a = k == 0 ? 0 : 1 + ((k - 1 + r) % (nn - 1));
        const int pb = nn - 1 - k;
        const int b = 1 + ((pb - 1 + r) % (nn - 1));
        int p = a < b ? a : b, q = a < b ? b : a;
        float c = 1.f, s = 0.f, c1 = 0.f;
        if (q < n) {
          const float apq = A[p * ld + q];
          // rotations below the rounding noise are skipped (they would only add noise)
          if (fabsf(apq) > 1e-8f * s_md) {
            const float th = (A[q * ld + q] - A[p * ld + p]) / (2.f * apq);
            const float t = fabsf(th) > 1e18f ? 0.5f / th
                                              : (th >= 0.f ? 1.f : -1.f) / (fabsf(th) + sqrtf(th * th + 1.f));
            c = 1.f / sqrtf(t * t + 1.f);
            s = t * c;
            c1 = -(s * s) / (1.f + c);
          }
        } else {
          p = q = -1;
        }
        pp[k] = p;
        qq[k] = q;
        cs[k] = c;
        sn[k] = s;
        cm1[k] = c1;
      }
      __syncthreads();
      // columns p, q of A and of X:  col_p <- c col_p - s col_q,  col_q <- s col_p + c col_q
      for (int e = tid; e < npair * n; e += nt) {
        const int k = e / n, i = e % n;
        const int p = pp[k], q = qq[k];
        if (p < 0 || sn[k] == 0.f) continue;
        const float c = cs[k], s = sn[k];
        const float ap = A[i * ld + p], aq = A[i * ld + q];
        A[i * ld + p] = c * ap - s * aq;
        A[i * ld + q] = s * ap + c * aq;
        const float xp = X[i * ld + p], xq = X[i * ld + q];
        // X = V - I: the identity's columns e_p, e_q rotate too
        X[i * ld + p] = xp - s * xq + cm1[k] * xp + (i == p ? cm1[k] : 0.f) - (i == q ? s : 0.f);
        X[i * ld + q] = xq + s * xp + cm1[k] * xq + (i == p ? s : 0.f) + (i == q ? cm1[k] : 0.f);
      }
      __syncthreads();
      // rows p, q of A
      for (int e = tid; e < npair * n; e += nt) {
        const int k = e / n, j = e % n;
        const int p = pp[k], q = qq[k];
        if (p < 0 || sn[k] == 0.f) continue;
        const float c = cs[k], s = sn[k];
        const float ap = A[p * ld + j], aq = A[q * ld + j];
        A[p * ld + j] = c * ap - s * aq;
        A[q * ld + j] = s * ap + c * aq;
      }
      __syncthreads();
    }
  }
  // eigenvalues ascending (rank sort, ties by index) and the permuted rotation in FP64
  __shared__ int perm[FL_MAXN];
  if (tid < n) {
    const float ei = A[tid * ld + tid];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const float ej = A[j * ld + j];
      rank += (ej < ei || (ej == ei && j < tid)) ? 1 : 0;
    }
    perm[rank] = tid;
  }
  __syncthreads();
  if (tid < n) eps[tid] = (double)A[perm[tid] * ld + perm[tid]];
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, k = e % n;
    const int j = perm[k];
    U[e] = (i == j ? 1.0 : 0.0) + (double)X[i * ld + j];  // U[i][k], row-major
  }
  if (tid == 0 && sweeps_out) *sweeps_out = sweep;
}

__global__ void fl_identity_axpy_kernel(int n, double a, double b, const double* X, double* M) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)n * n) return;
  const int r = (int)(i / n), c = (int)(i % n);
  M[i] = (r == c ? a : 0.0) + b * X[i];
}

// F^lambda in FP64 (the same construction as the FP32 kernel), row-major.
__global__ void fl_build_f64_kernel(int n, const double* lam, const double* dprev, int first, double bound,
                                    double* F) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int q = (int)(e / n), p = (int)(e % n);
  double v;
  if (q == p) {
    v = first ? lam[(size_t)p * n + p] : dprev[p];
  } else {
    const int hi = q > p ? q : p, lo = q > p ? p : q;
    double g = lam[(size_t)lo * n + hi] - lam[(size_t)hi * n + lo];
    double a = fabs(g);
    for (int k = 0; k < 700 && a > bound; ++k) {
      g *= 0.1;
      a *= 0.1;
    }
    v = isfinite(g) ? g : 0.0;
  }
  F[e] = v;
}

// First-order eigenvector correction from A' = U^T F U (nearly diagonal):
// K_qp = A'_qp / (A'_pp - A'_qq) (q != p), and the refined eigenvalues
// eps_p = A'_pp.  Where the pair is not resolved at this accuracy
// (|A'_qp| > |A'_pp - A'_qq| / 10, first-order theory would not hold) K_qp = 0:
// any basis of a (nearly) degenerate pair is an eigenbasis to that accuracy.
__global__ void fl_refine_kernel(int n, const double* Ap, double* K, double* eps) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int q = (int)(e / n), p = (int)(e % n);
  if (q == p) {
    K[e] = 0.0;
    eps[p] = Ap[e];
    return;
  }
  const double app = Ap[(size_t)p * n + p], aqq = Ap[(size_t)q * n + q];
  const double gap = app - aqq;
  const double a = Ap[e];
  K[e] = fabs(a) * 10.0 < fabs(gap) ? a / gap : 0.0;
}

__global__ void fl_add_kernel(long long n, const double* X, double* Y) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) Y[i] += X[i];
}

size_t flambda_scratch_doubles(int n) { return 6 * (size_t)n * n + (size_t)n + 2; }

// C = alpha op(A) op(B) + beta C for row-major n x n matrices.
static int fl_mm(donof_ri_ctx* ctx, int n, const double* A, bool at, const double* B, bool bt, double* C,
                 double alpha, double beta) {
  Gemm64 g{};
  g.M = n; g.N = n; g.K = n; g.batch = 1;
  g.A = A; g.sAm = at ? 1 : n; g.sAk = at ? n : 1;
  g.B = B; g.sBk = bt ? 1 : n; g.sBn = bt ? n : 1;
  g.C = C; g.sCm = n; g.sCn = 1;
  g.alpha = alpha; g.beta = beta;
  return launch_dgemm(ctx, g);
}

// U <- U (3 I - U^T U) / 2, then two refinements U <- orth(U (I + K)) against the
// FP64 matrix Fd; eps <- the refined eigenvalues.  T, W, Z, K: n x n scratch.
static int eig_refine(donof_ri_ctx* ctx, int n, const double* Fd, double* U, double* T, double* W, double* Z,
                      double* K, double* eps) {
  const long long n2 = (long long)n * n;
  const unsigned nblk = ceil_div_u(n2, 256);
  int rc;
  for (int pass = 0; pass < 3; ++pass) {
    if (pass > 0) {
      if ((rc = fl_mm(ctx, n, Fd, false, U, false, T, 1.0, 0.0))) return rc;   // T = F U
      if ((rc = fl_mm(ctx, n, U, true, T, false, W, 1.0, 0.0))) return rc;    // A' = U^T F U
      fl_refine_kernel<<<nblk, 256, 0, ctx->stream>>>(n, W, K, eps);
      DONOF_LAUNCH_CHECK(ctx);
      if ((rc = fl_mm(ctx, n, U, false, K, false, T, 1.0, 0.0))) return rc;   // T = U K
      fl_add_kernel<<<nblk, 256, 0, ctx->stream>>>(n2, T, U);
      DONOF_LAUNCH_CHECK(ctx);
    }
    if ((rc = fl_mm(ctx, n, U, true, U, false, W, 1.0, 0.0))) return rc;      // W = U^T U
    fl_identity_axpy_kernel<<<nblk, 256, 0, ctx->stream>>>(n, 1.5, -0.5, W, Z);
    DONOF_LAUNCH_CHECK(ctx);
    if ((rc = fl_mm(ctx, n, U, false, Z, false, T, 1.0, 0.0))) return rc;     // T = U Z
    DONOF_CUDA_TRY(cudaMemcpyAsync(U, T, n2 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  }
  return DONOF_RI_OK;
}

// One step on ctx->d_C (column-major = row-major C^T).  Scratch:
// flambda_scratch_doubles(n) doubles.  The FP32 eigenvectors are orthonormalised
// (Newton-Schulz) and refined twice in FP64 against the FP64 F^lambda by first-order
// perturbation theory, which brings them to FP64 accuracy wherever the eigenvalues
// are separated; the eigenvalues returned are those of the last refinement.
int flambda_step(donof_ri_ctx* ctx, const double* dprev, int first, double bound, double* scratch, double* gmax,
                 int* sweeps) {
  const int n = ctx->nbf;
  const long long n2 = (long long)n * n;
  double *U = scratch, *T = U + n2, *W = T + n2, *Z = W + n2, *Fd = Z + n2, *K = Fd + n2, *eps = K + n2,
         *gm = eps + n;
  int* sw = (int*)(gm + 1);
  const unsigned nblk = ceil_div_u(n2, 256);
  const size_t smem = 2 * (size_t)n * (n + 1) * sizeof(float);
  if (cudaFuncSetAttribute(flambda_jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return DONOF_RI_E_CUDA;
  fl_build_f64_kernel<<<nblk, 256, 0, ctx->stream>>>(n, ctx->d_lambda, dprev, first, bound, Fd);
  flambda_jacobi_kernel<<<1, 1024, smem, ctx->stream>>>(n, ctx->d_lambda, dprev, first, bound, U, eps, gm, sw);
  DONOF_LAUNCH_CHECK(ctx);
  ctx->launches++;
  int rc;
  if ((rc = eig_refine(ctx, n, Fd, U, T, W, Z, K, eps))) return rc;
  // (C U)^T = U^T C^T, then one Newton-Schulz step on its rows
  if ((rc = fl_mm(ctx, n, U, true, ctx->d_C, false, T, 1.0, 0.0))) return rc;
  if ((rc = fl_mm(ctx, n, T, false, T, true, W, 1.0, 0.0))) return rc;        // W = T T^T
  fl_identity_axpy_kernel<<<nblk, 256, 0, ctx->stream>>>(n, 1.5, -0.5, W, Z);
  DONOF_LAUNCH_CHECK(ctx);
  if ((rc = fl_mm(ctx, n, Z, false, T, false, ctx->d_C, 1.0, 0.0))) return rc;
  double hg = 0.0;
  int hs = 0;
  DONOF_CUDA_TRY(cudaMemcpyAsync(&hg, gm, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  DONOF_CUDA_TRY(cudaMemcpyAsync(&hs, sw, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  DONOF_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  *gmax = hg;
  *sweeps = hs;
  return DONOF_RI_OK;
}

}  // namespace donof
