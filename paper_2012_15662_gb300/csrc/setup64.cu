// Setup on the device, all FP64: s-type Gaussian integrals, the Cholesky
// factorisation of the Coulomb metric and the fitted three-index tensor.
//
// Paper: Table 2 / Table 3 steps 0-1 (evaluation of (mu nu|k), G_kl = (k|l)
// and the solve for b), Eq. (AOERI), Sec. 3 (integrals evaluated once and
// stored).  The engine factorises G = L L^T with a plain Cholesky (no
// pivoting, no eigenvalue correction) and forms B = L^-1 (Q|mu nu).
#include "common.cuh"

#include <math.h>

namespace donof {

// ---------------------------------------------------------------------------
// Generic strided batched FP64 GEMM (CUDA cores).  64x64 output tile per CTA,
// 256 threads, 4x4 outputs per thread, K staged through shared memory in
// slices of 16.  Loads are ordered along whichever operand stride is unit so
// that global reads coalesce for every layout the engine uses.
// ---------------------------------------------------------------------------
constexpr int DG_TM = 64, DG_TN = 64, DG_TK = 16;

__global__ void __launch_bounds__(256) dgemm_kernel(Gemm64 g) {
  __shared__ double As[DG_TK][DG_TM + 1];
  __shared__ double Bs[DG_TK][DG_TN + 1];
  const int b = blockIdx.z;
  const int m0 = blockIdx.y * DG_TM;
  const int n0 = blockIdx.x * DG_TN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const double* A = g.A + (long long)b * g.sAb;
  const double* B = g.B + (long long)b * g.sBb;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int k0 = 0; k0 < g.K; k0 += DG_TK) {
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      int e = threadIdx.x + it * 256;
      int mm, kk;
      if (g.sAm == 1) { mm = e % DG_TM; kk = e / DG_TM; } else { kk = e % DG_TK; mm = e / DG_TK; }
      int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < g.M && gk < g.K) ? A[(long long)gm * g.sAm + (long long)gk * g.sAk] : 0.0;
      int nn;
      if (g.sBn == 1) { nn = e % DG_TN; kk = e / DG_TN; } else { kk = e % DG_TK; nn = e / DG_TK; }
      int gn = n0 + nn;
      gk = k0 + kk;
      Bs[kk][nn] = (gn < g.N && gk < g.K) ? B[(long long)gk * g.sBk + (long long)gn * g.sBn] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < DG_TK; ++kk) {
      double a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
  double* C = g.C + (long long)b * g.sCb;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int m = m0 + ty + 16 * i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int n = n0 + tx + 16 * j;
      if (n >= g.N) continue;
      double* c = C + (long long)m * g.sCm + (long long)n * g.sCn;
      double v = g.alpha * acc[i][j];
      if (g.beta != 0.0) v += g.beta * (*c);
      *c = v;
    }
  }
}

int launch_dgemm(donof_ri_ctx* ctx, const Gemm64& g) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return DONOF_RI_OK;
  if (g.K <= 0) return DONOF_RI_E_ARG;
  long long gy = (g.M + DG_TM - 1) / DG_TM;
  if (gy > 65535 || g.batch > 65535) return DONOF_RI_E_ARG;
  dim3 grid(ceil_div_u(g.N, DG_TN), (unsigned)gy, (unsigned)g.batch);
  dgemm_kernel<<<grid, 256, 0, ctx->stream>>>(g);
  DONOF_LAUNCH_CHECK(ctx);
  return DONOF_RI_OK;
}

// ---------------------------------------------------------------------------
// Integrals over normalised s-type Gaussians.
//   orbital basis:   N_a = (2a/pi)^(3/4)
//   auxiliary basis: N_k = (2k/pi)^(3/4) sqrt(k / (4 pi))   ((k|k) = 1)
// Boys F0(T) = 1/2 sqrt(pi/T) erf(sqrt(T)), with the series 1 - T/3 + T^2/10
// below T = 1e-8.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double boys_f0(double t) {
  if (t < 1e-8) return 1.0 - t / 3.0 + t * t / 10.0;
  double st = sqrt(t);
  return 0.5 * sqrt(M_PI / t) * erf(st);
}

__device__ __forceinline__ double norm_orb(double a) { return pow(2.0 * a / M_PI, 0.75); }
__device__ __forceinline__ double norm_aux(double k) {
  return pow(2.0 * k / M_PI, 0.75) * sqrt(k / (4.0 * M_PI));
}

// S, H = T + V for every orbital pair.
__global__ void one_electron_kernel(int nbf, int n_atoms, const double* xyz, const double* charge,
                                    const int* bf_atom, const double* bf_alpha, double* S, double* H) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)nbf * nbf) return;
  int i = (int)(idx / nbf), j = (int)(idx % nbf);
  double a = bf_alpha[i], b = bf_alpha[j];
  const double* A = xyz + 3 * bf_atom[i];
  const double* Bc = xyz + 3 * bf_atom[j];
  double p = a + b, mu = a * b / p;
  double dx = A[0] - Bc[0], dy = A[1] - Bc[1], dz = A[2] - Bc[2];
  double r2 = dx * dx + dy * dy + dz * dz;
  double kab = exp(-mu * r2);
  double nn = norm_orb(a) * norm_orb(b);
  double s = nn * pow(M_PI / p, 1.5) * kab;
  double t = nn * mu * (3.0 - 2.0 * mu * r2) * pow(M_PI / p, 1.5) * kab;
  double Px = (a * A[0] + b * Bc[0]) / p, Py = (a * A[1] + b * Bc[1]) / p, Pz = (a * A[2] + b * Bc[2]) / p;
  double v = 0.0;
  for (int c = 0; c < n_atoms; ++c) {
    double ex = Px - xyz[3 * c], ey = Py - xyz[3 * c + 1], ez = Pz - xyz[3 * c + 2];
    v -= charge[c] * nn * (2.0 * M_PI / p) * kab * boys_f0(p * (ex * ex + ey * ey + ez * ez));
  }
  S[idx] = s;
  H[idx] = t + v;
}

// G_kl = (k|l) over the auxiliary basis.
__global__ void metric_kernel(int naux, const double* xyz, const int* aux_atom, const double* aux_alpha,
                              double* G) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)naux * naux) return;
  int k = (int)(idx / naux), l = (int)(idx % naux);
  double c = aux_alpha[k], d = aux_alpha[l];
  const double* X = xyz + 3 * aux_atom[k];
  const double* Y = xyz + 3 * aux_atom[l];
  double dx = X[0] - Y[0], dy = X[1] - Y[1], dz = X[2] - Y[2];
  double r2 = dx * dx + dy * dy + dz * dz;
  double pref = 2.0 * pow(M_PI, 2.5) / (c * d * sqrt(c + d));
  G[idx] = norm_aux(c) * norm_aux(d) * pref * boys_f0(c * d / (c + d) * r2);
}

// (k|mu nu) into out[k][mu][nu].
__global__ void eri3_kernel(int nbf, int naux, const double* xyz, const int* bf_atom, const double* bf_alpha,
                            const int* aux_atom, const double* aux_alpha, double* out) {
  long long nb2 = (long long)nbf * nbf;
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)naux * nb2) return;
  int k = (int)(idx / nb2);
  int rem = (int)(idx % nb2);
  int i = rem / nbf, j = rem % nbf;
  double a = bf_alpha[i], b = bf_alpha[j], c = aux_alpha[k];
  const double* A = xyz + 3 * bf_atom[i];
  const double* Bc = xyz + 3 * bf_atom[j];
  const double* Cc = xyz + 3 * aux_atom[k];
  double p = a + b, mu = a * b / p;
  double dx = A[0] - Bc[0], dy = A[1] - Bc[1], dz = A[2] - Bc[2];
  double kab = exp(-mu * (dx * dx + dy * dy + dz * dz));
  double Px = (a * A[0] + b * Bc[0]) / p, Py = (a * A[1] + b * Bc[1]) / p, Pz = (a * A[2] + b * Bc[2]) / p;
  double ex = Px - Cc[0], ey = Py - Cc[1], ez = Pz - Cc[2];
  double pref = 2.0 * pow(M_PI, 2.5) / (p * c * sqrt(p + c));
  out[idx] = norm_orb(a) * norm_orb(b) * norm_aux(c) * pref * kab *
             boys_f0(p * c / (p + c) * (ex * ex + ey * ey + ez * ez));
}

__global__ void enuc_kernel(int n_atoms, const double* xyz, const double* charge, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double e = 0.0;
  for (int i = 0; i < n_atoms; ++i)
    for (int j = 0; j < i; ++j) {
      double dx = xyz[3 * i] - xyz[3 * j], dy = xyz[3 * i + 1] - xyz[3 * j + 1], dz = xyz[3 * i + 2] - xyz[3 * j + 2];
      e += charge[i] * charge[j] / sqrt(dx * dx + dy * dy + dz * dz);
    }
  *out = e;
}

int setup_integrals(donof_ri_ctx* ctx) {
  const int nb = ctx->nbf, nx = ctx->naux;
  long long n1 = (long long)nb * nb;
  one_electron_kernel<<<ceil_div_u(n1, 256), 256, 0, ctx->stream>>>(
      nb, ctx->n_atoms, ctx->d_atom_xyz, ctx->d_atom_charge, ctx->d_bf_atom, ctx->d_bf_alpha, ctx->d_S, ctx->d_H);
  DONOF_LAUNCH_CHECK(ctx);
  long long n2 = (long long)nx * nx;
  metric_kernel<<<ceil_div_u(n2, 256), 256, 0, ctx->stream>>>(nx, ctx->d_atom_xyz, ctx->d_aux_atom,
                                                               ctx->d_aux_alpha, ctx->d_G);
  DONOF_LAUNCH_CHECK(ctx);
  long long n3 = (long long)nx * n1;
  eri3_kernel<<<ceil_div_u(n3, 256), 256, 0, ctx->stream>>>(nb, nx, ctx->d_atom_xyz, ctx->d_bf_atom,
                                                             ctx->d_bf_alpha, ctx->d_aux_atom,
                                                             ctx->d_aux_alpha, ctx->d_B);
  DONOF_LAUNCH_CHECK(ctx);
  enuc_kernel<<<1, 32, 0, ctx->stream>>>(ctx->n_atoms, ctx->d_atom_xyz, ctx->d_atom_charge, ctx->d_enuc);
  DONOF_LAUNCH_CHECK(ctx);
  return DONOF_RI_OK;
}

// ---------------------------------------------------------------------------
// Blocked right-looking Cholesky of G (row-major, lower factor in place).
// ---------------------------------------------------------------------------
constexpr int CH_NB = 64;

__global__ void max_diag_kernel(int n, const double* G, double* out) {
  __shared__ double red[256];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, G[(long long)i * n + i]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// Factor the nbk x nbk diagonal block at (k0, k0) in shared memory.  A pivot
// below rel_min * max(diag G) sets DEV_METRIC_NOT_PD (the factorisation then
// continues on a clamped pivot so that the kernel always terminates).
__global__ void __launch_bounds__(256) potrf_block_kernel(int n, double* G, int k0, int nbk, const double* maxdiag,
                                                          double rel_min, int* status) {
  __shared__ double s[CH_NB][CH_NB + 1];
  for (int e = threadIdx.x; e < nbk * nbk; e += blockDim.x) {
    int i = e / nbk, j = e % nbk;
    s[i][j] = G[(long long)(k0 + i) * n + k0 + j];
  }
  __syncthreads();
  const double thresh = rel_min * (*maxdiag);
  for (int j = 0; j < nbk; ++j) {
    if (threadIdx.x == 0) {
      double d = s[j][j];
      if (!(d > thresh)) {
        atomicCAS(status, 0, (int)DEV_METRIC_NOT_PD);
        d = fmax(thresh, 1e-300);
      }
      s[j][j] = sqrt(d);
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < nbk; i += blockDim.x) s[i][j] /= s[j][j];
    __syncthreads();
    int rem = nbk - j - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      int i = j + 1 + e / rem, k = j + 1 + e % rem;
      if (k <= i) s[i][k] -= s[i][j] * s[k][j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nbk * nbk; e += blockDim.x) {
    int i = e / nbk, j = e % nbk;
    G[(long long)(k0 + i) * n + k0 + j] = (j <= i) ? s[i][j] : 0.0;
  }
}

// L21 = A21 L11^-T for the rows below the diagonal block (one thread per row).
__global__ void trsm_panel_kernel(int n, double* G, int k0, int nbk) {
  __shared__ double L[CH_NB][CH_NB + 1];
  for (int e = threadIdx.x; e < nbk * nbk; e += blockDim.x) {
    int i = e / nbk, j = e % nbk;
    L[i][j] = G[(long long)(k0 + i) * n + k0 + j];
  }
  __syncthreads();
  int r = k0 + nbk + blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double* row = G + (long long)r * n + k0;
  for (int j = 0; j < nbk; ++j) {
    double x = row[j];
    for (int i = 0; i < j; ++i) x -= row[i] * L[j][i];
    row[j] = x / L[j][j];
  }
}

__global__ void zero_upper_kernel(int n, double* G) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  int i = (int)(idx / n), j = (int)(idx % n);
  if (j > i) G[idx] = 0.0;
}

// Solve L X = R in place for rows [i0, i0+nbk) of R (one thread per column):
// X_m = (R_m - sum_{j<m} L_{m j} X_j) / L_{m m} with the diagonal block of L
// staged in shared memory.
__global__ void trsm_rows_kernel(int nx, const double* L, double* R, long long ncol, int i0, int nbk) {
  __shared__ double Ls[CH_NB][CH_NB + 1];
  for (int e = threadIdx.x; e < nbk * nbk; e += blockDim.x) {
    int i = e / nbk, j = e % nbk;
    Ls[i][j] = L[(long long)(i0 + i) * nx + i0 + j];
  }
  __syncthreads();
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= ncol) return;
  double* col = R + (long long)i0 * ncol + c;
  for (int m = 0; m < nbk; ++m) {
    double x = col[(long long)m * ncol];
    for (int j = 0; j < m; ++j) x -= Ls[m][j] * col[(long long)j * ncol];
    col[(long long)m * ncol] = x / Ls[m][m];
  }
}

// A = L L^T in place for a symmetric positive definite n x n A (row-major; lower
// factor, upper triangle zeroed).  maxdiag: one device double of scratch.  A pivot
// below rel_min * max A_kk sets DEV_METRIC_NOT_PD in the context's status word.
int cholesky_lower(donof_ri_ctx* ctx, double* A, int n, double* maxdiag, double rel_min) {
  max_diag_kernel<<<1, 256, 0, ctx->stream>>>(n, A, maxdiag);
  DONOF_LAUNCH_CHECK(ctx);
  for (int k0 = 0; k0 < n; k0 += CH_NB) {
    int nbk = n - k0 < CH_NB ? n - k0 : CH_NB;
    potrf_block_kernel<<<1, 256, 0, ctx->stream>>>(n, A, k0, nbk, maxdiag, rel_min, ctx->d_status);
    DONOF_LAUNCH_CHECK(ctx);
    int rows = n - k0 - nbk;
    if (rows <= 0) break;
    trsm_panel_kernel<<<ceil_div_u(rows, 128), 128, 0, ctx->stream>>>(n, A, k0, nbk);
    DONOF_LAUNCH_CHECK(ctx);
    Gemm64 g{};
    g.M = rows; g.N = rows; g.K = nbk; g.batch = 1;
    g.A = A + (long long)(k0 + nbk) * n + k0; g.sAm = n; g.sAk = 1;
    g.B = A + (long long)(k0 + nbk) * n + k0; g.sBk = 1; g.sBn = n;
    g.C = A + (long long)(k0 + nbk) * n + (k0 + nbk); g.sCm = n; g.sCn = 1;
    g.alpha = -1.0; g.beta = 1.0;
    int rc = launch_dgemm(ctx, g);
    if (rc) return rc;
  }
  zero_upper_kernel<<<ceil_div_u((long long)n * n, 256), 256, 0, ctx->stream>>>(n, A);
  DONOF_LAUNCH_CHECK(ctx);
  return DONOF_RI_OK;
}

// R <- L^-1 R for a lower-triangular n x n L (row-major, zero upper triangle) and an
// n x ncol row-major R: forward substitution over row blocks of R.
int forward_subst(donof_ri_ctx* ctx, const double* L, int n, double* R, long long ncol) {
  for (int i0 = 0; i0 < n; i0 += CH_NB) {
    int nbk = n - i0 < CH_NB ? n - i0 : CH_NB;
    if (i0 > 0) {
      // N can exceed the grid limit in x only for ncol > 4e9; never for supported sizes.
      Gemm64 g{};
      g.M = nbk; g.N = (int)ncol; g.K = i0; g.batch = 1;
      g.A = L + (long long)i0 * n; g.sAm = n; g.sAk = 1;
      g.B = R; g.sBk = ncol; g.sBn = 1;
      g.C = R + (long long)i0 * ncol; g.sCm = ncol; g.sCn = 1;
      g.alpha = -1.0; g.beta = 1.0;
      int rc = launch_dgemm(ctx, g);
      if (rc) return rc;
    }
    trsm_rows_kernel<<<ceil_div_u(ncol, 128), 128, 0, ctx->stream>>>(n, L, R, ncol, i0, nbk);
    DONOF_LAUNCH_CHECK(ctx);
  }
  return DONOF_RI_OK;
}

int setup_cholesky_and_fit(donof_ri_ctx* ctx) {
  int rc = cholesky_lower(ctx, ctx->d_G, ctx->naux, ctx->d_scratch_max, 1e-14);
  if (rc) return rc;
  return fit_forward(ctx);
}

void max_diag_public(donof_ri_ctx* ctx, const double* G, double* out) {
  max_diag_kernel<<<1, 256, 0, ctx->stream>>>(ctx->naux, G, out);
  ctx->launches++;
}

// B <- L^-1 B for the lower-triangular L in ctx->d_G (row-major, zero upper
// triangle): forward substitution over row blocks of B.
int fit_forward(donof_ri_ctx* ctx) {
  return forward_subst(ctx, ctx->d_G, ctx->naux, ctx->d_B, (long long)ctx->nbf * ctx->nbf);
}

}  // namespace donof
