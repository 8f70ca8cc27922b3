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
// Device plan (nbf <= 160; larger bases: the block Jacobi further down): one CTA
// holds F^lambda and the accumulated rotation in shared memory (FP32) and
// diagonalises by cyclic Jacobi with round-robin pair
// ordering (every round rotates nbf/2 disjoint pairs: columns, then rows); the
// rotation is kept as X = V - I so that small rotations keep their relative
// precision.  The eigenvectors, sorted by eigenvalue, are then refined in FP64
// (orthonormalisation and two first-order corrections against F^lambda in FP64),
// C U is formed in FP64 and one Newton-Schulz step in the overlap metric restores
// C^T S C = I to FP64 rounding (the orbitals are orthonormal functions).
#include "common.cuh"

#include <math.h>
#include <string.h>

namespace donof {

constexpr int FL_MAXN = 160;

// Sort key of an eigenvalue: NaN orders last, so that the ranks stay a permutation.
__device__ __forceinline__ float fl_key(float x) { return x == x ? x : INFINITY; }

// With Fsrc set, the matrix is Fsrc (FP64, row-major, symmetric) instead of F^lambda
// (lam, dprev, first, bound and gmax are then unused): the general symmetric
// eigensolver of eigh_sym.
__global__ void __launch_bounds__(1024, 1) flambda_jacobi_kernel(int n, const double* lam, const double* dprev,
                                                                 int first, double bound, double* U, double* eps,
                                                                 double* gmax, int* sweeps_out,
                                                                 const double* Fsrc) {
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
    if (Fsrc) {
      v = (float)Fsrc[e];
    } else if (q == p) {
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
  if (tid == 0 && gmax && !Fsrc) {
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
    const float ei = fl_key(A[tid * ld + tid]);
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const float ej = fl_key(A[j * ld + j]);
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
// (|A'_qp| > |A'_pp - A'_qq| / 100) K_qp = 0: any basis of a (nearly) degenerate
// pair is an eigenbasis to that accuracy, and bounding every K_qp by 1/100 keeps
// the norm of K small even inside a cluster of close eigenvalues (U (I + K) is
// orthonormal to O(|K|^2), which the Newton-Schulz steps then remove).
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
  K[e] = fabs(a) * 100.0 < fabs(gap) ? a / gap : 0.0;
}

__global__ void fl_add_kernel(long long n, const double* X, double* Y) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) Y[i] += X[i];
}

// ---------------------------------------------------------------------------
// nbf > 160: two-sided block Jacobi on global memory (FP32, L2-resident).  The
// index range is cut into blocks of FLB = 32 (padded with zero rows and columns to
// an even count nbk; a zero row never rotates with a real one).  A sweep pairs
// every two blocks once, round-robin (nbk - 1 rounds of nbk / 2 disjoint pairs);
// in a round one CTA per pair gathers its 64 x 64 sub-problem and runs one cyclic
// Jacobi sweep on it, keeping its rotation Q as D = Q - I, and one CTA per
// (row group, column group) tile then applies A <- Q_g^T A Q_h and
// X <- X Q_h + [g = h] D_h, X = V - I.  Sweeps repeat until the largest
// off-diagonal element is below 1e-6 of the largest diagonal one (the FP32
// plateau, as on the one-CTA path); the FP64 refinement follows unchanged.
constexpr int FLB = 32, FLB2 = 2 * FLB, FL_LD = FLB2 + 1;

struct FlBig {
  int nbk, np, G;
};
static FlBig fl_big_dims(int n) {
  FlBig d;
  const int nb0 = (n + FLB - 1) / FLB;
  d.nbk = nb0 + (nb0 & 1);
  d.np = d.nbk * FLB;
  d.G = d.nbk / 2;
  return d;
}

// Round-robin (circle method) pairing of nn players: pair k of round r.
__host__ __device__ __forceinline__ void fl_rr_pair(int nn, int r, int k, int& a, int& b) {
  a = k == 0 ? 0 : 1 + ((k - 1 + r) % (nn - 1));
  const int pb = nn - 1 - k;
  b = 1 + ((pb - 1 + r) % (nn - 1));
}

// Global index of local index i (0..63) of the group made of blocks I, J.
__device__ __forceinline__ int fl_gidx(int I, int J, int i) { return (i < FLB ? I : J) * FLB + (i & (FLB - 1)); }

// A (np x np, FP32) from the FP64 F^lambda (n x n), zero padding; X = 0.
__global__ void fl_big_init_kernel(int n, int np, const double* Fd, float* A, float* X) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)np * np) return;
  const int i = (int)(e / np), j = (int)(e % np);
  A[e] = (i < n && j < n) ? (float)Fd[(size_t)i * n + j] : 0.f;
  X[e] = 0.f;
}

// max_{q != p} |lambda_qp - lambda_pq| (NaN entries ignored, as fmax does) as the
// bit pattern of a non-negative double (ordered like the value).
__global__ void fl_big_gmax_kernel(int n, const double* lam, unsigned long long* gbits) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int q = (int)(e / n), p = (int)(e % n);
  if (q <= p) return;
  const double a = fabs(lam[(size_t)p * n + q] - lam[(size_t)q * n + p]);
  if (a == a) atomicMax(gbits, (unsigned long long)__double_as_longlong(a));
}

// conv[0] = max off-diagonal |A_ij|, conv[1] = max |A_ii| over the real n x n block
// (FP32 bit patterns of non-negative values; zeroed before the launch).
__global__ void fl_big_conv_kernel(int n, int np, const float* A, unsigned int* conv) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  float off = 0.f, dia = 0.f;
  if (e < (long long)n * n) {
    const int i = (int)(e / n), j = (int)(e % n);
    const float a = fabsf(A[(size_t)i * np + j]);
    if (a == a) {
      if (i == j) dia = a;
      else off = a;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    off = fmaxf(off, __shfl_xor_sync(0xffffffffu, off, o));
    dia = fmaxf(dia, __shfl_xor_sync(0xffffffffu, dia, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(conv, __float_as_uint(off));
    atomicMax(conv + 1, __float_as_uint(dia));
  }
}

// One CTA per pair of blocks (I, J) of round r: one cyclic Jacobi sweep on the
// 64 x 64 sub-problem in shared memory (the same rotation formula and noise skip
// as the one-CTA path, md = the largest diagonal element of the last check); its
// rotation, kept as D = Q - I, goes to Dg[k].
__global__ void __launch_bounds__(256) fl_big_sub_kernel(int np, int nbk, int r, const float* A,
                                                         const unsigned int* conv, float* Dg) {
  __shared__ float S[FLB2][FL_LD], D[FLB2][FL_LD];
  __shared__ float cs[FLB], sn[FLB], cm1[FLB];
  __shared__ int pp[FLB], qq[FLB];
  const int k = blockIdx.x, tid = threadIdx.x;
  int I, J;
  fl_rr_pair(nbk, r, k, I, J);
  for (int e = tid; e < FLB2 * FLB2; e += blockDim.x) {
    const int i = e / FLB2, j = e % FLB2;
    S[i][j] = A[(size_t)fl_gidx(I, J, i) * np + fl_gidx(I, J, j)];
    D[i][j] = 0.f;
  }
  const float md = __uint_as_float(conv[1]);
  __syncthreads();
  for (int lr = 0; lr < FLB2 - 1; ++lr) {
    if (tid < FLB) {
      int a, b;
      fl_rr_pair(FLB2, lr, tid, a, b);
      const int p = a < b ? a : b, q = a < b ? b : a;
      float c = 1.f, s = 0.f, c1 = 0.f;
      const float apq = S[p][q];
      if (fabsf(apq) > 1e-8f * md) {
        const float th = (S[q][q] - S[p][p]) / (2.f * apq);
        const float t = fabsf(th) > 1e18f ? 0.5f / th : (th >= 0.f ? 1.f : -1.f) / (fabsf(th) + sqrtf(th * th + 1.f));
        c = 1.f / sqrtf(t * t + 1.f);
        s = t * c;
        c1 = -(s * s) / (1.f + c);
      }
      pp[tid] = p;
      qq[tid] = q;
      cs[tid] = c;
      sn[tid] = s;
      cm1[tid] = c1;
    }
    __syncthreads();
    for (int e = tid; e < FLB * FLB2; e += blockDim.x) {  // columns p, q of S and D
      const int kk = e / FLB2, i = e % FLB2;
      if (sn[kk] == 0.f) continue;
      const int p = pp[kk], q = qq[kk];
      const float c = cs[kk], s = sn[kk], c1 = cm1[kk];
      const float ap = S[i][p], aq = S[i][q];
      S[i][p] = c * ap - s * aq;
      S[i][q] = s * ap + c * aq;
      const float xp = D[i][p], xq = D[i][q];
      D[i][p] = xp - s * xq + c1 * xp + (i == p ? c1 : 0.f) - (i == q ? s : 0.f);
      D[i][q] = xq + s * xp + c1 * xq + (i == p ? s : 0.f) + (i == q ? c1 : 0.f);
    }
    __syncthreads();
    for (int e = tid; e < FLB * FLB2; e += blockDim.x) {  // rows p, q of S
      const int kk = e / FLB2, j = e % FLB2;
      if (sn[kk] == 0.f) continue;
      const int p = pp[kk], q = qq[kk];
      const float c = cs[kk], s = sn[kk];
      const float ap = S[p][j], aq = S[q][j];
      S[p][j] = c * ap - s * aq;
      S[q][j] = s * ap + c * aq;
    }
    __syncthreads();
  }
  float* out = Dg + (size_t)k * FLB2 * FLB2;
  for (int e = tid; e < FLB2 * FLB2; e += blockDim.x) out[e] = D[e / FLB2][e % FLB2];
}

// One CTA per (row group g, column group h) of round r, each thread a 4 x 4 piece
// of the 64 x 64 tile:  T = A_gh + A_gh D_h,  A_gh <- T + D_g^T T,  and
// X_gh <- X_gh + X_gh D_h + [g = h] D_h.  Each tile is read and written by its own
// CTA only.  Dynamic shared memory: four 64 x 65 FP32 tiles.
constexpr size_t FL_UPDATE_SMEM = 4 * (size_t)FLB2 * FL_LD * sizeof(float);
__global__ void __launch_bounds__(256) fl_big_update_kernel(int np, int nbk, int r, float* A, float* X,
                                                            const float* Dg) {
  extern __shared__ float fl_up[];
  float(*L)[FL_LD] = (float(*)[FL_LD])fl_up;  // the A tile, later the X tile
  float(*Tm)[FL_LD] = L + FLB2;
  float(*Dgs)[FL_LD] = Tm + FLB2;
  float(*Dhs)[FL_LD] = Dgs + FLB2;
  const int g = blockIdx.y, h = blockIdx.x, tid = threadIdx.x;
  int Ig, Jg, Ih, Jh;
  fl_rr_pair(nbk, r, g, Ig, Jg);
  fl_rr_pair(nbk, r, h, Ih, Jh);
  const float* dg = Dg + (size_t)g * FLB2 * FLB2;
  const float* dh = Dg + (size_t)h * FLB2 * FLB2;
  for (int e = tid; e < FLB2 * FLB2; e += blockDim.x) {
    const int i = e / FLB2, j = e % FLB2;
    L[i][j] = A[(size_t)fl_gidx(Ig, Jg, i) * np + fl_gidx(Ih, Jh, j)];
    Dgs[i][j] = dg[e];
    Dhs[i][j] = dh[e];
  }
  __syncthreads();
  const int ty = tid / 16, tx = tid % 16;
  float acc[4][4];
  // T = L + L D_h
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int kk = 0; kk < FLB2; ++kk) {
    float a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = L[ty * 4 + i][kk];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = Dhs[kk][tx * 4 + j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) Tm[ty * 4 + i][tx * 4 + j] = L[ty * 4 + i][tx * 4 + j] + acc[i][j];
  __syncthreads();
  // A_gh = T + D_g^T T; the X tile replaces the A tile in L meanwhile (L is no longer read)
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int kk = 0; kk < FLB2; ++kk) {
    float a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = Dgs[kk][ty * 4 + i];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = Tm[kk][tx * 4 + j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int row = ty * 4 + i, col = tx * 4 + j;
      A[(size_t)fl_gidx(Ig, Jg, row) * np + fl_gidx(Ih, Jh, col)] = Tm[row][col] + acc[i][j];
    }
  for (int e = tid; e < FLB2 * FLB2; e += blockDim.x) {
    const int i = e / FLB2, j = e % FLB2;
    L[i][j] = X[(size_t)fl_gidx(Ig, Jg, i) * np + fl_gidx(Ih, Jh, j)];
  }
  __syncthreads();
  // X_gh = X_gh + X_gh D_h + [g = h] D_h
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int kk = 0; kk < FLB2; ++kk) {
    float a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = L[ty * 4 + i][kk];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = Dhs[kk][tx * 4 + j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int row = ty * 4 + i, col = tx * 4 + j;
      X[(size_t)fl_gidx(Ig, Jg, row) * np + fl_gidx(Ih, Jh, col)] =
          L[row][col] + acc[i][j] + (g == h ? Dhs[row][col] : 0.f);
    }
}

// perm[rank] = i, the real diagonal elements in increasing order (ties by index).
__global__ void fl_big_rank_kernel(int n, int np, const float* A, int* perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float ei = fl_key(A[(size_t)i * np + i]);
  int rank = 0;
  for (int j = 0; j < n; ++j) {
    const float ej = fl_key(A[(size_t)j * np + j]);
    rank += (ej < ei || (ej == ei && j < i)) ? 1 : 0;
  }
  perm[rank] = i;
}

// U[i][k] = [i = perm_k] + X[i][perm_k] (FP64, row-major n x n), eps_k = A[perm_k][perm_k].
__global__ void fl_big_fill_kernel(int n, int np, const float* A, const float* X, const int* perm, double* U,
                                   double* eps) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e / n), k = (int)(e % n);
  const int j = perm[k];
  U[e] = (i == j ? 1.0 : 0.0) + (double)X[(size_t)i * np + j];
  if (i == 0) eps[k] = (double)A[(size_t)j * np + j];
}

size_t flambda_scratch_doubles(int n) {
  size_t s = 6 * (size_t)n * n + (size_t)n + 2;
  if (n > FL_MAXN) {
    const FlBig d = fl_big_dims(n);
    // A, X (np^2 floats each), D (G x 64 x 64 floats), conv (2 uint), gmax bits
    // (1 u64), perm (n int)
    const size_t bytes = 8 * (size_t)d.np * d.np + 4 * (size_t)d.G * FLB2 * FLB2 + 8 + 8 + 4 * (size_t)n;
    s += (bytes + 15) / 8;
  }
  return s;
}

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
// FP64 matrix Fd (orth: two Newton-Schulz steps); eps <- the refined eigenvalues.
// T, W, Z, K: n x n scratch.
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
    // U (I + K) is off orthonormality by O(|K|^2); two Newton-Schulz steps bring
    // that to FP64 rounding
    for (int ns = 0; ns < (pass > 0 ? 2 : 1); ++ns) {
      if ((rc = fl_mm(ctx, n, U, true, U, false, W, 1.0, 0.0))) return rc;    // W = U^T U
      fl_identity_axpy_kernel<<<nblk, 256, 0, ctx->stream>>>(n, 1.5, -0.5, W, Z);
      DONOF_LAUNCH_CHECK(ctx);
      if ((rc = fl_mm(ctx, n, U, false, Z, false, T, 1.0, 0.0))) return rc;   // T = U Z
      DONOF_CUDA_TRY(cudaMemcpyAsync(U, T, n2 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    }
  }
  return DONOF_RI_OK;
}

// Two-sided block Jacobi on the FP64 symmetric matrix Fd (n > FL_MAXN), FP32 on global
// memory, its buffers after the FP64 scratch; U (row-major, columns the eigenvectors in
// increasing order of eigenvalue) and eps.  With lam, the gradient norm max|lambda -
// lambda^T| goes to gm.  Returns the number of sweeps (or a negative status).
static int fl_big_solve(donof_ri_ctx* ctx, int n, const double* Fd, const double* lam, double* scratch, double* U,
                        double* eps, double* gm) {
  const long long n2 = (long long)n * n;
  const unsigned nblk = ceil_div_u(n2, 256);
  const FlBig d = fl_big_dims(n);
  char* base = (char*)(scratch + 6 * n2 + n + 2);
  float* A = (float*)base;
  float* X = A + (size_t)d.np * d.np;
  float* Dg = X + (size_t)d.np * d.np;
  unsigned int* conv = (unsigned int*)(Dg + (size_t)d.G * FLB2 * FLB2);
  unsigned long long* gbits = (unsigned long long*)(conv + 2);
  int* perm = (int*)(gbits + 1);
  if (cudaFuncSetAttribute(fl_big_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)FL_UPDATE_SMEM) != cudaSuccess)
    return DONOF_RI_E_CUDA;
  const long long np2 = (long long)d.np * d.np;
  DONOF_CUDA_TRY(cudaMemsetAsync(gbits, 0, sizeof(unsigned long long), ctx->stream));
  if (lam) {
    fl_big_gmax_kernel<<<nblk, 256, 0, ctx->stream>>>(n, lam, gbits);
    DONOF_LAUNCH_CHECK(ctx);
    DONOF_CUDA_TRY(cudaMemcpyAsync(gm, gbits, sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  }
  fl_big_init_kernel<<<ceil_div_u(np2, 256), 256, 0, ctx->stream>>>(n, d.np, Fd, A, X);
  DONOF_LAUNCH_CHECK(ctx);
  int sweep = 0;
  for (; sweep < 30; ++sweep) {
    DONOF_CUDA_TRY(cudaMemsetAsync(conv, 0, 2 * sizeof(unsigned int), ctx->stream));
    fl_big_conv_kernel<<<nblk, 256, 0, ctx->stream>>>(n, d.np, A, conv);
    DONOF_LAUNCH_CHECK(ctx);
    unsigned int hc[2] = {0u, 0u};
    DONOF_CUDA_TRY(cudaMemcpyAsync(hc, conv, sizeof(hc), cudaMemcpyDeviceToHost, ctx->stream));
    DONOF_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    float mo, mdia;
    memcpy(&mo, &hc[0], sizeof(float));
    memcpy(&mdia, &hc[1], sizeof(float));
    if (!(mo > 1e-6f * fmaxf(mdia, 1e-30f))) break;
    for (int r = 0; r < d.nbk - 1; ++r) {
      fl_big_sub_kernel<<<d.G, 256, 0, ctx->stream>>>(d.np, d.nbk, r, A, conv, Dg);
      DONOF_LAUNCH_CHECK(ctx);
      fl_big_update_kernel<<<dim3(d.G, d.G), 256, FL_UPDATE_SMEM, ctx->stream>>>(d.np, d.nbk, r, A, X, Dg);
      DONOF_LAUNCH_CHECK(ctx);
    }
  }
  fl_big_rank_kernel<<<ceil_div_u(n, 256), 256, 0, ctx->stream>>>(n, d.np, A, perm);
  DONOF_LAUNCH_CHECK(ctx);
  fl_big_fill_kernel<<<nblk, 256, 0, ctx->stream>>>(n, d.np, A, X, perm, U, eps);
  DONOF_LAUNCH_CHECK(ctx);
  return sweep;
}

// Eigen-decomposition of a symmetric FP64 matrix F (n x n row-major, n <=
// FLAMBDA_MAX_NBF): U (row-major; column k the eigenvector of the k-th smallest
// eigenvalue eps[k]), by the F^lambda step's solver (FP32 Jacobi, then FP64
// Newton-Schulz and two first-order refinements against F).  U and eps are device
// buffers outside scratch (flambda_scratch_doubles(n) doubles).
int eigh_sym(donof_ri_ctx* ctx, const double* F, int n, double* scratch, double* U_out, double* eps_out,
             int* sweeps) {
  const long long n2 = (long long)n * n;
  double *U = scratch, *T = U + n2, *W = T + n2, *Z = W + n2, *Fd = Z + n2, *K = Fd + n2, *eps = K + n2,
         *gm = eps + n;
  int* sw = (int*)(gm + 1);
  DONOF_CUDA_TRY(cudaMemcpyAsync(Fd, F, n2 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  int big_sweeps = -1;
  if (n <= FL_MAXN) {
    const size_t smem = 2 * (size_t)n * (n + 1) * sizeof(float);
    if (cudaFuncSetAttribute(flambda_jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return DONOF_RI_E_CUDA;
    flambda_jacobi_kernel<<<1, 1024, smem, ctx->stream>>>(n, (const double*)nullptr, (const double*)nullptr, 0, 0.0,
                                                          U, eps, (double*)nullptr, sw, (const double*)Fd);
    DONOF_LAUNCH_CHECK(ctx);
  } else {
    big_sweeps = fl_big_solve(ctx, n, Fd, (const double*)nullptr, scratch, U, eps, gm);
    if (big_sweeps < 0) return big_sweeps;
  }
  int rc;
  if ((rc = eig_refine(ctx, n, Fd, U, T, W, Z, K, eps))) return rc;
  DONOF_CUDA_TRY(cudaMemcpyAsync(U_out, U, n2 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  DONOF_CUDA_TRY(cudaMemcpyAsync(eps_out, eps, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  if (sweeps) {
    int hs = 0;
    if (big_sweeps < 0) {
      DONOF_CUDA_TRY(cudaMemcpyAsync(&hs, sw, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      DONOF_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    }
    *sweeps = big_sweeps >= 0 ? big_sweeps : hs;
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
  fl_build_f64_kernel<<<nblk, 256, 0, ctx->stream>>>(n, ctx->d_lambda, dprev, first, bound, Fd);
  DONOF_LAUNCH_CHECK(ctx);
  int big_sweeps = -1;
  if (n <= FL_MAXN) {
    const size_t smem = 2 * (size_t)n * (n + 1) * sizeof(float);
    if (cudaFuncSetAttribute(flambda_jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return DONOF_RI_E_CUDA;
    flambda_jacobi_kernel<<<1, 1024, smem, ctx->stream>>>(n, ctx->d_lambda, dprev, first, bound, U, eps, gm, sw,
                                                          (const double*)nullptr);
    DONOF_LAUNCH_CHECK(ctx);
  } else {
    big_sweeps = fl_big_solve(ctx, n, Fd, ctx->d_lambda, scratch, U, eps, gm);
    if (big_sweeps < 0) return big_sweeps;
  }
  int rc;
  if ((rc = eig_refine(ctx, n, Fd, U, T, W, Z, K, eps))) return rc;
  // (C U)^T = U^T C^T, then one Newton-Schulz step in the overlap metric:
  // W = (C U)^T S (C U) = T S T^T (K is free after the refinement)
  if ((rc = fl_mm(ctx, n, U, true, ctx->d_C, false, T, 1.0, 0.0))) return rc;
  if ((rc = fl_mm(ctx, n, ctx->d_S, false, T, true, K, 1.0, 0.0))) return rc;  // K = S T^T
  if ((rc = fl_mm(ctx, n, T, false, K, false, W, 1.0, 0.0))) return rc;        // W = T S T^T
  fl_identity_axpy_kernel<<<nblk, 256, 0, ctx->stream>>>(n, 1.5, -0.5, W, Z);
  DONOF_LAUNCH_CHECK(ctx);
  if ((rc = fl_mm(ctx, n, Z, false, T, false, ctx->d_C, 1.0, 0.0))) return rc;
  double hg = 0.0;
  int hs = 0;
  DONOF_CUDA_TRY(cudaMemcpyAsync(&hg, gm, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  DONOF_CUDA_TRY(cudaMemcpyAsync(&hs, sw, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  DONOF_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  *gmax = hg;
  *sweeps = big_sweeps >= 0 ? big_sweeps : hs;
  return DONOF_RI_OK;
}

}  // namespace donof
