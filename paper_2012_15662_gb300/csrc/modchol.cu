// Modified Cholesky factorisation of the Coulomb metric and the fit it defines
// (Sec. 2, "Occupancy Optimization with RI"), FP64 on the device:
//   G = P L D L^T P^T       Bunch-Kaufman partial pivoting (alpha = (1 + sqrt 17) / 8),
//                           L unit lower triangular, D with 1x1 and 2x2 blocks;
//   D -> D~                 every eigenvalue of a block below delta = tol max_k G_kk
//                           raised to delta (Cheng-Higham);
//   P L D~^(1/2) b^T = (mu nu|k)   b^T = D~^(-1/2) L^-1 P^T (mu nu|k), D~^(-1/2) the
//                           symmetric inverse square root of each block.
//
// The factorisation is right-looking, one pivot step per pair of launches: a
// one-CTA kernel chooses the pivot, interchanges, writes D's block and L's
// column(s) and keeps the pivot column(s) aside; a grid kernel applies the rank-1
// or rank-2 update to the trailing matrix.  The step counter lives on the
// device (a 2x2 pivot consumes two columns), so the host issues n step pairs
// and the surplus ones return at once.  G is kept as a full symmetric row-major
// matrix; the strict lower triangle ends up holding L.
#include "common.cuh"

#include <math.h>

namespace donof {

int fit_forward(donof_ri_ctx* ctx);  // setup64.cu: B <- L^-1 B by blocked forward substitution

struct BkState {
  int k;        // next column to eliminate
  int k_prev;   // column of the step just taken
  int size;     // its pivot size (0: no step)
  int n2x2;     // 2x2 pivots taken
  int nswap;    // interchanges made
  int nraised;  // eigenvalues raised by the correction
};

constexpr double BK_ALPHA = 0.6403882032022076;  // (1 + sqrt(17)) / 8

// Block-wide arg-max of v over the CTA (smallest index among equal maxima).
__device__ void block_argmax(double& v, int& idx, double* sv, int* si) {
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32, nw = blockDim.x / 32;
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, v, o);
    const int oi = __shfl_down_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  if (lane == 0) { sv[w] = v; si[w] = idx; }
  __syncthreads();
  if (w == 0) {
    v = lane < nw ? sv[lane] : -1.0;
    idx = lane < nw ? si[lane] : 0x7fffffff;
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, v, o);
      const int oi = __shfl_down_sync(0xffffffffu, idx, o);
      if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    if (lane == 0) { sv[0] = v; si[0] = idx; }
  }
  __syncthreads();
  v = sv[0];
  idx = si[0];
  __syncthreads();
}

// One pivot step (one CTA).  acol[0..n) and acol[n..2n) receive the pivot
// column(s) before they are overwritten by L; dd / de / bsz describe D's blocks.
__global__ void __launch_bounds__(1024) bk_pivot_kernel(int n, double* A, int* perm, BkState* st, double* acol,
                                                        double* dd, double* de, int* bsz) {
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int s_size, s_piv;
  const int k = st->k;
  if (k >= n) {
    __syncthreads();
    if (threadIdx.x == 0) st->size = 0;
    return;
  }
  // largest off-diagonal element of column k
  double v = -1.0;
  int idx = 0x7fffffff;
  for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
    const double a = fabs(A[(size_t)i * n + k]);
    if (a > v) { v = a; idx = i; }
  }
  block_argmax(v, idx, sv, si);
  const double colmax = k + 1 < n ? v : 0.0;
  const int imax = k + 1 < n ? idx : k;
  const double akk = fabs(A[(size_t)k * n + k]);
  int size = 1, piv = k;
  if (!(fmax(akk, colmax) == 0.0 || akk >= BK_ALPHA * colmax)) {
    // largest off-diagonal element of row / column imax in the active matrix
    double r = -1.0;
    int ri = 0;
    for (int j = k + threadIdx.x; j < n; j += blockDim.x) {
      if (j == imax) continue;
      const double a = j < imax ? fabs(A[(size_t)imax * n + j]) : fabs(A[(size_t)j * n + imax]);
      if (a > r) { r = a; ri = j; }
    }
    block_argmax(r, ri, sv, si);
    const double rowmax = r;
    if (akk * rowmax >= BK_ALPHA * colmax * colmax) {
      size = 1; piv = k;
    } else if (fabs(A[(size_t)imax * n + imax]) >= BK_ALPHA * rowmax) {
      size = 1; piv = imax;
    } else {
      size = 2; piv = imax;
    }
  }
  if (threadIdx.x == 0) { s_size = size; s_piv = piv; }
  __syncthreads();
  size = s_size;
  piv = s_piv;
  // symmetric interchange of r (k or k + 1) and piv: whole rows (this also swaps the
  // finished rows of L), then the columns of the active rows
  const int r = size == 1 ? k : k + 1;
  if (piv != r) {
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const double t = A[(size_t)r * n + c];
      A[(size_t)r * n + c] = A[(size_t)piv * n + c];
      A[(size_t)piv * n + c] = t;
    }
    __syncthreads();
    for (int row = k + threadIdx.x; row < n; row += blockDim.x) {
      const double t = A[(size_t)row * n + r];
      A[(size_t)row * n + r] = A[(size_t)row * n + piv];
      A[(size_t)row * n + piv] = t;
    }
    if (threadIdx.x == 0) {
      const int t = perm[r];
      perm[r] = perm[piv];
      perm[piv] = t;
    }
    __syncthreads();
  }
  if (size == 1) {
    const double d = A[(size_t)k * n + k];
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
      const double a = A[(size_t)i * n + k];
      acol[i] = a;
      A[(size_t)i * n + k] = d != 0.0 ? a / d : 0.0;
    }
    if (threadIdx.x == 0) {
      dd[k] = d;
      de[k] = 0.0;
      bsz[k] = 1;
    }
  } else {
    const double e00 = A[(size_t)k * n + k], e10 = A[(size_t)(k + 1) * n + k], e11 = A[(size_t)(k + 1) * n + k + 1];
    const double det = e00 * e11 - e10 * e10;  // < 0: a 2x2 pivot is indefinite
    for (int i = k + 2 + threadIdx.x; i < n; i += blockDim.x) {
      const double c0 = A[(size_t)i * n + k], c1 = A[(size_t)i * n + k + 1];
      acol[i] = c0;
      acol[n + i] = c1;
      A[(size_t)i * n + k] = (c0 * e11 - c1 * e10) / det;
      A[(size_t)i * n + k + 1] = (c1 * e00 - c0 * e10) / det;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      dd[k] = e00;
      dd[k + 1] = e11;
      de[k] = e10;
      de[k + 1] = 0.0;
      bsz[k] = 2;
      bsz[k + 1] = 0;
      A[(size_t)(k + 1) * n + k] = 0.0;  // L is the identity inside the block
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st->k_prev = k;
    st->size = size;
    st->k = k + size;
    st->n2x2 += size == 2;
    st->nswap += piv != r;
  }
}

// Trailing update of the step just taken: A_ij -= sum_t L_{i,k+t} a_{j,t} for
// i, j >= k + size.  The grid covers rows / columns from j_lo, a lower bound
// the host knows (the step index + 1).
__global__ void bk_update_kernel(int n, double* A, const BkState* st, const double* acol, int j_lo) {
  const int s = st->size;
  if (s == 0) return;
  const int k = st->k_prev, j0 = k + s;
  const int i = j_lo + blockIdx.y * 16 + threadIdx.y;
  const int j = j_lo + blockIdx.x * 16 + threadIdx.x;
  if (i < j0 || j < j0 || i >= n || j >= n) return;
  double* a = A + (size_t)i * n;
  double v = a[j] - a[k] * acol[j];
  if (s == 2) v -= a[k + 1] * acol[n + j];
  a[j] = v;
}

// Cheng-Higham correction and the blocks of D~^(-1/2): for a 1x1 block
// m00 = max(d, delta)^(-1/2); for a 2x2 block [[a, b], [b, c]] the Jacobi
// rotation J = [[cs, sn], [-sn, cs]] with J^T D J = diag(a - t b, c + t b) gives
// M = J diag(mu1, mu2) J^T, mu = max(lambda, delta)^(-1/2).
__global__ void ch_blocks_kernel(int n, const double* dd, const double* de, const int* bsz, const double* maxdiag,
                                 double tol, double* m00, double* m01, double* m11, BkState* st) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n || bsz[k] == 0) return;
  const double delta = tol * (*maxdiag);
  int raised = 0;
  if (bsz[k] == 1) {
    double lam = dd[k];
    if (!(lam >= delta)) { lam = delta; raised = 1; }
    m00[k] = 1.0 / sqrt(lam);
    m01[k] = 0.0;
    m11[k] = 0.0;
  } else {
    const double a = dd[k], b = de[k], c = dd[k + 1];
    double t = 0.0;
    if (b != 0.0) {
      const double th = (c - a) / (2.0 * b);
      t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
    }
    const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
    double l1 = a - t * b, l2 = c + t * b;
    if (!(l1 >= delta)) { l1 = delta; ++raised; }
    if (!(l2 >= delta)) { l2 = delta; ++raised; }
    const double mu1 = 1.0 / sqrt(l1), mu2 = 1.0 / sqrt(l2);
    m00[k] = cs * cs * mu1 + sn * sn * mu2;
    m01[k] = cs * sn * (mu2 - mu1);
    m11[k] = sn * sn * mu1 + cs * cs * mu2;
  }
  if (raised) atomicAdd(&st->nraised, raised);
}

// R[i] = X[perm[i]] (rows of ncol elements).
__global__ void gather_rows_kernel(int nrows, long long ncol, const int* perm, const double* X, double* R) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)nrows * ncol) return;
  const int i = (int)(e / ncol);
  const long long c = e % ncol;
  R[e] = X[(long long)perm[i] * ncol + c];
}

// Unit diagonal, zero upper triangle: the strict lower triangle is L.
__global__ void unit_lower_kernel(int n, double* A) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  if (j > i) A[e] = 0.0;
  else if (j == i) A[e] = 1.0;
}

// Rows of R times D~^(-1/2): a 2x2 block mixes its two rows.
__global__ void apply_dmh_kernel(int n, long long ncol, const int* bsz, const double* m00, const double* m01,
                                 const double* m11, double* R) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)n * ncol) return;
  const int k = (int)(e / ncol);
  const long long c = e % ncol;
  if (bsz[k] == 1) {
    R[e] *= m00[k];
  } else if (bsz[k] == 2) {
    const double x0 = R[e], x1 = R[e + ncol];
    R[e] = m00[k] * x0 + m01[k] * x1;
    R[e + ncol] = m01[k] * x0 + m11[k] * x1;
  }
}

__global__ void iota_kernel(int n, int* p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = i;
}

int setup_modified_and_fit(donof_ri_ctx* ctx, double tol) {
  const int n = ctx->naux;
  const long long nb2 = (long long)ctx->nbf * ctx->nbf;
  cudaStream_t s = ctx->stream;
  double* G = ctx->d_G;
  // scratch: state, perm, bsz (ints); pivot columns, dd, de, m00, m01, m11 (doubles)
  BkState* st = nullptr;
  int *perm = nullptr, *bsz = nullptr;
  double* work = nullptr;
  double* R = nullptr;
  int rc = DONOF_RI_OK;
  if (cudaMalloc((void**)&st, sizeof(BkState)) != cudaSuccess || cudaMalloc((void**)&perm, n * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&bsz, n * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&work, 7 * (size_t)n * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&R, (size_t)n * nb2 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    rc = DONOF_RI_E_OOM;
  }
  double *acol = work, *dd = work + 2 * n, *de = work + 3 * n, *m00 = work + 4 * n, *m01 = work + 5 * n,
         *m11 = work + 6 * n;
  if (!rc) {
    do {
      if (cudaMemsetAsync(st, 0, sizeof(BkState), s) != cudaSuccess) { rc = DONOF_RI_E_CUDA; break; }
      iota_kernel<<<ceil_div_u(n, 256), 256, 0, s>>>(n, perm);
      if (cudaGetLastError() != cudaSuccess) { rc = DONOF_RI_E_CUDA; break; }
      ctx->launches++;
      max_diag_public(ctx, G, ctx->d_scratch_max);
      for (int it = 0; it < n && !rc; ++it) {
        bk_pivot_kernel<<<1, 1024, 0, s>>>(n, G, perm, st, acol, dd, de, bsz);
        const int lo = it + 1, span = n - lo;
        if (span > 0) {
          dim3 g(ceil_div_u(span, 16), ceil_div_u(span, 16)), b(16, 16);
          bk_update_kernel<<<g, b, 0, s>>>(n, G, st, acol, lo);
        }
        if (cudaGetLastError() != cudaSuccess) rc = DONOF_RI_E_CUDA;
        ctx->launches += span > 0 ? 2 : 1;
      }
      if (rc) break;
      ch_blocks_kernel<<<ceil_div_u(n, 256), 256, 0, s>>>(n, dd, de, bsz, ctx->d_scratch_max, tol, m00, m01, m11, st);
      unit_lower_kernel<<<ceil_div_u((long long)n * n, 256), 256, 0, s>>>(n, G);
      gather_rows_kernel<<<ceil_div_u((long long)n * nb2, 256), 256, 0, s>>>(n, nb2, perm, ctx->d_B, R);
      if (cudaGetLastError() != cudaSuccess) { rc = DONOF_RI_E_CUDA; break; }
      ctx->launches += 3;
      // the permuted rows become the tensor that the forward substitution overwrites
      double* old = ctx->d_B;
      ctx->d_B = R;
      R = old;
      if ((rc = fit_forward(ctx))) break;
      apply_dmh_kernel<<<ceil_div_u((long long)n * nb2, 256), 256, 0, s>>>(n, nb2, bsz, m00, m01, m11, ctx->d_B);
      if (cudaGetLastError() != cudaSuccess) { rc = DONOF_RI_E_CUDA; break; }
      ctx->launches++;
      BkState h;
      if (cudaMemcpyAsync(&h, st, sizeof(BkState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        rc = DONOF_RI_E_CUDA;
        break;
      }
      ctx->metric_info[0] = h.n2x2;
      ctx->metric_info[1] = h.nraised;
      ctx->metric_info[2] = h.nswap;
    } while (0);
  }
  cudaStreamSynchronize(s);
  if (st) cudaFree(st);
  if (perm) cudaFree(perm);
  if (bsz) cudaFree(bsz);
  if (work) cudaFree(work);
  if (R) cudaFree(R);
  return rc;
}

}  // namespace donof
