// The plain FP64 form of the hot path (CUDA cores, DFMA), and the small
// kernels both precisions share: finiteness check, PNOF7 occupations and
// coupling coefficients, and the final energy reduction.
//
// Paper: Sec. 2, Tables 2 and 3 (RI transforms and J/K builders), Eq. (PNOF)
// (energy), orbital optimisation with RI (lambda).
#include "common.cuh"

namespace donof {

__global__ void check_finite_kernel(const double* x, long long n, int* status) {
  pdl_entry();
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n && !isfinite(x[i])) atomicCAS(status, 0, (int)DEV_NONFINITE);
}

int launch_check_finite(donof_ri_ctx* ctx, const double* x, long long n) {
  launch_pdl(check_finite_kernel, dim3(ceil_div_u(n, 256)), dim3(256), 0, ctx->stream, x, n, ctx->d_status);
  DONOF_LAUNCH_CHECK(ctx);
  return DONOF_RI_OK;
}

// b^P_pp = sum_nu C_{nu p} b^P_{p nu}: one warp per (P, p), lanes over nu.
__global__ void diag64_kernel(int nbf, int naux, int n_om, const double* bh, const double* C, double* d) {
  long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
  int lane = threadIdx.x % 32;
  if (w >= (long long)naux * n_om) return;
  int P = (int)(w / n_om), p = (int)(w % n_om);
  const double* row = bh + ((long long)P * n_om + p) * nbf;
  const double* c = C + (long long)p * nbf;
  double s = 0.0;
  for (int nu = lane; nu < nbf; nu += 32) s = fma(row[nu], c[nu], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) d[w] = s;
}

// K_pq = sum_P (b^P_pq)^2: one thread per (p, q), sequential over P.
__global__ void sqsum64_kernel(int naux, int n_om, const double* bf, double* K) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long m2 = (long long)n_om * n_om;
  if (i >= m2) return;
  double s = 0.0;
  for (int P = 0; P < naux; ++P) {
    double v = bf[(long long)P * m2 + i];
    s = fma(v, v, s);
  }
  K[i] = s;
}

int path64_transform(donof_ri_ctx* ctx, int mode) {
  const int nb = ctx->nbf, nx = ctx->naux, m = ctx->n_omega;
  const long long nb2 = (long long)nb * nb;
  int rc;
  // Table 2/3 step 2: b^P_{p nu} = sum_mu C_{mu p} B^P_{mu nu}
  {
    ProfScope ps(ctx, DONOF_RI_ROW_HALF);
    Gemm64 g{};
    g.M = m; g.N = nb; g.K = nb; g.batch = nx;
    g.A = ctx->d_C; g.sAb = 0; g.sAm = nb; g.sAk = 1;
    g.B = ctx->d_B; g.sBb = nb2; g.sBk = nb; g.sBn = 1;
    g.C = ctx->d_bh; g.sCb = (long long)m * nb; g.sCm = nb; g.sCn = 1;
    g.alpha = 1.0; g.beta = 0.0;
    if ((rc = launch_dgemm(ctx, g))) return rc;
  }
  // Table 3 step 3: b^P_pp
  {
    ProfScope ps(ctx, DONOF_RI_ROW_DIAG);
    diag64_kernel<<<ceil_div_u((long long)nx * m * 32, 256), 256, 0, ctx->stream>>>(nb, nx, m, ctx->d_bh, ctx->d_C,
                                                                                     ctx->d_d);
    DONOF_LAUNCH_CHECK(ctx);
  }
  if (mode == DONOF_RI_FULL) {
    // Table 2 step 3: b^P_pq = sum_nu C_{nu q} b^P_{p nu}
    ProfScope ps(ctx, DONOF_RI_ROW_FULL_K);
    Gemm64 g{};
    g.M = m; g.N = m; g.K = nb; g.batch = nx;
    g.A = ctx->d_bh; g.sAb = (long long)m * nb; g.sAm = nb; g.sAk = 1;
    g.B = ctx->d_C; g.sBb = 0; g.sBk = 1; g.sBn = nb;
    g.C = ctx->d_bf; g.sCb = (long long)m * m; g.sCm = m; g.sCn = 1;
    g.alpha = 1.0; g.beta = 0.0;
    if ((rc = launch_dgemm(ctx, g))) return rc;
    // Table 2 step 4: K_pq = sum_P (b^P_pq)^2
    sqsum64_kernel<<<ceil_div_u((long long)m * m, 256), 256, 0, ctx->stream>>>(nx, m, ctx->d_bf, ctx->d_K);
    DONOF_LAUNCH_CHECK(ctx);
  }
  if (mode == DONOF_RI_FULL) {
    // Table 2 step 4: J_pq = sum_P b^P_pp b^P_qq
    ProfScope ps(ctx, DONOF_RI_ROW_J);
    Gemm64 h{};
    h.M = m; h.N = m; h.K = nx; h.batch = 1;
    h.A = ctx->d_d; h.sAm = 1; h.sAk = m;
    h.B = ctx->d_d; h.sBk = m; h.sBn = 1;
    h.C = ctx->d_J; h.sCm = m; h.sCn = 1;
    h.alpha = 1.0; h.beta = 0.0;
    if ((rc = launch_dgemm(ctx, h))) return rc;
  }
  return DONOF_RI_OK;
}

int path64_jk_ao(donof_ri_ctx* ctx) {
  const int nb = ctx->nbf, nx = ctx->naux, m = ctx->n_omega;
  const long long nb2 = (long long)nb * nb;
  int rc;
  // Table 3 step 4: J^(q)_{mu nu} = sum_P b^P_qq B^P_{mu nu}
  {
    ProfScope ps(ctx, DONOF_RI_ROW_JAO);
    Gemm64 g{};
    g.M = m; g.N = (int)nb2; g.K = nx; g.batch = 1;
    g.A = ctx->d_d; g.sAm = 1; g.sAk = m;
    g.B = ctx->d_B; g.sBk = nb2; g.sBn = 1;
    g.C = ctx->d_Jao; g.sCm = nb2; g.sCn = 1;
    g.alpha = 1.0; g.beta = 0.0;
    if ((rc = launch_dgemm(ctx, g))) return rc;
  }
  // Table 3 step 3 (K): K^(q)_{mu nu} = sum_P b^P_{q mu} b^P_{q nu}
  {
    ProfScope ps(ctx, DONOF_RI_ROW_KAO);
    Gemm64 g{};
    g.M = nb; g.N = nb; g.K = nx; g.batch = m;
    g.A = ctx->d_bh; g.sAb = nb; g.sAm = 1; g.sAk = (long long)m * nb;
    g.B = ctx->d_bh; g.sBb = nb; g.sBk = (long long)m * nb; g.sBn = 1;
    g.C = ctx->d_Kao; g.sCb = nb2; g.sCm = nb; g.sCn = 1;
    g.alpha = 1.0; g.beta = 0.0;
    if ((rc = launch_dgemm(ctx, g))) return rc;
  }
  return DONOF_RI_OK;
}

// ---------------------------------------------------------------------------
// PNOF7 occupations and coupling coefficients (shared by both precisions).
//   n_g = (1 + cos^2 gamma_g)/2, h_g = 1 - n_g, weak n_{g,i} = h_g alpha_i with
//   alpha_i = prod_{j<i} sin^2 gamma_{g,j} cos^2 gamma_{g,i} (last: no cos factor).
//   A_pp = n_p; same subspace p != q: A = 0, B = -Pi_pq (Pi = -sqrt(n_p n_q) if
//   one is strong, +sqrt(n_p n_q) if both weak); different subspaces:
//   A = 2 n_p n_q, B = n_p n_q + Phi_p Phi_q, Phi = sqrt(n (1 - n)).
// ---------------------------------------------------------------------------
__global__ void occupations_kernel(int n_strong, int n_weak_per, int n_om, const int* subspace,
                                   const int* weak_rank, const double* gamma, double* n) {
  pdl_entry();
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_om) return;
  const int g = subspace[p];
  const int r = weak_rank[p];
  const double cg = cos(gamma[g]);
  const double ng = 0.5 * (1.0 + cg * cg);
  if (r < 0) {
    n[p] = ng;
    return;
  }
  double carry = 1.0, alpha = 0.0;
  for (int i = 0; i <= r; ++i) {
    if (i == n_weak_per - 1) {
      alpha = carry;
      break;
    }
    double th = gamma[n_strong + g * (n_weak_per - 1) + i];
    double c = cos(th), sn = sin(th);
    if (i == r) {
      alpha = carry * c * c;
      break;
    }
    carry *= sn * sn;
  }
  n[p] = (1.0 - ng) * alpha;
}

__global__ void coupling_kernel(int n_om, const int* subspace, const int* weak_rank, const double* n, double* A,
                                double* Bc) {
  pdl_entry();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_om * n_om) return;
  int p = i / n_om, q = i % n_om;
  double np_ = n[p], nq = n[q];
  double a = 0.0, b = 0.0;
  if (p == q) {
    a = np_;
  } else if (subspace[p] == subspace[q]) {
    double pi = (weak_rank[p] < 0 || weak_rank[q] < 0) ? -sqrt(np_ * nq) : sqrt(np_ * nq);
    b = -pi;
  } else {
    a = 2.0 * np_ * nq;
    b = np_ * nq + sqrt(np_ * (1.0 - np_)) * sqrt(nq * (1.0 - nq));
  }
  A[i] = a;
  Bc[i] = b;
}

int launch_occupations_coupling(donof_ri_ctx* ctx) {
  const int m = ctx->n_omega;
  launch_pdl(occupations_kernel, dim3(ceil_div_u(m, 128)), dim3(128), 0, ctx->stream, ctx->n_strong, ctx->n_weak_per, m,
             (const int*)ctx->d_subspace, (const int*)ctx->d_weak_rank, (const double*)ctx->d_gamma, ctx->d_n);
  DONOF_LAUNCH_CHECK(ctx);
  launch_pdl(coupling_kernel, dim3(ceil_div_u((long long)m * m, 256)), dim3(256), 0, ctx->stream, m,
             (const int*)ctx->d_subspace, (const int*)ctx->d_weak_rank, (const double*)ctx->d_n, ctx->d_A, ctx->d_Bc);
  DONOF_LAUNCH_CHECK(ctx);
  return DONOF_RI_OK;
}

// Y[mu][p] = n_p (H C)_{mu p} + sum_nu W[p][mu][nu] C_{nu p}: one warp per (mu, p).
__global__ void fock_apply64_kernel(int nbf, int n_om, const double* W, const double* C, const double* HC,
                                    const double* n, double* Y) {
  long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
  int lane = threadIdx.x % 32;
  if (w >= (long long)nbf * n_om) return;
  int p = (int)(w / nbf), mu = (int)(w % nbf);
  const double* row = W + ((long long)p * nbf + mu) * nbf;
  const double* c = C + (long long)p * nbf;
  double s = 0.0;
  for (int nu = lane; nu < nbf; nu += 32) s = fma(row[nu], c[nu], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) Y[(long long)mu * n_om + p] = n[p] * HC[(long long)mu * n_om + p] + s;
}

// E = E_nuc + sum_p (n_p H_pp + lambda_pp), H_pp = sum_mu C_{mu p} (H C)_{mu p}.
// One block; fixed reduction order, so the result is deterministic.
__global__ void energy_reduce_kernel(int nbf, int n_om, const double* C, const double* HC, const double* n,
                                     const double* lambda, const double* enuc, double* E) {
  __shared__ double red[256];
  double s = 0.0;
  for (int p = threadIdx.x; p < n_om; p += blockDim.x) {
    double hpp = 0.0;
    for (int mu = 0; mu < nbf; ++mu) hpp = fma(C[(long long)p * nbf + mu], HC[(long long)mu * n_om + p], hpp);
    s += n[p] * hpp + lambda[(long long)p * nbf + p];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *E = *enuc + red[0];
}

int launch_energy_reduce(donof_ri_ctx* ctx) {
  energy_reduce_kernel<<<1, 256, 0, ctx->stream>>>(ctx->nbf, ctx->n_omega, ctx->d_C, ctx->d_HC, ctx->d_n,
                                                   ctx->d_lambda, ctx->d_enuc, ctx->d_E);
  DONOF_LAUNCH_CHECK(ctx);
  return DONOF_RI_OK;
}

// out[i*so_i + j*so_j] = sum_k A[i*lda + k] B[j*ldb + k] (+ add[i*so_i + j*so_j] * scale[j] when add
// is given), FP64, one warp per output with a fixed shuffle tree (deterministic).  Used for the small
// products of the energy row, where a 64x64-tile GEMM would leave most SMs idle.
__global__ void dot64_kernel(int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* out,
                             long long so_i, long long so_j) {
  pdl_entry();
  long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
  int lane = threadIdx.x % 32;
  if (w >= (long long)M * N) return;
  int i = (int)(w / N), j = (int)(w % N);
  const double* a = A + (long long)i * lda;
  const double* b = B + (long long)j * ldb;
  double s = 0.0;
  for (int k = lane; k < K; k += 32) s = fma(a[k], b[k], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[i * so_i + j * so_j] = s;
}

int launch_dot64(donof_ri_ctx* ctx, int M, int N, int K, const double* A, int lda, const double* B, int ldb,
                 double* out, long long so_i, long long so_j) {
  launch_pdl(dot64_kernel, dim3(ceil_div_u((long long)M * N * 32, 256)), dim3(256), 0, ctx->stream, M, N, K, A, lda, B,
             ldb, out, so_i, so_j);
  DONOF_LAUNCH_CHECK(ctx);
  return DONOF_RI_OK;
}

// E = E_nuc + sum_p (n_p H_pp + lambda_pp) with H_pp = C_p^T (H C)_p taken from HCt[p][mu]
// (rows p, stride nbf).  One block, one warp per p, fixed reduction order.
__global__ void energy_rows_kernel(int nbf, int n_om, const double* C, const double* HCt, const double* n,
                                   const double* lambda, const double* enuc, double* E) {
  pdl_entry();
  __shared__ double part[32];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  double acc = 0.0;
  for (int p = warp; p < n_om; p += 32) {
    const double* c = C + (long long)p * nbf;
    const double* h = HCt + (long long)p * nbf;
    double s = 0.0;
    for (int mu = lane; mu < nbf; mu += 32) s = fma(c[mu], h[mu], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    acc += n[p] * s + lambda[(long long)p * nbf + p];
  }
  if (lane == 0) part[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    double v = part[lane];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) *E = *enuc + v;
  }
}

int launch_energy_rows(donof_ri_ctx* ctx, const double* HCt) {
  launch_pdl(energy_rows_kernel, dim3(1), dim3(1024), 0, ctx->stream, ctx->nbf, ctx->n_omega, (const double*)ctx->d_C,
             HCt, (const double*)ctx->d_n, (const double*)ctx->d_lambda, (const double*)ctx->d_enuc, ctx->d_E);
  DONOF_LAUNCH_CHECK(ctx);
  return DONOF_RI_OK;
}

// HC[mu][p] = sum_nu H_{mu nu} C_{nu p} (p < N_Omega).
static int launch_hc(donof_ri_ctx* ctx) {
  const int nb = ctx->nbf, m = ctx->n_omega;
  Gemm64 g{};
  g.M = nb; g.N = m; g.K = nb; g.batch = 1;
  g.A = ctx->d_H; g.sAm = nb; g.sAk = 1;
  g.B = ctx->d_C; g.sBk = 1; g.sBn = nb;
  g.C = ctx->d_HC; g.sCm = m; g.sCn = 1;
  g.alpha = 1.0; g.beta = 0.0;
  return launch_dgemm(ctx, g);
}

// lambda[p*nbf + q] = sum_mu C_{mu q} Y[mu][p]  (q < nbf, p < N_Omega).
int launch_lambda(donof_ri_ctx* ctx) {
  const int nb = ctx->nbf, m = ctx->n_omega;
  Gemm64 g{};
  g.M = nb; g.N = m; g.K = nb; g.batch = 1;
  g.A = ctx->d_C; g.sAm = nb; g.sAk = 1;
  g.B = ctx->d_Y; g.sBk = m; g.sBn = 1;
  g.C = ctx->d_lambda; g.sCm = 1; g.sCn = nb;
  g.alpha = 1.0; g.beta = 0.0;
  return launch_dgemm(ctx, g);
}

int launch_hc_public(donof_ri_ctx* ctx) { return launch_hc(ctx); }

// ---------------------------------------------------------------------------
// Contracted Lagrangian (FP64): F^(p) C_p straight from the RI transforms, without
// the per-orbital AO matrices.  With w_pP = sum_q A_pq b^P_qq,
//   F^(p) C_p = n_p H C_p + sum_P w_pP b^P_{p .} - sum_P sum_q B_pq b^P_qp b^P_{q .}
//             = n_p H C_p - sum_P sum_q b^P_{q .} X^P_qp,
//   X^P_qp = B_pq b^P_qp - [q = p] w_pP,
// one batched DGEMM over P (per P: N_b x N_Omega x N_Omega) and a fixed-order sum
// over P; then lambda = C^T Y and E as in the per-orbital form.
// ---------------------------------------------------------------------------
__global__ void contract_x_kernel(int naux, int n_om, const double* Bc, const double* bf, const double* w, double* X) {
  pdl_entry();
  const long long m2 = (long long)n_om * n_om;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)naux * m2) return;
  const int P = (int)(idx / m2);
  const long long r = idx % m2;
  const int q = (int)(r / n_om), p = (int)(r % n_om);
  double x = Bc[(long long)p * n_om + q] * bf[idx];
  if (q == p) x -= w[(long long)p * naux + P];
  X[idx] = x;
}

// Y[mu][p] = n_p HC[mu][p] - sum_P Yp[P][mu][p], P in increasing order.
__global__ void contract_sum_kernel(int naux, int nbf, int n_om, const double* Yp, const double* HC, const double* n,
                                    double* Y) {
  pdl_entry();
  const long long nm = (long long)nbf * n_om;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= nm) return;
  double s = 0.0;
  for (int P = 0; P < naux; ++P) s += Yp[(long long)P * nm + idx];
  Y[idx] = n[idx % n_om] * HC[idx] - s;
}

int path64_energy_contracted(donof_ri_ctx* ctx, double* w, double* X, double* Yp) {
  const int nb = ctx->nbf, nx = ctx->naux, m = ctx->n_omega;
  int rc;
  ProfScope ps(ctx, DONOF_RI_ROW_ENERGY);
  if ((rc = launch_occupations_coupling(ctx))) return rc;
  if ((rc = launch_hc(ctx))) return rc;
  // w[p][P] = sum_q A_pq b^P_qq
  Gemm64 g{};
  g.M = m; g.N = nx; g.K = m; g.batch = 1;
  g.A = ctx->d_A; g.sAm = m; g.sAk = 1;
  g.B = ctx->d_d; g.sBk = 1; g.sBn = m;
  g.C = w; g.sCm = nx; g.sCn = 1;
  g.alpha = 1.0; g.beta = 0.0;
  if ((rc = launch_dgemm(ctx, g))) return rc;
  launch_pdl(contract_x_kernel, dim3(ceil_div_u((long long)nx * m * m, 256)), dim3(256), 0, ctx->stream, nx, m,
             (const double*)ctx->d_Bc, (const double*)ctx->d_bf, (const double*)w, X);
  DONOF_LAUNCH_CHECK(ctx);
  // Yp[P][mu][p] = sum_q b^P_{q mu} X^P_qp
  Gemm64 h{};
  h.M = nb; h.N = m; h.K = m; h.batch = nx;
  h.A = ctx->d_bh; h.sAb = (long long)m * nb; h.sAm = 1; h.sAk = nb;
  h.B = X; h.sBb = (long long)m * m; h.sBk = m; h.sBn = 1;
  h.C = Yp; h.sCb = (long long)nb * m; h.sCm = m; h.sCn = 1;
  h.alpha = 1.0; h.beta = 0.0;
  if ((rc = launch_dgemm(ctx, h))) return rc;
  launch_pdl(contract_sum_kernel, dim3(ceil_div_u((long long)nb * m, 256)), dim3(256), 0, ctx->stream, nx, nb, m,
             (const double*)Yp, (const double*)ctx->d_HC, (const double*)ctx->d_n, ctx->d_Y);
  DONOF_LAUNCH_CHECK(ctx);
  if ((rc = launch_lambda(ctx))) return rc;
  return launch_energy_reduce(ctx);
}

int path64_energy(donof_ri_ctx* ctx, int part) {
  const int nb = ctx->nbf, m = ctx->n_omega;
  const long long nb2 = (long long)nb * nb;
  int rc;
  ProfScope ps(ctx, DONOF_RI_ROW_ENERGY);
  if (part & ENERGY_PREP) {
    if ((rc = launch_occupations_coupling(ctx))) return rc;
    if ((rc = launch_hc(ctx))) return rc;
  }
  if (!(part & ENERGY_MAIN)) return DONOF_RI_OK;
  // W[p] = sum_q A_pq J^(q) - B_pq K^(q)
  {
    Gemm64 g{};
    g.M = m; g.N = (int)nb2; g.K = m; g.batch = 1;
    g.A = ctx->d_A; g.sAm = m; g.sAk = 1;
    g.B = ctx->d_Jao; g.sBk = nb2; g.sBn = 1;
    g.C = ctx->d_W; g.sCm = nb2; g.sCn = 1;
    g.alpha = 1.0; g.beta = 0.0;
    if ((rc = launch_dgemm(ctx, g))) return rc;
    g.A = ctx->d_Bc;
    g.B = ctx->d_Kao;
    g.alpha = -1.0; g.beta = 1.0;
    if ((rc = launch_dgemm(ctx, g))) return rc;
  }
  fock_apply64_kernel<<<ceil_div_u((long long)nb * m * 32, 256), 256, 0, ctx->stream>>>(nb, m, ctx->d_W, ctx->d_C,
                                                                                       ctx->d_HC, ctx->d_n, ctx->d_Y);
  DONOF_LAUNCH_CHECK(ctx);
  if ((rc = launch_lambda(ctx))) return rc;
  return launch_energy_reduce(ctx);
}

}  // namespace donof
