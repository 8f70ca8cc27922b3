// Exact four-centre Coulomb / exchange for small orbital bases (FP64), the
// conventional algorithm that RI replaces (Table 1; Eqs. (Jpq), (Pmat), (Kpq)) and
// that the paper returns to for its RI -> exact restart (Sec. 1 and Sec. 4: a
// calculation converged with RI is finished with a few exact iterations):
//   (mu nu|l s)  exact s-type four-centre integrals, stored as [mu nu][l s]
//   J^(q)_{mu nu} = sum_{l s} (mu nu|l s) C_{l q} C_{s q}
//   K^(q)_{mu nu} = sum_{l s} (mu l|nu s) C_{l q} C_{s q}
//   J_pq = C_p^T J^(q) C_p,  K_pq = C_p^T K^(q) C_p.
// J^(q) is one DGEMM of the stored integrals with the orbital densities; K^(q)
// first contracts s with C (a batched DGEMM over mu) and then l.  The results go
// into an FP64 context's J^(q) / K^(q) and J / K buffers, so that the energy,
// Lagrangian and occupation optimisation calls that follow use exact integrals.
#include "common.cuh"

#include <math.h>

namespace donof {

__device__ __forceinline__ double boys_f0_x(double t) {
  if (t < 1e-8) return 1.0 - t / 3.0 + t * t / 10.0;
  return 0.5 * sqrt(M_PI / t) * erf(sqrt(t));
}

// Gaussian-product data of every orbital pair (a, b): p = a + b, the product
// centre, and N_a N_b exp(-a b |A - B|^2 / p).
__global__ void pairs_kernel(int nbf, const double* xyz, const int* bf_atom, const double* bf_alpha, double* pp,
                             double* pc, double* pk) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)nbf * nbf) return;
  const int i = (int)(idx / nbf), j = (int)(idx % nbf);
  const double a = bf_alpha[i], b = bf_alpha[j];
  const double* A = xyz + 3 * bf_atom[i];
  const double* B = xyz + 3 * bf_atom[j];
  const double p = a + b;
  const double dx = A[0] - B[0], dy = A[1] - B[1], dz = A[2] - B[2];
  const double na = pow(2.0 * a / M_PI, 0.75), nbn = pow(2.0 * b / M_PI, 0.75);
  pp[idx] = p;
  pc[3 * idx] = (a * A[0] + b * B[0]) / p;
  pc[3 * idx + 1] = (a * A[1] + b * B[1]) / p;
  pc[3 * idx + 2] = (a * A[2] + b * B[2]) / p;
  pk[idx] = na * nbn * exp(-a * b / p * (dx * dx + dy * dy + dz * dz));
}

// (ab|cd) = 2 pi^(5/2) / (p q sqrt(p + q)) K_ab K_cd F0(p q / (p + q) |P - Q|^2)
__global__ void eri4_kernel(long long npair, const double* pp, const double* pc, const double* pk, double* eri) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= npair * npair) return;
  const long long u = idx / npair, v = idx % npair;
  const double p = pp[u], q = pp[v];
  const double dx = pc[3 * u] - pc[3 * v], dy = pc[3 * u + 1] - pc[3 * v + 1], dz = pc[3 * u + 2] - pc[3 * v + 2];
  const double pref = 2.0 * pow(M_PI, 2.5) / (p * q * sqrt(p + q));
  eri[idx] = pref * pk[u] * pk[v] * boys_f0_x(p * q / (p + q) * (dx * dx + dy * dy + dz * dz));
}

// Orbital densities D[q][l s] = C_{l q} C_{s q} (C column-major).
__global__ void densities_kernel(int nbf, int m, const double* C, double* D) {
  const long long nb2 = (long long)nbf * nbf;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)m * nb2) return;
  const int q = (int)(idx / nb2);
  const long long r = idx % nb2;
  const int l = (int)(r / nbf), s = (int)(r % nbf);
  D[idx] = C[(size_t)q * nbf + l] * C[(size_t)q * nbf + s];
}

// K^(q)_{mu nu} = sum_l C_{l q} T[mu][l][nu][q], T[mu][l][nu][q] = sum_s (mu l|nu s) C_{s q}.
__global__ void exchange_finish_kernel(int nbf, int m, const double* C, const double* T, double* K) {
  const long long nb2 = (long long)nbf * nbf;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)m * nb2) return;
  const int q = (int)(idx / nb2);
  const long long r = idx % nb2;
  const int mu = (int)(r / nbf), nu = (int)(r % nbf);
  const double* c = C + (size_t)q * nbf;
  double s = 0.0;
  for (int l = 0; l < nbf; ++l) s += c[l] * T[(((size_t)mu * nbf + l) * nbf + nu) * m + q];
  K[idx] = s;
}

// X_pq = sum_mu C_{mu p} W[q][mu][p], W[q][mu][p] = (X^(q) C)_{mu p}; out row-major [p][q].
__global__ void mo_from_ao_kernel(int nbf, int m, const double* C, const double* W, double* out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * m) return;
  const int p = idx / m, q = idx % m;
  const double* c = C + (size_t)p * nbf;
  const double* w = W + (size_t)q * nbf * m;
  double s = 0.0;
  for (int mu = 0; mu < nbf; ++mu) s += c[mu] * w[(size_t)mu * m + p];
  out[(size_t)p * m + q] = s;
}

int exact_jk(donof_ri_ctx* ctx) {
  const int nb = ctx->nbf, m = ctx->n_omega;
  const long long nb2 = (long long)nb * nb;
  cudaStream_t s = ctx->stream;
  double *pp = nullptr, *pc = nullptr, *pk = nullptr, *eri = nullptr, *D = nullptr, *T = nullptr, *W = nullptr;
  int rc = DONOF_RI_OK;
  auto alloc = [&](double** ptr, size_t count) {
    if (!rc && cudaMalloc((void**)ptr, count * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      rc = DONOF_RI_E_OOM;
    }
  };
  alloc(&pp, nb2);
  alloc(&pc, 3 * nb2);
  alloc(&pk, nb2);
  alloc(&eri, (size_t)nb2 * nb2);
  alloc(&D, (size_t)m * nb2);
  alloc(&T, (size_t)nb2 * nb * m);
  alloc(&W, (size_t)m * nb * m);
  do {
    if (rc) break;
    pairs_kernel<<<ceil_div_u(nb2, 256), 256, 0, s>>>(nb, ctx->d_atom_xyz, ctx->d_bf_atom, ctx->d_bf_alpha, pp, pc, pk);
    eri4_kernel<<<ceil_div_u(nb2 * nb2, 256), 256, 0, s>>>(nb2, pp, pc, pk, eri);
    densities_kernel<<<ceil_div_u((long long)m * nb2, 256), 256, 0, s>>>(nb, m, ctx->d_C, D);
    if (cudaGetLastError() != cudaSuccess) { rc = DONOF_RI_E_CUDA; break; }
    ctx->launches += 3;
    // J^(q) [q][mu nu] = D [q][l s] x (l s|mu nu)
    Gemm64 g{};
    g.M = m; g.N = (int)nb2; g.K = (int)nb2; g.batch = 1;
    g.A = D; g.sAm = nb2; g.sAk = 1;
    g.B = eri; g.sBk = nb2; g.sBn = 1;
    g.C = ctx->d_Jao; g.sCm = nb2; g.sCn = 1;
    g.alpha = 1.0; g.beta = 0.0;
    if ((rc = launch_dgemm(ctx, g))) break;
    // T[mu][(l nu)][q] = sum_s (mu l|nu s) C_{s q}, batched over mu
    Gemm64 t{};
    t.M = (int)nb2; t.N = m; t.K = nb; t.batch = nb;
    t.A = eri; t.sAb = nb2 * nb; t.sAm = nb; t.sAk = 1;
    t.B = ctx->d_C; t.sBb = 0; t.sBk = 1; t.sBn = nb;
    t.C = T; t.sCb = nb2 * m; t.sCm = m; t.sCn = 1;
    t.alpha = 1.0; t.beta = 0.0;
    if ((rc = launch_dgemm(ctx, t))) break;
    exchange_finish_kernel<<<ceil_div_u((long long)m * nb2, 256), 256, 0, s>>>(nb, m, ctx->d_C, T, ctx->d_Kao);
    if (cudaGetLastError() != cudaSuccess) { rc = DONOF_RI_E_CUDA; break; }
    ctx->launches++;
    // J_pq, K_pq: W[q][mu][p] = sum_nu X^(q)_{mu nu} C_{nu p}, then the C_p^T contraction
    double* outs[2] = {ctx->d_J, ctx->d_K};
    double* aos[2] = {ctx->d_Jao, ctx->d_Kao};
    for (int k = 0; k < 2 && !rc; ++k) {
      Gemm64 w{};
      w.M = nb; w.N = m; w.K = nb; w.batch = m;
      w.A = aos[k]; w.sAb = nb2; w.sAm = nb; w.sAk = 1;
      w.B = ctx->d_C; w.sBb = 0; w.sBk = 1; w.sBn = nb;
      w.C = W; w.sCb = (long long)nb * m; w.sCm = m; w.sCn = 1;
      w.alpha = 1.0; w.beta = 0.0;
      if ((rc = launch_dgemm(ctx, w))) break;
      mo_from_ao_kernel<<<ceil_div_u((long long)m * m, 256), 256, 0, s>>>(nb, m, ctx->d_C, W, outs[k]);
      if (cudaGetLastError() != cudaSuccess) { rc = DONOF_RI_E_CUDA; break; }
      ctx->launches++;
    }
  } while (0);
  cudaStreamSynchronize(s);
  for (double* b : {pp, pc, pk, eri, D, T, W})
    if (b) cudaFree(b);
  return rc;
}

}  // namespace donof
