// Occupation optimisation for fixed orbitals (Sec. 2, "Occupancy Optimization
// with RI"): J_pq and K_pq of the current orbitals stay fixed while the PNOF7
// energy, Eq. (PNOF), is minimised over the unconstrained angles gamma that
// parametrise the occupations.  The paper names neither the optimiser nor the
// gradient.  Here the gradient is the chain rule
//   dE/dgamma_k = sum_p dE/dn_p dn_p/dgamma_k,
//   dE/dn_p = 2 H_pp + J_pp - sum_{q in g(p), q != p} s_pq K_pq sqrt(n_q / n_p)
//             + sum_{q not in g(p)} (4 n_q J_pq - 2 n_q K_pq - 2 Phi'_p Phi_q K_pq),
// (s_pq = +1 when p or q is the subspace's strong orbital, -1 when both are
// weak; Phi = sqrt(n (1 - n)), Phi' = (1 - 2n)/(2 Phi)), and the minimiser is
// L-BFGS (8 pairs of history, backtracking Armijo line search), all in FP64.
//
// The problem is small (N_Omega^2 terms per evaluation), so one CTA runs the whole
// optimisation on the device: one launch per outer iteration, no host round trips.
// Every loop has a fixed bound; __syncthreads() is only reached in uniform control
// flow (loop decisions are read from shared memory after a barrier).
#include "common.cuh"

namespace donof {

constexpr int ON_THREADS = 512;
constexpr int ON_HIST = 8;
constexpr int ON_MAX_WEAK = 16;

struct OnParams {
  int n_strong, n_weak_per, m, ng;
  const int* subspace;
  const int* weak_rank;
  const double* J;
  const double* K;
  const double* Hd;
  const double* enuc;
  double* gamma;     // in: start, out: result
  double* E_out;     // [1]
  double* grad_out;  // [ng]
  int* info_out;     // [2]: iterations, stop reason (0 gradient below gtol, 1 iteration cap,
                     //      2 line search found no decrease, 3 relative energy decrease below etol)
  int max_iter;
  double gtol, etol;
  int mode;  // 0: evaluate E and the gradient at gamma; 1: optimise
};

// H_pp = C_p^T (H C)_p for the pairing-space orbitals: one warp per p.
__global__ void on_hdiag_kernel(int nb, int m, const double* C, const double* HC, double* Hd) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
  if (w >= m) return;
  double s = 0.0;
  for (int mu = lane; mu < nb; mu += 32) s = fma(C[(size_t)w * nb + mu], HC[(size_t)mu * m + w], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) Hd[w] = s;
}

struct OnShared {
  double *n, *phi, *dphi, *dEdn, *red;
  double *x, *g, *xn, *gn, *d, *S, *Y, *rho, *al;
  int* orb;  // orb[g * (N_g + 1) + r + 1] = orbital of rank r (-1 strong) in subspace g
  double* scal;
};

// Block-wide sum of v over all threads (deterministic tree).
__device__ double on_block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = ON_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

__device__ double on_block_max(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = ON_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

__device__ double on_dot(const double* a, const double* b, int n, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += ON_THREADS) s = fma(a[i], b[i], s);
  return on_block_sum(s, red);
}

// alpha_i (i = 0..N_g-1) of subspace weak angles w[0..N_g-2] and d alpha_i / d w_j.
__device__ void on_alpha(const double* w, int Ng, double* alpha, double (*dalpha)[ON_MAX_WEAK]) {
  for (int i = 0; i < Ng; ++i) {
    const double tail = i < Ng - 1 ? cos(w[i]) * cos(w[i]) : 1.0;
    double prod = 1.0;
    for (int k = 0; k < i; ++k) prod *= sin(w[k]) * sin(w[k]);
    alpha[i] = prod * tail;
    for (int j = 0; j < Ng - 1; ++j) {
      double v = 0.0;
      if (j < i) {
        double others = 1.0;
        for (int k = 0; k < i; ++k)
          if (k != j) others *= sin(w[k]) * sin(w[k]);
        v = others * sin(2.0 * w[j]) * tail;
      } else if (j == i) {
        v = -prod * sin(2.0 * w[i]);
      }
      dalpha[i][j] = v;
    }
  }
}

// E(x) and dE/dx; every thread returns E.
__device__ double on_evaluate(const OnParams& p, const OnShared& sh, const double* x, double* gout) {
  const int NI = p.n_strong, Ng = p.n_weak_per, m = p.m, na = Ng - 1;
  // occupations, one thread per subspace
  for (int g = threadIdx.x; g < NI; g += ON_THREADS) {
    const double c = cos(x[g]);
    const double ngv = 0.5 * (1.0 + c * c), hg = 1.0 - ngv;
    double alpha[ON_MAX_WEAK], dal[ON_MAX_WEAK][ON_MAX_WEAK];
    on_alpha(x + NI + g * na, Ng, alpha, dal);
    sh.n[sh.orb[g * (Ng + 1)]] = ngv;
    for (int i = 0; i < Ng; ++i) sh.n[sh.orb[g * (Ng + 1) + i + 1]] = hg * alpha[i];
  }
  __syncthreads();
  for (int q = threadIdx.x; q < m; q += ON_THREADS) {
    const double nq = sh.n[q];
    const double ph = sqrt(nq * (1.0 - nq));
    sh.phi[q] = ph;
    sh.dphi[q] = ph > 0.0 ? (1.0 - 2.0 * nq) / (2.0 * ph) : 0.0;
  }
  __syncthreads();
  // dE/dn_p and the energy row sums, one thread per orbital p
  double epart = 0.0;
  for (int pp = threadIdx.x; pp < m; pp += ON_THREADS) {
    const double np_ = sh.n[pp], php = sh.phi[pp], dphp = sh.dphi[pp];
    const int gp = p.subspace[pp], rp = p.weak_rank[pp];
    const double* Jr = p.J + (size_t)pp * m;
    const double* Kr = p.K + (size_t)pp * m;
    double v = 2.0 * p.Hd[pp] + Jr[pp];
    double e = 2.0 * np_ * p.Hd[pp] + np_ * Jr[pp];
    for (int q = 0; q < m; ++q) {
      if (q == pp) continue;
      const double nq = sh.n[q];
      if (p.subspace[q] == gp) {
        const double s = (rp < 0 || p.weak_rank[q] < 0) ? 1.0 : -1.0;
        const double k = Kr[q];
        if (np_ > 0.0) v -= s * k * sqrt(nq / np_);
        e -= s * sqrt(np_ * nq) * k;
      } else {
        const double j = Jr[q], k = Kr[q], phq = sh.phi[q];
        v += 4.0 * nq * j - 2.0 * nq * k - 2.0 * dphp * phq * k;
        e += 2.0 * np_ * nq * j - (np_ * nq + php * phq) * k;
      }
    }
    sh.dEdn[pp] = v;
    epart += e;
  }
  const double E = on_block_sum(epart, sh.red) + p.enuc[0];  // (the sum's barriers also publish dEdn)
  // chain rule, one thread per subspace
  for (int g = threadIdx.x; g < NI; g += ON_THREADS) {
    const double dh = 0.5 * sin(2.0 * x[g]);
    const double c = cos(x[g]);
    const double hg = 1.0 - 0.5 * (1.0 + c * c);
    double alpha[ON_MAX_WEAK], dal[ON_MAX_WEAK][ON_MAX_WEAK];
    on_alpha(x + NI + g * na, Ng, alpha, dal);
    double gs = -dh * sh.dEdn[sh.orb[g * (Ng + 1)]];
    for (int i = 0; i < Ng; ++i) gs += dh * alpha[i] * sh.dEdn[sh.orb[g * (Ng + 1) + i + 1]];
    gout[g] = gs;
    for (int j = 0; j < na; ++j) {
      double gw = 0.0;
      for (int i = 0; i < Ng; ++i) gw += hg * dal[i][j] * sh.dEdn[sh.orb[g * (Ng + 1) + i + 1]];
      gout[NI + g * na + j] = gw;
    }
  }
  __syncthreads();
  return E;
}

__global__ void __launch_bounds__(ON_THREADS, 1) on_opt_kernel(const OnParams p) {
  extern __shared__ double onsm[];
  const int m = p.m, ng = p.ng;
  OnShared sh;
  double* ptr = onsm;
  sh.n = ptr; ptr += m;
  sh.phi = ptr; ptr += m;
  sh.dphi = ptr; ptr += m;
  sh.dEdn = ptr; ptr += m;
  sh.red = ptr; ptr += ON_THREADS;
  sh.x = ptr; ptr += ng;
  sh.g = ptr; ptr += ng;
  sh.xn = ptr; ptr += ng;
  sh.gn = ptr; ptr += ng;
  sh.d = ptr; ptr += ng;
  sh.S = ptr; ptr += (size_t)ON_HIST * ng;
  sh.Y = ptr; ptr += (size_t)ON_HIST * ng;
  sh.rho = ptr; ptr += ON_HIST;
  sh.al = ptr; ptr += ON_HIST;
  sh.scal = ptr; ptr += 8;
  sh.orb = (int*)ptr;

  for (int q = threadIdx.x; q < m; q += ON_THREADS) {
    const int r = p.weak_rank[q];
    sh.orb[p.subspace[q] * (p.n_weak_per + 1) + r + 1] = q;
  }
  for (int i = threadIdx.x; i < ng; i += ON_THREADS) sh.x[i] = p.gamma[i];
  __syncthreads();

  double E = on_evaluate(p, sh, sh.x, sh.g);
  int iters = 0, reason = 1, hist = 0, head = 0;
  if (p.mode == 1) {
    for (int it = 0; it < p.max_iter; ++it) {
      double gmax = 0.0;
      for (int i = threadIdx.x; i < ng; i += ON_THREADS) gmax = fmax(gmax, fabs(sh.g[i]));
      gmax = on_block_max(gmax, sh.red);
      if (gmax <= p.gtol) {
        reason = 0;
        break;
      }
      // two-loop recursion: d = -H g
      for (int i = threadIdx.x; i < ng; i += ON_THREADS) sh.d[i] = sh.g[i];
      __syncthreads();
      for (int k = 0; k < hist; ++k) {
        const int slot = (head - 1 - k + ON_HIST) % ON_HIST;
        const double a = sh.rho[slot] * on_dot(sh.S + (size_t)slot * ng, sh.d, ng, sh.red);
        if (threadIdx.x == 0) sh.al[slot] = a;
        for (int i = threadIdx.x; i < ng; i += ON_THREADS) sh.d[i] -= a * sh.Y[(size_t)slot * ng + i];
        __syncthreads();
      }
      double scale = 1.0;
      if (hist > 0) {
        const int slot = (head - 1 + ON_HIST) % ON_HIST;
        const double yy = on_dot(sh.Y + (size_t)slot * ng, sh.Y + (size_t)slot * ng, ng, sh.red);
        scale = yy > 0.0 ? 1.0 / (sh.rho[slot] * yy) : 1.0;
      } else {
        scale = gmax > 0.5 ? 0.5 / gmax : 1.0;  // first step: at most 0.5 rad in any angle
      }
      for (int i = threadIdx.x; i < ng; i += ON_THREADS) sh.d[i] *= scale;
      __syncthreads();
      for (int k = hist - 1; k >= 0; --k) {
        const int slot = (head - 1 - k + ON_HIST) % ON_HIST;
        const double b = sh.rho[slot] * on_dot(sh.Y + (size_t)slot * ng, sh.d, ng, sh.red);
        const double a = sh.al[slot];
        for (int i = threadIdx.x; i < ng; i += ON_THREADS) sh.d[i] += (a - b) * sh.S[(size_t)slot * ng + i];
        __syncthreads();
      }
      for (int i = threadIdx.x; i < ng; i += ON_THREADS) sh.d[i] = -sh.d[i];
      __syncthreads();
      double gd = on_dot(sh.g, sh.d, ng, sh.red);
      if (!(gd < 0.0)) {  // not a descent direction: restart from steepest descent
        hist = 0;
        const double sc = gmax > 0.5 ? 0.5 / gmax : 1.0;
        for (int i = threadIdx.x; i < ng; i += ON_THREADS) sh.d[i] = -sc * sh.g[i];
        __syncthreads();
        gd = on_dot(sh.g, sh.d, ng, sh.red);
      }
      // backtracking line search (Armijo, c1 = 1e-4)
      double t = 1.0, En = E;
      bool accepted = false;
      for (int ls = 0; ls < 40; ++ls) {
        for (int i = threadIdx.x; i < ng; i += ON_THREADS) sh.xn[i] = sh.x[i] + t * sh.d[i];
        __syncthreads();
        En = on_evaluate(p, sh, sh.xn, sh.gn);
        if (En <= E + 1e-4 * t * gd) {
          accepted = true;
          break;
        }
        t *= 0.5;
      }
      if (!accepted) {
        reason = 2;
        break;
      }
      // history update
      for (int i = threadIdx.x; i < ng; i += ON_THREADS) {
        sh.S[(size_t)head * ng + i] = sh.xn[i] - sh.x[i];
        sh.Y[(size_t)head * ng + i] = sh.gn[i] - sh.g[i];
      }
      __syncthreads();
      const double sy = on_dot(sh.S + (size_t)head * ng, sh.Y + (size_t)head * ng, ng, sh.red);
      if (sy > 0.0) {
        if (threadIdx.x == 0) sh.rho[head] = 1.0 / sy;
        head = (head + 1) % ON_HIST;
        hist = hist < ON_HIST ? hist + 1 : ON_HIST;
      }
      for (int i = threadIdx.x; i < ng; i += ON_THREADS) {
        sh.x[i] = sh.xn[i];
        sh.g[i] = sh.gn[i];
      }
      __syncthreads();
      const double dec = E - En;
      E = En;
      iters = it + 1;
      // Minima where an occupation reaches 0 or 1 sit on a kink of E(gamma) (the
      // sqrt(n) terms), where the gradient need not vanish: stop on the energy too.
      if (dec <= p.etol * fmax(1.0, fabs(E))) {
        reason = 3;
        break;
      }
    }
  }
  // E depends on the angles through cos^2 and sin^2 only: an optimised gamma is
  // returned folded into [0, pi/2] (and its gradient with the matching sign).
  for (int i = threadIdx.x; i < ng; i += ON_THREADS) {
    double xi = sh.x[i], gi = sh.g[i];
    if (p.mode == 1) {
      const double c = cos(xi), s = sin(xi);
      xi = atan2(fabs(s), fabs(c));
      if (s * c < 0.0) gi = -gi;
    }
    p.gamma[i] = xi;
    p.grad_out[i] = gi;
  }
  if (threadIdx.x == 0) {
    p.E_out[0] = E;
    p.info_out[0] = iters;
    p.info_out[1] = p.mode == 1 ? reason : 0;
  }
}

// Features of each pairing subspace g for the learned warm start (one row of
// 3 + 4 N_g values): [H_ss, J_ss, mf_s, then per weak orbital w in rank order:
// H_ww, J_ww, K_sw, mf_w], with mf_p = sum_{q outside g} n0_q (2 J_pq - K_pq)
// the mean field of the other subspaces at the standard-guess occupations n0
// (strong 0.98, weak 0.02 / N_g).  Thread per (subspace, member).
__global__ void on_features_kernel(int NI, int Ng, int m, const int* subspace, const int* weak_rank, const double* J,
                                   const double* K, const double* Hd, float* X) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NI * (Ng + 1)) return;
  const int g = t / (Ng + 1), k = t % (Ng + 1);
  int pp = -1, s = -1;
  for (int q = 0; q < m; ++q) {
    if (subspace[q] != g) continue;
    if (weak_rank[q] == k - 1) pp = q;
    if (weak_rank[q] < 0) s = q;
  }
  if (pp < 0 || s < 0) return;
  double mf = 0.0;
  for (int q = 0; q < m; ++q) {
    if (subspace[q] == g) continue;
    const double n0 = weak_rank[q] < 0 ? 0.98 : 0.02 / Ng;
    mf += n0 * (2.0 * J[(size_t)pp * m + q] - K[(size_t)pp * m + q]);
  }
  const int F = 3 + 4 * Ng;
  float* x = X + (size_t)g * F;
  if (k == 0) {
    x[0] = (float)Hd[pp];
    x[1] = (float)J[(size_t)pp * m + pp];
    x[2] = (float)mf;
  } else {
    float* y = x + 3 + 4 * (k - 1);
    y[0] = (float)Hd[pp];
    y[1] = (float)J[(size_t)pp * m + pp];
    y[2] = (float)K[(size_t)s * m + pp];
    y[3] = (float)mf;
  }
}

// Network outputs [N_I][N_g] -> gamma (strong angles, then the weak angles of each
// subspace), clipped to [clip, pi/2 - clip].
__global__ void on_unfold_kernel(const float* Y, int NI, int Ng, double clip, double* gamma) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NI * Ng) return;
  const int g = t / Ng, j = t % Ng;
  double v = (double)Y[t];
  const double hi = 1.5707963267948966 - clip;
  v = v < clip ? clip : (v > hi ? hi : v);
  if (j == 0) gamma[g] = v;
  else gamma[NI + g * (Ng - 1) + j - 1] = v;
}

int onopt_features(donof_ri_ctx* ctx, float* d_X) {
  const int m = ctx->n_omega, nb = ctx->nbf, NI = ctx->n_strong, Ng = ctx->n_weak_per;
  int rc;
  if ((rc = launch_hc_public(ctx))) return rc;
  on_hdiag_kernel<<<ceil_div_u((long long)m * 32, 256), 256, 0, ctx->stream>>>(nb, m, ctx->d_C, ctx->d_HC,
                                                                               ctx->d_Hd);
  DONOF_LAUNCH_CHECK(ctx);
  on_features_kernel<<<ceil_div_u((long long)NI * (Ng + 1), 128), 128, 0, ctx->stream>>>(
      NI, Ng, m, ctx->d_subspace, ctx->d_weak_rank, ctx->d_J, ctx->d_K, ctx->d_Hd, d_X);
  DONOF_LAUNCH_CHECK(ctx);
  return DONOF_RI_OK;
}

int onopt_unfold(donof_ri_ctx* ctx, const float* d_Y, double clip, double* d_gamma) {
  const int NI = ctx->n_strong, Ng = ctx->n_weak_per;
  on_unfold_kernel<<<ceil_div_u((long long)NI * Ng, 128), 128, 0, ctx->stream>>>(d_Y, NI, Ng, clip, d_gamma);
  DONOF_LAUNCH_CHECK(ctx);
  return DONOF_RI_OK;
}

// Runs the evaluation (mode 0) or the optimisation (mode 1) on the context's
// stream with gamma, E, grad and info in device memory.
int onopt_launch(donof_ri_ctx* ctx, double* d_gamma, double* d_E, double* d_grad, int* d_info, int mode,
                 int max_iter, double gtol, double etol) {
  const int m = ctx->n_omega, nb = ctx->nbf;
  const int ng = ctx->n_strong * ctx->n_weak_per;
  if (ctx->n_weak_per < 1 || ctx->n_weak_per > ON_MAX_WEAK) return DONOF_RI_E_UNSUPPORTED;
  int rc;
  if ((rc = launch_hc_public(ctx))) return rc;
  on_hdiag_kernel<<<ceil_div_u((long long)m * 32, 256), 256, 0, ctx->stream>>>(nb, m, ctx->d_C, ctx->d_HC,
                                                                               ctx->d_Hd);
  DONOF_LAUNCH_CHECK(ctx);
  OnParams p{};
  p.n_strong = ctx->n_strong;
  p.n_weak_per = ctx->n_weak_per;
  p.m = m;
  p.ng = ng;
  p.subspace = ctx->d_subspace;
  p.weak_rank = ctx->d_weak_rank;
  p.J = ctx->d_J;
  p.K = ctx->d_K;
  p.Hd = ctx->d_Hd;
  p.enuc = ctx->d_enuc;
  p.gamma = d_gamma;
  p.E_out = d_E;
  p.grad_out = d_grad;
  p.info_out = d_info;
  p.max_iter = max_iter;
  p.gtol = gtol;
  p.etol = etol;
  p.mode = mode;
  const size_t smem = sizeof(double) * ((size_t)4 * m + ON_THREADS + 5 * (size_t)ng + 2 * (size_t)ON_HIST * ng +
                                        2 * ON_HIST + 8) +
                      sizeof(int) * (size_t)ctx->n_strong * (ctx->n_weak_per + 1);
  if (smem > 227 * 1024) return DONOF_RI_E_UNSUPPORTED;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(on_opt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return DONOF_RI_E_CUDA;
  on_opt_kernel<<<1, ON_THREADS, smem, ctx->stream>>>(p);
  DONOF_LAUNCH_CHECK(ctx);
  return DONOF_RI_OK;
}

}  // namespace donof
