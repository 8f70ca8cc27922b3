// Split-precision tensor-core path (DONOF_RI_TF32X3) for sm_103a.
//
// Every dense contraction of the hot path (paper, Sec. 2, Tables 2 and 3)
// runs through one warp-specialised tcgen05 kernel:
//   warp 0 (one lane)  TMA producer: 128B-swizzled K-major tiles of the hi and
//                      lo parts of both operands into a ring of smem stages;
//   warp 1 (one lane)  MMA issuer: per 32-wide K block, 4 x 3 tcgen05.mma
//                      kind::tf32 (lo*hi, hi*lo, hi*hi) into a TMEM accumulator
//                      (two accumulators ping-pong so the epilogue of one work
//                      unit overlaps the MMAs of the next); also owns TMEM;
//   warps 2-5          epilogue: tcgen05.ld of the accumulator (one TMEM lane per
//                      thread = one output row) and a row-specific action.
// Operands are stored pre-split: x = hi + lo with hi = rna_tf32(x) and
// lo = rna_tf32(x - hi), so each product a*b is taken as
// a_lo b_hi + a_hi b_lo + a_hi b_hi (the a_lo b_lo term, ~2^-22 relative, is
// dropped) and accumulated in FP32.
//
// Rows of the hot path and their GEMM shapes (N_b = nbf, N_x = naux, N_O = N_Omega):
//   HALF   b^P_{p nu} = sum_mu C_{mu p} B^P_{mu nu}        (Tables 2/3 step 2)
//          M = (P, nu) blocks of 16 x 8, N = p, K = mu; writes b_half in two
//          layouts (for the full transform and for K^(p)), split hi/lo.
//   FULLSQ b^P_pq = sum_nu b^P_{p nu} C_{nu q}; K_pq += (b^P_pq)^2 (Table 2 steps 3-4)
//          M = p, N = q, K = nu, one work unit per P; squares summed in FP32
//          registers over the CTA's P range, FP32 partials summed in FP64.
//   JMO    J_pq = sum_P b^P_pp b^P_qq                      (Table 2 step 4)
//          M = p, N = q, K = P in chunks (one unit per chunk), FP64 reduction.
//   JAO    J^(q)_{mu nu} = sum_P B^P_{mu nu} b^P_qq        (Table 3 step 4)
//          M = (mu, nu) pairs, N = q, K = P.
//   KAO    K^(p)_{mu nu} = sum_P b^P_{p mu} b^P_{p nu}     (Table 3 step 3)
//          M = mu, N = nu, K = P, one unit per p.
//   FOCK   Y_{mu p} = sum_q [A_pq (J^(q) C)_{mu p} - B_pq (K^(q) C)_{mu p}]
//          M = mu, N = p, K = nu, one unit per q (2 N_O units: J then K),
//          weighted sum in FP32 registers, FP32 partials summed in FP64.
#include "common.cuh"
#include "tcgen05.cuh"

#include <atomic>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <mutex>
#include <stdlib.h>
#include <string.h>

namespace donof {
int launch_dot64(donof_ri_ctx* ctx, int M, int N, int K, const double* A, int lda, const double* B, int ldb,
                 double* out, long long so_i, long long so_j);
int launch_energy_rows(donof_ri_ctx* ctx, const double* HCt);

enum TcKind { K_HALF = 0, K_FULLSQ = 1, K_JMO = 2, K_JAO = 3, K_KAO = 4, K_FOCK = 5, K_NKINDS = 6 };
static_assert(DONOF_RI_GEMM_FOCK - DONOF_RI_GEMM_HALF == K_FOCK, "GEMM profile rows follow the kind order");

constexpr int TC_THREADS = 192;
constexpr int TC_BM = 128;   // rows per tile (TMEM lanes)
constexpr int TC_BK = 32;    // fp32 elements per K block (one 128-byte swizzle row)
constexpr int TC_SUM_MAXBN = 128;

struct TcParams {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;
  int N;            // valid columns of the unit's output (rows of the B operand)
  int K;            // reduction extent of one unit
  int BN;           // columns per tile (multiple of 16, <= 256)
  int stages;
  int tmem_cols;    // allocated TMEM columns (power of two >= 2*BN)
  int n_tiles;      // tiles along N
  int nbatch;       // work units per tile (batch entries or K chunks)
  int bpc;          // units per CTA
  int nsplit;       // CTAs per tile
  int kb_per_unit;  // K blocks per unit
  int nb, nx, m, nbp, nxp, mp;
  float* o0;
  float* o1;
  float* o2;
  float* o3;
  float* partial;   // [nsplit][prow][pcol]
  int prow, pcol;
  const float* w;   // FOCK weights [2 N_O][N_O]
  int* status;
};

// ---------------------------------------------------------------------------
// The GEMM kernel
// ---------------------------------------------------------------------------
template <int KIND>
__device__ __forceinline__ void issue_loads(const TcParams& p, uint8_t* st, uint64_t* bar, int mt, int nt, int b,
                                            int kb) {
  const uint32_t a_bytes = TC_BM * 128, b_bytes = (uint32_t)p.BN * 128;
  uint8_t* ah = st;
  uint8_t* al = st + a_bytes;
  uint8_t* bh = st + 2 * a_bytes;
  uint8_t* bl = st + 2 * a_bytes + b_bytes;
  const int k0 = kb * TC_BK;
  const int n0 = nt * p.BN;
  if (KIND == K_HALF) {
    const int nvb = (p.nb + 7) / 8;
    const int Pb = mt / nvb, vb = mt % nvb;
    tma_load_3d(ah, &p.a_hi, bar, k0, vb * 8, Pb * 16);
    tma_load_3d(al, &p.a_lo, bar, k0, vb * 8, Pb * 16);
    tma_load_2d(bh, &p.b_hi, bar, k0, n0);
    tma_load_2d(bl, &p.b_lo, bar, k0, n0);
  } else if (KIND == K_FULLSQ || KIND == K_FOCK) {
    tma_load_3d(ah, &p.a_hi, bar, k0, mt * TC_BM, b);
    tma_load_3d(al, &p.a_lo, bar, k0, mt * TC_BM, b);
    tma_load_2d(bh, &p.b_hi, bar, k0, n0);
    tma_load_2d(bl, &p.b_lo, bar, k0, n0);
  } else if (KIND == K_JMO) {
    const int kk = (b * p.kb_per_unit) * TC_BK + k0;
    tma_load_2d(ah, &p.a_hi, bar, kk, mt * TC_BM);
    tma_load_2d(al, &p.a_lo, bar, kk, mt * TC_BM);
    tma_load_2d(bh, &p.b_hi, bar, kk, n0);
    tma_load_2d(bl, &p.b_lo, bar, kk, n0);
  } else if (KIND == K_JAO) {
    tma_load_2d(ah, &p.a_hi, bar, k0, mt * TC_BM);
    tma_load_2d(al, &p.a_lo, bar, k0, mt * TC_BM);
    tma_load_2d(bh, &p.b_hi, bar, k0, n0);
    tma_load_2d(bl, &p.b_lo, bar, k0, n0);
  } else {  // K_KAO
    tma_load_3d(ah, &p.a_hi, bar, k0, mt * TC_BM, b);
    tma_load_3d(al, &p.a_lo, bar, k0, mt * TC_BM, b);
    tma_load_3d(bh, &p.b_hi, bar, k0, n0, b);
    tma_load_3d(bl, &p.b_lo, bar, k0, n0, b);
  }
}

template <int KIND>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm_kernel(const __grid_constant__ TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int S = p.stages;
  const uint32_t a_bytes = TC_BM * 128, b_bytes = (uint32_t)p.BN * 128;
  const uint32_t stage_bytes = 2 * (a_bytes + b_bytes);
  uint64_t* full = (uint64_t*)(smem + (size_t)S * stage_bytes);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;
  uint64_t* acce = accf + 2;
  uint64_t* drain = acce + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int tile = blockIdx.x / p.nsplit, split = blockIdx.x % p.nsplit;
  const int mt = tile / p.n_tiles, nt = tile % p.n_tiles;
  const int b0 = split * p.bpc;
  const int b1 = min(p.nbatch, b0 + p.bpc);
  const int nunits = max(0, b1 - b0);
  const int KB = p.kb_per_unit;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&accf[a], 1);
      mbar_init(&acce[a], 128);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, (uint32_t)p.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int it = 0;
      bool ok = true;
      for (int u = 0; u < nunits && ok; ++u) {
        for (int kb = 0; kb < KB; ++kb) {
          const int s = it % S;
          const uint32_t ph = (uint32_t)((it / S) & 1);
          if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, p.status)) { ok = false; break; }
          mbar_expect_tx(&full[s], stage_bytes);
          issue_loads<KIND>(p, smem + (size_t)s * stage_bytes, &full[s], mt, nt, b0 + u, kb);
          ++it;
        }
      }
      // Every issued copy must land before the CTA may exit.
      for (int j = max(0, it - S); j < it; ++j)
        mbar_wait(&full[j % S], (uint32_t)((j / S) & 1), nullptr, p.status);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t idesc = idesc_tf32(p.BN);
      int it = 0;
      bool ok = true;
      for (int u = 0; u < nunits && ok; ++u) {
        const int a = u & 1;
        if (!mbar_wait(&acce[a], (uint32_t)(((u >> 1) & 1) ^ 1), abort_flag, p.status)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(a * p.BN);
        for (int kb = 0; kb < KB; ++kb) {
          const int s = it % S;
          if (!mbar_wait(&full[s], (uint32_t)((it / S) & 1), abort_flag, p.status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + (size_t)s * stage_bytes);
          const uint32_t ah = st, al = st + a_bytes, bh = st + 2 * a_bytes, bl = st + 2 * a_bytes + b_bytes;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t off = (uint32_t)k * 32u;
            const uint64_t dah = sdesc_sw128(ah + off), dal = sdesc_sw128(al + off);
            const uint64_t dbh = sdesc_sw128(bh + off), dbl = sdesc_sw128(bl + off);
            mma_tf32(d_tmem, dal, dbh, idesc, (kb | k) != 0);
            mma_tf32(d_tmem, dah, dbl, idesc, 1u);
            mma_tf32(d_tmem, dah, dbh, idesc, 1u);
          }
          mma_commit(&empty[s]);
          ++it;
        }
        if (!ok) break;
        mma_commit(&accf[a]);
      }
      // All MMAs of this thread must complete before TMEM is released.
      mma_commit(drain);
      mbar_wait(drain, 0, nullptr, p.status);
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const int nchunks = p.BN / 16;
    float acc[(KIND == K_FULLSQ || KIND == K_JMO || KIND == K_FOCK) ? TC_SUM_MAXBN : 1];
    if (KIND == K_FULLSQ || KIND == K_JMO || KIND == K_FOCK) {
#pragma unroll
      for (int i = 0; i < TC_SUM_MAXBN; ++i) acc[i] = 0.f;
    }
    int units_done = 0;
    for (int u = 0; u < nunits; ++u) {
      const int a = u & 1;
      if (!mbar_wait(&accf[a], (uint32_t)((u >> 1) & 1), abort_flag, p.status)) break;
      tc_fence_after();
      const int b = b0 + u;
      const uint32_t tb = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * p.BN);
      if (KIND == K_FULLSQ || KIND == K_JMO || KIND == K_FOCK) {
#pragma unroll
        for (int c = 0; c < TC_SUM_MAXBN / 16; ++c) {
          if (c < nchunks) {
            float v[16];
            tmem_ld16(tb + (uint32_t)(c * 16), v);
            if (KIND == K_FULLSQ) {
#pragma unroll
              for (int j = 0; j < 16; ++j) acc[c * 16 + j] = fmaf(v[j], v[j], acc[c * 16 + j]);
            } else if (KIND == K_JMO) {
#pragma unroll
              for (int j = 0; j < 16; ++j) acc[c * 16 + j] += v[j];
            } else {
              const int col0 = nt * p.BN + c * 16;
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const int col = col0 + j;
                const float wt = col < p.m ? __ldg(&p.w[(size_t)b * p.m + col]) : 0.f;
                acc[c * 16 + j] = fmaf(wt, v[j], acc[c * 16 + j]);
              }
            }
          }
        }
      } else {
        for (int c = 0; c < nchunks; ++c) {
          float v[16];
          tmem_ld16(tb + (uint32_t)(c * 16), v);
          const int col0 = nt * p.BN + c * 16;
          if (KIND == K_HALF) {
            const int nvb = (p.nb + 7) / 8;
            const int P = (mt / nvb) * 16 + row / 8;
            const int nu = (mt % nvb) * 8 + row % 8;
            if (P < p.nx && nu < p.nb) {
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const int pc = col0 + j;
                if (pc < p.m) {
                  float hi, lo;
                  split_tf32(v[j], hi, lo);
                  const size_t i3 = ((size_t)P * p.mp + pc) * p.nbp + nu;
                  const size_t i6 = ((size_t)pc * p.nb + nu) * p.nxp + P;
                  p.o0[i3] = hi;
                  p.o1[i3] = lo;
                  p.o2[i6] = hi;
                  p.o3[i6] = lo;
                }
              }
            }
          } else if (KIND == K_JAO) {
            const int R = mt * TC_BM + row;
            if (R < p.nb * p.nb) {
              const int mu = R / p.nb, nu = R % p.nb;
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const int qc = col0 + j;
                if (qc < p.m) {
                  float hi, lo;
                  split_tf32(v[j], hi, lo);
                  const size_t i = ((size_t)qc * p.nb + mu) * p.nbp + nu;
                  p.o0[i] = hi;
                  p.o1[i] = lo;
                }
              }
            }
          } else {  // K_KAO
            const int mu = mt * TC_BM + row;
            if (mu < p.nb) {
              const size_t rb = ((size_t)(p.m + b) * p.nb + mu) * p.nbp;
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const int nu = col0 + j;
                if (nu < p.nb) {
                  float hi, lo;
                  split_tf32(v[j], hi, lo);
                  p.o0[rb + nu] = hi;
                  p.o1[rb + nu] = lo;
                }
              }
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&acce[a]);
      ++units_done;
    }
    if ((KIND == K_FULLSQ || KIND == K_JMO || KIND == K_FOCK) && units_done == nunits) {
      const int r = (KIND == K_FOCK ? mt * TC_BM : mt * TC_BM) + row;
      if (r < p.prow) {
        float* dst = p.partial + ((size_t)split * p.prow + r) * p.pcol;
#pragma unroll
        for (int c = 0; c < TC_SUM_MAXBN / 16; ++c) {
          if (c < nchunks) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int col = nt * p.BN + c * 16 + j;
              if (col < p.pcol) dst[col] = acc[c * 16 + j];
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, (uint32_t)p.tmem_cols);
  }
}

// ---------------------------------------------------------------------------
// Bandwidth-bound helpers
// ---------------------------------------------------------------------------
// B (FP64, [P][mu][nu], symmetric in mu nu) -> split layout [P][nu][mu] (row stride nbp).
__global__ void split_B_half_kernel(const double* B, int nb, int nbp, int nx, float* hi, float* lo) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long n = (long long)nx * nb * nb;
  if (i >= n) return;
  long long P = i / ((long long)nb * nb);
  int r = (int)(i % ((long long)nb * nb));
  int nu = r / nb, mu = r % nb;
  float h, l;
  split_tf32((float)B[i], h, l);
  // (float)B rounds to FP32 first; the residual B - (float)B is below the TF32 split error.
  size_t o = ((size_t)P * nb + nu) * nbp + mu;
  hi[o] = h;
  lo[o] = l;
}

// B (FP64, [P][mu nu]) -> split layout [mu nu][P] (row stride nxp), tiled transpose.
__global__ void split_B_jao_kernel(const double* B, int nb2, int nx, int nxp, float* hi, float* lo) {
  __shared__ float th[32][33], tl[32][33];
  int r0 = blockIdx.x * 32, P0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int P = P0 + k, r = r0 + threadIdx.x;
    float h = 0.f, l = 0.f;
    if (P < nx && r < nb2) split_tf32((float)B[(size_t)P * nb2 + r], h, l);
    th[k][threadIdx.x] = h;
    tl[k][threadIdx.x] = l;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int r = r0 + k, P = P0 + threadIdx.x;
    if (r < nb2 && P < nx) {
      hi[(size_t)r * nxp + P] = th[threadIdx.x][k];
      lo[(size_t)r * nxp + P] = tl[threadIdx.x][k];
    }
  }
}

// C (FP64 column-major [p][mu]) -> split C^T rows [p][mu] (row stride nbp), p < N_O.
__global__ void split_C_kernel(const double* C, int nb, int nbp, int m, float* hi, float* lo) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m * nb) return;
  int pc = i / nb, mu = i % nb;
  float h, l;
  split_tf32((float)C[(size_t)pc * nb + mu], h, l);
  hi[(size_t)pc * nbp + mu] = h;
  lo[(size_t)pc * nbp + mu] = l;
}

// Error-free transformations for the compensated dot product (Ogita-Rump-Oishi Dot2).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float z = s - a;
  e = (a - (s - z)) + (b - z);
}

// b^P_pp = sum_nu b^P_{p nu} C_{nu p} (Table 3 step 3) from the split half transform,
// compensated FP32 (Dot2) per warp; writes d split as [p][P] (row stride nxp).
__global__ void diag_mixed_kernel(const float* bh_hi, const float* bh_lo, const float* ct_hi, const float* ct_lo,
                                  int nb, int nbp, int nx, int m, int mp, int nxp, float* d_hi, float* d_lo) {
  long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
  int lane = threadIdx.x % 32;
  if (w >= (long long)nx * m) return;
  int P = (int)(w / m), pc = (int)(w % m);
  const size_t rb = ((size_t)P * mp + pc) * nbp;
  const size_t cb = (size_t)pc * nbp;
  float s = 0.f, c = 0.f;
  for (int nu = lane; nu < nb; nu += 32) {
    float xh = bh_hi[rb + nu], xl = bh_lo[rb + nu];
    float yh = ct_hi[cb + nu], yl = ct_lo[cb + nu];
    float t[3] = {xh * yh, xh * yl, xl * yh};
    float e0 = fmaf(xh, yh, -t[0]);
    c += e0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float ns, e;
      two_sum(s, t[k], ns, e);
      s = ns;
      c += e;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    float so = __shfl_xor_sync(0xffffffffu, s, o);
    float co = __shfl_xor_sync(0xffffffffu, c, o);
    float ns, e;
    two_sum(s, so, ns, e);
    s = ns;
    c += co + e;
  }
  if (lane == 0) {
    float tot = s + c;
    float hi, lo;
    hi = rna_tf32(tot);
    lo = rna_tf32((s - hi) + c);
    d_hi[(size_t)pc * nxp + P] = hi;
    d_lo[(size_t)pc * nxp + P] = lo;
  }
}

// sum_s partial[s][r][c] in FP64 (fixed order over s).
// mode 0: out[r][c] = sum.
// mode 1 (Fock rows): out[c][r] = n_c HCt[c][r] + sum, i.e. Y^T with Y_{mu p} = n_p (H C)_{mu p} + Z_{mu p}.
__global__ void reduce_partials_kernel(const float* partial, int nsplit, int rows, int cols, double* out, int mode,
                                       const double* n, const double* HCt) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long rc = (long long)rows * cols;
  if (i >= rc) return;
  double s = 0.0;
  for (int k = 0; k < nsplit; ++k) s += (double)partial[(size_t)k * rc + i];
  if (mode == 1) {
    int r = (int)(i / cols), c = (int)(i % cols);
    out[(size_t)c * rows + r] = n[c] * HCt[(size_t)c * rows + r] + s;
  } else {
    out[i] = s;
  }
}

// FOCK weights: W[q][p] = A_pq (q < N_O), W[N_O + q][p] = -B_pq.
__global__ void fock_weights_kernel(const double* A, const double* Bc, int m, float* W) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * m * m) return;
  int qq = i / m, pc = i % m;
  W[i] = qq < m ? (float)A[(size_t)pc * m + qq] : (float)(-Bc[(size_t)pc * m + (qq - m)]);
}

// hi + lo -> FP64 copy of a strided array: out[i] for i over (outer, inner), source row stride ld.
__global__ void join_kernel(const float* hi, const float* lo, long long rows, int cols, int ld, double* out) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  long long r = i / cols;
  int c = (int)(i % cols);
  size_t s = (size_t)r * ld + c;
  out[i] = (double)hi[s] + (double)lo[s];
}

// d split [p][P] (stride nxp) -> FP64 [P][p].
__global__ void join_diag_kernel(const float* hi, const float* lo, int nx, int m, int nxp, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx * m) return;
  int P = i / m, pc = i % m;
  size_t s = (size_t)pc * nxp + P;
  out[i] = (double)hi[s] + (double)lo[s];
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct TcPlan {
  TcParams p;
  int grid;
  size_t smem;
  bool valid;
};

}  // namespace donof

struct donof::MixedBuffers {
  int nbp, nxp, mp;
  float *Ba_hi, *Ba_lo;   // [nx][nb][nbp]       A operand of HALF
  float *B5_hi, *B5_lo;   // [nb*nb][nxp]        A operand of JAO
  float *Ct_hi, *Ct_lo;   // [m][nbp]            orbitals (rows p)
  float *bh3_hi, *bh3_lo; // [nx][mp][nbp]       b^P_{p nu}, rows p, K = nu
  float *bh6_hi, *bh6_lo; // [m][nb][nxp]        b^P_{p mu}, rows mu, K = P
  float *d_hi, *d_lo;     // [m][nxp]            b^P_pp, rows p, K = P
  float *JK_hi, *JK_lo;   // [2m][nb][nbp]       J^(q) then K^(q)
  float* W;               // [2m][m]             FOCK weights
  float* partial;         // split partial sums
  size_t partial_elems;
  double* HCt;            // [m][nb]   (H C)^T
  double* Yt;             // [m][nb]   Y^T
  donof::TcPlan plan[donof::K_NKINDS];
  PFN_cuTensorMapEncodeTiled_v12000 encode;
};

namespace donof {

static int get_encode(PFN_cuTensorMapEncodeTiled_v12000* fn) {
  void* f = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !f) {
    cudaGetLastError();
    return DONOF_RI_E_UNSUPPORTED;
  }
  *fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
  return DONOF_RI_OK;
}

// Tiled FP32 tensor map with a 128-byte swizzle; dims innermost first, strides in elements.
static int make_map(MixedBuffers* mb, CUtensorMap* map, const float* base, int rank, const long long* dims,
                    const long long* strides_el, const int* box) {
  cuuint64_t gd[3], gs[2];
  cuuint32_t bd[3], es[3] = {1, 1, 1};
  for (int i = 0; i < rank; ++i) {
    gd[i] = (cuuint64_t)dims[i];
    bd[i] = (cuuint32_t)box[i];
  }
  for (int i = 0; i < rank - 1; ++i) {
    gs[i] = (cuuint64_t)(strides_el[i] * 4);
    if (gs[i] % 16) return DONOF_RI_E_ARG;
  }
  if (((uintptr_t)base) % 16) return DONOF_RI_E_ARG;
  CUresult r = mb->encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, (void*)base, gd, gs, bd, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? DONOF_RI_OK : DONOF_RI_E_CUDA;
}

static int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Columns per tile: split n into the fewest tiles of at most cap columns, then round up to 16.
static int choose_bn(int n, int cap) {
  int tiles = (n + cap - 1) / cap;
  return round_up((n + tiles - 1) / tiles, 16);
}

static int pow2_at_least(int x) {
  int p = 32;
  while (p < x) p <<= 1;
  return p;
}

static void plan_common(TcPlan& pl, int BN, int m_tiles, int n_tiles, int nbatch, int nsplit, int kb_per_unit) {
  TcParams& p = pl.p;
  p.BN = BN;
  const size_t stage = 2 * (size_t)(TC_BM + BN) * 128;
  int S = (int)((220 * 1024) / stage);
  if (S > 4) S = 4;
  p.stages = S;
  p.tmem_cols = pow2_at_least(2 * BN);
  p.n_tiles = n_tiles;
  p.nbatch = nbatch;
  p.nsplit = nsplit;
  p.bpc = (nbatch + nsplit - 1) / nsplit;
  p.nsplit = (nbatch + p.bpc - 1) / p.bpc;  // drop CTAs that would get no unit
  p.kb_per_unit = kb_per_unit;
  pl.grid = m_tiles * n_tiles * p.nsplit;
  pl.smem = 1024 + (size_t)S * stage + 256;
  pl.valid = true;
}

int mixed_init(donof_ri_ctx* ctx) {
  MixedBuffers* mb = (MixedBuffers*)calloc(1, sizeof(MixedBuffers));
  if (!mb) return DONOF_RI_E_OOM;
  ctx->mixed = mb;
  int rc = get_encode(&mb->encode);
  if (rc) return rc;
  const int nb = ctx->nbf, nx = ctx->naux, m = ctx->n_omega;
  const int nbp = round_up(nb, 4), nxp = round_up(nx, 4), mp = round_up(m, 4);
  mb->nbp = nbp;
  mb->nxp = nxp;
  mb->mp = mp;
  const int sms = 152;

  // plans first: the partial buffer size depends on the splits
  TcPlan* P = mb->plan;
  int bn;
  // HALF: M = (P, nu) blocks, N = p, K = mu
  bn = choose_bn(m, 256);
  plan_common(P[K_HALF], bn, ((nx + 15) / 16) * ((nb + 7) / 8), (m + bn - 1) / bn, 1, 1, (nb + TC_BK - 1) / TC_BK);
  // FULLSQ: M = p, N = q, units = P
  {
    int b = choose_bn(m, TC_SUM_MAXBN);
    int tiles = ((m + TC_BM - 1) / TC_BM) * ((m + b - 1) / b);
    int ns = (2 * sms + tiles - 1) / tiles;
    if (ns > nx) ns = nx;
    plan_common(P[K_FULLSQ], b, (m + TC_BM - 1) / TC_BM, (m + b - 1) / b, nx, ns, (nb + TC_BK - 1) / TC_BK);
  }
  // JMO: M = p, N = q, units = K chunks of one K block
  {
    int b = choose_bn(m, TC_SUM_MAXBN);
    int kbt = (nx + TC_BK - 1) / TC_BK;
    plan_common(P[K_JMO], b, (m + TC_BM - 1) / TC_BM, (m + b - 1) / b, kbt, kbt, 1);
  }
  // JAO: M = mu nu pairs, N = q, K = P
  bn = choose_bn(m, 256);
  plan_common(P[K_JAO], bn, (nb * nb + TC_BM - 1) / TC_BM, (m + bn - 1) / bn, 1, 1, (nx + TC_BK - 1) / TC_BK);
  // KAO: M = mu, N = nu, units = p
  {
    int b = choose_bn(nb, 256);
    int tiles = ((nb + TC_BM - 1) / TC_BM) * ((nb + b - 1) / b);
    int ns = (sms + tiles - 1) / tiles;
    if (ns > m) ns = m;
    plan_common(P[K_KAO], b, (nb + TC_BM - 1) / TC_BM, (nb + b - 1) / b, m, ns, (nx + TC_BK - 1) / TC_BK);
  }
  // FOCK: M = mu, N = p, units = q (2m)
  {
    int b = choose_bn(m, TC_SUM_MAXBN);
    int tiles = ((nb + TC_BM - 1) / TC_BM) * ((m + b - 1) / b);
    int ns = (sms + tiles - 1) / tiles;
    if (ns > 2 * m) ns = 2 * m;
    plan_common(P[K_FOCK], b, (nb + TC_BM - 1) / TC_BM, (m + b - 1) / b, 2 * m, ns, (nb + TC_BK - 1) / TC_BK);
  }
  size_t pe = 0;
  pe = (size_t)P[K_FULLSQ].p.nsplit * m * m;
  if ((size_t)P[K_JMO].p.nsplit * m * m > pe) pe = (size_t)P[K_JMO].p.nsplit * m * m;
  if ((size_t)P[K_FOCK].p.nsplit * nb * m > pe) pe = (size_t)P[K_FOCK].p.nsplit * nb * m;
  mb->partial_elems = pe;

#define MALLOC(ptr, n)                                                      \
  do {                                                                      \
    if (cudaMalloc((void**)&(ptr), (size_t)(n) * sizeof(float)) != cudaSuccess) { \
      cudaGetLastError();                                                   \
      return DONOF_RI_E_OOM;                                                \
    }                                                                       \
  } while (0)
  const size_t nxs = nx, nbs = nb, ms = m;
  MALLOC(mb->Ba_hi, nxs * nbs * nbp);
  MALLOC(mb->Ba_lo, nxs * nbs * nbp);
  MALLOC(mb->B5_hi, nbs * nbs * nxp);
  MALLOC(mb->B5_lo, nbs * nbs * nxp);
  MALLOC(mb->Ct_hi, ms * nbp);
  MALLOC(mb->Ct_lo, ms * nbp);
  MALLOC(mb->bh3_hi, nxs * mp * nbp);
  MALLOC(mb->bh3_lo, nxs * mp * nbp);
  MALLOC(mb->bh6_hi, ms * nbs * nxp);
  MALLOC(mb->bh6_lo, ms * nbs * nxp);
  MALLOC(mb->d_hi, ms * nxp);
  MALLOC(mb->d_lo, ms * nxp);
  MALLOC(mb->JK_hi, 2 * ms * nbs * nbp);
  MALLOC(mb->JK_lo, 2 * ms * nbs * nbp);
  MALLOC(mb->W, 2 * ms * ms);
  MALLOC(mb->partial, pe);
#undef MALLOC
  if (cudaMalloc((void**)&mb->HCt, ms * nbs * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&mb->Yt, ms * nbs * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return DONOF_RI_E_OOM;
  }

  // split B into both operand layouts (one-time)
  {
    long long n = (long long)nx * nb * nb;
    split_B_half_kernel<<<ceil_div_u(n, 256), 256, 0, ctx->stream>>>(ctx->d_B, nb, nbp, nx, mb->Ba_hi, mb->Ba_lo);
    DONOF_LAUNCH_CHECK(ctx);
    dim3 g(ceil_div_u((long long)nb * nb, 32), ceil_div_u(nx, 32));
    split_B_jao_kernel<<<g, dim3(32, 8), 0, ctx->stream>>>(ctx->d_B, nb * nb, nx, nxp, mb->B5_hi, mb->B5_lo);
    DONOF_LAUNCH_CHECK(ctx);
  }

  // tensor maps (all buffers are fixed for the context's lifetime)
  for (int k = 0; k < K_NKINDS; ++k) {
    TcParams& p = P[k].p;
    p.nb = nb; p.nx = nx; p.m = m; p.nbp = nbp; p.nxp = nxp; p.mp = mp;
    p.status = ctx->d_status;
    p.partial = mb->partial;
    p.w = mb->W;
  }
  {
    TcParams& p = P[K_HALF].p;
    long long dA[3] = {nb, nb, nx}, sA[2] = {nbp, (long long)nb * nbp};
    int bA[3] = {TC_BK, 8, 16};
    long long dB[2] = {nb, m}, sB[1] = {nbp};
    int bB[2] = {TC_BK, p.BN};
    if ((rc = make_map(mb, &p.a_hi, mb->Ba_hi, 3, dA, sA, bA))) return rc;
    if ((rc = make_map(mb, &p.a_lo, mb->Ba_lo, 3, dA, sA, bA))) return rc;
    if ((rc = make_map(mb, &p.b_hi, mb->Ct_hi, 2, dB, sB, bB))) return rc;
    if ((rc = make_map(mb, &p.b_lo, mb->Ct_lo, 2, dB, sB, bB))) return rc;
    p.N = m; p.K = nb;
    p.o0 = mb->bh3_hi; p.o1 = mb->bh3_lo; p.o2 = mb->bh6_hi; p.o3 = mb->bh6_lo;
  }
  {
    TcParams& p = P[K_FULLSQ].p;
    long long dA[3] = {nb, m, nx}, sA[2] = {nbp, (long long)mp * nbp};
    int bA[3] = {TC_BK, TC_BM, 1};
    long long dB[2] = {nb, m}, sB[1] = {nbp};
    int bB[2] = {TC_BK, p.BN};
    if ((rc = make_map(mb, &p.a_hi, mb->bh3_hi, 3, dA, sA, bA))) return rc;
    if ((rc = make_map(mb, &p.a_lo, mb->bh3_lo, 3, dA, sA, bA))) return rc;
    if ((rc = make_map(mb, &p.b_hi, mb->Ct_hi, 2, dB, sB, bB))) return rc;
    if ((rc = make_map(mb, &p.b_lo, mb->Ct_lo, 2, dB, sB, bB))) return rc;
    p.N = m; p.K = nb; p.prow = m; p.pcol = m;
  }
  {
    TcParams& p = P[K_JMO].p;
    long long dA[2] = {nx, m}, sA[1] = {nxp};
    int bA[2] = {TC_BK, TC_BM};
    int bB[2] = {TC_BK, p.BN};
    if ((rc = make_map(mb, &p.a_hi, mb->d_hi, 2, dA, sA, bA))) return rc;
    if ((rc = make_map(mb, &p.a_lo, mb->d_lo, 2, dA, sA, bA))) return rc;
    if ((rc = make_map(mb, &p.b_hi, mb->d_hi, 2, dA, sA, bB))) return rc;
    if ((rc = make_map(mb, &p.b_lo, mb->d_lo, 2, dA, sA, bB))) return rc;
    p.N = m; p.K = nx; p.prow = m; p.pcol = m;
  }
  {
    TcParams& p = P[K_JAO].p;
    long long dA[2] = {nx, (long long)nb * nb}, sA[1] = {nxp};
    int bA[2] = {TC_BK, TC_BM};
    long long dB[2] = {nx, m}, sB[1] = {nxp};
    int bB[2] = {TC_BK, p.BN};
    if ((rc = make_map(mb, &p.a_hi, mb->B5_hi, 2, dA, sA, bA))) return rc;
    if ((rc = make_map(mb, &p.a_lo, mb->B5_lo, 2, dA, sA, bA))) return rc;
    if ((rc = make_map(mb, &p.b_hi, mb->d_hi, 2, dB, sB, bB))) return rc;
    if ((rc = make_map(mb, &p.b_lo, mb->d_lo, 2, dB, sB, bB))) return rc;
    p.N = m; p.K = nx;
    p.o0 = mb->JK_hi; p.o1 = mb->JK_lo;
  }
  {
    TcParams& p = P[K_KAO].p;
    long long dA[3] = {nx, nb, m}, sA[2] = {nxp, (long long)nb * nxp};
    int bA[3] = {TC_BK, TC_BM, 1};
    int bB[3] = {TC_BK, p.BN, 1};
    if ((rc = make_map(mb, &p.a_hi, mb->bh6_hi, 3, dA, sA, bA))) return rc;
    if ((rc = make_map(mb, &p.a_lo, mb->bh6_lo, 3, dA, sA, bA))) return rc;
    if ((rc = make_map(mb, &p.b_hi, mb->bh6_hi, 3, dA, sA, bB))) return rc;
    if ((rc = make_map(mb, &p.b_lo, mb->bh6_lo, 3, dA, sA, bB))) return rc;
    p.N = nb; p.K = nx;
    p.o0 = mb->JK_hi; p.o1 = mb->JK_lo;
  }
  {
    TcParams& p = P[K_FOCK].p;
    long long dA[3] = {nb, nb, 2LL * m}, sA[2] = {nbp, (long long)nb * nbp};
    int bA[3] = {TC_BK, TC_BM, 1};
    long long dB[2] = {nb, m}, sB[1] = {nbp};
    int bB[2] = {TC_BK, p.BN};
    if ((rc = make_map(mb, &p.a_hi, mb->JK_hi, 3, dA, sA, bA))) return rc;
    if ((rc = make_map(mb, &p.a_lo, mb->JK_lo, 3, dA, sA, bA))) return rc;
    if ((rc = make_map(mb, &p.b_hi, mb->Ct_hi, 2, dB, sB, bB))) return rc;
    if ((rc = make_map(mb, &p.b_lo, mb->Ct_lo, 2, dB, sB, bB))) return rc;
    p.N = m; p.K = nb; p.prow = nb; p.pcol = m;
  }
  // opt in to the dynamic shared memory each kind needs
#define OPTIN(KIND)                                                                                     \
  if (cudaFuncSetAttribute(tc_gemm_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,          \
                           (int)P[KIND].smem) != cudaSuccess)                                           \
    return DONOF_RI_E_CUDA;
  OPTIN(K_HALF) OPTIN(K_FULLSQ) OPTIN(K_JMO) OPTIN(K_JAO) OPTIN(K_KAO) OPTIN(K_FOCK)
#undef OPTIN
  return DONOF_RI_OK;
}

void mixed_free(donof_ri_ctx* ctx) {
  MixedBuffers* mb = ctx->mixed;
  if (!mb) return;
  float* bufs[] = {mb->Ba_hi, mb->Ba_lo, mb->B5_hi, mb->B5_lo, mb->Ct_hi, mb->Ct_lo, mb->bh3_hi, mb->bh3_lo,
                   mb->bh6_hi, mb->bh6_lo, mb->d_hi, mb->d_lo, mb->JK_hi, mb->JK_lo, mb->W, mb->partial};
  for (float* b : bufs)
    if (b) cudaFree(b);
  if (mb->HCt) cudaFree(mb->HCt);
  if (mb->Yt) cudaFree(mb->Yt);
  free(mb);
  ctx->mixed = nullptr;
}

template <int KIND>
static int launch_tc(donof_ri_ctx* ctx) {
  const TcPlan& pl = ctx->mixed->plan[KIND];
  if (pl.grid <= 0) return DONOF_RI_OK;
  ProfScope ps(ctx, DONOF_RI_GEMM_HALF + KIND);
  tc_gemm_kernel<KIND><<<pl.grid, TC_THREADS, pl.smem, ctx->stream>>>(pl.p);
  DONOF_LAUNCH_CHECK(ctx);
  return DONOF_RI_OK;
}

static int launch_reduce(donof_ri_ctx* ctx, int kind, double* out, int mode) {
  const TcParams& p = ctx->mixed->plan[kind].p;
  long long n = (long long)p.prow * p.pcol;
  reduce_partials_kernel<<<ceil_div_u(n, 256), 256, 0, ctx->stream>>>(ctx->mixed->partial, p.nsplit, p.prow, p.pcol,
                                                                       out, mode, ctx->d_n, ctx->mixed->HCt);
  DONOF_LAUNCH_CHECK(ctx);
  return DONOF_RI_OK;
}

int mixed_transform(donof_ri_ctx* ctx, int mode) {
  MixedBuffers* mb = ctx->mixed;
  const int nb = ctx->nbf, nx = ctx->naux, m = ctx->n_omega;
  int rc;
  {
    ProfScope ps(ctx, DONOF_RI_ROW_OTHER);
    split_C_kernel<<<ceil_div_u((long long)m * nb, 256), 256, 0, ctx->stream>>>(ctx->d_C, nb, mb->nbp, m, mb->Ct_hi,
                                                                                 mb->Ct_lo);
    DONOF_LAUNCH_CHECK(ctx);
  }
  {
    ProfScope ps(ctx, DONOF_RI_ROW_HALF);
    if ((rc = launch_tc<K_HALF>(ctx))) return rc;
  }
  {
    ProfScope ps(ctx, DONOF_RI_ROW_DIAG);
    diag_mixed_kernel<<<ceil_div_u((long long)nx * m * 32, 256), 256, 0, ctx->stream>>>(
        mb->bh3_hi, mb->bh3_lo, mb->Ct_hi, mb->Ct_lo, nb, mb->nbp, nx, m, mb->mp, mb->nxp, mb->d_hi, mb->d_lo);
    DONOF_LAUNCH_CHECK(ctx);
  }
  if (mode == DONOF_RI_FULL) {
    {
      ProfScope ps(ctx, DONOF_RI_ROW_FULL_K);
      if ((rc = launch_tc<K_FULLSQ>(ctx))) return rc;
      if ((rc = launch_reduce(ctx, K_FULLSQ, ctx->d_K, 0))) return rc;
    }
    {
      ProfScope ps(ctx, DONOF_RI_ROW_J);
      if ((rc = launch_tc<K_JMO>(ctx))) return rc;
      if ((rc = launch_reduce(ctx, K_JMO, ctx->d_J, 0))) return rc;
    }
  }
  return DONOF_RI_OK;
}

int mixed_jk_ao(donof_ri_ctx* ctx) {
  int rc;
  {
    ProfScope ps(ctx, DONOF_RI_ROW_JAO);
    if ((rc = launch_tc<K_JAO>(ctx))) return rc;
  }
  {
    ProfScope ps(ctx, DONOF_RI_ROW_KAO);
    if ((rc = launch_tc<K_KAO>(ctx))) return rc;
  }
  return DONOF_RI_OK;
}

int mixed_energy(donof_ri_ctx* ctx, int part) {
  MixedBuffers* mb = ctx->mixed;
  const int m = ctx->n_omega;
  const int nb = ctx->nbf;
  int rc;
  ProfScope ps(ctx, DONOF_RI_ROW_ENERGY);
  if (part & ENERGY_PREP) {
    if ((rc = launch_occupations_coupling(ctx))) return rc;
    fock_weights_kernel<<<ceil_div_u(2LL * m * m, 256), 256, 0, ctx->stream>>>(ctx->d_A, ctx->d_Bc, m, mb->W);
    DONOF_LAUNCH_CHECK(ctx);
    // (H C)^T[p][mu] = sum_nu C_{nu p} H_{mu nu}
    if ((rc = launch_dot64(ctx, m, nb, nb, ctx->d_C, nb, ctx->d_H, nb, mb->HCt, nb, 1))) return rc;
  }
  if (!(part & ENERGY_MAIN)) return DONOF_RI_OK;
  if ((rc = launch_tc<K_FOCK>(ctx))) return rc;
  if ((rc = launch_reduce(ctx, K_FOCK, mb->Yt, 1))) return rc;
  // lambda_qp = sum_mu C_{mu q} Y_{mu p}, column-major lambda[p*nb + q]
  if ((rc = launch_dot64(ctx, m, nb, nb, mb->Yt, nb, ctx->d_C, nb, ctx->d_lambda, nb, 1))) return rc;
  return launch_energy_rows(ctx, mb->HCt);
}

int mixed_fetch(donof_ri_ctx* ctx, int what, double* dst, size_t count) {
  MixedBuffers* mb = ctx->mixed;
  const int nb = ctx->nbf, nx = ctx->naux, m = ctx->n_omega;
  double* tmp = nullptr;
  if (cudaMalloc((void**)&tmp, count * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return DONOF_RI_E_OOM;
  }
  if (what == DONOF_RI_FETCH_BHALF) {
    // [P][p][nu] from the rows-p layout (row stride nbp, P stride mp*nbp)
    for (int P = 0; P < nx; ++P) {
      join_kernel<<<ceil_div_u((long long)m * nb, 256), 256, 0, ctx->stream>>>(
          mb->bh3_hi + (size_t)P * mb->mp * mb->nbp, mb->bh3_lo + (size_t)P * mb->mp * mb->nbp, m, nb, mb->nbp,
          tmp + (size_t)P * m * nb);
    }
  } else {
    join_diag_kernel<<<ceil_div_u((long long)nx * m, 256), 256, 0, ctx->stream>>>(mb->d_hi, mb->d_lo, nx, m, mb->nxp,
                                                                                   tmp);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(dst, tmp, count * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(tmp);
  return e == cudaSuccess ? DONOF_RI_OK : DONOF_RI_E_CUDA;
}

int mixed_copy_ao(donof_ri_ctx* ctx, double* Jao, double* Kao, bool jao_dev, bool kao_dev) {
  MixedBuffers* mb = ctx->mixed;
  const int nb = ctx->nbf, m = ctx->n_omega;
  const size_t n = (size_t)m * nb * nb;
  double* tmp = nullptr;
  if (cudaMalloc((void**)&tmp, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return DONOF_RI_E_OOM;
  }
  cudaError_t e = cudaSuccess;
  for (int which = 0; which < 2 && e == cudaSuccess; ++which) {
    double* dst = which == 0 ? Jao : Kao;
    bool dev = which == 0 ? jao_dev : kao_dev;
    if (!dst) continue;
    size_t off = (size_t)which * m * nb * mb->nbp;
    join_kernel<<<ceil_div_u((long long)n, 256), 256, 0, ctx->stream>>>(mb->JK_hi + off, mb->JK_lo + off,
                                                                         (long long)m * nb, nb, mb->nbp, tmp);
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dst, tmp, n * sizeof(double), dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  }
  cudaFree(tmp);
  return e == cudaSuccess ? DONOF_RI_OK : DONOF_RI_E_CUDA;
}

}  // namespace donof

// ---------------------------------------------------------------------------
// donof_ri_jmo_noalloc: J_pq = sum_P b^P_pp b^P_qq without any device allocation.
//
// For callers that cannot allocate device memory themselves or through this
// library (for example code running inside a memory pool or allocator that
// forbids cudaMalloc, or a host that must not grow its device footprint after
// start-up).  The split operands and the split-K partial sums live in the
// file-scope array below, which every GPU that loads this library holds until
// the process exits.
// ---------------------------------------------------------------------------
namespace donof {

constexpr size_t NOALLOC_SCRATCH_FLOATS = (size_t)6 << 20;  // 24 MiB
static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_SCRATCH_FLOATS];

struct NoallocDevice {
  std::atomic<bool> ready;
  float* scratch;  // device address of g_noalloc_scratch on this device
  PFN_cuTensorMapEncodeTiled_v12000 encode;
};
static NoallocDevice g_noalloc_dev[64];
// Serialises the one-time set-up of a device when several host threads make their
// first call at once; later calls read `ready` (acquire) and take no lock.
static std::mutex g_noalloc_setup_mu;

// J = sum of the chunk partials (fixed order), or NaN everywhere when a device-side
// wait of the GEMM timed out (its status word is non-zero): an aborted CTA leaves its
// partials unwritten, and the scratch array still holds an earlier call's.
__global__ void noalloc_reduce_kernel(const float* partial, int nsplit, int m, const int* status, double* J) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long mm = (long long)m * m;
  if (i >= mm) return;
  if (*status != 0) {
    J[i] = __longlong_as_double(0x7FF8000000000000LL);
    return;
  }
  double s = 0.0;
  for (int k = 0; k < nsplit; ++k) s += (double)partial[(size_t)k * mm + i];
  J[i] = s;
}

// d (FP64 [naux][m]) -> split rows [m][nxp] (hi, lo).
__global__ void noalloc_split_diag_kernel(const double* d, int nx, int m, int nxp, float* hi, float* lo) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx * m) return;
  int P = i / m, pc = i % m;
  float h, l;
  split_tf32((float)d[i], h, l);
  hi[(size_t)pc * nxp + P] = h;
  lo[(size_t)pc * nxp + P] = l;
}

static int noalloc_map(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap* map, const float* base, int nx, int m,
                       int nxp, int box_rows) {
  cuuint64_t gd[2] = {(cuuint64_t)nx, (cuuint64_t)m};
  cuuint64_t gs[1] = {(cuuint64_t)nxp * 4};
  cuuint32_t bd[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, gd, gs, bd, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? DONOF_RI_OK : DONOF_RI_E_CUDA;
}

}  // namespace donof

extern "C" int donof_ri_jmo_noalloc(const double* d, int naux, int n_omega, double* J, void* stream) {
  using namespace donof;
  if (!d || !J || naux < 1 || n_omega < 1 || naux > 65535 || n_omega > 4096) return DONOF_RI_E_ARG;
  const int nx = naux, m = n_omega;
  const int nxp = round_up(nx, 4);
  const int kbt = (nx + TC_BK - 1) / TC_BK;
  const int kbc = (kbt + 15) / 16;               // K blocks per chunk: at most 16 chunks
  const int nchunk = (kbt + kbc - 1) / kbc;
  const size_t split_floats = (size_t)round_up(m * nxp, 64);
  const size_t need = 2 * split_floats + (size_t)nchunk * m * m + 64;
  if (need > NOALLOC_SCRATCH_FLOATS) return DONOF_RI_E_ARG;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return DONOF_RI_E_CUDA;
  }
  NoallocDevice& nd = g_noalloc_dev[dev];
  if (!nd.ready.load(std::memory_order_acquire)) {
    // One-time set-up for this device (the current one): the device address of the
    // scratch array and the tensor-map encoder.
    std::lock_guard<std::mutex> lock(g_noalloc_setup_mu);
    if (!nd.ready.load(std::memory_order_relaxed)) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return DONOF_RI_E_CUDA;
      }
      if (get_encode(&nd.encode)) return DONOF_RI_E_UNSUPPORTED;
      nd.scratch = (float*)ptr;
      nd.ready.store(true, std::memory_order_release);
    }
  }
  float* d_hi = nd.scratch;
  float* d_lo = nd.scratch + split_floats;
  float* partial = nd.scratch + 2 * split_floats;
  int* status = (int*)(nd.scratch + NOALLOC_SCRATCH_FLOATS - 64);

  TcPlan pl{};
  const int bn = choose_bn(m, TC_SUM_MAXBN);
  plan_common(pl, bn, (m + TC_BM - 1) / TC_BM, (m + bn - 1) / bn, nchunk, nchunk, kbc);
  TcParams& p = pl.p;
  p.nb = 0; p.nx = nx; p.m = m; p.nbp = 0; p.nxp = nxp; p.mp = m;
  p.partial = partial;
  p.prow = m;
  p.pcol = m;
  p.N = m;
  p.K = nx;
  p.status = status;
  if (noalloc_map(nd.encode, &p.a_hi, d_hi, nx, m, nxp, TC_BM) || noalloc_map(nd.encode, &p.a_lo, d_lo, nx, m, nxp, TC_BM) ||
      noalloc_map(nd.encode, &p.b_hi, d_hi, nx, m, nxp, bn) || noalloc_map(nd.encode, &p.b_lo, d_lo, nx, m, nxp, bn))
    return DONOF_RI_E_CUDA;
  if (cudaFuncSetAttribute(tc_gemm_kernel<K_JMO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return DONOF_RI_E_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return DONOF_RI_E_CUDA;
  noalloc_split_diag_kernel<<<ceil_div_u((long long)nx * m, 256), 256, 0, s>>>(d, nx, m, nxp, d_hi, d_lo);
  tc_gemm_kernel<K_JMO><<<pl.grid, TC_THREADS, pl.smem, s>>>(p);
  noalloc_reduce_kernel<<<ceil_div_u((long long)m * m, 256), 256, 0, s>>>(partial, p.nsplit, m, status, J);
  return cudaGetLastError() == cudaSuccess ? DONOF_RI_OK : DONOF_RI_E_CUDA;
}
