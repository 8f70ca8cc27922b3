// Exact-accumulation BF16 digit-plane path (DONOF_RI_SLICE4) for sm_103a.
//
// Every GEMM operand row r is stored as a power-of-two exponent e_r and four
// balanced base-256 digits: X_rk = 2^(e_r - 31) Xint_rk with
//   Xint = d0 2^24 + d1 2^16 + d2 2^8 + d3,  |Xint| < 2^30,
//   d0 in [-64, 64], d1..d3 in [-128, 127],
// so the digits are small integers, exact in BF16, and the int32 Xint turns into
// digits with one addition (Xint + 0x808080: the top byte is d0, the others are
// d_t + 128).  The four digits of a row are stored interleaved per row:
// element (r, t, k) at [(r*4 + t)*ld + k], one TMA coordinate selecting t.
//
// A product of operand rows i and j is
//   sum_k A_ik B_jk = 2^(ea_i + eb_j - 62) sum_{t,u} 256^(6-t-u) sum_k dA_t dB_u,
// and the digit-pair products with t + u <= 4 (13 of the 16) are issued as
// tcgen05.mma kind::f16 into five FP32 TMEM accumulators, one per g = t + u.  The
// g = 4 group lies 2^-32 below the leading pair but is kept: for a row multiplied
// by itself (J_pp, K^(p)_{mu mu}) its (2,2) product is a sum of squares whose bias
// grows with K.  With |d0| <= 64 and |d1..d3| <= 128 one K element adds at most
// 2^12, 2^14, 2^15, 3 2^14, 3 2^14 to groups 0..4, so over a 512-wide K chunk
// every partial sum of groups 0..2 is an integer of magnitude <= 2^24 and their
// FP32 accumulation is exact; groups 3 and 4 may round once they pass 2^24, an
// error below 2^-38 of the leading group's scale.  After every chunk the
// epilogue combines the five sums: J_pq and the multi-chunk J^(q), K^(q) and full
// transform fold them into one int64 per output (v = sum_g G_g 2^(32 - 8g); the
// value is 2^(ea + eb - 46) v), so the reduction over K is exact in its leading
// 38 bits and independent of order; single-chunk units convert them straight to
// a double-float pair (groups_to_df); the half transform rounds each group term
// to an integer at its output scale (half_fold) and adds the chunks' integers.
// The other errors are the 31-bit digit representation of the operands and the
// dropped pair products (g >= 5).
// Outputs feeding another GEMM are re-digitised in integer arithmetic, with
// bound-based exponents (b_half) or exact row maxima (d, J^(q), K^(q)).
//
// Rows of the hot path as in tc.cu (HALF, FULLSQ, JMO, JAO, KAO, FOCK); the paper's
// equations: Sec. 2, Tables 2 and 3, Eq. (PNOF).
#include "common.cuh"
#include "tcgen05.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <stdlib.h>

#include <vector>

namespace donof {

// S_HALF1: the half transform with one CTA per SM, two accumulator sets and two
// epilogue warpgroups (the layout of the other kinds); the autotuner chooses
// between it and the two-CTA S_HALF.
// S_JKAO: J^(q) and K^(q) of one orbital iteration in one persistent launch (the
// J^(q) tiles, then the K^(q) (tile, orbital) units).
// S_CTR: the contracted Lagrangian's F^(p) C_p without J^(q), K^(q): one GEMM over
// K = (q, P), sum_q sum_P X^P_qp b^P_{q mu}, as one unit per orbital q (rows p of the
// X digits, columns mu of the b_half digits in the K^(q) layout, both over P) whose
// chunks are converted to double-float and summed across the CTA's orbitals.
enum S4Kind {
  S_HALF = 0, S_FULLSQ = 1, S_JMO = 2, S_JAO = 3, S_KAO = 4, S_FOCK = 5, S_HALF1 = 6, S_JKAO = 7, S_CTR = 8,
  S_NKINDS = 9
};
__host__ __device__ constexpr bool s4_half(int kind) { return kind == S_HALF || kind == S_HALF1; }

static_assert(DONOF_RI_GEMM_FOCK - DONOF_RI_GEMM_HALF == S_FOCK, "GEMM profile rows follow the kind order");

constexpr int S4_BM = 128;      // rows per tile
constexpr int S4_BK = 32;       // BF16 elements per K block (one 64-byte swizzle row)
constexpr int S4_KS = S4_BK / 16;  // MMA K steps per K block
constexpr int S4_CHUNK_KB = 16; // K blocks per chunk (512 elements; groups 0..2 exact)
// The kinds that contract over the orbital basis (K = nbf: the half and full
// transforms and F^(p) C_p) take chunks of up to 23 blocks (736 elements), so that
// a basis of up to 736 functions needs one epilogue drain per unit.  Past 512
// elements group 2's FP32 sum may round once it exceeds 2^24, which needs most of
// the chunk's top-digit products near their maximum; each rounding is at most one
// unit of the group, and the 3 K/16 accumulations into it add at most
// 3 K/16 2^(32-16) to the 2^(32 + 24.5)-scale sums: below 2^-30 of the largest
// value the chunk can hold (the operands' 31-bit digits already cost 2^-31).
constexpr int S4_CHUNK_KB_NB = 23;
// K blocks per epilogue chunk of a kind
__host__ __device__ constexpr int s4_chunk_kb(int kind) {
  return (s4_half(kind) || kind == S_FULLSQ || kind == S_FOCK) ? S4_CHUNK_KB_NB : S4_CHUNK_KB;
}
constexpr int S4_PLANES = 4;
constexpr int S4_NG = 5;        // digit-pair groups g = t + u = 0..4
constexpr int S4_SHIFT = 46;    // value = 2^(ea + eb - 46) v

// Columns per tile: five groups of BN columns per accumulator set.  The half
// transform runs two CTAs per SM, each with one set (5 x 48 = 240 of TMEM's 512
// columns): one MMA-issuing thread cannot keep the tensor pipe busy (each
// tcgen05.mma has a fixed issue latency), two can, and while one CTA drains its
// accumulators the other one's MMAs run.  The other kinds keep running sums in
// registers and run one CTA per SM with two ping-pong sets.  The full transform
// uses 32 columns.
template <int KIND>
struct S4Cfg {
  static constexpr int BN = 48;
  static constexpr int CTAS = (KIND == S_HALF) ? 2 : 1;  // CTAs per SM
  static constexpr int NSETS = CTAS == 2 ? 1 : 2;        // accumulator sets per CTA
  static constexpr int TMEM_COLS = CTAS == 2 ? 256 : 512;
  // Epilogue warpgroups: the kinds that carry running sums (int64 across K chunks
  // for J^(q), K^(q), J; double-float across units for a3 and a7) split the
  // columns over two warpgroups in 8-column blocks so that the sums stay in
  // registers; the half transform uses one.
  static constexpr int NWG = (KIND == S_HALF) ? 1 : 2;
  static constexpr int CW = NWG == 2 ? 8 : 16;
  static constexpr int THREADS = 64 + 128 * NWG;
  static constexpr int ES_WARP_BYTES = BN * 4 + BN * 8 + 4 * BN * 4 + BN * 16 * 4;
};

struct S4Params {
  CUtensorMap a, b;  // digit planes; coordinate 1 selects the digit
  CUtensorMap a2, b2;  // S_JKAO: the K^(q) operands (a, b: the J^(q) ones)
  int stages, tmem_cols;
  int n_tiles, nbatch, bpc, nsplit;
  int nb, nx, m, nbp, nxp, mp;  // nbp / nxp: BF16 row strides (multiples of 8)
  const int* ea;
  const int* eb;
  __nv_bfloat16* o3;  // HALF: L3 digits [nx][mp][4][nbp]
  const int* e3;
  int* x6;            // HALF: b_half integers [nx][m][nbp] at scale min(e3, e6) (xf_to_digits_kernel)
  const int* e6;
  float* ohi;
  float* olo;
  int ldo;
  void* partial;
  int prow, pcol;
  const float2* w;  // FOCK weights as double-float pairs [2m][m]
  int* status;
  int persist;      // 1: units are whole tiles, CTA c takes tiles c, c + grid, ...
  int ntiles;       // total tiles (persistent kinds)
  const int* tmap;  // optional list of the tiles to compute, (mt << 16) | nt (K^(q): upper triangle)
  // S_JKAO: units [0, u_split) are J^(q) tiles (tmap, exponents ea / eb), the rest
  // (tile, orbital) units of K^(q) (tmap2 of ntiles2 tiles, exponents ea2 / eb2)
  const int* tmap2;
  const int* ea2;
  const int* eb2;
  int ntiles2, u_split;
  double* bfull;    // FULLSQ: when set, b^P_qp is also stored, [P][q][p] (FP64)
};

// ---------------------------------------------------------------------------
// integer / double-float helpers
// ---------------------------------------------------------------------------
// Four balanced digits of |X| < 2^30 as BF16 values.  U = X + 0x80808080 holds
// digit + 128 in each byte (the top digit lies in [-64, 64]).  A byte b placed
// under the exponent of 2^23 reads as the float 2^23 + b, and subtracting
// 2^23 + 128 leaves the digit exactly; an integer of at most 8 significant bits
// is exact in BF16, so its BF16 pattern is the top half of the FP32 pattern.
__device__ __forceinline__ void digits_bf16(int X, __nv_bfloat16 d[4]) {
  const unsigned int U = (unsigned int)X + 0x80808080u;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const float x = __uint_as_float(__byte_perm(U, 0x4B000000u, 0x7440u | (unsigned int)(3 - t))) - 8388736.0f;
    d[t] = __ushort_as_bfloat16((unsigned short)(__float_as_uint(x) >> 16));
  }
}

// The digits of two integers at once, as BF16 pairs (d[t].x from X0, d[t].y from X1):
// the same exact digit values, each pair rounded to BF16 by one packed conversion
// (exact: every digit has at most 8 significant bits).
__device__ __forceinline__ void digits_bf16x2(int X0, int X1, __nv_bfloat162 d[4]) {
  const unsigned int U0 = (unsigned int)X0 + 0x80808080u, U1 = (unsigned int)X1 + 0x80808080u;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const unsigned int sel = 0x7440u | (unsigned int)(3 - t);
    const float x0 = __uint_as_float(__byte_perm(U0, 0x4B000000u, sel)) - 8388736.0f;
    const float x1 = __uint_as_float(__byte_perm(U1, 0x4B000000u, sel)) - 8388736.0f;
    d[t] = __floats2bfloat162_rn(x0, x1);
  }
}

// Exponent e with |x| < 2^(e-1) for every |x| <= amax (amax >= 0); 0 for amax == 0.
__device__ __forceinline__ int expo_of(double amax) {
  if (!(amax > 0.0)) return 0;
  int k;
  frexp(amax, &k);
  return k + 1;
}

// expo_of((double)mx * (1 + 2^-16)) for an FP32 bound mx, in integer arithmetic
// (the product is exact in FP64: 24 x 17 significant bits).  With mx = I0 2^(E-150),
// I0 = 2^23 + mantissa, the product is I0 (2^16 + 1) 2^(E-166), whose frexp
// exponent is E - 126, or E - 125 once I0 (2^16 + 1) reaches 2^40.  Zero,
// subnormal and non-finite bounds take the FP64 route.  (FP64 instructions run
// at a small fraction of the FP32 rate; these bounds are taken once per row.)
__device__ __forceinline__ int expo_of_inflated(float mx) {
  const unsigned int b = __float_as_uint(mx);
  const int E = (int)((b >> 23) & 0xFFu);
  if (mx > 0.f && E > 0 && E < 255) {
    const unsigned long long I = (unsigned long long)((b & 0x7FFFFFu) | 0x800000u) * 65537ull;
    return E - 125 + (I >= (1ull << 40) ? 1 : 0);
  }
  return expo_of((double)mx * (1.0 + 1.0 / 65536.0));
}

// x 2^k for FP64 x: one multiplication by an exact power of two while 2^k is a
// normal double (the same correctly rounded result as ldexp), ldexp beyond.
__device__ __forceinline__ double scale_pow2(double x, int k) {
  if (k >= -1022 && k <= 1023) return x * __longlong_as_double((long long)(k + 1023) << 52);
  return ldexp(x, k);
}

// FP64 -> double-float pair (h + l = x to about 2^-48 relative).
__device__ __forceinline__ float2 to_df(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}
__device__ __forceinline__ float2 to_df(float2 x) { return x; }

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (sh, sl) += (ph, pl) in double-float arithmetic.
__device__ __forceinline__ void df_add(float& sh, float& sl, float ph, float pl) {
  float s, e;
  two_sum_f(sh, ph, s, e);
  e += sl + pl;
  sh = s + e;
  sl = e - (sh - s);
}

// 2^k as an FP32 value for k in [-126, 127] (k is clamped to that range).
__device__ __forceinline__ float exp2_int(int k) {
  k = k < -126 ? -126 : (k > 127 ? 127 : k);
  return __int_as_float((k + 127) << 23);
}

// (h, l) *= 2^k: one multiplication each while 2^k is a normal float, ldexpf beyond.
__device__ __forceinline__ void df_scale(float& h, float& l, int k) {
  if (k >= -126 && k <= 127) {
    const float sc = exp2_int(k);
    h *= sc;
    l *= sc;
  } else {
    h = ldexpf(h, k);
    l = ldexpf(l, k);
  }
}

// int64 * 2^k as a double-float pair, built from 32-bit pieces only (|v| < 2^55):
// v = a 2^32 + b1 2^16 + b0 with every piece exact in FP32, summed with TwoSum.
__device__ __forceinline__ void ll_to_df(long long v, int k, float& h, float& l) {
  const int a = (int)(v >> 32);
  const unsigned int lo = (unsigned int)v;
  const float fa = ldexpf((float)a, 32), f1 = ldexpf((float)(lo >> 16), 16), f0 = (float)(lo & 0xFFFFu);
  float s, e;
  two_sum_f(fa, f1, s, e);
  float s2, e2;
  two_sum_f(s, f0, s2, e2);
  const float t = e + e2;
  h = s2 + t;
  l = t - (h - s2);
  df_scale(h, l, k);
}

// Double-float value of one chunk's five group sums, sum_g G_g 2^(32 - 8g + k),
// without the int64 fold: every term G_g 2^(-8g) is exact in FP32 (a power-of-two
// scaling), a TwoSum chain adds them with the rounding errors collected in e, and
// the pair is scaled by 2^(32 + k) at the end.  Relative error about 2^-48, the same
// order as the int64 fold followed by its conversion.
__device__ __forceinline__ void groups_to_df(const uint32_t* G, int k, float& h, float& l) {
  float sum = __uint_as_float(G[0]), e = 0.f;
#pragma unroll
  for (int g = 1; g < S4_NG; ++g) {
    float t, err;
    two_sum_f(sum, __uint_as_float(G[g]) * exp2_int(-8 * g), t, err);
    sum = t;
    e += err;
  }
  h = sum + e;
  l = e - (h - sum);
  df_scale(h, l, 32 + k);
}

// Output integer of the half transform from one chunk's group sums:
// X = sum_g rint(G_g 2^(sigma - 8 g)), clamped to [-2^30, 2^30], with
// H_g = G_g 2^(-8 g) (exact).  Each term is rounded on its own, so X differs
// from round(v 2^(sigma - 32)) by at most 2.5; the row exponents guarantee
// |X| < 2^30 (the leading term is X to within a few per cent), so no term
// reaches the int32 range.
__device__ __forceinline__ int half_fold(const float H[S4_NG], int sigma) {
  const float sc = exp2_int(sigma);
  int X = 0;
#pragma unroll
  for (int g = 0; g < S4_NG; ++g) X += __float2int_rn(H[g] * sc);
  X = X > (1 << 30) ? (1 << 30) : X;
  X = X < -(1 << 30) ? -(1 << 30) : X;
  return X;
}

// round(X 2^-d) for d >= 0 (halves rounded up), without overflow.
__device__ __forceinline__ int rshift_round(int X, int d) {
  if (d <= 0) return X;
  const int sh = d - 1 > 31 ? 31 : d - 1;
  return ((X >> sh) + 1) >> 1;
}

// ---------------------------------------------------------------------------
// The digit-plane GEMM kernel
// ---------------------------------------------------------------------------
template <int KIND>
__device__ __forceinline__ void s4_unit(const S4Params& p, int b, int& batch, int& kb0, int& nkb) {
  const int KBb = (p.nb + S4_BK - 1) / S4_BK, KBx = (p.nx + S4_BK - 1) / S4_BK;
  if (s4_half(KIND)) { batch = 0; kb0 = 0; nkb = KBb; }
  else if (KIND == S_FULLSQ) { batch = b; kb0 = 0; nkb = KBb; }
  else if (KIND == S_JMO) { batch = 0; kb0 = b * S4_CHUNK_KB; nkb = min(S4_CHUNK_KB, KBx - kb0); }
  else if (KIND == S_JAO || KIND == S_JKAO) { batch = 0; kb0 = 0; nkb = KBx; }
  else if (KIND == S_KAO || KIND == S_CTR) { batch = b; kb0 = 0; nkb = KBx; }
  else {
    constexpr int CKB = s4_chunk_kb(KIND);
    const int nc = (KBb + CKB - 1) / CKB;
    batch = b / nc;
    kb0 = (b % nc) * CKB;
    nkb = min(CKB, KBb - kb0);
  }
}

// Persistent unit U -> (K^(q) unit?, batch entry, tile (mt, nt)).
template <int KIND>
__device__ __forceinline__ void s4_persist_unit(const S4Params& p, int U, bool& kao, int& batch, int& mt, int& nt) {
  const int* tm = p.tmap;
  int ntl = p.ntiles, V = U;
  kao = (KIND == S_KAO);
  if (KIND == S_JKAO) {
    if (U >= p.u_split) {
      kao = true;
      V = U - p.u_split;
      tm = p.tmap2;
      ntl = p.ntiles2;
    } else {
      ntl = p.u_split;
    }
  }
  batch = V / ntl;
  const int tl = V % ntl;
  mt = tm ? tm[tl] >> 16 : tl / p.n_tiles;
  nt = tm ? tm[tl] & 0xFFFF : tl % p.n_tiles;
}

template <int KIND>
__device__ __forceinline__ void s4_loads(const S4Params& p, uint8_t* st, uint64_t* bar, int mt, int nt, int batch,
                                         int kb, bool kao) {
  constexpr int BN = S4Cfg<KIND>::BN;
  const int k0 = kb * S4_BK, n0 = nt * BN;
#pragma unroll
  for (int t = 0; t < S4_PLANES; ++t) {
    uint8_t* da = st + t * (S4_BM * S4_BK * 2);
    uint8_t* db = st + S4_PLANES * (S4_BM * S4_BK * 2) + t * (BN * S4_BK * 2);
    if (s4_half(KIND)) {
      const int nvb = (p.nb + 15) / 16;
      tma_load_4d(da, &p.a, bar, k0, t, (mt % nvb) * 16, (mt / nvb) * 8);
      tma_load_3d(db, &p.b, bar, k0, t, n0);
    } else if (KIND == S_FULLSQ) {
      tma_load_4d(da, &p.a, bar, k0, t, mt * S4_BM, batch);
      tma_load_3d(db, &p.b, bar, k0, t, n0);
    } else if (KIND == S_FOCK) {
      tma_load_3d(da, &p.a, bar, k0, t, mt * S4_BM);
      tma_load_4d(db, &p.b, bar, k0, t, n0, batch);
    } else if (KIND == S_JMO || KIND == S_JAO || (KIND == S_JKAO && !kao)) {
      tma_load_3d(da, &p.a, bar, k0, t, mt * S4_BM);
      tma_load_3d(db, &p.b, bar, k0, t, n0);
    } else if (KIND == S_JKAO) {  // K^(q) unit of the merged launch
      tma_load_4d(da, &p.a2, bar, k0, t, mt * S4_BM, batch);
      tma_load_4d(db, &p.b2, bar, k0, t, n0, batch);
    } else {  // S_KAO, S_CTR
      tma_load_4d(da, &p.a, bar, k0, t, mt * S4_BM, batch);
      tma_load_4d(db, &p.b, bar, k0, t, n0, batch);
    }
  }
}

template <int KIND, int ONE>
__global__ void __launch_bounds__(S4Cfg<KIND>::THREADS, S4Cfg<KIND>::CTAS) s4_gemm_kernel(const __grid_constant__ S4Params p) {
  // ONE: every unit is a single K chunk (K <= 512, and always for F^(p) C_p), so the
  // epilogue converts group sums straight to double-float pairs and carries no int64
  // running sums; chosen at launch from the problem's K extent.
  constexpr int BN = S4Cfg<KIND>::BN;
  constexpr int NWG = S4Cfg<KIND>::NWG, CW = S4Cfg<KIND>::CW;
  constexpr int NCBT = BN / CW / NWG;  // column blocks per epilogue thread
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int S = p.stages;
  constexpr int NSETS = S4Cfg<KIND>::NSETS;
  constexpr uint32_t a_bytes = S4_PLANES * S4_BM * S4_BK * 2, b_bytes = S4_PLANES * BN * S4_BK * 2;
  constexpr uint32_t stage_bytes = a_bytes + b_bytes;
  uint64_t* full = (uint64_t*)(smem + (size_t)S * stage_bytes);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;
  uint64_t* acce = accf + 2;
  uint64_t* drain = acce + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  // Epilogue scratch (after the 256-byte barrier block), one copy per epilogue warp so
  // that staging needs only __syncwarp: the current unit's per-column exponents /
  // weights and, for HALF, the output exponents of the warp's rows.
  constexpr int ES_WARP_BYTES = S4Cfg<KIND>::ES_WARP_BYTES;
  const int ew = threadIdx.x / 32 >= 2 ? threadIdx.x / 32 - 2 : 0;  // epilogue warp index
  uint8_t* es_base = smem + (size_t)S * stage_bytes + 256 + (size_t)ew * ES_WARP_BYTES;
  int* es_b = (int*)es_base;              // [BN]
  float2* es_w = (float2*)(es_b + BN);    // [BN]
  int* es_3 = (int*)(es_w + BN);          // [4][BN]: the warp's 4 auxiliary rows P
  int* es_6 = es_3 + 4 * BN;              // [BN][16]

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  // Work assignment.  Persistent kinds (no sums across units): unit U = blockIdx.x +
  // u*gridDim.x of ntiles x nbatch, tile U % ntiles of batch entry U / ntiles.  Other
  // kinds: the CTA owns one tile and a contiguous range of its batch entries, with the
  // tile fastest in blockIdx so that the CTAs running at the same time cover every
  // tile of the same batch range and share its A rows through L2.
  const int tile0 = p.persist ? (int)blockIdx.x : (int)blockIdx.x % p.ntiles;
  const int split = p.persist ? 0 : (int)blockIdx.x / p.ntiles;
  const int b0 = split * p.bpc;
  const int nunits = p.persist ? max(0, (p.ntiles * p.nbatch - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x)
                               : max(0, min(p.nbatch, b0 + p.bpc) - b0);
  int mt = tile0 / p.n_tiles, nt = tile0 % p.n_tiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&accf[a], 1);
      mbar_init(&acce[a], 128 * NWG);
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
  // barriers and TMEM are set up; global memory only from here on
  pdl_entry();

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int it = 0;
      bool ok = true;
      for (int u = 0; u < nunits && ok; ++u) {
        int batch, kb0, nkb;
        bool kao = (KIND == S_KAO);
        const int U = tile0 + u * (int)gridDim.x;
        s4_unit<KIND>(p, p.persist ? U / p.ntiles : b0 + u, batch, kb0, nkb);
        if (p.persist) s4_persist_unit<KIND>(p, U, kao, batch, mt, nt);
        for (int kb = 0; kb < nkb; ++kb) {
          const int s = it % S;
          if (!mbar_wait(&empty[s], (uint32_t)(((it / S) & 1) ^ 1), abort_flag, p.status)) { ok = false; break; }
          mbar_expect_tx(&full[s], stage_bytes);
          s4_loads<KIND>(p, smem + (size_t)s * stage_bytes, &full[s], mt, nt, batch, kb0 + kb, kao);
          ++it;
        }
      }
      for (int j = max(0, it - S); j < it; ++j) mbar_wait(&full[j % S], (uint32_t)((j / S) & 1), nullptr, p.status);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      // The B planes of a stage sit one above the other (plane u at rows u*BN), so one
      // MMA of N = 4*BN multiplies digit plane t of A by all four B planes and, with the
      // accumulator window shifted by t*BN columns, adds product (t,u) to group t+u.
      // Window t covers groups t..min(t+3,4): four MMAs per K step instead of 13.
      const uint32_t id1 = idesc_bf16(BN), id2 = idesc_bf16(2 * BN), id3 = idesc_bf16(3 * BN),
                     id4 = idesc_bf16(4 * BN);
      int it = 0, cc = 0;
      bool ok = true;
      for (int u = 0; u < nunits && ok; ++u) {
        int batch, kb0, nkb;
        s4_unit<KIND>(p, p.persist ? (tile0 + u * (int)gridDim.x) / p.ntiles : b0 + u, batch, kb0, nkb);
        constexpr int CKB = s4_chunk_kb(KIND);
        for (int ch = 0; ch * CKB < nkb && ok; ++ch) {
          const int set = cc % NSETS;
          if (!mbar_wait(&acce[set], (uint32_t)(((cc / NSETS) & 1) ^ 1), abort_flag, p.status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t dbase = tmem_base + (uint32_t)(set * S4_NG * BN);
          const int kbs = min(CKB, nkb - ch * CKB);
          for (int j = 0; j < kbs; ++j) {
            const int s = it % S;
            if (!mbar_wait(&full[s], (uint32_t)((it / S) & 1), abort_flag, p.status)) { ok = false; break; }
            tc_fence_after();
            const uint32_t st = smem_u32(smem + (size_t)s * stage_bytes);
            uint64_t dA[S4_PLANES], dB[S4_PLANES];
#pragma unroll
            for (int t = 0; t < S4_PLANES; ++t) {
              dA[t] = sdesc_sw64(st + (uint32_t)t * (S4_BM * S4_BK * 2));
              dB[t] = sdesc_sw64(st + a_bytes + (uint32_t)t * (BN * S4_BK * 2));
            }
            // K step ks: +32 bytes inside the 64-byte swizzle row (+2 in the descriptor's address field)
#pragma unroll
            for (int ks = 0; ks < S4_KS; ++ks) {
              const uint64_t o = (uint64_t)(2 * ks);
              if (j == 0 && ks == 0) {
                // First step of a chunk: every group block must be written once with
                // accumulate = 0 before any MMA adds to it.  Window 1 initialises groups
                // 1..4; group 0 is initialised by (0,0) alone and (0,1..3) then adds.
                mma_bf16(dbase + (uint32_t)BN, dA[1] + o, dB[0] + o, id4, 0u);
                mma_bf16(dbase, dA[0] + o, dB[0] + o, id1, 0u);
                mma_bf16(dbase + (uint32_t)BN, dA[0] + o, dB[1] + o, id3, 1u);
              } else {
                mma_bf16(dbase, dA[0] + o, dB[0] + o, id4, 1u);
                mma_bf16(dbase + (uint32_t)BN, dA[1] + o, dB[0] + o, id4, 1u);
              }
              mma_bf16(dbase + (uint32_t)(2 * BN), dA[2] + o, dB[0] + o, id3, 1u);
              mma_bf16(dbase + (uint32_t)(3 * BN), dA[3] + o, dB[0] + o, id2, 1u);
            }
            mma_commit(&empty[s]);
            ++it;
          }
          if (!ok) break;
          mma_commit(&accf[set]);
          ++cc;
        }
      }
      // All MMAs of this thread must complete before TMEM is released.
      mma_commit(drain);
      mbar_wait(drain, 0, nullptr, p.status);
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    // Each thread owns one output row (its TMEM lane).  Per 16-column block the five
    // exact group sums of a chunk are folded into int64 values; a block is finalised
    // (stored, squared or weighted) as soon as the last chunk of its unit is drained.
    // HALF / JAO / KAO / JMO keep the column-block loop rolled (their per-output code
    // is long) with running int64 sums in small per-thread arrays; FULLSQ and FOCK
    // unroll it and keep their sums in registers.
    const int q = warp & 3;     // TMEM lane quarter this warp may access
    const int wg = ew / 4;      // epilogue warpgroup: column blocks wg, wg + NWG, ...
    const int row = q * 32 + lane;
    constexpr bool SUM_DF = (KIND == S_FULLSQ || KIND == S_FOCK || KIND == S_CTR);
    // FOCK units are single chunks, CTR converts every chunk on its own, and the half
    // transform keeps its partial sums in its output: none carries int64 running sums
    constexpr int NACC = (KIND == S_FOCK || KIND == S_CTR || s4_half(KIND)) ? 1 : BN / NWG;
    long long acc[NACC];
    float sh[SUM_DF ? BN / NWG : 1], sl[SUM_DF ? BN / NWG : 1];
#pragma unroll
    for (int i = 0; i < NACC; ++i) acc[i] = 0;
#pragma unroll
    for (int i = 0; i < (SUM_DF ? BN / NWG : 1); ++i) {
      sh[i] = 0.f;
      sl[i] = 0.f;
    }
    int cc = 0, units_done = 0;
    bool ok = true;
    for (int u = 0; u < nunits && ok; ++u) {
      int batch, kb0, nkb;
      bool kao = (KIND == S_KAO);
      const int U = tile0 + u * (int)gridDim.x;
      s4_unit<KIND>(p, p.persist ? U / p.ntiles : b0 + u, batch, kb0, nkb);
      if (p.persist) s4_persist_unit<KIND>(p, U, kao, batch, mt, nt);
      // the merged kind's exponents for this unit
      const int* eA = (KIND == S_JKAO && kao) ? p.ea2 : p.ea;
      const int* eB = (KIND == S_JKAO && kao) ? p.eb2 : p.eb;
      // Stage this unit's column exponents (and weights) in shared memory: one pass of
      // coalesced loads per warp instead of a dependent global load per output column.
      if (KIND != S_JMO) {
        // All of a lane's loads are issued before any of them is stored, so the warp
        // waits for one memory latency rather than one per element.
        __syncwarp();
        constexpr int NLB = (BN + 31) / 32;
        int rb[NLB];
#pragma unroll
        for (int k = 0; k < NLB; ++k) {
          const int i = lane + 32 * k, col = nt * BN + i;
          rb[k] = 0;
          if (i < BN) {
            if (KIND == S_KAO || KIND == S_FOCK || KIND == S_CTR || (KIND == S_JKAO && kao))
              rb[k] = col < p.nb ? eB[(size_t)batch * p.nb + col] : 0;
            else rb[k] = col < p.m ? eB[col] : 0;
          }
        }
        if (s4_half(KIND)) {
          const int nvb = (p.nb + 15) / 16;
          const int Pb = mt / nvb, vb = mt % nvb;
          constexpr int N3 = 2 * BN / 32, N6 = BN * 16 / 32;
          static_assert(!s4_half(KIND) || (2 * BN) % 32 == 0, "staging assumes 2*BN divisible by 32");
          int r3[N3], r6[N6];
#pragma unroll
          for (int k = 0; k < N3; ++k) {
            const int i = lane + 32 * k;
            const int P = Pb * 8 + q * 2 + i / BN, pc = nt * BN + i % BN;
            r3[k] = (P < p.nx && pc < p.m) ? p.e3[(size_t)P * p.m + pc] : 0;
          }
#pragma unroll
          for (int k = 0; k < N6; ++k) {
            const int i = lane + 32 * k;
            const int pc = nt * BN + i / 16, nu = vb * 16 + i % 16;
            r6[k] = (pc < p.m && nu < p.nb) ? p.e6[(size_t)pc * p.nb + nu] : 0;
          }
#pragma unroll
          for (int k = 0; k < N3; ++k) es_3[lane + 32 * k] = r3[k];
#pragma unroll
          for (int k = 0; k < N6; ++k) es_6[lane + 32 * k] = r6[k];
        }
#pragma unroll
        for (int k = 0; k < NLB; ++k) {
          const int i = lane + 32 * k;
          if (i < BN) es_b[i] = rb[k];
        }
        __syncwarp();
      }
      // row-dependent data of the unit
      int ea = 0;
      bool rvalid = false;
      int P = 0, nu = 0, mu = 0;
      if (s4_half(KIND)) {
        // M tile = 16 nu x 8 P with nu fastest: a warp holds 16 consecutive nu of two
        // auxiliary rows, so each L3 digit row it stores is one full 32-byte sector.
        const int nvb = (p.nb + 15) / 16;
        P = (mt / nvb) * 8 + row / 16;
        nu = (mt % nvb) * 16 + row % 16;
        rvalid = P < p.nx && nu < p.nb;
        ea = rvalid ? p.ea[(size_t)P * p.nb + nu] : 0;
      } else if (KIND == S_FULLSQ) {
        mu = mt * S4_BM + row;
        rvalid = mu < p.m;
        ea = rvalid ? p.ea[(size_t)batch * p.m + mu] : 0;
      } else if (KIND == S_JAO || (KIND == S_JKAO && !kao)) {
        const int r = mt * S4_BM + row;
        rvalid = r < p.nb * p.nb;
        mu = r / p.nb;
        nu = r % p.nb;
        ea = rvalid ? eA[r] : 0;
      } else if (KIND == S_KAO || KIND == S_JKAO) {
        mu = mt * S4_BM + row;
        rvalid = mu < p.nb;
        ea = rvalid ? eA[(size_t)batch * p.nb + mu] : 0;
      } else if (KIND == S_CTR) {
        // the row is orbital p of the X digits of orbital q = batch
        mu = mt * S4_BM + row;
        rvalid = mu < p.m;
        ea = rvalid ? p.ea[(size_t)batch * p.m + mu] : 0;
      }
      // FOCK: the row is orbital p (C^T digits), the unit's weight W[batch][p] is per row
      float2 wrow = make_float2(0.f, 0.f);
      if (KIND == S_FOCK) {
        mu = mt * S4_BM + row;
        rvalid = mu < p.m;
        ea = rvalid ? p.ea[mu] : 0;
        wrow = rvalid ? p.w[(size_t)batch * p.m + mu] : wrow;
      }
      const int nch = (nkb + s4_chunk_kb(KIND) - 1) / s4_chunk_kb(KIND);
      for (int ch = 0; ch < nch; ++ch) {
        const int set = cc % NSETS;
        if (!mbar_wait(&accf[set], (uint32_t)((cc / NSETS) & 1), abort_flag, p.status)) { ok = false; break; }
        tc_fence_after();
        const uint32_t tb = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(set * S4_NG * BN);
        const bool last = (ch == nch - 1);
#pragma unroll(SUM_DF || NWG == 2 ? NCBT : 1)
        for (int cb = 0; cb < NCBT; ++cb) {
          const int c = cb * NWG + wg;  // column block (CW columns)
          // group g holds digit pairs with t + u = g; its weight is 2^(32 - 8 g) in units of 2^(ea+eb-46)
          uint32_t gr[S4_NG][CW];
#pragma unroll
          for (int g = 0; g < S4_NG; ++g) {
            if (CW == 16) tmem_ld16_issue(tb + (uint32_t)(g * BN + c * CW), gr[g]);
            else tmem_ld8_issue(tb + (uint32_t)(g * BN + c * CW), gr[g]);
          }
#pragma unroll
          for (int g = 0; g < S4_NG; ++g) {
            if (CW == 16) tmem_wait16(gr[g]);
            else tmem_wait8(gr[g]);
          }
          if (s4_half(KIND)) {
            // Half transform: one output integer at the finer of the two output scales
            // (exponents e3, e6), X = sum_g rint(G_g 2^(sigma - 8g)) in int32 per chunk
            // (see half_fold), without an int64 fold.  A unit of several K chunks adds
            // each chunk's integer to the one the same thread stored for the previous
            // chunk of this unit (a read of its own write, held in L2) and clamps the
            // sum, so no running sums occupy registers or local memory; each chunk adds
            // at most 2.5 units of rounding.  xf_to_digits_kernel derives both digit
            // layouts from the final integer.
            if (!rvalid) continue;
            const int lrow = lane / 16, l16 = lane % 16;
            int* basef = p.x6 + (size_t)P * p.m * p.nbp + nu;
            int prev[ONE ? 1 : CW];
            if (!ONE && ch > 0) {
#pragma unroll
              for (int j = 0; j < CW; ++j) {
                const int col = nt * BN + c * CW + j;
                prev[j] = col < p.m ? basef[(size_t)col * p.nbp] : 0;
              }
            }
#pragma unroll
            for (int j = 0; j < CW; ++j) {
              const int i = c * CW + j;
              const int col = nt * BN + i;
              if (col < p.m) {
                float H[S4_NG];
#pragma unroll
                for (int g = 0; g < S4_NG; ++g) H[g] = __uint_as_float(gr[g][j]) * exp2_int(-8 * g);
                const int emin = min(es_3[lrow * BN + i], es_6[i * 16 + l16]);
                int X = half_fold(H, ea + es_b[i] + 17 - emin);
                if (!ONE && ch > 0) {
                  long long t = (long long)prev[j] + X;
                  t = t > (1LL << 30) ? (1LL << 30) : (t < -(1LL << 30) ? -(1LL << 30) : t);
                  X = (int)t;
                }
                basef[(size_t)col * p.nbp] = X;
              }
            }
            continue;
          }
          if (KIND == S_JMO) {
            // int64 fold: running sums over K chunks (J_pq's partials stay integers)
            long long v[CW];
#pragma unroll
            for (int j = 0; j < CW; ++j) v[j] = (ch > 0 || KIND == S_JMO) ? acc[NACC == 1 ? 0 : cb * CW + j] : 0;
#pragma unroll
            for (int g = 0; g < S4_NG; ++g) {
#pragma unroll
              for (int j = 0; j < CW; ++j) v[j] += (long long)__float2int_rn(__uint_as_float(gr[g][j])) << (32 - 8 * g);
            }
            if (!last || KIND == S_JMO) {
#pragma unroll
              for (int j = 0; j < CW; ++j) acc[NACC == 1 ? 0 : cb * CW + j] = v[j];
              continue;
            }
            continue;
          }
          // The value of every output of the block as a double-float pair (h, l).  A
          // single-chunk unit converts its five group sums directly (groups_to_df); a
          // multi-chunk one keeps exact int64 running sums until its last chunk.  CTR
          // converts every chunk and adds it to the CTA's running double-float sums
          // (the exponents are the same for the chunks of a unit, not across units).
          float hv[CW], lv[CW];
          if (ONE || KIND == S_CTR) {
#pragma unroll
            for (int j = 0; j < CW; ++j) {
              const uint32_t G[S4_NG] = {gr[0][j], gr[1][j], gr[2][j], gr[3][j], gr[4][j]};
              groups_to_df(G, ea + es_b[c * CW + j] - S4_SHIFT, hv[j], lv[j]);
            }
          } else {
            long long v[CW];
#pragma unroll
            for (int j = 0; j < CW; ++j) v[j] = ch > 0 ? acc[NACC == 1 ? 0 : cb * CW + j] : 0;
#pragma unroll
            for (int g = 0; g < S4_NG; ++g) {
#pragma unroll
              for (int j = 0; j < CW; ++j) v[j] += (long long)__float2int_rn(__uint_as_float(gr[g][j])) << (32 - 8 * g);
            }
            if (!last) {
#pragma unroll
              for (int j = 0; j < CW; ++j) acc[NACC == 1 ? 0 : cb * CW + j] = v[j];
              continue;
            }
#pragma unroll
            for (int j = 0; j < CW; ++j) ll_to_df(v[j], ea + es_b[c * CW + j] - S4_SHIFT, hv[j], lv[j]);
          }
          // ---- the block's values are final: unit action ----
          if (!rvalid) continue;
          if (KIND == S_FULLSQ) {
#pragma unroll
            for (int j = 0; j < CW; ++j) {
              const int i = c * CW + j;
              if (nt * BN + i < p.m) {
                const float xh = hv[j], xl = lv[j];
                const float ph = xh * xh;
                const float pl = fmaf(xh, xh, -ph) + 2.f * xh * xl;
                df_add(sh[SUM_DF ? cb * CW + j : 0], sl[SUM_DF ? cb * CW + j : 0], ph, pl);
                if (p.bfull) p.bfull[((size_t)batch * p.m + mu) * p.m + nt * BN + i] = (double)xh + (double)xl;
              }
            }
          } else if (KIND == S_FOCK) {
#pragma unroll
            for (int j = 0; j < CW; ++j) {
              const int i = c * CW + j;
              if (nt * BN + i < p.nb) {
                const float xh = hv[j], xl = lv[j];
                const float2 wv = wrow;
                const float ph = xh * wv.x;
                const float pl = fmaf(xh, wv.x, -ph) + (xh * wv.y + xl * wv.x);
                df_add(sh[SUM_DF ? cb * CW + j : 0], sl[SUM_DF ? cb * CW + j : 0], ph, pl);
              }
            }
          } else if (KIND == S_CTR) {
#pragma unroll
            for (int j = 0; j < CW; ++j) {
              if (nt * BN + c * CW + j < p.nb) df_add(sh[SUM_DF ? cb * CW + j : 0], sl[SUM_DF ? cb * CW + j : 0], hv[j], lv[j]);
            }
          } else if (KIND == S_JAO || (KIND == S_JKAO && !kao)) {
#pragma unroll
            for (int j = 0; j < CW; ++j) {
              const int i = c * CW + j;
              const int col = nt * BN + i;
              if (col < p.m) {
                const size_t o = ((size_t)col * p.nb + mu) * p.ldo + nu;
                p.ohi[o] = hv[j];
                p.olo[o] = lv[j];
              }
            }
          } else if (KIND == S_KAO || KIND == S_JKAO) {
            // A thread's CW = 8 consecutive columns of one output row are one 32-byte
            // sector of hi and one of lo (ldo is a multiple of 8): two 16-byte vector
            // stores each instead of eight scattered 4-byte ones.
            const int col0 = nt * BN + c * CW;
            const size_t o = ((size_t)(p.m + batch) * p.nb + mu) * p.ldo + col0;
            if (CW == 8 && col0 + CW <= p.nb) {
              float4* dh = (float4*)(p.ohi + o);
              float4* dl = (float4*)(p.olo + o);
              dh[0] = make_float4(hv[0], hv[1], hv[2], hv[3]);
              dh[1] = make_float4(hv[4], hv[5], hv[6], hv[7]);
              dl[0] = make_float4(lv[0], lv[1], lv[2], lv[3]);
              dl[1] = make_float4(lv[4], lv[5], lv[6], lv[7]);
            } else {
#pragma unroll
              for (int j = 0; j < CW; ++j) {
                if (col0 + j < p.nb) {
                  p.ohi[o + j] = hv[j];
                  p.olo[o + j] = lv[j];
                }
              }
            }
          }
        }
        tc_fence_before();
        mbar_arrive(&acce[set]);
        ++cc;
      }
      if (!ok) break;
      ++units_done;
    }
    // ---- CTA results of the summing kinds ----
    if (ok && units_done == nunits) {
      const int r = mt * S4_BM + row;
      if (r < p.prow) {
        if (KIND == S_JMO) {
          long long* dst = (long long*)p.partial + ((size_t)split * p.prow + r) * p.pcol;
#pragma unroll 1
          for (int i = 0; i < BN / NWG; ++i) {
            const int col = nt * BN + ((i / CW) * NWG + wg) * CW + i % CW;
            if (col < p.pcol) dst[col] = acc[NACC == 1 ? 0 : i];
          }
        } else if (SUM_DF) {
          float2* dst = (float2*)p.partial + ((size_t)split * p.prow + r) * p.pcol;
#pragma unroll
          for (int i = 0; i < BN / NWG; ++i) {
            const int col = nt * BN + ((i / CW) * NWG + wg) * CW + i % CW;
            if (col < p.pcol) dst[col] = make_float2(sh[SUM_DF ? i : 0], sl[SUM_DF ? i : 0]);
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
// digitisation and bound kernels
// ---------------------------------------------------------------------------
// Rows of an FP64 matrix (element (r, k) at X[r*rs + k*cs]) -> interleaved digits
// [(r*4 + t)*ldp + k] with the row's exact exponent.  One warp per row.  Optionally
// writes |X| (absout[r*cols + k] and absT[k*rows + r]) and a double-float copy.
__global__ void slice_f64_kernel(const double* X, long long rows, int cols, long long rs, long long cs,
                                 __nv_bfloat16* planes, int ldp, int* exps, float* absout, float* absT,
                                 float2* dfout) {
  pdl_entry();
  long long r = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
  int lane = threadIdx.x % 32;
  if (r >= rows) return;
  const double* x = X + r * rs;
  double mx = 0.0;
  for (int k = lane; k < cols; k += 32) mx = fmax(mx, fabs(x[k * cs]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const int e = expo_of(mx);
  if (lane == 0) exps[r] = e;
  __nv_bfloat16* out = planes + (size_t)r * 4 * ldp;
  for (int k = lane; k < cols; k += 32) {
    const double v = x[k * cs];
    __nv_bfloat16 d[4];
    digits_bf16(__double2int_rn(scale_pow2(v, 31 - e)), d);
#pragma unroll
    for (int t = 0; t < 4; ++t) out[t * ldp + k] = d[t];
    if (absout) absout[r * cols + k] = (float)fabs(v);
    if (absT) absT[(long long)k * rows + r] = (float)fabs(v);
    if (dfout) {
      const float h = (float)v;
      dfout[r * cols + k] = make_float2(h, (float)(v - (double)h));
    }
  }
}

// The per-iteration form of slice_f64_kernel (unit column stride): one block per
// row, so that a row's loads are spread over many threads and its FP64 work over
// the SMs.  Rows r in [rows, rows_df) only write their double-float copy.
constexpr int SLICE_ROWS_THREADS = 128;
__global__ void __launch_bounds__(SLICE_ROWS_THREADS) slice_rows_kernel(const double* __restrict__ X, int rows,
                                                                        int cols, long long rs,
                                                                        __nv_bfloat16* __restrict__ planes, int ldp,
                                                                        int* __restrict__ exps, float* absout,
                                                                        float* absT, float2* dfout) {
  pdl_entry();
  __shared__ double wmax[SLICE_ROWS_THREADS / 32];
  __shared__ int se;
  const int r = blockIdx.x, tid = threadIdx.x;
  const double* x = X + (long long)r * rs;
  if (r >= rows) {
    for (int k = tid; k < cols; k += SLICE_ROWS_THREADS) dfout[(long long)r * cols + k] = to_df(x[k]);
    return;
  }
  double mx = 0.0;
#pragma unroll 4
  for (int k = tid; k < cols; k += SLICE_ROWS_THREADS) mx = fmax(mx, fabs(x[k]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0) wmax[tid >> 5] = mx;
  __syncthreads();
  if (tid == 0) {
    double m2 = wmax[0];
    for (int w = 1; w < SLICE_ROWS_THREADS / 32; ++w) m2 = fmax(m2, wmax[w]);
    se = expo_of(m2);
    exps[r] = se;
  }
  __syncthreads();
  const int e = se;
  __nv_bfloat16* out = planes + (size_t)r * 4 * ldp;
#pragma unroll 4
  for (int k = tid; k < cols; k += SLICE_ROWS_THREADS) {
    const double v = x[k];
    __nv_bfloat16 d[4];
    digits_bf16(__double2int_rn(scale_pow2(v, 31 - e)), d);
#pragma unroll
    for (int t = 0; t < 4; ++t) out[t * ldp + k] = d[t];
    if (absout) absout[(long long)r * cols + k] = (float)fabs(v);
    if (absT) absT[(long long)k * rows + r] = (float)fabs(v);
    if (dfout) dfout[(long long)r * cols + k] = to_df(v);
  }
}

// FP64 -> double-float pairs, elementwise.
__global__ void to_df_kernel(const double* __restrict__ x, long long n, float2* __restrict__ out) {
  pdl_entry();
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = to_df(x[i]);
}

// Rows of a double-float matrix (hi, lo; row stride ld, a multiple of 2) ->
// interleaved digits with exact row exponents.  One warp per row, two adjacent
// columns per lane (8-byte loads, BF16 pairs stored as 4 bytes; ldp even).
__device__ __forceinline__ float scale_pow2f(float x, int k) {
  return (k >= -126 && k <= 127) ? x * exp2_int(k) : ldexpf(x, k);
}
__device__ __forceinline__ int pair_to_int(float h, float l, int k) {
  const float hs = scale_pow2f(h, k), ls = scale_pow2f(l, k);  // |hs| < 2^30
  const float ih = rintf(hs);
  return __float2int_rn(ih) + __float2int_rn((hs - ih) + ls);
}
__global__ void slice_pair_kernel(const float* hi, const float* lo, long long rows, int cols, int ld,
                                  __nv_bfloat16* planes, int ldp, int* exps) {
  pdl_entry();
  long long r = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
  int lane = threadIdx.x % 32;
  if (r >= rows) return;
  const float* h = hi + r * ld;
  const float* l = lo + r * ld;
  float mx = 0.f;
  for (int k = 2 * lane; k < cols; k += 64) {
    if (k + 1 < cols) {
      const float2 hv = *(const float2*)(h + k), lv = *(const float2*)(l + k);
      mx = fmaxf(mx, fmaxf(fabsf(hv.x) + fabsf(lv.x), fabsf(hv.y) + fabsf(lv.y)));
    } else {
      mx = fmaxf(mx, fabsf(h[k]) + fabsf(l[k]));
    }
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const int e = expo_of_inflated(mx);
  if (lane == 0) exps[r] = e;
  __nv_bfloat16* out = planes + (size_t)r * 4 * ldp;
  for (int k = 2 * lane; k < cols; k += 64) {
    if (k + 1 < cols) {
      const float2 hv = *(const float2*)(h + k), lv = *(const float2*)(l + k);
      __nv_bfloat162 dd[4];
      digits_bf16x2(pair_to_int(hv.x, lv.x, 31 - e), pair_to_int(hv.y, lv.y, 31 - e), dd);
#pragma unroll
      for (int t = 0; t < 4; ++t) *(__nv_bfloat162*)(out + (size_t)t * ldp + k) = dd[t];
    } else {
      __nv_bfloat16 d[4];
      digits_bf16(pair_to_int(h[k], l[k], 31 - e), d);
#pragma unroll
      for (int t = 0; t < 4; ++t) out[(size_t)t * ldp + k] = d[t];
    }
  }
}

// Upper bounds on |b^P_{p nu}| (Table 2/3 step 2), FP32 sums inflated by (1 + 2^-16):
//   e3[P][p] = expo(sum_mu rmaxB[P][mu] |C_{mu p}|)   (rows (P,p) of the full-transform operand)
//   e6[p][nu] = expo(sum_mu |C_{mu p}| maxB[mu][nu])   (rows (p,nu) of the K^(p) operand)
// Both are out[i][j] = expo(sum_k A[i][k] B[k][j]) over a small FP32 product: 16 x 16
// outputs per block, K staged through shared memory in slices of 64, every sum
// taken in k order with one FMA chain (the bounds do not depend on the launch).
constexpr int BOUND_TILE = 16, BOUND_KC = 64;
__global__ void __launch_bounds__(256) bound_kernel(int M, int N, int K, const float* __restrict__ A, int lda,
                                                    const float* __restrict__ B, int ldb, int* __restrict__ out,
                                                    int ldo) {
  pdl_entry();
  __shared__ float As[BOUND_TILE][BOUND_KC + 1];
  __shared__ float Bs[BOUND_KC][BOUND_TILE + 1];
  const int tid = threadIdx.x, tx = tid % BOUND_TILE, ty = tid / BOUND_TILE;
  const int i0 = blockIdx.y * BOUND_TILE, j0 = blockIdx.x * BOUND_TILE;
  float acc = 0.f;
  for (int k0 = 0; k0 < K; k0 += BOUND_KC) {
#pragma unroll
    for (int u = 0; u < BOUND_TILE * BOUND_KC / 256; ++u) {
      const int idx = tid + 256 * u;
      const int ar = idx / BOUND_KC, ac = idx % BOUND_KC;  // A: row i0 + ar, column k0 + ac
      As[ar][ac] = (i0 + ar < M && k0 + ac < K) ? A[(size_t)(i0 + ar) * lda + k0 + ac] : 0.f;
      const int br = idx / BOUND_TILE, bc = idx % BOUND_TILE;  // B: row k0 + br, column j0 + bc
      Bs[br][bc] = (k0 + br < K && j0 + bc < N) ? B[(size_t)(k0 + br) * ldb + j0 + bc] : 0.f;
    }
    __syncthreads();
    const int kn = K - k0 < BOUND_KC ? K - k0 : BOUND_KC;
    for (int kk = 0; kk < kn; ++kk) acc = fmaf(As[ty][kk], Bs[kk][tx], acc);
    __syncthreads();
  }
  if (i0 + ty < M && j0 + tx < N) out[(size_t)(i0 + ty) * ldo + j0 + tx] = expo_of_inflated(acc);
}

// max over nu of |B^P_{mu nu}| -> rmaxB[P][mu], max over P -> maxB[mu][nu] (FP32, rounded up).
__global__ void bmax_rows_kernel(const double* B, int nx, int nb, float* rmaxB) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)nx * nb) return;
  const double* x = B + i * nb;
  double mx = 0.0;
  for (int k = 0; k < nb; ++k) mx = fmax(mx, fabs(x[k]));
  rmaxB[i] = __double2float_ru(mx);
}

__global__ void bmax_aux_kernel(const double* B, int nx, int nb, float* maxB) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long nb2 = (long long)nb * nb;
  if (i >= nb2) return;
  double mx = 0.0;
  for (int P = 0; P < nx; ++P) mx = fmax(mx, fabs(B[P * nb2 + i]));
  maxB[i] = __double2float_ru(mx);
}

// J_pq = 2^(ed_p + ed_q - 46) x (sum over splits of the exact int64 partials).
__global__ void reduce_jmo_kernel(const long long* partial, int nsplit, int m, const int* ed, double* J) {
  pdl_entry();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m * m) return;
  long long s = 0;
#pragma unroll 8
  for (int k = 0; k < nsplit; ++k) s += partial[(size_t)k * m * m + i];
  J[i] = ldexp((double)s, ed[i / m] + ed[i % m] - S4_SHIFT);
}

// Sum over splits of double-float partials, in double-float arithmetic (FP64 only
// for the final value).  Without outdf: out[i] = the sum (FP64).  With outdf: the
// [rows = p][cols = mu] partials of F^(p) C_p, written as the double-float Y^T
// [p][mu] with n_p (H C)^T added (HCt double-float).
__global__ void __launch_bounds__(256) reduce_df_kernel(const float2* partial, int nsplit, int rows, int cols,
                                                       double* out, float2* outdf, const double* n,
                                                       const float2* HCt) {
  pdl_entry();
  // 32 outputs per block, their splits dealt to 8 thread rows (split k to row
  // k % 8), each row summing its share in split order; the 8 row sums are then
  // added in row order, so the result does not depend on the launch beyond that
  // fixed order.
  __shared__ float2 part[8][32];
  const long long rc = (long long)rows * cols;
  const long long i = blockIdx.x * 32LL + threadIdx.x;
  float sh = 0.f, sl = 0.f;
  if (i < rc) {
    for (int k = threadIdx.y; k < nsplit; k += 8) {
      const float2 v = partial[(size_t)k * rc + i];
      df_add(sh, sl, v.x, v.y);
    }
  }
  part[threadIdx.y][threadIdx.x] = make_float2(sh, sl);
  __syncthreads();
  if (threadIdx.y != 0 || i >= rc) return;
  float th = part[0][threadIdx.x].x, tl = part[0][threadIdx.x].y;
#pragma unroll
  for (int y = 1; y < 8; ++y) df_add(th, tl, part[y][threadIdx.x].x, part[y][threadIdx.x].y);
  if (outdf) {
    const float2 np = to_df(n[i / cols]), h = HCt[i];
    const float ph = np.x * h.x;
    const float pl = fmaf(np.x, h.x, -ph) + fmaf(np.x, h.y, np.y * h.x);
    df_add(th, tl, ph, pl);
    outdf[i] = make_float2(th, tl);
  } else {
    out[i] = (double)th + (double)tl;
  }
}

// The contracted Lagrangian's first operand,
//   X^P_qp = [q = p] w_pP - B_pq b^P_qp,  w_pP = sum_r A_pr b^P_rr,
// as digit rows (q, p) over P with the row's exact exponent: X digits
// [q][p][4][nxp], eX[q][p].  b^P_qp from bf [P][q][p] (FP64), w [p][P], B [p][q].
// Block (32, 8) per orbital q and 32 consecutive p: one pass for the row maxima,
// a second that rounds each value to its integer, turns a 32 x 32 (P, p) block
// around in shared memory and writes each digit row's 32 consecutive P at once.
__global__ void __launch_bounds__(256) ctr_digits_kernel(const double* __restrict__ bf, const double* __restrict__ Bc,
                                                         const double* __restrict__ w, int m, int nx, int nxp,
                                                         __nv_bfloat16* __restrict__ Xd, int* __restrict__ eX) {
  pdl_entry();
  __shared__ double red[8][32];
  __shared__ int tile[32][33];
  __shared__ int es[32];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int q = blockIdx.y, p0 = blockIdx.x * 32, p = p0 + tx;
  const bool pv = p < m;
  const double bqp = pv ? Bc[(size_t)p * m + q] : 0.0;
  const bool diag = pv && p == q;
  double mx = 0.0;
  if (pv) {
    for (int P = ty; P < nx; P += 8) {
      double x = -bqp * bf[((size_t)P * m + q) * m + p];
      if (diag) x += w[(size_t)p * nx + P];
      mx = fmax(mx, fabs(x));
    }
  }
  red[ty][tx] = mx;
  __syncthreads();
  if (ty == 0) {
#pragma unroll
    for (int y = 1; y < 8; ++y) mx = fmax(mx, red[y][tx]);
    const int e = expo_of(mx);
    es[tx] = e;
    if (pv) eX[(size_t)q * m + p] = e;
  }
  __syncthreads();
  const int e = es[tx];
  for (int P0 = 0; P0 < nx; P0 += 32) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int P = P0 + ty + 8 * k;
      int X = 0;
      if (pv && P < nx) {
        double x = -bqp * bf[((size_t)P * m + q) * m + p];
        if (diag) x += w[(size_t)p * nx + P];
        X = __double2int_rn(scale_pow2(x, 31 - e));
      }
      tile[ty + 8 * k][tx] = X;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int pr = ty + 8 * k, P = P0 + tx;
      if (p0 + pr < m && P < nx) {
        __nv_bfloat16 d[4];
        digits_bf16(tile[tx][pr], d);
        __nv_bfloat16* o = Xd + ((size_t)q * m + p0 + pr) * 4 * nxp + P;
#pragma unroll
        for (int t = 0; t < 4; ++t) o[(size_t)t * nxp] = d[t];
      }
    }
    __syncthreads();
  }
}

// out[i][j] = sum_k A[i][k] B[j][k] in double-float arithmetic: each product as
// an FP32 pair (about 2^-46 relative), the high parts summed with TwoSum in k
// order and the low parts and rounding errors collected beside them.  A and B are
// double-float; out double-float or FP64.  The small products of the energy row
// (H C, lambda = Y^T C) run here rather than in DFMA, whose rate is a small
// fraction of FP32's on this part.  16 x 16 outputs per block, K staged through
// shared memory in slices of 64, the loads of a slice issued together.
__device__ __forceinline__ void df_store(float2& o, float h, float l) { o = make_float2(h, l); }
__device__ __forceinline__ void df_store(double& o, float h, float l) { o = (double)h + (double)l; }

constexpr int DFG_KC = 64, DFG_TI = 16, DFG_TJ = 16, DFG_THREADS = DFG_TI * DFG_TJ;
template <typename TO>
__global__ void __launch_bounds__(DFG_THREADS) df_gemm_nt_kernel(int M, int N, int K, const float2* __restrict__ A,
                                                                 int lda, const float2* __restrict__ B, int ldb,
                                                                 TO* __restrict__ out, int ldo) {
  pdl_entry();
  __shared__ float2 As[DFG_TI][DFG_KC + 1];  // [i][k]
  __shared__ float2 Bs[DFG_KC][DFG_TJ + 1];  // [k][j]
  const int tid = threadIdx.x, tx = tid % DFG_TJ, ty = tid / DFG_TJ;
  const int i0 = blockIdx.y * DFG_TI, j0 = blockIdx.x * DFG_TJ;
  constexpr int NA = DFG_TI * DFG_KC / DFG_THREADS, NB = DFG_TJ * DFG_KC / DFG_THREADS;
  float sum = 0.f, cmp = 0.f;
  for (int k0 = 0; k0 < K; k0 += DFG_KC) {
    float2 av[NA], bv[NB];
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      const int idx = tid + DFG_THREADS * u, r = idx / DFG_KC, c = idx % DFG_KC;
      av[u] = (i0 + r < M && k0 + c < K) ? A[(size_t)(i0 + r) * lda + k0 + c] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int idx = tid + DFG_THREADS * u, r = idx / DFG_KC, c = idx % DFG_KC;
      bv[u] = (j0 + r < N && k0 + c < K) ? B[(size_t)(j0 + r) * ldb + k0 + c] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      const int idx = tid + DFG_THREADS * u;
      As[idx / DFG_KC][idx % DFG_KC] = av[u];
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int idx = tid + DFG_THREADS * u;
      Bs[idx % DFG_KC][idx / DFG_KC] = bv[u];
    }
    __syncthreads();
    const int kn = K - k0 < DFG_KC ? K - k0 : DFG_KC;
#pragma unroll 8
    for (int kk = 0; kk < kn; ++kk) {
      const float2 a = As[ty][kk], b = Bs[kk][tx];
      const float ph = a.x * b.x;
      const float pl = fmaf(a.x, b.x, -ph) + fmaf(a.x, b.y, a.y * b.x);
      float ns, e;
      two_sum_f(sum, ph, ns, e);
      sum = ns;
      cmp += e + pl;
    }
    __syncthreads();
  }
  if (i0 + ty < M && j0 + tx < N) {
    const float h = sum + cmp;
    df_store(out[(size_t)(i0 + ty) * ldo + j0 + tx], h, cmp - (h - sum));
  }
}

// E = E_nuc + sum_p (n_p H_pp + lambda_pp).  One warp per p: H_pp = C_p . (H C)_p
// in double-float arithmetic (lanes over mu, a fixed shuffle tree), the term in
// FP64 into eterm[p].  The last warp to finish (a ticket counter, which that warp
// resets for the next launch) adds the terms in a fixed order (lanes over p, then
// a shuffle tree).  No FP64 loop runs on one SM over a whole matrix, and no block
// waits for another.
__global__ void energy_terms_kernel(int nbf, int n_om, const float2* Cdf, const float2* HCt, const double* n,
                                    const double* lambda, const double* enuc, double* eterm, unsigned int* ticket,
                                    double* E) {
  pdl_entry();
  __shared__ int last;
  const int p = blockIdx.x, lane = threadIdx.x;
  float sum = 0.f, cmp = 0.f;
  for (int mu = lane; mu < nbf; mu += 32) {
    const float2 c = Cdf[(size_t)p * nbf + mu], h = HCt[(size_t)p * nbf + mu];
    const float ph = c.x * h.x;
    const float pl = fmaf(c.x, h.x, -ph) + fmaf(c.x, h.y, c.y * h.x);
    float ns, e;
    two_sum_f(sum, ph, ns, e);
    sum = ns;
    cmp += e + pl;
  }
  float sh = sum + cmp, sl = cmp - (sh - sum);
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, sh, o), ol = __shfl_xor_sync(0xffffffffu, sl, o);
    df_add(sh, sl, oh, ol);
  }
  if (lane == 0) {
    eterm[p] = n[p] * ((double)sh + (double)sl) + lambda[(size_t)p * nbf + p];
    __threadfence();
    last = atomicAdd(ticket, 1u) == (unsigned int)(n_om - 1);
  }
  __syncwarp();
  if (!last) return;
  __threadfence();
  // lane l adds the terms q = l, l + 32, ... in order; then a fixed shuffle tree
  double v = 0.0;
  for (int q = lane; q < n_om; q += 32) v += __ldcg(eterm + q);
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) {
    *E = *enuc + v;
    *ticket = 0u;
  }
}

// FOCK weights as double-float pairs: W[q][p] = A_pq, W[N_O + q][p] = -B_pq.
__global__ void fock_weights_df_kernel(const double* A, const double* Bc, int m, float2* W) {
  pdl_entry();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * m * m) return;
  int qq = i / m, pc = i % m;
  const double v = qq < m ? A[(size_t)pc * m + qq] : -Bc[(size_t)pc * m + (qq - m)];
  const float h = (float)v;
  W[i] = make_float2(h, (float)(v - (double)h));
}

// Interleaved digits + row exponents -> FP64 values (fetch / copy-out paths).
// Both digit layouts of b_half from the half transform's integers Xf [P][p][nu]
// (scale 2^(min(e3, e6) - 31)): L3 [P][p][t][nu] with exponent e3[P][p] and L6
// [p][nu][t][P] with exponent e6[p][nu], each a rounding right shift of Xf by
// the exponent difference.  A 64 x 64 (P, nu) tile per block, two adjacent
// elements per thread (8-byte loads, BF16 pairs stored as 4 bytes); L6 goes
// through a shared-memory transposition, so the reads and both digit stores are
// 128 contiguous bytes per warp.  Row strides (nbp, nxp) are even.
//
// The same pass accumulates the diagonal b^P_pp = sum_nu C_{nu p} b^P_{p nu} (Table 3
// step 3) from the L3 integers it has in hand: in the transposed half each thread
// sums its two rows P over its eight nu in double-float arithmetic (X3 = xh + xl
// exactly, C as a double-float pair), the eight thread rows are added in a fixed
// order through shared memory, and one partial per (nu tile, p, P) goes to dpart;
// diag_reduce_kernel adds the tiles in a fixed order and applies the row scale.
__global__ void __launch_bounds__(256) xf_to_digits_kernel(const int* Xf, const int* e3, const int* e6, int nx, int nb,
                                                           int m, int mp, int nbp, int nxp, __nv_bfloat16* L3,
                                                           __nv_bfloat16* L6, const float2* Cdf, float2* dpart) {
  pdl_entry();
  __shared__ int tile[64][65];   // the integers Xf of the tile
  __shared__ int ytile[64][65];  // their L3 values (scale e3), for the diagonal partials
  __shared__ int s3[64], s6[64];
  __shared__ float2 sc[64];
  __shared__ float2 red[8][64];
  const int p = blockIdx.z, nu0 = blockIdx.x * 64, P0 = blockIdx.y * 64;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if (tid < 64) s3[tid] = (P0 + tid < nx) ? e3[(size_t)(P0 + tid) * m + p] : 0;
  else if (tid < 128) s6[tid - 64] = (nu0 + tid - 64 < nb) ? e6[(size_t)p * nb + nu0 + tid - 64] : 0;
  else if (tid < 192) sc[tid - 128] = (nu0 + tid - 128 < nb) ? Cdf[(size_t)p * nb + nu0 + tid - 128] : make_float2(0.f, 0.f);
  __syncthreads();
  const int c0 = 2 * threadIdx.x;  // this thread's column pair within the tile
  // rows P of the tile: L3 digits (nu contiguous).  The eight rows' loads are
  // issued before any of their stores, so that they are in flight together.
  int2 xv[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int P = P0 + threadIdx.y + 8 * i, nu = nu0 + c0;
    xv[i] = make_int2(0, 0);
    if (P < nx && nu < nb) {
      const int* src = Xf + ((size_t)P * m + p) * nbp + nu;
      if (nu + 1 < nb) xv[i] = *(const int2*)src;
      else xv[i].x = src[0];
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = threadIdx.y + 8 * i;
    const int P = P0 + r, nu = nu0 + c0;
    const int x0 = xv[i].x, x1 = xv[i].y;
    if (P < nx && nu < nb) {
      int d = s3[r] - s6[c0];
      const int y0 = rshift_round(x0, d > 0 ? d : 0);
      d = s3[r] - s6[c0 + 1];
      const int y1 = rshift_round(x1, d > 0 ? d : 0);
      __nv_bfloat162 dd[4];
      digits_bf16x2(y0, y1, dd);
      __nv_bfloat16* o = L3 + (((size_t)P * mp + p) * 4) * nbp + nu;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (nu + 1 < nb) *(__nv_bfloat162*)(o + (size_t)t * nbp) = dd[t];
        else o[(size_t)t * nbp] = dd[t].x;
      }
      ytile[r][c0] = y0;
      ytile[r][c0 + 1] = y1;
    } else {
      ytile[r][c0] = 0;
      ytile[r][c0 + 1] = 0;
    }
    tile[r][c0] = x0;
    tile[r][c0 + 1] = x1;
  }
  __syncthreads();
  // columns nu of the tile: L6 digits (P contiguous), and the diagonal partials of the
  // thread's two rows P over its eight nu in double-float arithmetic (the L3 value
  // y = yh + yl exactly in FP32, C as a double-float pair)
  float sum[2] = {0.f, 0.f}, cmp[2] = {0.f, 0.f};
  for (int r = threadIdx.y; r < 64; r += 8) {
    const int nu = nu0 + r, P = P0 + c0;
    if (nu < nb && P < nx) {
      int d = s6[r] - s3[c0];
      const int z0 = rshift_round(tile[c0][r], d > 0 ? d : 0);
      d = s6[r] - s3[c0 + 1];
      const int z1 = rshift_round(tile[c0 + 1][r], d > 0 ? d : 0);
      __nv_bfloat162 dd[4];
      digits_bf16x2(z0, z1, dd);
      __nv_bfloat16* o = L6 + ((size_t)p * nb + nu) * 4 * nxp + P;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (P + 1 < nx) *(__nv_bfloat162*)(o + (size_t)t * nxp) = dd[t];
        else o[(size_t)t * nxp] = dd[t].x;
      }
      const float2 cv = sc[r];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int y = ytile[c0 + k][r];
        const float yh = (float)(y >> 8) * 256.f, yl = (float)(y & 255);
        const float p0 = yh * cv.x;
        const float e0 = fmaf(yh, cv.x, -p0) + (yh * cv.y + yl * cv.x);
        float ns, e;
        two_sum_f(sum[k], p0, ns, e);
        sum[k] = ns;
        cmp[k] += e + e0;
      }
    }
  }
  red[threadIdx.y][c0] = make_float2(sum[0], cmp[0]);
  red[threadIdx.y][c0 + 1] = make_float2(sum[1], cmp[1]);
  __syncthreads();
  if (tid < 64 && P0 + tid < nx) {
    float sh = red[0][tid].x, sl = red[0][tid].y;
#pragma unroll
    for (int y = 1; y < 8; ++y) {
      float ns, e;
      two_sum_f(sh, red[y][tid].x, ns, e);
      sh = ns;
      sl += e + red[y][tid].y;
    }
    dpart[((size_t)blockIdx.x * m + p) * nx + P0 + tid] = make_float2(sh, sl);
  }
}

// d[p][P] = 2^(e3[P][p] - 31) sum over the nu tiles of the pass's double-float
// partials, added in tile order in double-float arithmetic; FP64 only for the
// final value.
__global__ void diag_reduce_kernel(const float2* dpart, int ntiles, int nx, int m, const int* e3, double* d) {
  pdl_entry();
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)nx * m) return;
  const int pc = (int)(i / nx), P = (int)(i % nx);
  float sh = 0.f, sl = 0.f;
  for (int t = 0; t < ntiles; ++t) {
    const float2 v = dpart[((size_t)t * m + pc) * nx + P];
    df_add(sh, sl, v.x, v.y);
  }
  d[i] = scale_pow2((double)sh + (double)sl, e3[(size_t)P * m + pc] - 31);
}

// J^(q) and K^(q) are symmetric: their GEMMs skip the tiles that lie wholly below
// the diagonal, and this kernel fills those elements from the transposed ones,
// through a shared-memory tile so that reads and writes are coalesced.
// hi/lo: [2m][nb][ldo] with J^(q) at rows q and K^(q) at rows m + q.
//   K^(q) tiles: 128 mu x bn nu; skipped when the tile's last nu is below its first mu.
//   J^(q) tiles: 128 consecutive rows r = mu nb + nu of the output (one tile per
//   row block); skipped when all of its rows lie in one mu and have nu < mu.
__host__ __device__ __forceinline__ bool kao_tile_computed(int mu, int nu, int bn) {
  return (nu / bn) * bn + bn - 1 >= (mu / 128) * 128;
}

__host__ __device__ __forceinline__ bool jao_block_skipped(long long r0, int nb) {
  const long long r1 = r0 + 127 < (long long)nb * nb ? r0 + 127 : (long long)nb * nb - 1;
  const long long mu0 = r0 / nb, mu1 = r1 / nb;
  return mu0 == mu1 && (r1 - mu0 * nb) < mu0;
}

// Launched over the 32 x 32 destination blocks that hold skipped elements only
// (tiles[] = (bi << 16) | bj, built on the host from the same predicates), one
// grid row per matrix.
__global__ void sym_mirror_kernel(float* hi, float* lo, int nb, int row0, int ldo, int bn, int jao, const int* tiles) {
  pdl_entry();
  __shared__ float th[32][33], tl[32][33];
  const int bi = tiles[blockIdx.x] >> 16, bj = tiles[blockIdx.x] & 0xFFFF;  // rows mu (bi), columns nu (bj)
  if (bj > bi) return;
  // most blocks below the diagonal were computed by the GEMM: leave before any load
  int work = 0;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int mu = bi * 32 + r, nu = bj * 32 + threadIdx.x;
    if (mu < nb && nu < nb && nu < mu)
      work |= !(jao ? !jao_block_skipped(((long long)mu * nb + nu) / 128 * 128, nb) : kao_tile_computed(mu, nu, bn));
  }
  if (!__syncthreads_or(work)) return;
  const size_t base = (size_t)(row0 + blockIdx.y) * nb * ldo;
  for (int r = threadIdx.y; r < 32; r += 8) {  // source rows nu = bj*32 + r, columns mu = bi*32 + x
    const int nu = bj * 32 + r, mu = bi * 32 + threadIdx.x;
    if (nu < nb && mu < nb) {
      th[r][threadIdx.x] = hi[base + (size_t)nu * ldo + mu];
      tl[r][threadIdx.x] = lo[base + (size_t)nu * ldo + mu];
    }
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int mu = bi * 32 + r, nu = bj * 32 + threadIdx.x;
    const bool computed = jao ? !jao_block_skipped(((long long)mu * nb + nu) / 128 * 128, nb)
                              : kao_tile_computed(mu, nu, bn);
    if (mu < nb && nu < nb && nu < mu && !computed) {
      hi[base + (size_t)mu * ldo + nu] = th[threadIdx.x][r];
      lo[base + (size_t)mu * ldo + nu] = tl[threadIdx.x][r];
    }
  }
}

__global__ void unslice_kernel(const __nv_bfloat16* planes, int ldp, const int* exps, long long rows, int cols,
                               double* out) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  long long r = i / cols;
  int k = (int)(i % cols);
  const __nv_bfloat16* pr = planes + r * 4 * ldp + k;
  long long X = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t) X = X * 256 + (long long)__bfloat162float(pr[t * ldp]);
  out[i] = ldexp((double)X, exps[r] - 31);
}

__global__ void join_pair_kernel(const float* hi, const float* lo, long long rows, int cols, int ld, double* out) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  long long r = i / cols;
  int c = (int)(i % cols);
  out[i] = (double)hi[r * ld + c] + (double)lo[r * ld + c];
}

}  // namespace donof

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct donof::S4Buffers {
  int nbp, nxp, mp, ldo;
  __nv_bfloat16 *B1, *B5, *Ct, *L3, *L6, *Dp, *JKp;  // interleaved digits
  int* X6;                                            // L6 integers [nx][m][nbp] before digitisation
  int* kao_tmap;                                      // K^(q) tiles on or above the diagonal
  int* jao_tmap;                                      // J^(q) row blocks on or above the diagonal
  int* jao_tmap_full;                                 // every J^(q) row block
  int jao_ntiles_sym, jao_ntiles_full;
  int jao_sym;                                        // 1: J^(q) lower row blocks skipped and mirrored
  int *mir_jao, *mir_kao;                             // 32 x 32 blocks the mirrors fill, (bi << 16) | bj
  int mir_n_jao, mir_n_kao;
  int half_variant;                                   // 1: the half transform runs as S_HALF1
  int jk_merged;                                      // 1: J^(q) and K^(q) in one launch (S_JKAO)
  int max_stages[donof::S_NKINDS];                    // pipeline depth that fits the shared memory
  int target[donof::S_NKINDS];                        // CTA count the split kinds aim at
  int *eB1, *eB5, *eC, *e3, *e6, *ed, *eJK;          // row exponents
  float *rmaxB, *maxB, *absC, *absCt;
  // Working basis: the orbital basis orthonormalised by the Cholesky factor of the
  // overlap, chi' = chi L^-T with S = L L^T.  Orbitals are C' = L^T C (C'^T C' = I),
  // the fitted tensor B'^P = L^-1 B^P L^-T and H' = L^-1 H L^-T; every GEMM operand
  // and the energy row work in it, and AO outputs are transformed back.
  double* Ls;     // L [mu][nu] row-major, lower triangle (FP64)
  float2* LsTdf;  // L^T [nu][mu] as double-float pairs
  float2* Cin;    // C^T rows [p][mu] (every p < nbf) as double-float pairs
  double* Cp;     // C'^T rows [p][mu'] (every p < nbf), FP64
  float2* Cinp;   // the energy prep's own double-float C^T rows (p < N_O)
  float2* Cdf;    // C' rows p (every p < nbf) as double-float pairs
  float2* Hdf;    // H' as double-float pairs (fixed at init)
  float2* Cdfp;   // C' rows p (< N_O) as double-float pairs, the energy prep's own copy (its stream
                  // may run ahead of the transform that writes Cdf)
  float2* dpart;  // diagonal partials [nu tile][m][nx] from the digit pass
  double* dmat;   // d [m][nx] FP64
  float *JKhi, *JKlo;
  float2* W;
  float2* HCt;  // (H C)^T [p][mu], double-float
  float2* Yt;   // Y^T [p][mu] = (F^(p) C_p)^T, double-float
  // contracted Lagrangian (allocated on its first call)
  double* bf;          // b^P_qp [P][q][p]
  double* wP;          // w [p][P]
  __nv_bfloat16* Xd;   // X digits [q][p][4][nxp]
  int* eX;             // their row exponents [q][p]
  double* eterm;          // the energy's per-orbital terms
  unsigned int* ticket;   // energy_terms_kernel's completion counter (zero between launches)
  void* partial;
  void* partial_j;  // J_pq's int64 partials (its launch group may run beside a3's)
  donof::S4Params plan[donof::S_NKINDS];
  int grid[donof::S_NKINDS];
  size_t smem[donof::S_NKINDS];
  PFN_cuTensorMapEncodeTiled_v12000 encode;
};

namespace donof {

static int s4_round_up(int a, int b) { return (a + b - 1) / b * b; }

// BF16 tensor map, 64-byte swizzle; dims innermost first, strides in elements.
static int s4_map(S4Buffers* sb, CUtensorMap* map, const void* base, int rank, const long long* dims,
                  const long long* strides_el, const int* box) {
  cuuint64_t gd[5], gs[4];
  cuuint32_t bd[5], es[5] = {1, 1, 1, 1, 1};
  for (int i = 0; i < rank; ++i) {
    gd[i] = (cuuint64_t)dims[i];
    bd[i] = (cuuint32_t)box[i];
  }
  for (int i = 0; i < rank - 1; ++i) {
    gs[i] = (cuuint64_t)(strides_el[i] * 2);
    if (gs[i] % 16) return DONOF_RI_E_ARG;
  }
  if (((uintptr_t)base) % 16) return DONOF_RI_E_ARG;
  CUresult r = sb->encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, (void*)base, gd, gs, bd, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? DONOF_RI_OK : DONOF_RI_E_CUDA;
}

template <int KIND>
static void s4_plan(S4Buffers* sb, int m_tiles, int n_tiles, int nbatch, int target_ctas, int persist_ctas = 0) {
  constexpr int BN = S4Cfg<KIND>::BN;
  S4Params& p = sb->plan[KIND];
  const size_t stage = (size_t)S4_PLANES * (S4_BM + BN) * S4_BK * 2;
  // Two CTAs per SM share its 228 KB of shared memory (1 KB of it reserved per CTA).
  const size_t fixed = 1024 + 256 + 4 * S4Cfg<KIND>::NWG * (size_t)S4Cfg<KIND>::ES_WARP_BYTES;
  const size_t budget = (S4Cfg<KIND>::CTAS == 2 ? (size_t)112 * 1024 : (size_t)220 * 1024) - fixed;
  int S = (int)(budget / stage);
  if (S > 6) S = 6;
  p.stages = S;
  p.tmem_cols = S4Cfg<KIND>::TMEM_COLS;
  p.n_tiles = n_tiles;
  p.nbatch = nbatch;
  const int tiles = m_tiles * n_tiles;
  // At most one wave: a second, partial wave would double the time of its CTAs' share.
  int ns = target_ctas / tiles;
  if (ns < 1) ns = 1;
  if (ns > nbatch) ns = nbatch;
  p.bpc = (nbatch + ns - 1) / ns;
  p.nsplit = (nbatch + p.bpc - 1) / p.bpc;
  sb->grid[KIND] = tiles * p.nsplit;
  sb->smem[KIND] = fixed + (size_t)S * stage;
  p.persist = 0;
  p.ntiles = tiles;
  if (persist_ctas > 0) {
    p.persist = 1;
    p.nsplit = 1;
    p.bpc = 1;
    const long long units = (long long)tiles * nbatch;
    sb->grid[KIND] = units < persist_ctas ? (int)units : persist_ctas;
  }
}

// The merged J^(q) + K^(q) launch: the current J^(q) plan (tile list, symmetric or
// full) and the K^(q) plan in one persistent grid, one CTA per SM.
static void s4_plan_jkao(S4Buffers* sb) {
  const S4Params& pj = sb->plan[S_JAO];
  const S4Params& pk = sb->plan[S_KAO];
  S4Params& p = sb->plan[S_JKAO];
  const int stages = p.stages > 0 ? p.stages : pj.stages;
  p = pj;
  p.a2 = pk.a;
  p.b2 = pk.b;
  p.ea2 = pk.ea;
  p.eb2 = pk.eb;
  p.tmap2 = pk.tmap;
  p.ntiles2 = pk.ntiles;
  p.u_split = pj.ntiles * pj.nbatch;
  p.ntiles = p.u_split + pk.ntiles * pk.nbatch;  // every unit of the launch
  p.nbatch = 1;
  p.persist = 1;
  p.stages = stages;
  const int pc = S4Cfg<S_JKAO>::CTAS * 152;
  sb->grid[S_JKAO] = p.ntiles < pc ? p.ntiles : pc;
  sb->smem[S_JKAO] = sb->smem[S_JAO] > sb->smem[S_KAO] ? sb->smem[S_JAO] : sb->smem[S_KAO];
  // the shared memory holds the deeper of the two pipelines' stages
  const int sj = sb->plan[S_JAO].stages, sk = sb->plan[S_KAO].stages;
  if (p.stages > (sj > sk ? sj : sk)) p.stages = sj > sk ? sj : sk;
}

// L L^T = S (FP64 Cholesky of the overlap) into sb->Ls, Li = L^-1, and the fitted
// tensor and core Hamiltonian in the working basis: Bw^P = Li B^P Li^T (Tb: scratch
// of the same size), Hw = Li H Li^T; L^T as double-float pairs into sb->LsTdf.
__global__ void transpose_df_kernel(const double* X, int n, float2* out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)n * n) return;
  const int r = (int)(i / n), c = (int)(i % n);
  out[i] = to_df(X[(size_t)c * n + r]);
}

__global__ void identity64_kernel(int n, double* X) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)n * n) return;
  X[i] = (i / n == i % n) ? 1.0 : 0.0;
}

// X^P <- (X^P + X^P^T) / 2 for each of `batch` n x n matrices: the two-sided products
// below are symmetric only up to rounding, and the digit layouts take B' as symmetric.
__global__ void symmetrize_kernel(double* X, int n, long long batch) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n2 = (long long)n * n;
  if (i >= batch * n2) return;
  const long long b = i / n2;
  const int r = (int)((i % n2) / n), c = (int)(i % n);
  if (c <= r) return;
  double* M = X + b * n2;
  const double v = 0.5 * (M[(size_t)r * n + c] + M[(size_t)c * n + r]);
  M[(size_t)r * n + c] = v;
  M[(size_t)c * n + r] = v;
}

static int s4_working_basis(donof_ri_ctx* ctx, double* Li, double* Tb, double* Bw, double* Hw) {
  S4Buffers* sb = ctx->s4;
  const int nb = ctx->nbf, nx = ctx->naux;
  const long long n2 = (long long)nb * nb;
  cudaStream_t s = ctx->stream;
  int rc;
  DONOF_CUDA_TRY(cudaMemcpyAsync(sb->Ls, ctx->d_S, n2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if ((rc = cholesky_lower(ctx, sb->Ls, nb, ctx->d_scratch_max, 1e-14))) return rc;
  identity64_kernel<<<ceil_div_u(n2, 256), 256, 0, s>>>(nb, Li);
  DONOF_LAUNCH_CHECK(ctx);
  if ((rc = forward_subst(ctx, sb->Ls, nb, Li, nb))) return rc;  // Li = L^-1
  transpose_df_kernel<<<ceil_div_u(n2, 256), 256, 0, s>>>(sb->Ls, nb, sb->LsTdf);
  DONOF_LAUNCH_CHECK(ctx);
  for (int which = 0; which < 2; ++which) {
    // X <- Li X (one matrix per auxiliary function), then X Li^T
    const double* X = which == 0 ? ctx->d_B : ctx->d_H;
    double* T = Tb;  // free again for H once Bw is formed
    double* out = which == 0 ? Bw : Hw;
    const int batch = which == 0 ? nx : 1;
    Gemm64 g{};
    g.M = nb; g.N = nb; g.K = nb; g.batch = batch;
    g.A = Li; g.sAb = 0; g.sAm = nb; g.sAk = 1;
    g.B = X; g.sBb = n2; g.sBk = nb; g.sBn = 1;
    g.C = T; g.sCb = n2; g.sCm = nb; g.sCn = 1;
    g.alpha = 1.0; g.beta = 0.0;
    if ((rc = launch_dgemm(ctx, g))) return rc;
    Gemm64 h{};
    h.M = nb; h.N = nb; h.K = nb; h.batch = batch;
    h.A = T; h.sAb = n2; h.sAm = nb; h.sAk = 1;
    h.B = Li; h.sBb = 0; h.sBk = 1; h.sBn = nb;  // element (k, n) of Li^T = Li[n][k]
    h.C = out; h.sCb = n2; h.sCm = nb; h.sCn = 1;
    h.alpha = 1.0; h.beta = 0.0;
    if ((rc = launch_dgemm(ctx, h))) return rc;
    symmetrize_kernel<<<ceil_div_u((long long)batch * n2, 256), 256, 0, s>>>(out, nb, batch);
    DONOF_LAUNCH_CHECK(ctx);
  }
  return DONOF_RI_OK;
}

int s4_init(donof_ri_ctx* ctx) {
  S4Buffers* sb = (S4Buffers*)calloc(1, sizeof(S4Buffers));
  if (!sb) return DONOF_RI_E_OOM;
  ctx->s4 = sb;
  {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !f) {
      cudaGetLastError();
      return DONOF_RI_E_UNSUPPORTED;
    }
    sb->encode = (PFN_cuTensorMapEncodeTiled_v12000)f;
  }
  const int nb = ctx->nbf, nx = ctx->naux, m = ctx->n_omega;
  // Digit rows padded to 16 elements (32 bytes) so that full-sector stores stay aligned.
  const int nbp = s4_round_up(nb, 16), nxp = s4_round_up(nx, 16), mp = s4_round_up(m, 4), ldo = s4_round_up(nb, 8);
  sb->nbp = nbp; sb->nxp = nxp; sb->mp = mp; sb->ldo = ldo;
  const long long nbs = nb, nxs = nx, ms = m;
  const int sms = 152;
  const int KBb = (nb + S4_BK - 1) / S4_BK, KBx = (nx + S4_BK - 1) / S4_BK;
  const int bn = S4Cfg<S_HALF>::BN;  // 48 for every kind but the full transform (32)
  s4_plan<S_HALF>(sb, ((nx + 7) / 8) * ((nb + 15) / 16), (m + bn - 1) / bn, 1, 1, S4Cfg<S_HALF>::CTAS * sms);
  s4_plan<S_HALF1>(sb, ((nx + 7) / 8) * ((nb + 15) / 16), (m + bn - 1) / bn, 1, 1, S4Cfg<S_HALF1>::CTAS * sms);
  s4_plan<S_FULLSQ>(sb, (m + S4_BM - 1) / S4_BM, (m + bn - 1) / bn, nx, S4Cfg<S_FULLSQ>::CTAS * sms);
  s4_plan<S_JMO>(sb, (m + S4_BM - 1) / S4_BM, (m + bn - 1) / bn, (KBx + S4_CHUNK_KB - 1) / S4_CHUNK_KB,
                 S4Cfg<S_JMO>::CTAS * sms);
  // J^(q): only the row blocks that reach the diagonal or lie above it, once the
  // saving outweighs the extra mirror pass (default from nbf 256 on; s4_autotune
  // measures both).
  sb->jao_sym = nb >= 256;
  std::vector<int> jao_tiles, jao_full;
  for (long long mt = 0; mt < ((long long)nb * nb + S4_BM - 1) / S4_BM; ++mt)
    for (int nt = 0; nt < (m + bn - 1) / bn; ++nt) {
      jao_full.push_back((int)((mt << 16) | nt));
      if (!jao_block_skipped(mt * S4_BM, nb)) jao_tiles.push_back((int)((mt << 16) | nt));
    }
  sb->jao_ntiles_sym = (int)jao_tiles.size();
  sb->jao_ntiles_full = (int)jao_full.size();
  s4_plan<S_JAO>(sb, 1, sb->jao_sym ? sb->jao_ntiles_sym : sb->jao_ntiles_full, 1, 1, S4Cfg<S_JAO>::CTAS * sms);
  // K^(q): only the tiles that reach the diagonal or lie above it (the rest is mirrored).
  std::vector<int> kao_tiles;
  for (int mt = 0; mt < (nb + S4_BM - 1) / S4_BM; ++mt)
    for (int nt = 0; nt < (nb + bn - 1) / bn; ++nt)
      if (nt * bn + bn - 1 >= mt * S4_BM) kao_tiles.push_back((mt << 16) | nt);
  s4_plan<S_KAO>(sb, 1, (int)kao_tiles.size(), m, S4Cfg<S_KAO>::CTAS * sms, S4Cfg<S_KAO>::CTAS * sms);
  s4_plan<S_FOCK>(sb, (m + S4_BM - 1) / S4_BM, (nb + bn - 1) / bn,
                  2 * m * ((KBb + s4_chunk_kb(S_FOCK) - 1) / s4_chunk_kb(S_FOCK)), sms);
  s4_plan<S_CTR>(sb, (m + S4_BM - 1) / S4_BM, (nb + bn - 1) / bn, m, sms);
  for (int k = 0; k < S_NKINDS; ++k) sb->max_stages[k] = sb->plan[k].stages;
  sb->target[S_FULLSQ] = S4Cfg<S_FULLSQ>::CTAS * sms;
  sb->target[S_JMO] = S4Cfg<S_JMO>::CTAS * sms;
  sb->target[S_FOCK] = sms;
  // partial sums sized for twice the default split count (the autotuner may pick it)
  size_t pbytes = 2 * (size_t)sb->plan[S_FULLSQ].nsplit * m * m * sizeof(float2);
  const size_t jbytes = 2 * (size_t)sb->plan[S_JMO].nsplit * m * m * sizeof(long long);
  size_t t = 2 * (size_t)sb->plan[S_FOCK].nsplit * nb * m * sizeof(float2);
  if (t > pbytes) pbytes = t;
  t = (size_t)sb->plan[S_CTR].nsplit * nb * m * sizeof(float2);
  if (t > pbytes) pbytes = t;

#define ALLOC(ptr, bytes)                                             \
  do {                                                                \
    if (cudaMalloc((void**)&(ptr), (size_t)(bytes)) != cudaSuccess) { \
      cudaGetLastError();                                             \
      return DONOF_RI_E_OOM;                                          \
    }                                                                 \
  } while (0)
  ALLOC(sb->B1, nxs * nbs * 4 * nbp * 2);
  ALLOC(sb->B5, nbs * nbs * 4 * nxp * 2);
  ALLOC(sb->Ct, ms * 4 * nbp * 2);
  ALLOC(sb->L3, nxs * mp * 4 * nbp * 2);
  ALLOC(sb->L6, ms * nbs * 4 * nxp * 2);
  ALLOC(sb->X6, nxs * ms * nbp * 4);
  ALLOC(sb->kao_tmap, kao_tiles.size() * sizeof(int));
  ALLOC(sb->jao_tmap, jao_tiles.size() * sizeof(int));
  ALLOC(sb->jao_tmap_full, jao_full.size() * sizeof(int));
  if (cudaMemcpy(sb->jao_tmap_full, jao_full.data(), jao_full.size() * sizeof(int), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return DONOF_RI_E_CUDA;
  if (cudaMemcpy(sb->jao_tmap, jao_tiles.data(), jao_tiles.size() * sizeof(int), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return DONOF_RI_E_CUDA;
  if (cudaMemcpy(sb->kao_tmap, kao_tiles.data(), kao_tiles.size() * sizeof(int), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return DONOF_RI_E_CUDA;
  {
    // the 32 x 32 destination blocks of the mirrors: those holding an element below
    // the diagonal that the J^(q) (resp. K^(q)) GEMM skips
    std::vector<int> lists[2];
    const int nbk = (nb + 31) / 32;
    for (int jao = 0; jao < 2; ++jao) {
      const int bn = jao ? S4Cfg<S_JAO>::BN : S4Cfg<S_KAO>::BN;
      for (int bi = 0; bi < nbk; ++bi)
        for (int bj = 0; bj <= bi; ++bj) {
          bool work = false;
          for (int r = 0; r < 32 && !work; ++r)
            for (int x = 0; x < 32 && !work; ++x) {
              const int mu = bi * 32 + r, nu = bj * 32 + x;
              if (mu < nb && nu < nb && nu < mu)
                work = jao ? jao_block_skipped(((long long)mu * nb + nu) / 128 * 128, nb) : !kao_tile_computed(mu, nu, bn);
            }
          if (work) lists[jao].push_back((bi << 16) | bj);
        }
    }
    sb->mir_n_kao = (int)lists[0].size();
    sb->mir_n_jao = (int)lists[1].size();
    ALLOC(sb->mir_kao, (lists[0].size() + 1) * sizeof(int));
    ALLOC(sb->mir_jao, (lists[1].size() + 1) * sizeof(int));
    if ((!lists[0].empty() && cudaMemcpy(sb->mir_kao, lists[0].data(), lists[0].size() * sizeof(int),
                                         cudaMemcpyHostToDevice) != cudaSuccess) ||
        (!lists[1].empty() && cudaMemcpy(sb->mir_jao, lists[1].data(), lists[1].size() * sizeof(int),
                                         cudaMemcpyHostToDevice) != cudaSuccess))
      return DONOF_RI_E_CUDA;
  }
  ALLOC(sb->Dp, ms * 4 * nxp * 2);
  ALLOC(sb->JKp, 2 * ms * nbs * 4 * nbp * 2);
  ALLOC(sb->eB1, nxs * nbs * 4);
  ALLOC(sb->eB5, nbs * nbs * 4);
  ALLOC(sb->eC, ms * 4);
  ALLOC(sb->e3, nxs * ms * 4);
  ALLOC(sb->e6, ms * nbs * 4);
  ALLOC(sb->ed, ms * 4);
  ALLOC(sb->eJK, 2 * ms * nbs * 4);
  ALLOC(sb->rmaxB, nxs * nbs * 4);
  ALLOC(sb->maxB, nbs * nbs * 4);
  ALLOC(sb->absC, ms * nbs * 4);
  ALLOC(sb->absCt, ms * nbs * 4);
  ALLOC(sb->Ls, nbs * nbs * 8);
  ALLOC(sb->LsTdf, nbs * nbs * 8);
  ALLOC(sb->Cin, nbs * nbs * 8);
  ALLOC(sb->Cp, nbs * nbs * 8);
  ALLOC(sb->Cinp, ms * nbs * 8);
  ALLOC(sb->Cdf, nbs * nbs * 8);
  ALLOC(sb->Hdf, nbs * nbs * 8);
  ALLOC(sb->Cdfp, ms * nbs * 8);
  ALLOC(sb->eterm, ms * 8);
  ALLOC(sb->ticket, 4);
  ALLOC(sb->dpart, (size_t)((nb + 63) / 64) * ms * nxs * 8);
  ALLOC(sb->dmat, ms * nxs * 8);
  ALLOC(sb->JKhi, 2 * ms * nbs * ldo * 4);
  ALLOC(sb->JKlo, 2 * ms * nbs * ldo * 4);
  ALLOC(sb->W, 2 * ms * ms * 8);
  ALLOC(sb->HCt, ms * nbs * 8);
  ALLOC(sb->Yt, ms * nbs * 8);
  ALLOC(sb->partial, pbytes);
  ALLOC(sb->partial_j, jbytes);
#undef ALLOC

  // The working basis (see S4Buffers): L from the overlap, then B' = L^-1 B L^-T and
  // H' = L^-1 H L^-T in FP64 (temporaries freed after the digitisation), L^T as
  // double-float pairs for the per-iteration C' = L^T C.
  cudaStream_t s = ctx->stream;
  double *Li = nullptr, *Tb = nullptr, *Bw = nullptr, *Hw = nullptr;
  int rc;
  auto free_tmp = [&]() {
    if (Li) cudaFree(Li);
    if (Tb) cudaFree(Tb);
    if (Bw) cudaFree(Bw);
    if (Hw) cudaFree(Hw);
  };
  if (cudaMalloc((void**)&Li, nbs * nbs * 8) != cudaSuccess || cudaMalloc((void**)&Tb, nxs * nbs * nbs * 8) != cudaSuccess ||
      cudaMalloc((void**)&Bw, nxs * nbs * nbs * 8) != cudaSuccess || cudaMalloc((void**)&Hw, nbs * nbs * 8) != cudaSuccess) {
    cudaGetLastError();
    free_tmp();
    return DONOF_RI_E_OOM;
  }
  if ((rc = s4_working_basis(ctx, Li, Tb, Bw, Hw))) {
    cudaStreamSynchronize(s);
    free_tmp();
    return rc;
  }
  // one-time digitisation of B' in both operand layouts, and its maxima for the bounds
  to_df_kernel<<<ceil_div_u(nbs * nbs, 256), 256, 0, s>>>(Hw, nbs * nbs, sb->Hdf);
  if (cudaMemsetAsync(sb->ticket, 0, sizeof(unsigned int), s) != cudaSuccess) return DONOF_RI_E_CUDA;
  {
    long long rows = nxs * nbs;  // rows (P, nu) over mu (B' symmetric)
    slice_f64_kernel<<<ceil_div_u(rows * 32, 256), 256, 0, s>>>(Bw, rows, nb, nb, 1, sb->B1, nbp, sb->eB1,
                                                                 nullptr, nullptr, nullptr);
    DONOF_LAUNCH_CHECK(ctx);
    long long rows5 = nbs * nbs;  // rows (mu nu) over P
    slice_f64_kernel<<<ceil_div_u(rows5 * 32, 256), 256, 0, s>>>(Bw, rows5, nx, 1, nbs * nbs, sb->B5, nxp,
                                                                  sb->eB5, nullptr, nullptr, nullptr);
    DONOF_LAUNCH_CHECK(ctx);
    bmax_rows_kernel<<<ceil_div_u(nxs * nbs, 256), 256, 0, s>>>(Bw, nx, nb, sb->rmaxB);
    DONOF_LAUNCH_CHECK(ctx);
    bmax_aux_kernel<<<ceil_div_u(nbs * nbs, 256), 256, 0, s>>>(Bw, nx, nb, sb->maxB);
    DONOF_LAUNCH_CHECK(ctx);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    free_tmp();
    return DONOF_RI_E_CUDA;
  }
  free_tmp();

  for (int k = 0; k < S_NKINDS; ++k) {
    S4Params& p = sb->plan[k];
    p.nb = nb; p.nx = nx; p.m = m; p.nbp = nbp; p.nxp = nxp; p.mp = mp;
    p.status = ctx->d_status;
    p.partial = k == S_JMO ? sb->partial_j : sb->partial;
    p.ldo = ldo;
  }
  {  // HALF: A = B1 [nx][nb][4][nbp] rows (P, nu) over mu; B = C^T digits [m][4][nbp]
    S4Params& p = sb->plan[S_HALF];
    long long dA[4] = {nb, 4, nb, nx}, sA[3] = {nbp, 4LL * nbp, nbs * 4 * nbp};
    int bA[4] = {S4_BK, 1, 16, 8};
    long long dB[3] = {nb, 4, m}, sB[2] = {nbp, 4LL * nbp};
    int bB[3] = {S4_BK, 1, bn};
    if ((rc = s4_map(sb, &p.a, sb->B1, 4, dA, sA, bA))) return rc;
    if ((rc = s4_map(sb, &p.b, sb->Ct, 3, dB, sB, bB))) return rc;
    p.ea = sb->eB1; p.eb = sb->eC;
    p.o3 = sb->L3; p.e3 = sb->e3;
    p.x6 = sb->X6; p.e6 = sb->e6;
    // the one-CTA variant: same operands, its own schedule
    S4Params& p1 = sb->plan[S_HALF1];
    const int st1 = p1.stages, tc1 = p1.tmem_cols, pe1 = p1.persist, nt1 = p1.ntiles, ntl1 = p1.n_tiles;
    p1 = p;
    p1.stages = st1; p1.tmem_cols = tc1; p1.persist = pe1; p1.ntiles = nt1; p1.n_tiles = ntl1;
  }
  {  // FULLSQ: A = L3 [nx][mp][4][nbp] rows p (per P) over nu; B = C^T digits
    S4Params& p = sb->plan[S_FULLSQ];
    long long dA[4] = {nb, 4, m, nx}, sA[3] = {nbp, 4LL * nbp, (long long)mp * 4 * nbp};
    int bA[4] = {S4_BK, 1, S4_BM, 1};
    long long dB[3] = {nb, 4, m}, sB[2] = {nbp, 4LL * nbp};
    int bB[3] = {S4_BK, 1, bn};
    if ((rc = s4_map(sb, &p.a, sb->L3, 4, dA, sA, bA))) return rc;
    if ((rc = s4_map(sb, &p.b, sb->Ct, 3, dB, sB, bB))) return rc;
    p.ea = sb->e3; p.eb = sb->eC;
    p.prow = m; p.pcol = m;
  }
  {  // JMO: A = B = d digits [m][4][nxp] rows p over P
    S4Params& p = sb->plan[S_JMO];
    long long dA[3] = {nx, 4, m}, sA[2] = {nxp, 4LL * nxp};
    int bA[3] = {S4_BK, 1, S4_BM};
    int bB[3] = {S4_BK, 1, bn};
    if ((rc = s4_map(sb, &p.a, sb->Dp, 3, dA, sA, bA))) return rc;
    if ((rc = s4_map(sb, &p.b, sb->Dp, 3, dA, sA, bB))) return rc;
    p.ea = sb->ed; p.eb = sb->ed;
    p.prow = m; p.pcol = m;
  }
  {  // JAO: A = B5 [nb*nb][4][nxp] rows (mu nu) over P; B = d digits
    S4Params& p = sb->plan[S_JAO];
    long long dA[3] = {nx, 4, nbs * nbs}, sA[2] = {nxp, 4LL * nxp};
    int bA[3] = {S4_BK, 1, S4_BM};
    long long dB[3] = {nx, 4, m}, sB[2] = {nxp, 4LL * nxp};
    int bB[3] = {S4_BK, 1, bn};
    if ((rc = s4_map(sb, &p.a, sb->B5, 3, dA, sA, bA))) return rc;
    if ((rc = s4_map(sb, &p.b, sb->Dp, 3, dB, sB, bB))) return rc;
    p.ea = sb->eB5; p.eb = sb->ed;
    p.ohi = sb->JKhi; p.olo = sb->JKlo;
    p.tmap = sb->jao_sym ? sb->jao_tmap : sb->jao_tmap_full;
  }
  {  // KAO: A = B = L6 [m][nb][4][nxp] rows (p, mu) over P
    S4Params& p = sb->plan[S_KAO];
    long long dA[4] = {nx, 4, nb, m}, sA[3] = {nxp, 4LL * nxp, nbs * 4 * nxp};
    int bA[4] = {S4_BK, 1, S4_BM, 1};
    int bB[4] = {S4_BK, 1, bn, 1};
    if ((rc = s4_map(sb, &p.a, sb->L6, 4, dA, sA, bA))) return rc;
    if ((rc = s4_map(sb, &p.b, sb->L6, 4, dA, sA, bB))) return rc;
    p.ea = sb->e6; p.eb = sb->e6;
    p.ohi = sb->JKhi; p.olo = sb->JKlo;
    p.tmap = sb->kao_tmap;
  }
  {  // FOCK: A = C^T digits [m][4][nbp] rows p over nu; B = JK digits [2m][nb][4][nbp]
     // rows mu (per q') over nu.  Orbitals on the rows: N_Omega <= N_b fills the
     // 128-row tiles at least as well as mu would, and the weight W[q'][p] is per row.
    S4Params& p = sb->plan[S_FOCK];
    long long dA[3] = {nb, 4, m}, sA[2] = {nbp, 4LL * nbp};
    int bA[3] = {S4_BK, 1, S4_BM};
    long long dB[4] = {nb, 4, nb, 2 * ms}, sB[3] = {nbp, 4LL * nbp, nbs * 4 * nbp};
    int bB[4] = {S4_BK, 1, bn, 1};
    if ((rc = s4_map(sb, &p.a, sb->Ct, 3, dA, sA, bA))) return rc;
    if ((rc = s4_map(sb, &p.b, sb->JKp, 4, dB, sB, bB))) return rc;
    p.ea = sb->eC; p.eb = sb->eJK;
    p.w = sb->W;
    p.prow = m; p.pcol = nb;
  }
  sb->plan[S_JKAO].stages = 0;
  s4_plan_jkao(sb);
  // J^(q) and K^(q) in one persistent launch while every unit is one K chunk (it
  // saves a launch and its tail); beyond 512 auxiliary functions two launches are
  // faster (C20H40: 14.4 against 15.7 ms).  s4_autotune measures both.
  sb->jk_merged = nx <= S4_CHUNK_KB * S4_BK ? 1 : 0;
#define OPTIN(KIND, ONE)                                                                                      \
  if (cudaFuncSetAttribute(s4_gemm_kernel<KIND, ONE>, cudaFuncAttributeMaxDynamicSharedMemorySize,           \
                           (int)sb->smem[KIND]) != cudaSuccess ||                                             \
      cudaFuncSetAttribute(s4_gemm_kernel<KIND, ONE>, cudaFuncAttributePreferredSharedMemoryCarveout,        \
                           (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)                               \
    return DONOF_RI_E_CUDA;
  OPTIN(S_HALF, 0) OPTIN(S_HALF, 1) OPTIN(S_HALF1, 0) OPTIN(S_HALF1, 1) OPTIN(S_FULLSQ, 0) OPTIN(S_FULLSQ, 1) OPTIN(S_JMO, 0) OPTIN(S_JAO, 0) OPTIN(S_JAO, 1)
  OPTIN(S_KAO, 0) OPTIN(S_KAO, 1) OPTIN(S_FOCK, 1) OPTIN(S_JKAO, 0) OPTIN(S_JKAO, 1) OPTIN(S_CTR, 0)
#undef OPTIN
  return DONOF_RI_OK;
}

void s4_free(donof_ri_ctx* ctx) {
  S4Buffers* sb = ctx->s4;
  if (!sb) return;
  void* bufs[] = {sb->mir_jao, sb->mir_kao, sb->jao_tmap_full, sb->jao_tmap, sb->kao_tmap, sb->X6,    sb->B1,   sb->B5,   sb->Ct,   sb->L3,   sb->L6, sb->Dp,  sb->JKp,  sb->eB1,   sb->eB5,
                  sb->eC,    sb->e3,   sb->e6,   sb->ed,   sb->eJK, sb->rmaxB, sb->maxB, sb->absC, sb->absCt,
                  sb->Ls,    sb->LsTdf, sb->Cin,   sb->Cp,   sb->Cinp,
                  sb->Cdf,   sb->Hdf,   sb->Cdfp,  sb->eterm, sb->ticket, sb->dpart, sb->dmat, sb->JKhi, sb->JKlo, sb->W,  sb->HCt, sb->Yt,   sb->partial, sb->partial_j,
                  sb->bf,    sb->wP,    sb->Xd,    sb->eX};
  for (void* b : bufs)
    if (b) cudaFree(b);
  free(sb);
  ctx->s4 = nullptr;
}

template <int KIND>
static int launch_s4(donof_ri_ctx* ctx) {
  S4Buffers* sb = ctx->s4;
  if (sb->grid[KIND] <= 0) return DONOF_RI_OK;
  ProfScope ps(ctx, KIND == S_JKAO  ? DONOF_RI_GEMM_JAO
                    : KIND == S_CTR ? DONOF_RI_GEMM_FOCK
                                    : DONOF_RI_GEMM_HALF + KIND);
  // single-chunk epilogue where every unit's K fits one chunk (F^(p) C_p: always)
  const int kext = (KIND == S_JAO || KIND == S_KAO || KIND == S_JKAO) ? ctx->naux : ctx->nbf;
  const bool one =
      KIND == S_FOCK ||
      ((KIND == S_HALF || KIND == S_FULLSQ || KIND == S_JAO || KIND == S_KAO || KIND == S_JKAO) &&
       kext <= s4_chunk_kb(KIND) * S4_BK);
  if constexpr (KIND == S_HALF) {
    const S4Params& p1 = sb->plan[S_HALF1];
    const int g1 = sb->grid[S_HALF1];
    const size_t m1 = sb->smem[S_HALF1];
    constexpr int T1 = S4Cfg<S_HALF1>::THREADS;
    const dim3 g0(sb->grid[KIND]), t0(S4Cfg<KIND>::THREADS);
    const size_t m0 = sb->smem[KIND];
    if (sb->half_variant && one) launch_pdl(s4_gemm_kernel<S_HALF1, 1>, dim3(g1), dim3(T1), m1, ctx->stream, p1);
    else if (sb->half_variant) launch_pdl(s4_gemm_kernel<S_HALF1, 0>, dim3(g1), dim3(T1), m1, ctx->stream, p1);
    else if (one) launch_pdl(s4_gemm_kernel<S_HALF, 1>, g0, t0, m0, ctx->stream, sb->plan[KIND]);
    else launch_pdl(s4_gemm_kernel<S_HALF, 0>, g0, t0, m0, ctx->stream, sb->plan[KIND]);
  } else {
    const dim3 g0(sb->grid[KIND]), t0(S4Cfg<KIND>::THREADS);
    const size_t m0 = sb->smem[KIND];
    if constexpr (KIND == S_FOCK) {
      (void)one;
      launch_pdl(s4_gemm_kernel<KIND, 1>, g0, t0, m0, ctx->stream, sb->plan[KIND]);
    } else if constexpr (KIND == S_FULLSQ || KIND == S_JAO || KIND == S_KAO || KIND == S_JKAO) {
      if (one) launch_pdl(s4_gemm_kernel<KIND, 1>, g0, t0, m0, ctx->stream, sb->plan[KIND]);
      else launch_pdl(s4_gemm_kernel<KIND, 0>, g0, t0, m0, ctx->stream, sb->plan[KIND]);
    } else {
      (void)one;
      launch_pdl(s4_gemm_kernel<KIND, 0>, g0, t0, m0, ctx->stream, sb->plan[KIND]);
    }
  }
  DONOF_LAUNCH_CHECK(ctx);
  return DONOF_RI_OK;
}

int s4_transform(donof_ri_ctx* ctx, int mode) {
  S4Buffers* sb = ctx->s4;
  const int nb = ctx->nbf, nx = ctx->naux, m = ctx->n_omega;
  cudaStream_t s = ctx->stream;
  int rc;
  {
    ProfScope ps(ctx, DONOF_RI_ROW_OTHER);
    // the orbitals in the working basis, C' = L^T C: rows of C'^T [p][mu'] =
    // sum_mu C^T[p][mu] L[mu][mu'] (C column-major = rows p contiguous), in double-float
    launch_pdl(to_df_kernel, dim3(ceil_div_u((long long)nb * nb, 256)), dim3(256), 0, s, (const double*)ctx->d_C,
               (long long)nb * nb, sb->Cin);
    DONOF_LAUNCH_CHECK(ctx);
    launch_pdl(df_gemm_nt_kernel<double>, dim3((nb + DFG_TJ - 1) / DFG_TJ, (nb + DFG_TI - 1) / DFG_TI),
               dim3(DFG_THREADS), 0, s, nb, nb, nb, (const float2*)sb->Cin, nb, (const float2*)sb->LsTdf, nb, sb->Cp,
               nb);
    DONOF_LAUNCH_CHECK(ctx);
    // C'^T rows p over mu' (and every row of C' as double-float pairs, for lambda)
    launch_pdl(slice_rows_kernel, dim3(nb), dim3(SLICE_ROWS_THREADS), 0, s, (const double*)sb->Cp, m, nb,
               (long long)nb, sb->Ct, sb->nbp, sb->eC, sb->absC, sb->absCt, sb->Cdf);
    DONOF_LAUNCH_CHECK(ctx);
    // the two bound passes are independent: e6 on the second stream
    cudaStream_t main_stream;
    const bool forked = fork_begin(ctx, &main_stream);
    launch_pdl(bound_kernel, dim3((nb + BOUND_TILE - 1) / BOUND_TILE, (m + BOUND_TILE - 1) / BOUND_TILE), dim3(256), 0,
               ctx->stream, m, nb, nb, (const float*)sb->absC, nb, (const float*)sb->maxB, nb, sb->e6, nb);
    rc = cudaGetLastError() == cudaSuccess ? DONOF_RI_OK : DONOF_RI_E_CUDA;
    ctx->launches++;
    if (forked) fork_end(ctx, main_stream);
    launch_pdl(bound_kernel, dim3((m + BOUND_TILE - 1) / BOUND_TILE, (nx + BOUND_TILE - 1) / BOUND_TILE), dim3(256), 0, s,
               nx, m, nb, (const float*)sb->rmaxB, nb, (const float*)sb->absCt, m, sb->e3, m);
    DONOF_LAUNCH_CHECK(ctx);
    if (forked && (rc = fork_join(ctx))) return rc;
    if (rc) return rc;
  }
  {
    ProfScope ps(ctx, DONOF_RI_ROW_HALF);
    if ((rc = launch_s4<S_HALF>(ctx))) return rc;
    dim3 g((nb + 63) / 64, (nx + 63) / 64, m), b(32, 8);
    ProfScope pm(ctx, DONOF_RI_MEM_DIGITS);
    launch_pdl(xf_to_digits_kernel, g, b, 0, s, (const int*)sb->X6, (const int*)sb->e3, (const int*)sb->e6, nx, nb, m,
               sb->mp, sb->nbp, sb->nxp, sb->L3, sb->L6, (const float2*)sb->Cdf, sb->dpart);
    DONOF_LAUNCH_CHECK(ctx);
  }
  {
    ProfScope ps(ctx, DONOF_RI_ROW_DIAG);
    launch_pdl(diag_reduce_kernel, dim3(ceil_div_u((long long)nx * m, 256)), dim3(256), 0, s, (const float2*)sb->dpart,
               (nb + 63) / 64, nx, m, (const int*)sb->e3, sb->dmat);
    DONOF_LAUNCH_CHECK(ctx);
    launch_pdl(slice_rows_kernel, dim3(m), dim3(SLICE_ROWS_THREADS), 0, s, (const double*)sb->dmat, m, nx,
               (long long)nx, sb->Dp, sb->nxp, sb->ed, (float*)nullptr, (float*)nullptr, (float2*)nullptr);
    DONOF_LAUNCH_CHECK(ctx);
  }
  if (mode == DONOF_RI_FULL) {
    // J_pq (a few CTAs, its own partial buffer) runs on the second stream beside the
    // full transform, on the SMs the latter leaves free; the shared-memory footprint
    // of both kinds keeps their CTAs off each other's SMs.
    cudaStream_t main_stream;
    const bool forked = fork_begin(ctx, &main_stream);
    int rcj;
    {
      ProfScope ps(ctx, DONOF_RI_ROW_J);
      rcj = launch_s4<S_JMO>(ctx);
      if (!rcj) {
        const S4Params& p = sb->plan[S_JMO];
        launch_pdl(reduce_jmo_kernel, dim3(ceil_div_u((long long)m * m, 256)), dim3(256), 0, ctx->stream,
                   (const long long*)p.partial, p.nsplit, m, (const int*)sb->ed, ctx->d_J);
        rcj = cudaGetLastError() == cudaSuccess ? DONOF_RI_OK : DONOF_RI_E_CUDA;
        ctx->launches++;
      }
    }
    if (forked) fork_end(ctx, main_stream);
    {
      ProfScope ps(ctx, DONOF_RI_ROW_FULL_K);
      if ((rc = launch_s4<S_FULLSQ>(ctx))) return rc;
      const S4Params& p = sb->plan[S_FULLSQ];
      launch_pdl(reduce_df_kernel, dim3(ceil_div_u((long long)m * m, 32)), dim3(32, 8), 0, s, (const float2*)p.partial,
                 p.nsplit, m, m, ctx->d_K, (float2*)nullptr, (const double*)nullptr, (const float2*)nullptr);
      DONOF_LAUNCH_CHECK(ctx);
    }
    if (forked && (rc = fork_join(ctx))) return rc;
    if (rcj) return rcj;
  }
  return DONOF_RI_OK;
}

// The mirrors after the J^(q) (jao = 1) or K^(q) GEMM: only the blocks in the list.
static int launch_mirror(donof_ri_ctx* ctx, int jao, bool pdl) {
  S4Buffers* sb = ctx->s4;
  const int n = jao ? sb->mir_n_jao : sb->mir_n_kao;
  if (n == 0) return DONOF_RI_OK;
  const dim3 g(n, ctx->n_omega), b(32, 8);
  const int* tl = jao ? sb->mir_jao : sb->mir_kao;
  const int row0 = jao ? 0 : ctx->n_omega;
  const int bn = jao ? S4Cfg<S_JAO>::BN : S4Cfg<S_KAO>::BN;
  if (pdl)
    launch_pdl(sym_mirror_kernel, g, b, 0, ctx->stream, sb->JKhi, sb->JKlo, ctx->nbf, row0, sb->ldo, bn, jao, tl);
  else
    sym_mirror_kernel<<<g, b, 0, ctx->stream>>>(sb->JKhi, sb->JKlo, ctx->nbf, row0, sb->ldo, bn, jao, tl);
  DONOF_LAUNCH_CHECK(ctx);
  return DONOF_RI_OK;
}

int s4_jk_ao(donof_ri_ctx* ctx) {
  S4Buffers* sb = ctx->s4;
  const int nb = ctx->nbf, m = ctx->n_omega;
  int rc;
  if (sb->jk_merged && !ctx->prof_enabled) {
    // one persistent launch for every J^(q) and K^(q) unit, then the mirrors.  Per-row
    // profiling keeps the two launches apart so that each row has its own events.
    if ((rc = launch_s4<S_JKAO>(ctx))) return rc;
    if (sb->jao_sym && (rc = launch_mirror(ctx, 1, true))) return rc;
    if ((rc = launch_mirror(ctx, 0, true))) return rc;
  } else {
  {
    ProfScope ps(ctx, DONOF_RI_ROW_JAO);
    if ((rc = launch_s4<S_JAO>(ctx))) return rc;
    if (sb->jao_sym && (rc = launch_mirror(ctx, 1, true))) return rc;
  }
  {
    ProfScope ps(ctx, DONOF_RI_ROW_KAO);
    if ((rc = launch_s4<S_KAO>(ctx))) return rc;
    if ((rc = launch_mirror(ctx, 0, true))) return rc;
  }
  }
  {
    ProfScope ps(ctx, DONOF_RI_ROW_OTHER);
    long long rows = 2LL * m * nb;
    ProfScope pm(ctx, DONOF_RI_MEM_SPLIT);
    launch_pdl(slice_pair_kernel, dim3(ceil_div_u(rows * 32, 256)), dim3(256), 0, ctx->stream, (const float*)sb->JKhi,
               (const float*)sb->JKlo, rows, nb, sb->ldo, sb->JKp, sb->nbp, sb->eJK);
    DONOF_LAUNCH_CHECK(ctx);
  }
  return DONOF_RI_OK;
}

int s4_energy(donof_ri_ctx* ctx, int part) {
  S4Buffers* sb = ctx->s4;
  const int nb = ctx->nbf, m = ctx->n_omega;
  cudaStream_t s = ctx->stream;
  int rc;
  ProfScope ps(ctx, DONOF_RI_ROW_ENERGY);
  if (part & ENERGY_PREP) {
    if ((rc = launch_occupations_coupling(ctx))) return rc;
    launch_pdl(fock_weights_df_kernel, dim3(ceil_div_u(2LL * m * m, 256)), dim3(256), 0, s, (const double*)ctx->d_A,
               (const double*)ctx->d_Bc, m, sb->W);
    DONOF_LAUNCH_CHECK(ctx);
    // (H' C')^T [p][mu'] as double-float pairs, from the prep's own double-float copy of
    // C' = L^T C (this part may run on a second stream beside the transform)
    launch_pdl(to_df_kernel, dim3(ceil_div_u((long long)m * nb, 256)), dim3(256), 0, s, (const double*)ctx->d_C,
               (long long)m * nb, sb->Cinp);
    DONOF_LAUNCH_CHECK(ctx);
    launch_pdl(df_gemm_nt_kernel<float2>, dim3((nb + DFG_TJ - 1) / DFG_TJ, (m + DFG_TI - 1) / DFG_TI), dim3(DFG_THREADS),
               0, s, m, nb, nb, (const float2*)sb->Cinp, nb, (const float2*)sb->LsTdf, nb, sb->Cdfp, nb);
    DONOF_LAUNCH_CHECK(ctx);
    launch_pdl(df_gemm_nt_kernel<float2>, dim3((nb + DFG_TJ - 1) / DFG_TJ, (m + DFG_TI - 1) / DFG_TI), dim3(DFG_THREADS),
               0, s, m, nb, nb,
               (const float2*)sb->Cdfp, nb, (const float2*)sb->Hdf, nb, sb->HCt, nb);
    DONOF_LAUNCH_CHECK(ctx);
  }
  if (!(part & ENERGY_MAIN)) return DONOF_RI_OK;
  if ((rc = launch_s4<S_FOCK>(ctx))) return rc;
  const S4Params& p = sb->plan[S_FOCK];
  launch_pdl(reduce_df_kernel, dim3(ceil_div_u((long long)nb * m, 32)), dim3(32, 8), 0, s, (const float2*)p.partial,
             p.nsplit, m, nb, (double*)nullptr, sb->Yt, (const double*)ctx->d_n, (const float2*)sb->HCt);
  DONOF_LAUNCH_CHECK(ctx);
  // lambda[p][q] = Y^T_p . C_q for every q < nbf
  launch_pdl(df_gemm_nt_kernel<double>, dim3((nb + DFG_TJ - 1) / DFG_TJ, (m + DFG_TI - 1) / DFG_TI), dim3(DFG_THREADS),
             0, s, m, nb, nb,
             (const float2*)sb->Yt, nb, (const float2*)sb->Cdf, nb, ctx->d_lambda, nb);
  DONOF_LAUNCH_CHECK(ctx);
  launch_pdl(energy_terms_kernel, dim3(m), dim3(32), 0, s, nb, m, (const float2*)sb->Cdf, (const float2*)sb->HCt,
             (const double*)ctx->d_n, (const double*)ctx->d_lambda, (const double*)ctx->d_enuc, sb->eterm, sb->ticket,
             ctx->d_E);
  DONOF_LAUNCH_CHECK(ctx);
  return DONOF_RI_OK;
}

// ---------------------------------------------------------------------------
// Contracted Lagrangian on the digit path.  With w_pP = sum_q A_pq b^P_qq and
// X^P_qp = [q = p] w_pP - B_pq b^P_qp,
//   F^(p) C_p = n_p H C_p + sum_q sum_P X^P_qp b^P_{q .}
// (J^(q) C_p = sum_P b^P_qq b^P_{p .}, K^(q) C_p = sum_P b^P_{q .} b^P_qp), one
// digit-plane GEMM of N_b N_Omega^2 N_aux products (S_CTR) in place of J^(q),
// K^(q) and the Fock sum.  b^P_qp comes from the full transform's GEMM run once more
// with its store switched on, w from an FP64 GEMM, X's digits from
// ctr_digits_kernel; Y, lambda and E then as in s4_energy.
// ---------------------------------------------------------------------------
static int s4_ctr_setup(donof_ri_ctx* ctx) {
  S4Buffers* sb = ctx->s4;
  const long long nb = ctx->nbf, nx = ctx->naux, m = ctx->n_omega, nxp = sb->nxp;
  // every buffer and both tensor maps first, then the context's pointers: a failed
  // set-up leaves nothing behind and the next call starts again
  double *bf = nullptr, *wP = nullptr;
  __nv_bfloat16* Xd = nullptr;
  int* eX = nullptr;
  auto release = [&]() {
    cudaFree(bf);
    cudaFree(wP);
    cudaFree(Xd);
    cudaFree(eX);
  };
  if (cudaMalloc((void**)&bf, (size_t)(nx * m * m * 8)) != cudaSuccess ||
      cudaMalloc((void**)&wP, (size_t)(m * nx * 8)) != cudaSuccess ||
      cudaMalloc((void**)&Xd, (size_t)(m * m * 4 * nxp * 2)) != cudaSuccess ||
      cudaMalloc((void**)&eX, (size_t)(m * m * 4)) != cudaSuccess) {
    cudaGetLastError();
    release();
    return DONOF_RI_E_OOM;
  }
  // A = X digits [m][m][4][nxp] rows p (per q) over P; B = L6 [m][nb][4][nxp] rows mu (per q) over P
  const int bn = S4Cfg<S_CTR>::BN;
  long long dA[4] = {nx, 4, m, m}, sA[3] = {nxp, 4 * nxp, m * 4 * nxp};
  int bA[4] = {S4_BK, 1, S4_BM, 1};
  long long dB[4] = {nx, 4, nb, m}, sB[3] = {nxp, 4 * nxp, nb * 4 * nxp};
  int bB[4] = {S4_BK, 1, bn, 1};
  CUtensorMap ma, mb;
  int rc;
  if ((rc = s4_map(sb, &ma, Xd, 4, dA, sA, bA)) || (rc = s4_map(sb, &mb, sb->L6, 4, dB, sB, bB))) {
    release();
    return rc;
  }
  S4Params& p = sb->plan[S_CTR];
  p.a = ma; p.b = mb;
  p.ea = eX; p.eb = sb->e6;
  p.prow = (int)m; p.pcol = (int)nb;
  sb->bf = bf; sb->wP = wP; sb->Xd = Xd; sb->eX = eX;
  return DONOF_RI_OK;
}

int s4_energy_contracted(donof_ri_ctx* ctx) {
  S4Buffers* sb = ctx->s4;
  const int nb = ctx->nbf, nx = ctx->naux, m = ctx->n_omega;
  cudaStream_t s = ctx->stream;
  int rc;
  if (!sb->Xd && (rc = s4_ctr_setup(ctx))) return rc;
  // occupations, couplings A and B, (H' C')^T
  if ((rc = s4_energy(ctx, ENERGY_PREP))) return rc;
  ProfScope ps(ctx, DONOF_RI_ROW_ENERGY);
  {
    S4Params& pf = sb->plan[S_FULLSQ];
    pf.bfull = sb->bf;
    rc = launch_s4<S_FULLSQ>(ctx);
    pf.bfull = nullptr;
    if (rc) return rc;
  }
  Gemm64 g{};  // w[p][P] = sum_q A_pq d[q][P]
  g.M = m; g.N = nx; g.K = m; g.batch = 1;
  g.A = ctx->d_A; g.sAm = m; g.sAk = 1;
  g.B = sb->dmat; g.sBk = nx; g.sBn = 1;
  g.C = sb->wP; g.sCm = nx; g.sCn = 1;
  g.alpha = 1.0; g.beta = 0.0;
  if ((rc = launch_dgemm(ctx, g))) return rc;
  launch_pdl(ctr_digits_kernel, dim3((m + 31) / 32, m), dim3(32, 8), 0, s, (const double*)sb->bf,
             (const double*)ctx->d_Bc, (const double*)sb->wP, m, nx, sb->nxp, sb->Xd, sb->eX);
  DONOF_LAUNCH_CHECK(ctx);
  if ((rc = launch_s4<S_CTR>(ctx))) return rc;
  const S4Params& p = sb->plan[S_CTR];
  launch_pdl(reduce_df_kernel, dim3(ceil_div_u((long long)nb * m, 32)), dim3(32, 8), 0, s, (const float2*)p.partial,
             p.nsplit, m, nb, (double*)nullptr, sb->Yt, (const double*)ctx->d_n, (const float2*)sb->HCt);
  DONOF_LAUNCH_CHECK(ctx);
  launch_pdl(df_gemm_nt_kernel<double>, dim3((nb + DFG_TJ - 1) / DFG_TJ, (m + DFG_TI - 1) / DFG_TI), dim3(DFG_THREADS),
             0, s, m, nb, nb,
             (const float2*)sb->Yt, nb, (const float2*)sb->Cdf, nb, ctx->d_lambda, nb);
  DONOF_LAUNCH_CHECK(ctx);
  launch_pdl(energy_terms_kernel, dim3(m), dim3(32), 0, s, nb, m, (const float2*)sb->Cdf, (const float2*)sb->HCt,
             (const double*)ctx->d_n, (const double*)ctx->d_lambda, (const double*)ctx->d_enuc, sb->eterm, sb->ticket,
             ctx->d_E);
  DONOF_LAUNCH_CHECK(ctx);
  return DONOF_RI_OK;
}

// ---------------------------------------------------------------------------
// Autotuning: every digit-plane GEMM kind is timed on the live problem for each
// pipeline depth that fits its shared memory, the split kinds (a3, a4, a7) also
// for one and two waves of CTAs, and J^(q) with and without the symmetric
// skip-and-mirror.  Each timed launch starts from a flushed L2 (a 256 MB write
// outside the events), as inside an iteration, and a setting replaces the
// default only when it is at least 3 % faster.  Each launch rewrites its
// outputs, so the inputs stay valid.
// ---------------------------------------------------------------------------
template <int KIND>
static int s4_split(S4Buffers* sb, int target) {
  S4Params& p = sb->plan[KIND];
  const int tiles = p.ntiles;
  int ns = target / tiles;
  if (ns < 1) ns = 1;
  if (ns > p.nbatch) ns = p.nbatch;
  p.bpc = (p.nbatch + ns - 1) / ns;
  p.nsplit = (p.nbatch + p.bpc - 1) / p.bpc;
  sb->grid[KIND] = tiles * p.nsplit;
  return p.nsplit;
}

template <int KIND>
static int s4_time(donof_ri_ctx* ctx, int reps, cudaEvent_t a, cudaEvent_t b, void* flush, size_t flush_bytes,
                   float* ms) {
  S4Buffers* sb = ctx->s4;
  int rc;
  if ((rc = launch_s4<KIND>(ctx))) return rc;  // warm-up
  float total = 0.f;
  for (int r = 0; r < reps; ++r) {
    DONOF_CUDA_TRY(cudaMemsetAsync(flush, r & 255, flush_bytes, ctx->stream));
    DONOF_CUDA_TRY(cudaEventRecord(a, ctx->stream));
    if ((rc = launch_s4<KIND>(ctx))) return rc;
    if (KIND == S_JAO && sb->jao_sym && (rc = launch_mirror(ctx, 1, false))) return rc;
    DONOF_CUDA_TRY(cudaEventRecord(b, ctx->stream));
    DONOF_CUDA_TRY(cudaEventSynchronize(b));
    float t = 0.f;
    DONOF_CUDA_TRY(cudaEventElapsedTime(&t, a, b));
    total += t;
  }
  *ms = total / reps;
  return DONOF_RI_OK;
}

template <int KIND>
static int s4_tune_kind(donof_ri_ctx* ctx, int reps, cudaEvent_t a, cudaEvent_t b, void* flush, size_t fbytes,
                        int* report, int* tried) {
  S4Buffers* sb = ctx->s4;
  S4Params& p = sb->plan[KIND];
  const bool split = (KIND == S_FULLSQ || KIND == S_JMO || KIND == S_FOCK);
  // J^(q): symmetric skip on / off; half transform: the two-CTA or the one-CTA kernel
  const int nsym = (KIND == S_JAO || KIND == S_HALF) ? 2 : 1;
  float best = 1e30f, dflt = 1e30f;
  const int dS = p.stages, dT = split ? sb->target[KIND] : 0;
  const int dSym = KIND == S_HALF ? sb->half_variant : sb->jao_sym;
  const int dS1 = sb->plan[S_HALF1].stages;
  int bestS = dS, bestT = dT, bestSym = dSym;
  const int targets[2] = {split ? sb->target[KIND] : 0, split ? 2 * sb->target[KIND] : 0};
  int rc;
  for (int sym = 0; sym < nsym; ++sym) {
    if (KIND == S_JAO) {
      sb->jao_sym = sym;
      p.tmap = sym ? sb->jao_tmap : sb->jao_tmap_full;
      p.ntiles = p.n_tiles = sym ? sb->jao_ntiles_sym : sb->jao_ntiles_full;
      const int units = p.ntiles * p.nbatch, pc = S4Cfg<S_JAO>::CTAS * 152;
      sb->grid[KIND] = units < pc ? units : pc;
    }
    if (KIND == S_HALF) sb->half_variant = sym;
    S4Params& pv = (KIND == S_HALF && sym) ? sb->plan[S_HALF1] : p;
    const int maxS = (KIND == S_HALF && sym) ? sb->max_stages[S_HALF1] : sb->max_stages[KIND];
    const int defS = (KIND == S_HALF && sym) ? dS1 : dS;
    for (int ti = 0; ti < (split ? 2 : 1); ++ti) {
      if (split) s4_split<KIND>(sb, targets[ti]);
      for (int S = 2; S <= maxS; ++S) {
        pv.stages = S;
        float ms = 0.f;
        if ((rc = s4_time<KIND>(ctx, reps, a, b, flush, fbytes, &ms))) return rc;
        ++*tried;
        if (S == defS && targets[ti] == dT && ((KIND != S_JAO && KIND != S_HALF) || sym == dSym)) dflt = ms;
        if (ms < best) {
          best = ms;
          bestS = S;
          bestT = targets[ti];
          bestSym = sym;
        }
      }
    }
    pv.stages = defS;
  }
  if (!(best < 0.97f * dflt)) {  // keep the default unless clearly beaten
    best = dflt;
    bestS = (KIND == S_HALF && dSym) ? dS1 : dS;
    bestT = dT;
    bestSym = dSym;
  }
  if (KIND == S_JAO) {
    sb->jao_sym = bestSym;
    p.tmap = bestSym ? sb->jao_tmap : sb->jao_tmap_full;
    p.ntiles = p.n_tiles = bestSym ? sb->jao_ntiles_sym : sb->jao_ntiles_full;
    const int units = p.ntiles * p.nbatch, pc = S4Cfg<S_JAO>::CTAS * 152;
    sb->grid[KIND] = units < pc ? units : pc;
  }
  if (KIND == S_HALF) {
    sb->half_variant = bestSym;
    (bestSym ? sb->plan[S_HALF1] : p).stages = bestS;
  } else {
    p.stages = bestS;
  }
  if (split) s4_split<KIND>(sb, bestT);
  if (report) {
    report[KIND * 4 + 0] = bestS;
    report[KIND * 4 + 1] = split ? p.nsplit : ((KIND == S_JAO || KIND == S_HALF) ? bestSym : 0);
    report[KIND * 4 + 2] = (KIND == S_HALF && bestSym) ? sb->grid[S_HALF1] : sb->grid[KIND];
    report[KIND * 4 + 3] = (int)(best * 1000.f + 0.5f);  // microseconds
  }
  return DONOF_RI_OK;
}

// A kind's schedule set by the caller (the choices the autotuner makes): pipeline
// depth, and option = waves of CTAs (1 or 2) for the split kinds, the symmetric
// skip (0 / 1) for J^(q), the kernel variant (0: two CTAs per SM, 1: one) for the
// half transform, 0 otherwise.
int s4_set_schedule(donof_ri_ctx* ctx, int kind, int stages, int option) {
  S4Buffers* sb = ctx->s4;
  if (kind < 0 || kind > S_FOCK) return DONOF_RI_E_ARG;
  const bool split = (kind == S_FULLSQ || kind == S_JMO || kind == S_FOCK);
  const int var_kind = (kind == S_HALF && option == 1) ? S_HALF1 : kind;
  if (stages < 2 || stages > sb->max_stages[var_kind]) return DONOF_RI_E_ARG;
  if (split ? (option != 1 && option != 2)
            : ((kind == S_JAO || kind == S_HALF || kind == S_KAO) ? (option != 0 && option != 1) : option != 0))
    return DONOF_RI_E_ARG;
  S4Params& p = sb->plan[kind];
  if (kind == S_HALF) {
    sb->half_variant = option;
    sb->plan[var_kind].stages = stages;
    return DONOF_RI_OK;
  }
  p.stages = stages;
  if (kind == S_KAO) sb->jk_merged = option;
  if (kind == S_JAO) {
    sb->jao_sym = option;
    p.tmap = option ? sb->jao_tmap : sb->jao_tmap_full;
    p.ntiles = p.n_tiles = option ? sb->jao_ntiles_sym : sb->jao_ntiles_full;
    const int units = p.ntiles * p.nbatch, pc = S4Cfg<S_JAO>::CTAS * 152;
    sb->grid[kind] = units < pc ? units : pc;
  }
  if (split) {
    const int target = option * sb->target[kind];
    if (kind == S_FULLSQ) s4_split<S_FULLSQ>(sb, target);
    if (kind == S_JMO) s4_split<S_JMO>(sb, target);
    if (kind == S_FOCK) s4_split<S_FOCK>(sb, target);
  }
  if (kind == S_JAO || kind == S_KAO) s4_plan_jkao(sb);
  return DONOF_RI_OK;
}

// J^(q) and K^(q) as one launch or as two (with their mirrors), each timed from a
// flushed L2; the merged launch stays unless the pair of launches is 3 % faster.
static int s4_tune_jk_merge(donof_ri_ctx* ctx, int reps, cudaEvent_t a, cudaEvent_t b, void* flush, size_t fbytes,
                            int* tried) {
  S4Buffers* sb = ctx->s4;
  float t[2] = {0.f, 0.f};
  int rc;
  for (int merged = 0; merged < 2; ++merged) {
    sb->jk_merged = merged;
    for (int r = 0; r <= reps; ++r) {  // r = 0: warm-up
      DONOF_CUDA_TRY(cudaMemsetAsync(flush, r & 255, fbytes, ctx->stream));
      DONOF_CUDA_TRY(cudaEventRecord(a, ctx->stream));
      if (merged) {
        if ((rc = launch_s4<S_JKAO>(ctx))) return rc;
      } else {
        if ((rc = launch_s4<S_JAO>(ctx))) return rc;
        if ((rc = launch_s4<S_KAO>(ctx))) return rc;
      }
      if (sb->jao_sym && (rc = launch_mirror(ctx, 1, false))) return rc;
      if ((rc = launch_mirror(ctx, 0, false))) return rc;
      DONOF_CUDA_TRY(cudaEventRecord(b, ctx->stream));
      DONOF_CUDA_TRY(cudaEventSynchronize(b));
      float ms = 0.f;
      DONOF_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
      if (r > 0) t[merged] += ms;
    }
    ++*tried;
  }
  sb->jk_merged = (t[0] < 0.97f * t[1]) ? 0 : 1;
  return DONOF_RI_OK;
}

int s4_autotune(donof_ri_ctx* ctx, int reps, int* report, int* tried) {
  const size_t fbytes = (size_t)256 << 20;
  void* flush = nullptr;
  if (cudaMalloc(&flush, fbytes) != cudaSuccess) {
    cudaGetLastError();
    return DONOF_RI_E_OOM;
  }
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) {
    cudaFree(flush);
    return DONOF_RI_E_CUDA;
  }
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    cudaFree(flush);
    return DONOF_RI_E_CUDA;
  }
  int rc = DONOF_RI_OK;
  *tried = 0;
  if (!rc) rc = s4_tune_kind<S_HALF>(ctx, reps, a, b, flush, fbytes, report, tried);
  if (!rc) rc = s4_tune_kind<S_FULLSQ>(ctx, reps, a, b, flush, fbytes, report, tried);
  if (!rc) rc = s4_tune_kind<S_JMO>(ctx, reps, a, b, flush, fbytes, report, tried);
  if (!rc) rc = s4_tune_kind<S_JAO>(ctx, reps, a, b, flush, fbytes, report, tried);
  if (!rc) rc = s4_tune_kind<S_KAO>(ctx, reps, a, b, flush, fbytes, report, tried);
  if (!rc) rc = s4_tune_kind<S_FOCK>(ctx, reps, a, b, flush, fbytes, report, tried);
  s4_plan_jkao(ctx->s4);  // the merged J^(q) + K^(q) launch follows the tuned tile lists
  if (!rc) rc = s4_tune_jk_merge(ctx, reps, a, b, flush, fbytes, tried);
  if (!rc && report) report[S_KAO * 4 + 1] = ctx->s4->jk_merged;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(flush);
  return rc;
}

int s4_fetch(donof_ri_ctx* ctx, int what, double* dst, size_t count) {
  S4Buffers* sb = ctx->s4;
  const int nb = ctx->nbf, nx = ctx->naux, m = ctx->n_omega;
  cudaError_t e = cudaSuccess;
  if (what == DONOF_RI_FETCH_BHALF) {
    double* tmp = nullptr;
    if (cudaMalloc((void**)&tmp, count * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return DONOF_RI_E_OOM;
    }
    double* ao = nullptr;
    if (cudaMalloc((void**)&ao, count * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(tmp);
      return DONOF_RI_E_OOM;
    }
    // rows (P, p) of the L3 digits over nu'; consecutive P are mp rows apart
    for (int P = 0; P < nx && e == cudaSuccess; ++P) {
      unslice_kernel<<<ceil_div_u((long long)m * nb, 256), 256, 0, ctx->stream>>>(
          sb->L3 + (size_t)P * sb->mp * 4 * sb->nbp, sb->nbp, sb->e3 + (size_t)P * m, m, nb,
          tmp + (size_t)P * m * nb);
      e = cudaGetLastError();
    }
    // back to the AO basis: b^P_{p nu} = sum_nu' b'^P_{p nu'} L_{nu nu'}
    int rc = DONOF_RI_OK;
    if (e == cudaSuccess) {
      Gemm64 g{};
      g.M = nx * m; g.N = nb; g.K = nb; g.batch = 1;
      g.A = tmp; g.sAm = nb; g.sAk = 1;
      g.B = sb->Ls; g.sBk = 1; g.sBn = nb;
      g.C = ao; g.sCm = nb; g.sCn = 1;
      g.alpha = 1.0; g.beta = 0.0;
      rc = launch_dgemm(ctx, g);
    }
    if (e == cudaSuccess && !rc) e = cudaMemcpyAsync(dst, ao, count * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(tmp);
    cudaFree(ao);
    if (rc) return rc;
    return e == cudaSuccess ? DONOF_RI_OK : DONOF_RI_E_CUDA;
  }
  // d is kept as FP64 [p][P]; the fetch layout is [P][p]
  double* hostbuf = (double*)malloc(count * sizeof(double));
  if (!hostbuf) return DONOF_RI_E_OOM;
  e = cudaMemcpyAsync(hostbuf, sb->dmat, count * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess)
    for (int P = 0; P < nx; ++P)
      for (int pc = 0; pc < m; ++pc) dst[(size_t)P * m + pc] = hostbuf[(size_t)pc * nx + P];
  free(hostbuf);
  return e == cudaSuccess ? DONOF_RI_OK : DONOF_RI_E_CUDA;
}

int s4_copy_ao(donof_ri_ctx* ctx, double* Jao, double* Kao, bool jao_dev, bool kao_dev) {
  S4Buffers* sb = ctx->s4;
  const int nb = ctx->nbf, m = ctx->n_omega;
  const size_t n = (size_t)m * nb * nb;
  double *tmp = nullptr, *tmp2 = nullptr;
  if (cudaMalloc((void**)&tmp, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&tmp2, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    if (tmp) cudaFree(tmp);
    return DONOF_RI_E_OOM;
  }
  cudaError_t e = cudaSuccess;
  for (int which = 0; which < 2 && e == cudaSuccess; ++which) {
    double* dst = which == 0 ? Jao : Kao;
    bool dev = which == 0 ? jao_dev : kao_dev;
    if (!dst) continue;
    size_t off = (size_t)which * m * nb * sb->ldo;
    join_pair_kernel<<<ceil_div_u((long long)n, 256), 256, 0, ctx->stream>>>(sb->JKhi + off, sb->JKlo + off,
                                                                              (long long)m * nb, nb, sb->ldo, tmp);
    e = cudaGetLastError();
    // back to the AO basis: X^(q) = L X'^(q) L^T for every orbital q
    if (e == cudaSuccess) {
      const long long n2 = (long long)nb * nb;
      Gemm64 g{};
      g.M = nb; g.N = nb; g.K = nb; g.batch = m;
      g.A = sb->Ls; g.sAb = 0; g.sAm = nb; g.sAk = 1;
      g.B = tmp; g.sBb = n2; g.sBk = nb; g.sBn = 1;
      g.C = tmp2; g.sCb = n2; g.sCm = nb; g.sCn = 1;
      g.alpha = 1.0; g.beta = 0.0;
      int rc = launch_dgemm(ctx, g);
      Gemm64 h{};
      h.M = nb; h.N = nb; h.K = nb; h.batch = m;
      h.A = tmp2; h.sAb = n2; h.sAm = nb; h.sAk = 1;
      h.B = sb->Ls; h.sBb = 0; h.sBk = 1; h.sBn = nb;  // element (k, n) of L^T = L[n][k]
      h.C = tmp; h.sCb = n2; h.sCm = nb; h.sCn = 1;
      h.alpha = 1.0; h.beta = 0.0;
      if (!rc) rc = launch_dgemm(ctx, h);
      if (rc) {
        cudaFree(tmp);
        cudaFree(tmp2);
        return rc;
      }
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dst, tmp, n * sizeof(double), dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  }
  cudaFree(tmp);
  cudaFree(tmp2);
  return e == cudaSuccess ? DONOF_RI_OK : DONOF_RI_E_CUDA;
}

}  // namespace donof
