// TOA contractions on the tcgen05 tensor cores at FP32 accuracy, same quantities as
// k_toa_simt (the projected residual of Eq. raw_det_posterior with N~^-1 of Eq.
// Gmatrix_proj, whitened by Eq. WN_cov):
//   y  = [F | M | F~_lo] coef,  r~ = dt'' - y,  w~ = N^-1 r~,  chi2 = sum r~ w~,
//   ghat = F^T w~.
//
// Why an exact split.  The tensor cores accumulate in FP32 without round-to-nearest,
// and the products of one residual cancel 16-100 fold (the coefficients of low
// frequencies, the timing model and DM are nearly degenerate), so an FP32-accuracy
// result needs most of the sum to be computed without rounding at all.  Both operands
// are scaled to a common power-of-two grid and cut into fp16 pieces:
//   v = v0 + v1 + r2,  v0 on the 2^7 grid, v1 on the 2^-1 grid (|v0/2^7|, |2 v1| <= 128),
//   r = v - v0 and r2 = v - v0 - v1 rounded to fp16,
// for |v| <= 2^14.  Products of grid pieces are integers times a fixed quantum, so
//   L0 = sum X0 C0            (quantum 2^14, at most K 2^14 quanta)
//   L1 = sum X1 C0 + X0 C1    (quantum 2^6,  at most 2 K 2^14 quanta)
// stay below 2^24 quanta for K <= 511 columns and are exact in the FP32 accumulator
// whatever its rounding; the rest,
//   L2 = sum X2 C0 + X0 C2 + Xr Cr   (2^-16 of the leading terms),
// carries rounding relative to its own small size.  Six MMAs per K step represent
// both operands to about 2^-27 of their scale.  y = (L0 + L1 + L2) 2^(scale).
//
// Scaling (k_f16_pack): basis column q is normalised to 2^14 by a power of two from
// its largest value over the pulsar's TOAs (|sin|, |cos| <= 1, the largest DM weight,
// stored maxima of the timing-model and projected low-frequency columns); the
// coefficients carry the inverse factor and each chain row is normalised to 2^14 by
// its own exponent, so a chain's accuracy does not depend on the other chains.
//
// k_f16_res: F a, the residual, chi2 and w~.  One CTA per (work unit, block of NC
// chains).  The MMA's M is 128 TOAs and its A operand (the basis, 32 columns per
// chunk) is written into tensor memory by generator warps with tcgen05.st; its N is
// the NC chains and its B operand (the block's coefficients, all columns) is resident
// in shared memory.  Accumulators and basis chunks are double-buffered in tensor
// memory.  Epilogue warps read the three accumulators per TOA lane, form the
// residual, write w~ to global memory (TOA-major per chain) and reduce chi2 over the
// TOAs in FP64.
//
// k_f16_ftw: ghat = F^T w~ over the unit.  One CTA per (work unit, block of 128
// chains, chunk of <= 144 basis columns).  M = 128 chains with A = w~ in tensor memory
// (scaled per chain and unit by its largest |w~|, from k_f16_res), N = the chunk's
// columns with B = the basis in shared memory (MN-major), K = TOAs, 32 per stage.
// w~ = W0 + Wr (Wr as fp16 hi + lo), basis likewise; L0 = sum W0 X0 is exact (7-bit
// grid pieces: at most 2048 2^12 quanta), the other five products go to a second
// accumulator.
//
// Every mbarrier wait is bounded; a wait that gives up marks the CTA's chains with
// status bit 4 and the CTA drains its own MMAs before it frees tensor memory.
#include <cuda_fp16.h>

#include "pta_internal.cuh"
#include "tc_ptx.cuh"

namespace pta {
namespace {

constexpr int TTA = 128;   // TOAs per tile in k_f16_res (MMA M)
constexpr int KCA = 32;    // basis columns per chunk in k_f16_res
constexpr int KWB = 32;    // TOAs per stage in k_f16_ftw
constexpr int QWB = 144;   // basis columns per chunk in k_f16_ftw (MMA N)
constexpr int NSB = 4;     // stages in k_f16_ftw
constexpr uint32_t kWaitLimit = 4000000u;
constexpr uint32_t kDrainLimit = 4000000u;

// fp16 A and B, FP32 accumulator; A K-major, B K-major (b_mn = 0) or MN-major (1)
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, int b_mn) {
  return (1u << 4) | ((uint32_t)b_mn << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (tensor memory) (+)= A (tensor memory) x B (shared-memory descriptor)
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(d),
      "r"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// 32 lanes x 16 columns of 32-bit values (waits for completion)
__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(mbar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(mbar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          tc::smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(tc::smem_u32(mbar))
      : "memory");
}
__device__ __forceinline__ void named_bar(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

__device__ __forceinline__ uint32_t h2(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ float f16r(float v) { return __half2float(__float2half_rn(v)); }

// |v| <= 2^14: v0 on the 2^7 grid, v1 on the 2^-1 grid (round to nearest by the
// magic-number additions), r = v - v0, r2 = v - v0 - v1 (all exact in FP32)
__device__ __forceinline__ void split_grid(float v, float& v0, float& v1, float& r, float& r2) {
  v0 = __fsub_rn(__fadd_rn(v, 1610612736.f), 1610612736.f);  // 1.5 x 2^30: ulp 2^7
  r = __fsub_rn(v, v0);
  v1 = __fsub_rn(__fadd_rn(r, 6291456.f), 6291456.f);        // 1.5 x 2^22: ulp 2^-1
  r2 = __fsub_rn(r, v1);
}

// 2^e as a float for -126 <= e <= 127 (exact)
__device__ __forceinline__ float pow2f(int e) {
  e = max(-126, min(127, e));
  return __int_as_float((e + 127) << 23);
}

// s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
  return s;
}

// sin and cos of harmonic k+1 from those of harmonic k by one rotation with the
// fundamental (s1, c1): two FMA-rounded products, so a run of three rotations after an
// exactly reduced anchor stays within a few ulp of the exact values
__device__ __forceinline__ void rotate(float& s, float& c, float s1, float c1) {
  const float sn = fmaf(s, c1, c * s1);
  c = fmaf(c, c1, -(s * s1));
  s = sn;
}

// exponent e with |v| <= 2^e (frexp); 0 for v == 0
__device__ __forceinline__ int exp_up(float v) {
  int e = 0;
  frexpf(v, &e);
  return v == 0.f ? 0 : e;
}

__device__ __forceinline__ int round_up_d(int a, int b) { return (a + b - 1) / b * b; }
__device__ __forceinline__ int kx_of(const DevModel& m, int I) { return round_up_d(m.P + m.m[I] + m.NL, KCA); }

// Column maxima of the basis over pulsar I's TOAs (sin/cos: 1; DM: largest weight;
// fixed columns: stored)
__device__ __forceinline__ float basis_colmax(const DevModel& m, int I, int q) {
  if (q < 2 * m.na) return 1.f;
  if (q < m.P) return m.wmaxp[I];
  const int j = q - m.P;
  return j < m.m[I] + m.NL ? m.colmaxf[(size_t)I * (m.m_max + m.NL) + (j < m.m[I] ? j : m.m_max + j - m.m[I])] : 0.f;
}

// ---------------------------------------------------------------------------
// Pack: per (pulsar, block of NC chains) the basis column factors, the chain
// exponents and the four fp16 pieces of the scaled coefficients in the MMA's K-major
// layout: element (chain n, column k) of piece a at a PM NC 2 + (k/8) NC 16 + (n/8) 128
// + (n%8) 16 + (k%8) 2 bytes.  Pieces: 0 C0, 1 C1, 2 C2 (fp16 of r2), 3 Cr.
// Column q of the basis is normalised by its own largest value over the pulsar's TOAs,
// X' = X 2^(14 - c_q), and the coefficients carry the inverse factor, C' = C 2^c_q,
// each chain row normalised to 2^14 by its own exponent E_n: so every chain's accuracy
// is relative to its own largest term, independent of the other chains of the block.
// ---------------------------------------------------------------------------
template <int NC>
__global__ void __launch_bounds__(256)
    k_f16_pack(DevModel m, const float* __restrict__ a32, unsigned char* __restrict__ c16, float* __restrict__ spf,
               int* __restrict__ yexp, int B, int nCB) {
  extern __shared__ float sh[];
  float* cf = sh;                 // [PM] coefficient factors 2^c_q
  __shared__ int s_e[NC];
  const int I = blockIdx.x, cb = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b0 = cb * NC, nvalid = min(NC, B - b0), KX = kx_of(m, I), PM = m.PM;
  const float* rows = a32 + ((size_t)I * B + b0) * PM;
  float* spo = spf + ((size_t)I * nCB + cb) * PM;
  for (int q = tid; q < KX; q += 256) {
    const int c = exp_up(basis_colmax(m, I, q));
    cf[q] = ldexpf(1.f, c);
    spo[q] = ldexpf(1.f, 14 - c);
  }
  __syncthreads();
  // per-chain exponent of max_q |C_nq 2^c_q| (one warp per chain)
  for (int n = warp; n < NC; n += 8) {
    float mx = 0.f;
    if (n < nvalid)
      for (int q = lane; q < KX; q += 32) mx = fmaxf(mx, fabsf(rows[(size_t)n * PM + q]) * cf[q]);
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
      s_e[n] = exp_up(mx);
      if (n < nvalid) yexp[(size_t)I * B + b0 + n] = exp_up(mx) - 28;
    }
  }
  __syncthreads();
  unsigned char* out = c16 + ((size_t)I * nCB + cb) * 4 * (size_t)PM * NC * 2;
  const size_t asz = (size_t)PM * NC * 2;
  for (int e = tid; e < NC * (KX / 8); e += 256) {
    const int n = e % NC, g = e / NC;  // consecutive threads: consecutive chains
    float c0[8], c1[8], c2[8], cr[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int q = 8 * g + i;
      const float v = n < nvalid ? ldexpf(rows[(size_t)n * PM + q] * cf[q], 14 - s_e[n]) : 0.f;
      float r;
      split_grid(v, c0[i], c1[i], r, c2[i]);
      cr[i] = r;
    }
    const size_t off = (size_t)g * NC * 16 + (n >> 3) * 128 + (n & 7) * 16;
    *reinterpret_cast<uint4*>(out + off) = make_uint4(h2(c0[0], c0[1]), h2(c0[2], c0[3]), h2(c0[4], c0[5]), h2(c0[6], c0[7]));
    *reinterpret_cast<uint4*>(out + asz + off) =
        make_uint4(h2(c1[0], c1[1]), h2(c1[2], c1[3]), h2(c1[4], c1[5]), h2(c1[6], c1[7]));
    *reinterpret_cast<uint4*>(out + 2 * asz + off) =
        make_uint4(h2(c2[0], c2[1]), h2(c2[2], c2[3]), h2(c2[4], c2[5]), h2(c2[6], c2[7]));
    *reinterpret_cast<uint4*>(out + 3 * asz + off) =
        make_uint4(h2(cr[0], cr[1]), h2(cr[2], cr[3]), h2(cr[4], cr[5]), h2(cr[6], cr[7]));
  }
}

// ---------------------------------------------------------------------------
// k_f16_res
// ---------------------------------------------------------------------------
template <int NC>
struct ResCfg {
  static constexpr int DB = 3 * NC;               // tensor-memory columns of one accumulator set
  static constexpr int XBASE = 2 * DB;            // first basis-chunk column
  static constexpr int XST = 4 * (KCA / 2);       // columns of one basis chunk (4 pieces)
  static constexpr int NXS = (512 - XBASE) / XST; // basis-chunk stages
  static_assert(NXS >= 2, "tensor memory");
};

template <int NC>
__global__ void __launch_bounds__(448, 1)
    k_f16_res(DevModel m, const unsigned char* __restrict__ c16, const float* __restrict__ spf,
              const int* __restrict__ yexp, float* __restrict__ wres, float* __restrict__ wmx,
              double* __restrict__ c2part, int32_t* __restrict__ stat, const float* __restrict__ cwsig, int B,
              int nCB) {
  using CF = ResCfg<NC>;
  constexpr int NXS = CF::NXS;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t cfull, xfull[NXS], xfree[NXS], dfull[2], dempty[2], drain;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_bad;
  const int u = blockIdx.x, cb = blockIdx.y, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int I = m.unit_psr[u], start = m.unit_start[u], len = m.unit_len[u];
  const int mI = m.m[I], PM = m.PM, KX = kx_of(m, I), nch = KX / KCA, ntile = len / TTA;
  const int b0 = cb * NC, nvalid = min(NC, B - b0);
  const size_t asz = (size_t)PM * NC * 2;
  unsigned char* Cs = smem;                                            // 4 pieces x PM x NC fp16
  float* sp = reinterpret_cast<float*>(smem + 4 * asz);               // [PM] basis column factors
  double* redc = reinterpret_cast<double*>(sp + round_up_d(PM, 2));   // [4][NC] chi2 partials
  float* redm = reinterpret_cast<float*>(redc + 4 * NC);              // [4][NC] max |w|
  float* ysc = redm + 4 * NC;                                         // [NC] 2^(exponent of y) per chain

  if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
  if (tid == 0) {
    tc::mbar_init(&cfull, 1);
    for (int s = 0; s < NXS; ++s) {
      tc::mbar_init(&xfull[s], 8);
      tc::mbar_init(&xfree[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&dfull[b], 1);
      tc::mbar_init(&dempty[b], 4);
    }
    tc::mbar_init(&drain, 1);
    s_bad = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  const float* spg = spf + ((size_t)I * nCB + cb) * PM;
  for (int q = tid; q < KX; q += blockDim.x) sp[q] = spg[q];
  for (int n = tid; n < NC; n += blockDim.x) ysc[n] = pow2f(n < nvalid ? yexp[(size_t)I * B + b0 + n] : 0);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
    if (s_bad) return false;
    if (tc::mbar_wait(bar, parity, kWaitLimit)) return true;
    s_bad = 1;
    return false;
  };

  if (warp == 0) {
    // ------------------------------------------------ MMA issue (lane 0)
    if (lane == 0) {
      constexpr uint32_t ID = idesc_f16(TTA, NC, 0);
      bool ok = wait(&cfull, 0);
      if (ok) tc::fence_after();
      const uint32_t cbase = tc::smem_u32(Cs);
      int g = 0;
      for (int i = 0; i < ntile && ok; ++i) {
        const int buf = i & 1;
        if (i >= 2 && !(ok = wait(&dempty[buf], ((i >> 1) - 1) & 1))) break;
        tc::fence_after();
        const uint32_t d0 = tmem + buf * CF::DB, d1 = d0 + NC, d2 = d0 + 2 * NC;
        for (int c = 0; c < nch; ++c, ++g) {
          const int s = g % NXS;
          if (!(ok = wait(&xfull[s], (g / NXS) & 1))) break;
          tc::fence_after();
          const uint32_t xa = tmem + CF::XBASE + s * CF::XST;
#pragma unroll
          for (int ks = 0; ks < KCA / 16; ++ks) {
            const uint32_t kg = (uint32_t)(c * (KCA / 8) + 2 * ks);
            uint64_t bd[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) bd[a] = tc::desc(cbase + a * (uint32_t)asz + kg * NC * 16, NC * 16, 128);
            const uint32_t ax0 = xa + 8 * ks, ax1 = ax0 + KCA / 2, ax2 = ax0 + KCA, ax3 = ax0 + 3 * (KCA / 2);
            const uint32_t acc = (c | ks) ? 1u : 0u;
            mma_ts(d0, ax0, bd[0], ID, acc);  // L0 = X0 C0
            mma_ts(d1, ax1, bd[0], ID, acc);  // L1 = X1 C0 + X0 C1
            mma_ts(d1, ax0, bd[1], ID, 1u);
            mma_ts(d2, ax2, bd[0], ID, acc);  // L2 = X2 C0 + X0 C2 + Xr Cr
            mma_ts(d2, ax0, bd[2], ID, 1u);
            mma_ts(d2, ax3, bd[3], ID, 1u);
          }
          tc::commit(&xfree[s]);
        }
        if (!ok) break;
        tc::commit(&dfull[buf]);
      }
      tc::commit(&drain);  // every MMA issued here has completed before the CTA may exit
      if (!tc::mbar_wait(&drain, 0, kDrainLimit)) s_bad = 1;
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------ resident coefficient block
    if (lane == 0) {
      const unsigned char* src = c16 + ((size_t)I * nCB + cb) * 4 * asz;
      const uint32_t bytes = (uint32_t)KX * NC * 2;
      mbar_expect_tx(&cfull, 4 * bytes);
      for (int a = 0; a < 4; ++a) bulk_g2s(Cs + a * asz, src + a * asz, bytes, &cfull);
      if (!tc::mbar_wait(&cfull, 0, kDrainLimit)) s_bad = 1;  // landed before the CTA may exit
    }
    __syncwarp();
  } else if (warp < 10) {
    // ------------------------------------------------ basis generation into tensor memory
    // Harmonics come in runs of consecutive k along the columns: each run of four
    // pairs starts from an exactly reduced sin/cos and rotates by the fundamental.
    // Column factors: every achromatic column shares one (|sin|, |cos| <= 1), every DM
    // column another (the pulsar's largest weight), fixed columns their own.
    const int qw = warp & 3, hf = (warp - 2) >> 2, t = 32 * qw + lane;
    const uint32_t lanef = (uint32_t)(32 * qw) << 16;
    const int na2 = 2 * m.na, P = m.P, NL = m.NL;
    const float fa = sp[0], fd = m.nd ? sp[na2] : 0.f;
    int g = 0;
    bool ok = true;
    for (int i = 0; i < ntile && ok; ++i) {
      const int ta = start + i * TTA + t;
      const uint64_t U = m.phase[ta];
      const float wd = m.chrom[ta] * fd;  // DM weight times the DM column factor (a power of two)
      float s1, c1;
      sincos_turns64(U, &s1, &c1);
      const long long row = (long long)(start - m.toa_off[I] + i * TTA + t);
      const float* Mr = m.M32 + m.m_off[I] + row * mI;
      const float* Lr = m.Flo + m.flo_off[I] + row * NL;
      for (int c = 0; c < nch; ++c, ++g) {
        const int s = g % NXS;
        if (g >= NXS && !(ok = __all_sync(0xffffffffu, wait(&xfree[s], ((g / NXS) - 1) & 1)))) break;
        uint32_t w0[8], w1[8], w2[8], wr[8];
        const int q0 = c * KCA + hf * (KCA / 2);
        float sn = 0.f, cs = 1.f;
        int kprev = -8;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int q = q0 + 2 * j;  // warp-uniform: every branch below is uniform
          float xa, xb;
          if (q < P) {
            const bool dm = q >= na2;
            const int k = dm ? (q - na2) / 2 + 1 : q / 2 + 1;
            if ((j & 3) == 0 || k != kprev + 1)
              sincos_turns64(U * (uint64_t)k, &sn, &cs);
            else
              rotate(sn, cs, s1, c1);
            kprev = k;
            const float f = dm ? wd : fa;
            xa = sn * f;
            xb = cs * f;
          } else {
            const int j0 = q - P, j1 = j0 + 1;
            xa = (j0 < mI ? Mr[j0] : (j0 < mI + NL ? Lr[j0 - mI] : 0.f)) * sp[q];
            xb = (j1 < mI ? Mr[j1] : (j1 < mI + NL ? Lr[j1 - mI] : 0.f)) * sp[q + 1];
          }
          float a0, a1, ar, a2, b0_, b1, br, b2;
          split_grid(xa, a0, a1, ar, a2);
          split_grid(xb, b0_, b1, br, b2);
          w0[j] = h2(a0, b0_);
          w1[j] = h2(a1, b1);
          w2[j] = h2(a2, b2);
          wr[j] = h2(ar, br);
        }
        const uint32_t col = tmem + lanef + CF::XBASE + s * CF::XST + hf * 8;
        st8(col, w0);
        st8(col + KCA / 2, w1);
        st8(col + KCA, w2);
        st8(col + 3 * (KCA / 2), wr);
        wait_st();
        tc::fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&xfull[s]);
      }
    }
  } else {
    // ------------------------------------------------ epilogue (lane = TOA)
    const int qe = warp & 3, t = 32 * qe + lane;
    const uint32_t lanef = (uint32_t)(32 * qe) << 16;
    // per-warp partials in this warp's own slots of redc / redm (even lanes write)
    double* myc = redc + qe * NC;
    float* mym = redm + qe * NC;
    for (int n = lane; n < NC; n += 32) {
      myc[n] = 0.0;
      mym[n] = 0.f;
    }
    __syncwarp();
    for (int i = 0; i < ntile; ++i) {
      const int buf = i & 1;
      if (!__all_sync(0xffffffffu, wait(&dfull[buf], (i >> 1) & 1))) break;
      tc::fence_after();
      const int ta = start + i * TTA + t;
      // dt'' as an unevaluated float pair: the residual dt'' - y is formed with
      // error-free sums from the exact level sums L0 and L1, so it is accurate to its
      // own size, not to the size of dt'' or y
      const double d64 = m.dt64[ta];
      const float dh = (float)d64, dl = (float)(d64 - (double)dh), ni = m.ninv[ta];
      const uint32_t d0 = tmem + lanef + buf * CF::DB;
#pragma unroll 1
      for (int gq = 0; gq < NC / 16; ++gq) {
        uint32_t l0[16], l1[16], l2[16];
        ld16(d0 + 16 * gq, l0);
        ld16(d0 + NC + 16 * gq, l1);
        ld16(d0 + 2 * NC + 16 * gq, l2);
        float ch[16], am[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = 16 * gq + j;
          const int bb = b0 + n;
          const float sc = ysc[n];  // 2^(exponent of y): the products below are exact
          float ea, eb;
          const float a = two_sum(dh, -__uint_as_float(l0[j]) * sc, ea);
          const float b = two_sum(a, -__uint_as_float(l1[j]) * sc, eb);
          float r = __fadd_rn(b, __fadd_rn(__fadd_rn(ea, eb), __fsub_rn(dl, __uint_as_float(l2[j]) * sc)));
          if (cwsig && n < nvalid) r -= cwsig[(size_t)bb * m.ntoa_pad + ta];
          const float w = r * ni;
          if (n < nvalid) wres[(size_t)bb * m.ntoa_pad + ta] = w;
          ch[j] = n < nvalid ? r * w : 0.f;
          am[j] = n < nvalid ? fabsf(w) : 0.f;
        }
        // transpose-reduce over the 32 lanes: lanes 2c and 2c + 1 end with chain 16 gq + c
#pragma unroll
        for (int hw = 8; hw >= 1; hw >>= 1) {
          const int msk = 2 * hw;
          const bool up = lane & msk;
#pragma unroll
          for (int j = 0; j < hw; ++j) {
            const float sc = up ? ch[j] : ch[j + hw], kc = up ? ch[j + hw] : ch[j];
            const float sm = up ? am[j] : am[j + hw], km = up ? am[j + hw] : am[j];
            ch[j] = kc + __shfl_xor_sync(0xffffffffu, sc, msk);
            am[j] = fmaxf(km, __shfl_xor_sync(0xffffffffu, sm, msk));
          }
        }
        ch[0] += __shfl_xor_sync(0xffffffffu, ch[0], 1);
        am[0] = fmaxf(am[0], __shfl_xor_sync(0xffffffffu, am[0], 1));
        if ((lane & 1) == 0) {
          myc[16 * gq + (lane >> 1)] += (double)ch[0];
          mym[16 * gq + (lane >> 1)] = fmaxf(mym[16 * gq + (lane >> 1)], am[0]);
        }
      }
      tc::fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&dempty[buf]);
    }
    // fixed-order combination of the four epilogue warps
    named_bar(1, 128);
    for (int n = tid - 320; n < nvalid; n += 128) {
      c2part[(size_t)u * B + b0 + n] = ((redc[n] + redc[NC + n]) + redc[2 * NC + n]) + redc[3 * NC + n];
      wmx[(size_t)u * B + b0 + n] = fmaxf(fmaxf(redm[n], redm[NC + n]), fmaxf(redm[2 * NC + n], redm[3 * NC + n]));
    }
  }
  tc::fence_before();
  __syncthreads();
  if (s_bad && tid < nvalid) atomicOr(&stat[b0 + tid], 4);
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------------------
// k_f16_ftw
// ---------------------------------------------------------------------------
constexpr int FW_D0 = 0, FW_DR = QWB, FW_WB = 2 * QWB;  // tensor-memory columns
constexpr int FW_WST = 3 * (KWB / 2);                   // columns of one w~ stage (3 pieces)
static_assert(FW_WB + NSB * FW_WST <= 512, "tensor memory");
constexpr int FW_XARR = KWB * QWB * 2;                  // bytes of one basis piece per stage
constexpr int FW_XST = 3 * FW_XARR;
constexpr int FW_WROW = KWB + 4;                        // floats per staged w~ row (padded: no bank conflicts)
constexpr int FW_SMEM = NSB * FW_XST + NSB * 128 * FW_WROW * 4;

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void split_w(float v, float& v0, float& rh, float& rl) {
  v0 = __fsub_rn(__fadd_rn(v, 1610612736.f), 1610612736.f);
  const float r = __fsub_rn(v, v0);
  rh = f16r(r);
  rl = __fsub_rn(r, rh);
}

__global__ void __launch_bounds__(416, 1)
    k_f16_ftw(DevModel m, const float* __restrict__ wres, const float* __restrict__ wmx, float* __restrict__ gpart,
              int32_t* __restrict__ stat, int B) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t wfull[NSB], xfull[NSB], wfree[NSB], xfree[NSB], dfull, drain;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_bad;
  // column chunk fastest: the chunks of one (unit, chain block) run together and the
  // second one reads w~ from L2
  const int qc = blockIdx.x, cb = blockIdx.y, u = blockIdx.z, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int I = m.unit_psr[u], start = m.unit_start[u], len = m.unit_len[u], nst = len / KWB;
  const int b0 = cb * 128, nvalid = min(128, B - b0);
  const int q0 = qc * QWB, qw = min(QWB, m.P - q0), NQ = round_up_d(qw, 16);
  // column exponent: |F| <= 1 (achromatic), <= the largest DM weight (DM columns)
  const int cdm = exp_up(m.wmaxp[I]);

  if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
  if (tid == 0) {
    for (int s = 0; s < NSB; ++s) {
      tc::mbar_init(&wfull[s], 4);
      tc::mbar_init(&xfull[s], 8);
      tc::mbar_init(&wfree[s], 1);
      tc::mbar_init(&xfree[s], 1);
    }
    tc::mbar_init(&dfull, 1);
    tc::mbar_init(&drain, 1);
    s_bad = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
    if (s_bad) return false;
    if (tc::mbar_wait(bar, parity, kWaitLimit)) return true;
    s_bad = 1;
    return false;
  };

  if (warp == 0) {
    // ------------------------------------------------ MMA issue (lane 0)
    if (lane == 0) {
      const uint32_t ID = idesc_f16(128, NQ, 1);
      const uint32_t xbase = tc::smem_u32(smem);
      bool ok = true;
      for (int g = 0; g < nst && ok; ++g) {
        const int s = g % NSB;
        if (!(ok = wait(&wfull[s], (g / NSB) & 1))) break;
        if (!(ok = wait(&xfull[s], (g / NSB) & 1))) break;
        tc::fence_after();
        const uint32_t wa = tmem + FW_WB + s * FW_WST;
#pragma unroll
        for (int ks = 0; ks < KWB / 16; ++ks) {
          uint64_t bx[3];
#pragma unroll
          for (int j = 0; j < 3; ++j)
            bx[j] = tc::desc(xbase + s * FW_XST + j * FW_XARR + ks * 256, 128, (KWB / 8) * 128);
          const uint32_t a0 = wa + 8 * ks, ah = a0 + KWB / 2, al = a0 + KWB;
          const uint32_t acc = (g | ks) ? 1u : 0u;
          mma_ts(tmem + FW_D0, a0, bx[0], ID, acc);  // L0 = W0 X0
          mma_ts(tmem + FW_DR, a0, bx[1], ID, acc);  // rest
          mma_ts(tmem + FW_DR, ah, bx[0], ID, 1u);
          mma_ts(tmem + FW_DR, a0, bx[2], ID, 1u);
          mma_ts(tmem + FW_DR, al, bx[0], ID, 1u);
          mma_ts(tmem + FW_DR, ah, bx[1], ID, 1u);
        }
        tc::commit(&wfree[s]);
        tc::commit(&xfree[s]);
      }
      if (ok) tc::commit(&dfull);
      tc::commit(&drain);
      if (!tc::mbar_wait(&drain, 0, kDrainLimit)) s_bad = 1;
    }
    __syncwarp();
  } else if (warp < 5) {
    // ------------------------------------------------ w~ into tensor memory (lane = chain), epilogue
    const int qwp = warp & 3, n = 32 * qwp + lane;
    const uint32_t lanef = (uint32_t)(32 * qwp) << 16;
    const bool valid = n < nvalid;
    const int ew = valid ? exp_up(wmx[(size_t)u * B + b0 + n]) : 0;
    const float wsc = pow2f(13 - ew);
    const float* wrow = wres + (size_t)(valid ? b0 + n : 0) * m.ntoa_pad + start;
    // w~ rows stream in through cp.async, NSB stages ahead; each thread copies and reads
    // only its own chain's row, so its own wait_group orders them
    float* wsm = reinterpret_cast<float*>(smem + NSB * FW_XST);
    auto issue = [&](int g) {
      if (valid && g < nst) {
        float* dst = wsm + ((g % NSB) * 128 + n) * FW_WROW;
#pragma unroll
        for (int j = 0; j < KWB / 4; ++j) cp_async16(dst + 4 * j, wrow + g * KWB + 4 * j);
      }
      cp_async_commit();
    };
    for (int g = 0; g < NSB; ++g) issue(g);
    bool ok = true;
    for (int g = 0; g < nst; ++g) {
      const int s = g % NSB;
      if (g >= NSB && !(ok = __all_sync(0xffffffffu, wait(&wfree[s], ((g / NSB) - 1) & 1)))) break;
      asm volatile("cp.async.wait_group %0;" ::"n"(NSB - 1) : "memory");
      const float* src = wsm + (s * 128 + n) * FW_WROW;
      uint32_t p0[16], ph[16], pl[16];
#pragma unroll
      for (int j = 0; j < KWB / 4; ++j) {
        const float4 v = valid ? *reinterpret_cast<const float4*>(src + 4 * j) : make_float4(0, 0, 0, 0);
        const float vv[4] = {v.x, v.y, v.z, v.w};
        float a0[4], ah[4], al[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split_w(vv[e] * wsc, a0[e], ah[e], al[e]);
        p0[2 * j] = h2(a0[0], a0[1]);
        p0[2 * j + 1] = h2(a0[2], a0[3]);
        ph[2 * j] = h2(ah[0], ah[1]);
        ph[2 * j + 1] = h2(ah[2], ah[3]);
        pl[2 * j] = h2(al[0], al[1]);
        pl[2 * j + 1] = h2(al[2], al[3]);
      }
      issue(g + NSB);  // into the buffer just read
      const uint32_t col = tmem + lanef + FW_WB + s * FW_WST;
      st16(col, p0);
      st16(col + KWB / 2, ph);
      st16(col + KWB, pl);
      wait_st();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&wfull[s]);
    }
    // ghat rows of this unit and column chunk
    asm volatile("cp.async.wait_group 0;" ::: "memory");  // no copy in flight at exit
    const float sa = pow2f(ew - 26), sd = pow2f(ew + cdm - 26);  // undo the w~ and column scales
    if (ok && __all_sync(0xffffffffu, wait(&dfull, 0))) {
      tc::fence_after();
      for (int c0 = 0; c0 < NQ; c0 += 16) {
        uint32_t l0[16], lr[16];
        ld16(tmem + lanef + FW_D0 + c0, l0);
        ld16(tmem + lanef + FW_DR + c0, lr);
        if (valid) {
          float* dst = gpart + ((size_t)u * B + b0 + n) * m.Qs + q0;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int q = c0 + j;
            if (q < qw)
              dst[q] = __fadd_rn(__uint_as_float(l0[j]), __uint_as_float(lr[j])) * (q0 + q >= 2 * m.na ? sd : sa);
          }
        }
      }
    }
  } else {
    // ------------------------------------------------ basis chunk into shared memory (MN-major)
    const int gw = warp - 5;  // 8 warps; lane = TOA of the stage
    const int na2 = 2 * m.na, P = m.P;
    const float fa = 8192.f, fd = pow2f(13 - cdm);  // |sin|, |cos| <= 1; DM columns <= 2^cdm
    for (int g = 0; g < nst; ++g) {
      const int s = g % NSB;
      if (g >= NSB && !__all_sync(0xffffffffu, wait(&xfree[s], ((g / NSB) - 1) & 1))) break;
      const int ta = start + g * KWB + lane;
      const uint64_t U = m.phase[ta];
      const float wd = m.chrom[ta] * fd;
      float s1, c1;
      sincos_turns64(U, &s1, &c1);
      unsigned char* xs = smem + s * FW_XST;
      for (int grp = gw; grp < NQ / 8; grp += 8) {
        float v0[8], vh[8], vl[8];
        float sn = 0.f, cs = 1.f;
        int kprev = -8;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int q = q0 + 8 * grp + 2 * j;  // warp-uniform
          float xa = 0.f, xb = 0.f;
          if (q < P) {
            const bool dm = q >= na2;
            const int k = dm ? (q - na2) / 2 + 1 : q / 2 + 1;
            if (j == 0 || k != kprev + 1)
              sincos_turns64(U * (uint64_t)k, &sn, &cs);
            else
              rotate(sn, cs, s1, c1);
            kprev = k;
            const float f = dm ? wd : fa;
            xa = sn * f;
            xb = cs * f;
          }
          split_w(xa, v0[2 * j], vh[2 * j], vl[2 * j]);
          split_w(xb, v0[2 * j + 1], vh[2 * j + 1], vl[2 * j + 1]);
        }
        const int off = grp * ((KWB / 8) * 128) + (lane >> 3) * 128 + (lane & 7) * 16;
        *reinterpret_cast<uint4*>(xs + off) = make_uint4(h2(v0[0], v0[1]), h2(v0[2], v0[3]), h2(v0[4], v0[5]), h2(v0[6], v0[7]));
        *reinterpret_cast<uint4*>(xs + FW_XARR + off) =
            make_uint4(h2(vh[0], vh[1]), h2(vh[2], vh[3]), h2(vh[4], vh[5]), h2(vh[6], vh[7]));
        *reinterpret_cast<uint4*>(xs + 2 * FW_XARR + off) =
            make_uint4(h2(vl[0], vl[1]), h2(vl[2], vl[3]), h2(vl[4], vl[5]), h2(vl[6], vl[7]));
      }
      tc::fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&xfull[s]);
    }
  }
  tc::fence_before();
  __syncthreads();
  if (s_bad && tid < nvalid) atomicOr(&stat[b0 + tid], 4);
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

template <int NC>
size_t res_smem(const DevModel& m) {
  return 4 * (size_t)m.PM * NC * 2 + sizeof(float) * round_up(m.PM, 2) + 4 * NC * (sizeof(double) + sizeof(float)) +
         NC * sizeof(int);
}

// chains per CTA of k_f16_res: 64 when the coefficient block fits in shared memory
int res_nc(const DevModel& m) { return res_smem<64>(m) <= 200 * 1024 ? 64 : 32; }

template <int NC>
cudaError_t launch_f16_nc(const DevModel& m, const Scratch& s, int B, cudaStream_t st) {
  const int nCB = (B + NC - 1) / NC;
  k_f16_pack<NC><<<dim3(m.npsr, nCB), 256, sizeof(float) * m.PM, st>>>(m, s.a32, s.c16, s.spf, s.yexp, B, nCB);
  const size_t sm = res_smem<NC>(m);
  if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(k_f16_res<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  float* w = m.cw ? s.cwwt : s.wres;
  k_f16_res<NC><<<dim3(m.n_units, nCB), 448, sm, st>>>(m, s.c16, s.spf, s.yexp, w, s.wmx, s.c2part, s.stat,
                                                      m.cw ? s.cwsig : nullptr, B, nCB);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_f16_ftw, cudaFuncAttributeMaxDynamicSharedMemorySize, FW_SMEM);
  if (e != cudaSuccess) return e;
  k_f16_ftw<<<dim3((m.P + QWB - 1) / QWB, (B + 127) / 128, m.n_units), 416, FW_SMEM, st>>>(m, w, s.wmx, s.gpart,
                                                                                           s.stat, B);
  return cudaGetLastError();
}

}  // namespace

// The exact levels need K = P + m + n_low <= 480 columns per tile (2 K 2^14 < 2^24 quanta
// with margin) and the coefficient block of 32 chains in shared memory.
bool f16_supported(const DevModel& m) { return res_smem<32>(m) <= 227 * 1024 && m.PM <= 480; }

size_t f16_pack_bytes(const DevModel& m, int cap) {
  const int nc = res_nc(m), nCB = (cap + nc - 1) / nc;
  return (size_t)m.npsr * nCB * 4 * m.PM * nc * 2;
}
size_t f16_scale_floats(const DevModel& m, int cap) {
  const int nc = res_nc(m), nCB = (cap + nc - 1) / nc;
  return (size_t)m.npsr * nCB * m.PM;
}

cudaError_t launch_toa_f16(const DevModel& m, const Scratch& s, int B, cudaStream_t st) {
  if (!f16_supported(m) || !s.c16 || !s.spf || !s.yexp || !s.wmx || (!m.cw && !s.wres)) return cudaErrorInvalidValue;
  return res_nc(m) == 64 ? launch_f16_nc<64>(m, s, B, st) : launch_f16_nc<32>(m, s, B, st);
}

}  // namespace pta
