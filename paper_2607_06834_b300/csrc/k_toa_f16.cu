// TOA contractions on the tcgen05 tensor cores at FP32 accuracy or better, same
// quantities as k_toa_simt (the projected residual of Eq. raw_det_posterior with N~^-1
// of Eq. Gmatrix_proj, whitened by Eq. WN_cov), written with the fully projected basis
//   F~ = F - M (M^T N^-1 M)^-1 M^T N^-1 F   (N^-1-orthogonal to the timing model):
//   y  = F~ (a - a_ref) [+ M c_s],  r~ = dt'' - y,  w~ = N^-1 r~,  chi2 = sum r~ w~,
//   ghat = F~^T w~ = F^T w~   (M^T w~ = 0).
// With a deterministic signal s the projection of s enters through the timing-model
// columns, c_s = -(M^T N^-1 M)^-1 M^T N^-1 s, and the kernel subtracts s itself.
//
// Why an exact split.  The tensor cores accumulate in FP32 without round-to-nearest,
// and the terms of one residual cancel 20-400 fold, so an FP32-accuracy result needs
// most of the sum formed without rounding.  Both operands are scaled to a common
// power-of-two grid (|v| < 2^14) and cut into fp16 pieces, three on fixed grids and
// the rest:
//   v = v0 + v1 + v2 + v3,  v0, v1, v2 on the 2^7, 2^-1, 2^-9 grids (round to nearest),
//   v3 the fp16 of what is left (|v3| <= 2^-10),
// so |v0| <= 2^14, |v1| <= 2^6, |v2| <= 2^-2 are exact fp16 numbers of at most 8
// significant bits.  Products of grid pieces are integers times a fixed quantum, so
//   L0 = sum X0 C0            (quantum 2^14, at most K 2^14 quanta)
//   L1 = sum X1 C0 + X0 C1    (quantum 2^6,  at most 2 K 2^14 quanta)
// stay within 2^24 quanta for K <= 512 columns and are exact in the FP32 accumulator
// whatever its rounding; the rest,
//   L2 = X2 C0 + X1 C1 + X0 C2 + X3 C0 + X0 C3 + X2 C1 + X1 C2   (2^-16 of the scale),
// carries rounding relative to its own small size.  Ten MMAs per K step represent the
// product to about 2^-35 of its largest term.  y = (L0 + L1 + L2) 2^(scale).
//
// The basis is fixed, so it is built once per model in FP64 (k_f16_image): F~ from
// FP64 sines and cosines of the exactly reduced phases minus the FP64 timing-model
// projection, each column normalised by a power of two from its largest value over
// the pulsar's TOAs, cut into the four pieces and stored in the order the residual
// kernel reads it.  The coefficients are cut from the FP64 rows of the prior stage,
// each chain normalised to 2^14 by its own exponent (k_f16_pack), so a chain's accuracy
// does not depend on the other chains.
//
// k_f16_res: F~ a, the residual, chi2 and w~.  One CTA per (block of NC chains, work
// unit).  The MMA's M is 128 TOAs and its A operand (32 basis columns per chunk) sits
// in tensor memory, written there by loader warps from the stored pieces; its N is the
// NC chains and its B operand (the block's coefficient pieces, all columns) is resident
// in shared memory.  Accumulators and basis chunks are double-buffered in tensor
// memory.  Epilogue warps read the three accumulators per TOA lane, form the residual
// with error-free sums, write w~ (TOA-major per chain) and reduce chi2 in FP64.
//
// k_f16_ftw: ghat = F~^T w~ over the unit.  One CTA per (chunk of <= 144 basis columns,
// block of 128 chains, work unit).  M = 128 chains with A = w~ in tensor memory (scaled
// per chain and unit by its largest |w~|), N = the chunk's columns with B = the pieces
// X0, X1, X2 in shared memory (MN-major), K = TOAs, 32 per stage.  w~ = W0 + Wh + Wl
// (W0 on the 2^7 grid for |w~| < 2^12, Wh and Wl fp16); L0 = sum W0 X0 is exact (at most
// 2048 2^12 quanta), W0 X1 + Wh X0 + W0 X2 + Wh X1 + Wl X0 go to a second accumulator
// (about 2^-23 of the largest term: the gradient's tolerance is 1e-4).
//
// Every mbarrier wait is bounded; a wait that gives up marks the CTA's chains with
// status bit 4 and the CTA drains its own MMAs before it frees tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include "dwarith.cuh"
#include "pta_internal.cuh"
#include "tc_ptx.cuh"

namespace pta {
namespace {

constexpr int TTA = 128;                  // TOAs per tile in k_f16_res (MMA M) and per stored basis tile
constexpr int KCA = 32;                   // basis columns per chunk
constexpr int KCB = 16;                   // basis columns per stored block (one MMA K step)
constexpr int XBW = 4 * (KCB / 2) * TTA;  // 32-bit words of one stored (tile, column block): 4 pieces
constexpr int RES_XSB = XBW * 4;          // bytes of one stored block (16 KB)
constexpr int KWB = 32;                   // TOAs per stage in k_f16_ftw
constexpr int QWB = 144;                  // basis columns per chunk in k_f16_ftw (MMA N)
constexpr int NSB = 4;                    // tensor-memory (w~) stages in k_f16_ftw
constexpr int NSM = 5;                    // shared-memory (TMA landing) stages in k_f16_ftw
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
__device__ __forceinline__ void st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
// 32 lanes x 16 columns of 32-bit values, completion awaited by wait_ld
__device__ __forceinline__ void ld16_nw(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// ties registers written by ld16_nw to a point after wait_ld, so that no use of them is
// scheduled before the wait
template <int N>
__device__ __forceinline__ void after_wait(uint32_t (&r)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) asm volatile("" : "+r"(r[i]));
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

// exponent e with |v| < 2^e (frexp); 0 for v == 0
__device__ __forceinline__ int exp_up(float v) {
  int e = 0;
  frexpf(v, &e);
  return v == 0.f ? 0 : e;
}
__device__ __forceinline__ int exp_up64(double v) {
  int e = 0;
  frexp(v, &e);
  return v == 0.0 ? 0 : e;
}

// |v| < 2^14 (FP64): v0, v1, v2 on the 2^7, 2^-1, 2^-9 grids, each rounded to nearest
// from what the previous ones leave (exact in FP64), v3 the rest; as floats (v0, v1, v2
// exact, fp16-exact too; v3 is rounded to fp16 when packed)
__device__ __forceinline__ void split4(double v, float& v0, float& v1, float& v2, float& v3) {
  const double a0 = rint(v * 0x1p-7) * 0x1p7;
  double r = v - a0;
  const double a1 = rint(r * 2.0) * 0.5;
  r -= a1;
  const double a2 = rint(r * 0x1p9) * 0x1p-9;
  r -= a2;
  v0 = (float)a0;
  v1 = (float)a1;
  v2 = (float)a2;
  v3 = (float)r;
}

// |v| < 2^12: v0 on the 2^7 grid (round to nearest by the magic-number addition),
// rh = fp16(v - v0), rl = the rest (exact in FP32; rounded to fp16 when packed)
__device__ __forceinline__ void split_w(float v, float& v0, float& rh, float& rl) {
  v0 = __fsub_rn(__fadd_rn(v, 1610612736.f), 1610612736.f);  // 1.5 x 2^30: ulp 2^7
  const float r = __fsub_rn(v, v0);
  rh = f16r(r);
  rl = __fsub_rn(r, rh);
}

__host__ __device__ __forceinline__ int round_up_hd(int a, int b) { return (a + b - 1) / b * b; }
// stored basis columns of pulsar I: P Fourier columns, then its timing-model columns
// when a deterministic signal is modelled, padded to whole chunks
__host__ __device__ __forceinline__ int kx_cols(int P, int mI, int cw) { return round_up_hd(P + (cw ? mI : 0), KCA); }
__device__ __forceinline__ int kx_of(const DevModel& m, int I) { return kx_cols(m.P, m.m[I], m.cw); }

// ---------------------------------------------------------------------------
// Stored basis.  Pulsar I's pieces start at word x16_off[I]; its tile tau (TOAs
// 128 tau .. 128 tau + 127 of the pulsar) and column block kc (columns 16 kc ..
// 16 kc + 15) form one block of XBW words (16 KB) at x16_off[I] + (tau nkc + kc) XBW.
// Inside it, piece a, 8-column half h, TOA t and word w (columns 16 kc + 8 h + 2 w (low
// half) and + 1 (high half)) is word  ((2 a + h) 128 + t) 4 + w:  one 16-byte row per
// (piece, half, TOA).  Piece a of a block is then the K-major, unswizzled A operand of
// one M = 128, K = 16 MMA in shared memory as it stands (8 x 16-byte core matrices,
// 128 bytes between 8-TOA groups, 2048 bytes between the two 8-column halves), and the
// 16-byte rows of 32 consecutive TOAs (512 bytes) are the core-matrix rows of the
// MN-major B operand of k_f16_ftw.
// ---------------------------------------------------------------------------

// Column q of pulsar I's stored basis at padded TOA ta (FP64).  F~ = F - M K^-1 H^T for
// q < P (DM columns weighted by (nu_ref/nu)^2), the normalised timing-model column
// q - P beyond (signal models only); 0 on padding rows.  kih: this chunk's 32 columns
// of K^-1 H^T as kih[32 j + (q mod 32)].
__device__ double basis64(const DevModel& m, int I, int ta, int q, const double* kih, double s, double c) {
  if (m.ninv64[ta] == 0.0) return 0.0;
  const int mI = m.m[I], P = m.P;
  const long long row = ta - m.toa_off[I];
  const double* Mr = m.M64 + m.m_off[I] + row * mI;
  if (q >= P) return q - P < mI ? Mr[q - P] : 0.0;
  double v = (q & 1) ? c : s;
  if (q >= 2 * m.na) v *= m.chrom64[ta];
  const double* kq = kih + (q & (KCA - 1));
  for (int j = 0; j < mI; ++j) v = fma(-Mr[j], kq[KCA * j], v);
  return v;
}

// sin and cos of column pair (q, q + 1) at TOA ta: harmonic k of the exactly reduced
// phase, FP64 sincospi (zero beyond the Fourier columns)
__device__ __forceinline__ void pair_sincos(const DevModel& m, int ta, int q, double& s, double& c) {
  s = 0.0;
  c = 0.0;
  if (q >= m.P) return;
  const int k = q < 2 * m.na ? q / 2 + 1 : (q - 2 * m.na) / 2 + 1;
  const uint64_t ph = m.phase[ta] * (uint64_t)k;  // mod 2^64: the fraction of a turn
  sincospi(2.0 * ((double)(ph >> 11) * 0x1p-53), &s, &c);
}

__device__ void load_kih(const DevModel& m, int I, int c, double* kih) {
  const int mI = m.m[I], P = m.P;
  for (int e = threadIdx.x; e < KCA * mI; e += blockDim.x) {
    const int j = e / KCA, q = KCA * c + e % KCA;
    kih[e] = q < P ? m.KiH[m.h_off[I] + (size_t)j * P + q] : 0.0;
  }
}

// Pass 1: largest |column| over each pulsar's TOAs (as the bits of a non-negative
// double, which order like the values).  Grid (unit, chunk), 128 threads (one TOA each).
__global__ void __launch_bounds__(128) k_f16_colmax(DevModel m, unsigned long long* cmax, int kxm) {
  __shared__ double kih[KCA * 128];
  const int u = blockIdx.x, c = blockIdx.y, t = threadIdx.x, lane = t & 31;
  const int I = m.unit_psr[u], start = m.unit_start[u], len = m.unit_len[u];
  if (c >= kx_of(m, I) / KCA) return;
  load_kih(m, I, c, kih);
  __syncthreads();
#pragma unroll 1
  for (int j = 0; j < KCA; j += 2) {
    const int q = KCA * c + j;
    double m0 = 0.0, m1 = 0.0;
    for (int i = t; i < len; i += 128) {
      const int ta = start + i;
      double s, cs;
      pair_sincos(m, ta, q, s, cs);
      m0 = fmax(m0, fabs(basis64(m, I, ta, q, kih, s, cs)));
      m1 = fmax(m1, fabs(basis64(m, I, ta, q + 1, kih, s, cs)));
    }
    for (int o = 16; o; o >>= 1) {
      m0 = fmax(m0, __shfl_xor_sync(0xffffffffu, m0, o));
      m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    }
    if (lane == 0) {
      atomicMax(&cmax[(size_t)I * kxm + q], (unsigned long long)__double_as_longlong(m0));
      atomicMax(&cmax[(size_t)I * kxm + q + 1], (unsigned long long)__double_as_longlong(m1));
    }
  }
}

// Pass 2: the column exponents and the four pieces of every stored word.
__global__ void __launch_bounds__(128)
    k_f16_image(DevModel m, const unsigned long long* __restrict__ cmax, int kxm, uint32_t* __restrict__ img,
                int* __restrict__ cexp) {
  __shared__ double kih[KCA * 128];
  __shared__ double fac[KCA];
  const int u = blockIdx.x, c = blockIdx.y, t = threadIdx.x;
  const int I = m.unit_psr[u], start = m.unit_start[u], len = m.unit_len[u];
  const int nch = kx_of(m, I) / KCA;
  if (c >= nch) return;
  load_kih(m, I, c, kih);
  if (t < KCA) {
    const int e = exp_up64(__longlong_as_double((long long)cmax[(size_t)I * kxm + KCA * c + t]));
    fac[t] = ldexp(1.0, 14 - e);  // |column| < 2^e: scaled columns stay below 2^14
    if (u == m.unit0[I]) cexp[(size_t)I * kxm + KCA * c + t] = e;
  }
  __syncthreads();
  const int tau0 = (start - m.toa_off[I]) / TTA, nkc = nch * (KCA / KCB);
  for (int i = 0; i < len / TTA; ++i) {
    const int ta = start + i * TTA + t;
    uint4* dst = reinterpret_cast<uint4*>(img + m.x16_off[I] + (size_t)(tau0 + i) * nkc * XBW) + t;
#pragma unroll 1
    for (int g = 0; g < KCA / 8; ++g) {  // 8 columns: one 16-byte row per piece
      uint32_t w[4][4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int q = KCA * c + 8 * g + 2 * jj;
        double s, cs;
        pair_sincos(m, ta, q, s, cs);
        float a0, a1, a2, a3, b0, b1, b2, b3;
        split4(basis64(m, I, ta, q, kih, s, cs) * fac[8 * g + 2 * jj], a0, a1, a2, a3);
        split4(basis64(m, I, ta, q + 1, kih, s, cs) * fac[8 * g + 2 * jj + 1], b0, b1, b2, b3);
        w[0][jj] = h2(a0, b0);
        w[1][jj] = h2(a1, b1);
        w[2][jj] = h2(a2, b2);
        w[3][jj] = h2(a3, b3);
      }
      const int kc = (KCA * c + 8 * g) / KCB, h = g & 1;
#pragma unroll
      for (int a = 0; a < 4; ++a)
        dst[(size_t)kc * (XBW / 4) + (2 * a + h) * TTA] = make_uint4(w[a][0], w[a][1], w[a][2], w[a][3]);
    }
  }
}

constexpr int PACK_THREADS = 512;  // 16 warps per (pulsar, chain block): the loads' latency needs the warps

// ---------------------------------------------------------------------------
// Pack: per (pulsar, block of NC chains) the chain exponents and the four fp16 pieces
// of the scaled coefficients as one K-major B operand of 4 NC rows, the pieces stacked
// along N (row a NC + n is piece a of chain n): element (row r, column k) at
// (k/8) 4 NC 16 + (r/8) 128 + (r%8) 16 + (k%8) 2 bytes.  Rows [0, j NC) are then the
// pieces c0 .. c(j-1), so one MMA with A = X_i and N = (4 - i) NC forms X_i c0 ..
// X_i c(3-i) at once.  Coefficient q is a_q - a_ref,q for q < P and, with a signal,
// the FP64 c_s that k_tm_prologue wrote after them.  Stored basis column q carries
// 2^(14 - c_q), so coefficient q carries 2^c_q, and each chain row is normalised to
// 2^14 by its own exponent E_n (y = L 2^(E_n - 28)).  The FP64 value is carried as an
// unevaluated float pair, split off its encoding with integer operations, and cut with
// FP32 operations (B300's FP64 rate is 1/64 of FP32).
// ---------------------------------------------------------------------------

// hi + lo (|hi| <= 2^14, |lo| <= ulp(hi) / 2) = v0 + v1 + v2 + v3: v0, v1 on the 2^7 and
// 2^-1 grids (from hi alone, so |v0| <= 2^14 and |v1| <= 2^6 as in the exact split), v2 on
// the 2^-9 grid, v3 the rest; every step is exact except the one rounding that adds lo
// (2^-26 of 2^-2, far below v3's fp16 rounding)
__device__ __forceinline__ void split4_ff(float hi, float lo, float& v0, float& v1, float& v2, float& v3) {
  v0 = __fsub_rn(__fadd_rn(hi, 1610612736.f), 1610612736.f);  // 1.5 x 2^30: ulp 2^7
  float r = __fsub_rn(hi, v0);
  v1 = __fsub_rn(__fadd_rn(r, 6291456.f), 6291456.f);         // 1.5 x 2^22: ulp 2^-1
  r = __fadd_rn(__fsub_rn(r, v1), lo);
  v2 = __fsub_rn(__fadd_rn(r, 24576.f), 24576.f);             // 1.5 x 2^14: ulp 2^-9
  v3 = __fsub_rn(r, v2);
}

template <int NC>
__global__ void __launch_bounds__(PACK_THREADS)
    k_f16_pack(DevModel m, const double* __restrict__ a64, unsigned char* __restrict__ c16, int* __restrict__ yexp,
               int B, int nCB) {
  extern __shared__ int ce[];  // [KX] column exponents c_q
  __shared__ int s_e[NC];
  const int I = blockIdx.x, cb = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b0 = cb * NC, nvalid = min(NC, B - b0), KX = kx_of(m, I), PM = m.PM, P = m.P, KXM = m.x16_kxm;
  const int ncol = P + (m.cw ? m.m[I] : 0);  // columns with coefficients; the rest of the block is 0
  const double* rows = a64 + ((size_t)I * B + b0) * PM;
  const double* ar = m.aref + (size_t)I * P;
  for (int q = tid; q < KX; q += PACK_THREADS) ce[q] = m.x16_cexp[(size_t)I * KXM + q];
  __syncthreads();
  auto coef = [&](int n, int q) -> double { return q < P ? rows[(size_t)n * PM + q] - ar[q] : rows[(size_t)n * PM + q]; };
  // per-chain exponent of max_q |C_nq 2^c_q| (one warp per chain).  |C| is truncated to a
  // float, and frexpf's exponent of a truncated value still bounds the exact one
  // strictly, which keeps |v| < 2^14.
  for (int n = warp; n < NC; n += PACK_THREADS / 32) {
    float mx = 0.f;
    if (n < nvalid)
      for (int q = lane; q < ncol; q += 32) mx = fmaxf(mx, fabsf(d2f_trunc(coef(n, q))) * pow2f(ce[q]));
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
      s_e[n] = exp_up(mx);
      if (n < nvalid) yexp[(size_t)I * B + b0 + n] = exp_up(mx) - 28;
    }
  }
  __syncthreads();
  unsigned char* out = c16 + ((size_t)I * nCB + cb) * 4 * (size_t)KXM * NC * 2;
  constexpr int PS = NC * 16;  // bytes between the pieces' row blocks within one K group
  for (int e = tid; e < NC * (KX / 8); e += PACK_THREADS) {
    const int n = e % NC, g = e / NC;  // consecutive threads: consecutive chains
    float c0[8], c1[8], c2[8], c3[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int q = 8 * g + i;
      float hi = 0.f, lo = 0.f;
      if (n < nvalid && q < ncol) {
        const float2 d = d2dw_bits(coef(n, q));      // integer split, off the FP64 pipe
        const float sc = pow2f(ce[q] + 14 - s_e[n]);  // exact: a power of two
        hi = d.x * sc;
        lo = d.y * sc;
      }
      split4_ff(hi, lo, c0[i], c1[i], c2[i], c3[i]);
    }
    const size_t off = (size_t)g * 4 * NC * 16 + (n >> 3) * 128 + (n & 7) * 16;
    *reinterpret_cast<uint4*>(out + off) = make_uint4(h2(c0[0], c0[1]), h2(c0[2], c0[3]), h2(c0[4], c0[5]), h2(c0[6], c0[7]));
    *reinterpret_cast<uint4*>(out + PS + off) =
        make_uint4(h2(c1[0], c1[1]), h2(c1[2], c1[3]), h2(c1[4], c1[5]), h2(c1[6], c1[7]));
    *reinterpret_cast<uint4*>(out + 2 * PS + off) =
        make_uint4(h2(c2[0], c2[1]), h2(c2[2], c2[3]), h2(c2[4], c2[5]), h2(c2[6], c2[7]));
    *reinterpret_cast<uint4*>(out + 3 * PS + off) =
        make_uint4(h2(c3[0], c3[1]), h2(c3[2], c3[3]), h2(c3[4], c3[5]), h2(c3[6], c3[7]));
  }
}

// ---------------------------------------------------------------------------
// k_f16_res
// ---------------------------------------------------------------------------
constexpr int RES_NXS = 3;             // shared-memory stages: up to three stored basis blocks and their coefficient slices
constexpr int RES_KB = 3;              // stored blocks per stage, at most
constexpr int RES_THREADS = 320;       // warp 0 MMA, warp 1 copies, warps 2-9 epilogue
constexpr int RES_EPI0 = 64;           // first epilogue thread

// Accumulator blocks (NC columns each) of one tile: after every K step
//   block 0 = X0 c0 (L0, exact), block 1 = X0 c1 + X1 c0 (L1, exact),
//   block 2 = X0 c2 + X1 c1 + X2 c0, block 3 = X0 c3 + X1 c2 + X2 c1 + X3 c0 (L2 = 2 + 3),
// from four MMAs: A = X_i, B = the first 4 - i pieces, D = blocks i .. 3.
template <int NC>
struct ResCfg {
  static constexpr int DB = 4 * NC;  // tensor-memory columns of one accumulator set (double-buffered)
  static_assert(2 * DB <= 512, "tensor memory");
};

template <int NC>
__global__ void __launch_bounds__(RES_THREADS, 1)
    k_f16_res(DevModel m, const unsigned char* __restrict__ c16, const int* __restrict__ yexp,
              float* __restrict__ wres, float* __restrict__ wmx, double* __restrict__ c2part,
              int32_t* __restrict__ stat, const float* __restrict__ cwsig, int B, int nCB) {
  using CF = ResCfg<NC>;
  constexpr int NXS = RES_NXS;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t xfull[NXS], xfree[NXS], dfull[2], dempty[2], drain;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_bad;
  // chain block fastest: the blocks of one unit run together and share its basis in L2
  const int cb = blockIdx.x, u = blockIdx.y, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int I = m.unit_psr[u], start = m.unit_start[u], len = m.unit_len[u];
  const int KXM = m.x16_kxm, KX = kx_of(m, I), nkc = KX / KCB, ntile = len / TTA, G = ntile * nkc;
  const bool unit_ok = PTA_IN(m.chk, start - m.toa_off[I], m.n_pad[I] - len + 1, kChkUnit) &&
                       PTA_ALIGNED(m.chk, start - m.toa_off[I], TTA, kChkUnit);
  const int b0 = cb * NC, nvalid = min(NC, B - b0);
  const size_t csz = 4 * (size_t)KXM * NC * 2;
  constexpr int CSL = 2 * 4 * NC * 16;                              // coefficient slice of one 16-column step
  constexpr int STB = RES_XSB + CSL;                                // one step: basis block + slice
  constexpr int STG = RES_KB * STB;                                 // one stage: up to RES_KB steps
  const int kb = nkc % 3 == 0 ? 3 : 2;                              // steps per stage (nkc is even)
  const int G2 = G / kb;                                            // stages; a tile is nkc / kb of them
  unsigned char* Xs = smem;                                         // NXS stages
  double* redc = reinterpret_cast<double*>(smem + NXS * STG);       // [8][NC/2] chi2 partials
  float* redm = reinterpret_cast<float*>(redc + 4 * NC);            // [8][NC/2] max |w|
  float* ysc = redm + 4 * NC;                                       // [NC] 2^(exponent of y) per chain

  if (warp == 0) tc::tmem_alloc(&tmem_base, 2 * CF::DB <= 256 ? 256 : 512);
  if (tid == 0) {
    for (int s = 0; s < NXS; ++s) {
      tc::mbar_init(&xfull[s], 1);
      tc::mbar_init(&xfree[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&dfull[b], 1);
      tc::mbar_init(&dempty[b], 8);
    }
    tc::mbar_init(&drain, 1);
    s_bad = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
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
      bool ok = true;
      const uint32_t xbase = tc::smem_u32(Xs);
      int g = 0;
      for (int i = 0; i < ntile && ok; ++i) {
        const int buf = i & 1;
        if (i >= 2 && !(ok = wait(&dempty[buf], ((i >> 1) - 1) & 1))) break;
        tc::fence_after();
        const uint32_t dbase = tmem + buf * CF::DB;
        for (int kc = 0; kc < nkc; kc += kb, ++g) {
          const int s = g % NXS;
          if (!(ok = wait(&xfull[s], (g / NXS) & 1))) break;
          tc::fence_after();
#pragma unroll 1
          for (int h = 0; h < kb; ++h) {
            const uint32_t sb = xbase + s * STG + h * STB;
            const uint64_t cd = tc::desc(sb + RES_XSB, 4 * NC * 16, 128);
#pragma unroll
            for (int a = 0; a < 4; ++a)
              tc::mma_f16(dbase + a * NC, tc::desc(sb + a * (RES_XSB / 4), 2048, 128), cd,
                          idesc_f16(TTA, (4 - a) * NC, 0), (kc | h | a) ? 1u : 0u);
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
    // ------------------------------------------------ bulk copies: basis block + coefficient slice per step
    // (the coefficient block, 147 KB at 64 chains and 288 columns, would halve the ring's
    // depth if it stayed resident; its slices come from L2, where the whole batch's
    // pieces stay)
    if (lane == 0) {
      const unsigned char* csrc = c16 + ((size_t)I * nCB + cb) * csz;
      // the unit's blocks are consecutive: (tile i, column block kc) is block i nkc + kc
      const unsigned char* xsrc = reinterpret_cast<const unsigned char*>(
          m.x16 + m.x16_off[I] + (size_t)((start - m.toa_off[I]) / TTA) * nkc * XBW);
      int g = 0;
      for (; g < G2; ++g) {
        const int s = g % NXS;
        if (g >= NXS && !wait(&xfree[s], ((g / NXS) - 1) & 1)) break;
        mbar_expect_tx(&xfull[s], kb * STB);
        for (int h = 0; h < kb; ++h) {
          const int gb = kb * g + h;  // stored block: (tile gb / nkc, column block gb % nkc)
          if (unit_ok &&
              PTA_IN(m.chk, (start - m.toa_off[I]) / TTA * nkc + gb, m.n_pad[I] / TTA * nkc, kChkResBasis) &&
              PTA_IN(m.chk, (size_t)(gb % nkc) * CSL + CSL - 1, csz, kChkResCoef) &&
              PTA_ALIGNED(m.chk, reinterpret_cast<uintptr_t>(xsrc + (size_t)gb * RES_XSB), 16, kChkBulkAlign) &&
              PTA_ALIGNED(m.chk, reinterpret_cast<uintptr_t>(csrc + (size_t)(gb % nkc) * CSL), 16, kChkBulkAlign) &&
              PTA_ALIGNED(m.chk, tc::smem_u32(Xs + s * STG + h * STB), 16, kChkBulkAlign)) {
            bulk_g2s(Xs + s * STG + h * STB, xsrc + (size_t)gb * RES_XSB, RES_XSB, &xfull[s]);
            bulk_g2s(Xs + s * STG + h * STB + RES_XSB, csrc + (size_t)(gb % nkc) * CSL, CSL, &xfull[s]);
          }
        }
      }
      // no copy in flight into this CTA's shared memory at exit (bounded waits)
      for (int h = max(0, g - NXS); h < g; ++h)
        if (!tc::mbar_wait(&xfull[h % NXS], (h / NXS) & 1, kDrainLimit)) s_bad = 1;
    }
    __syncwarp();
  } else {
    // ------------------------------------------------ epilogue (lane = TOA)
    // Eight warps: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (its 32 TOAs) and
    // chains NH h .. NH h + NH - 1 of the block (h = (w - 2) / 4), 16 at a time.
    constexpr int NH = NC / 2;
    const int qe = warp & 3, hq = (warp - 2) >> 2, t = 32 * qe + lane, n0 = NH * hq;
    const uint32_t lanef = (uint32_t)(32 * qe) << 16;
    // per-warp partials in this warp's own slots of redc / redm (even lanes write)
    double* myc = redc + (warp - 2) * NH;
    float* mym = redm + (warp - 2) * NH;
    for (int n = lane; n < NH; n += 32) {
      myc[n] = 0.0;
      mym[n] = 0.f;
    }
    __syncwarp();
    double d64n = m.dt64[start + t];
    float nin = m.ninv[start + t];
    for (int i = 0; i < ntile; ++i) {
      const int buf = i & 1;
      if (!__all_sync(0xffffffffu, wait(&dfull[buf], (i >> 1) & 1))) break;
      tc::fence_after();
      const int ta = start + i * TTA + t;
      // dt'' as an unevaluated float pair: the residual dt'' - y is formed with
      // error-free sums from the exact level sums L0 and L1, so it is accurate to its
      // own size, not to the size of dt'' or y
      const double d64 = d64n;
      const float dh = (float)d64, dl = (float)(d64 - (double)dh), ni = nin;
      if (i + 1 < ntile) {  // the next tile's TOA data, in flight during this one
        d64n = m.dt64[ta + TTA];
        nin = m.ninv[ta + TTA];
      }
      const uint32_t d0 = tmem + lanef + buf * CF::DB + n0;
#pragma unroll 1
      for (int gq = 0; gq < NH / 16; ++gq) {
        uint32_t l0[16], l1[16], l2[16], l3[16];
        ld16_nw(d0 + 16 * gq, l0);
        ld16_nw(d0 + NC + 16 * gq, l1);
        ld16_nw(d0 + 2 * NC + 16 * gq, l2);
        ld16_nw(d0 + 3 * NC + 16 * gq, l3);
        wait_ld();
        after_wait(l0);
        after_wait(l1);
        after_wait(l2);
        after_wait(l3);
        float ch[16], am[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int nl = 16 * gq + j, n = n0 + nl;
          const int bb = b0 + n;
          const float sc = ysc[n];  // 2^(exponent of y): the products below are exact
          float ea, eb;
          const float a = two_sum(dh, -__uint_as_float(l0[j]) * sc, ea);
          const float b = two_sum(a, -__uint_as_float(l1[j]) * sc, eb);
          const float l2s = __fadd_rn(__uint_as_float(l2[j]), __uint_as_float(l3[j]));
          float r = __fadd_rn(b, __fadd_rn(__fadd_rn(ea, eb), __fsub_rn(dl, l2s * sc)));
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
    // fixed-order combination of the four warps of each chain half
    named_bar(1, RES_THREADS - RES_EPI0);
    for (int n = tid - RES_EPI0; n < nvalid; n += RES_THREADS - RES_EPI0) {
      const int h = n / NH, j = n % NH;
      const double* c = redc + 4 * h * NH + j;
      const float* mm = redm + 4 * h * NH + j;
      c2part[(size_t)u * B + b0 + n] = ((c[0] + c[NH]) + c[2 * NH]) + c[3 * NH];
      wmx[(size_t)u * B + b0 + n] = fmaxf(fmaxf(mm[0], mm[NH]), fmaxf(mm[2 * NH], mm[3 * NH]));
    }
  }
  tc::fence_before();
  __syncthreads();
  if (s_bad && tid < nvalid) atomicOr(&stat[b0 + tid], 4);
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, 2 * CF::DB <= 256 ? 256 : 512);
  }
}


// ---------------------------------------------------------------------------
// k_f16_ftw
// ---------------------------------------------------------------------------
constexpr int FW_D0 = 0, FW_DR = QWB, FW_WB = 2 * QWB;  // tensor-memory columns
constexpr int FW_WST = 3 * (KWB / 2);                   // columns of one w~ stage (3 pieces)
static_assert(FW_WB + NSB * FW_WST <= 512, "tensor memory");
constexpr int FW_XARR = KWB * QWB * 2;                  // bytes of one basis piece per stage
constexpr int FW_XST = 3 * FW_XARR;                     // one stage: pieces X0, X1, X2
constexpr int FW_WSB = 128 * KWB * 4;                   // w~ stage: two halves of 128 chains x 32 TOAs (128-byte swizzled rows)
constexpr int FW_WHB = 128 * 32 * 4;                    // one half
constexpr int FW_SMEM = NSM * FW_XST + NSM * FW_WSB;
constexpr int FW_THREADS = 320;                         // warp 0 MMA, warps 1-8 w~ and epilogue, warp 9 copies
static_assert(KWB == 32, "the w~ producers take 16 TOAs of a stage each");
static_assert((NSM * FW_XST) % 1024 == 0, "swizzled w~ stages start on 1024-byte boundaries");
static_assert(FW_SMEM + 2048 <= 227 * 1024, "shared memory");

// TMA tile loads (tensor maps built on the host; coordinates innermost first)
__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(tc::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(tc::smem_u32(mbar))
      : "memory");
}
__device__ __forceinline__ void tma_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                       uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(tc::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(tc::smem_u32(mbar))
      : "memory");
}

// Tensor maps: tw over w~ [chains][ntoa_pad] (FP32, box 32 TOAs x 128 chains per 32-TOA half, 128-byte
// swizzle: 16-byte chunk j of chain row n sits at chunk j ^ (n % 8)); tx over the stored
// basis as (TOA x 8 halves 1024, half h 2, block, piece a 4) with byte strides 2048,
// 16384, 4096 (box 256 x 2 x 9 x 3: one stage's X0, X1, X2 rows of 144 columns as 512-byte
// runs of 32 TOAs, in the MN-major order [a][column group][TOA][8 columns]).
__global__ void __launch_bounds__(FW_THREADS, 1)
    k_f16_ftw(DevModel m, const __grid_constant__ CUtensorMap tw, const __grid_constant__ CUtensorMap tx,
              const float* __restrict__ wmx, float* __restrict__ gpart, int32_t* __restrict__ stat, int B) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // shared-memory stages (NSM: TMA landings of w~ and basis rows) and tensor-memory stages
  // (NSB: w~ pieces) run as separate rings
  __shared__ __align__(8) uint64_t wland[NSM], wread[NSM], xfull[NSM], xfree[NSM], wfull[NSB], wfree[NSB], dfull,
      drain;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_bad;
  // column chunk fastest: the chunks of one (unit, chain block) run together and the
  // second one reads w~ from L2
  const int qc = blockIdx.x, cb = blockIdx.y, u = blockIdx.z, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int I = m.unit_psr[u], start = m.unit_start[u], len = m.unit_len[u], nst = len / KWB;
  const int b0 = cb * 128, nvalid = min(128, B - b0);
  const int q0 = qc * QWB, qw = min(QWB, m.P - q0), NQ = round_up_hd(qw, 16);
  unsigned char* wsm = smem + NSM * FW_XST;

  if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
  if (tid == 0) {
    for (int s = 0; s < NSM; ++s) {
      tc::mbar_init(&wland[s], 1);
      tc::mbar_init(&wread[s], 8);
      tc::mbar_init(&xfull[s], 1);
      tc::mbar_init(&xfree[s], 1);
    }
    for (int s = 0; s < NSB; ++s) {
      tc::mbar_init(&wfull[s], 8);
      tc::mbar_init(&wfree[s], 1);
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
        const int s = g % NSB, sx = g % NSM;
        if (!(ok = wait(&wfull[s], (g / NSB) & 1))) break;
        if (!(ok = wait(&xfull[sx], (g / NSM) & 1))) break;
        tc::fence_after();
        const uint32_t wa = tmem + FW_WB + s * FW_WST;
#pragma unroll
        for (int ks = 0; ks < KWB / 16; ++ks) {
          uint64_t bx[3];
#pragma unroll
          for (int j = 0; j < 3; ++j)
            bx[j] = tc::desc(xbase + sx * FW_XST + j * FW_XARR + ks * 256, 128, (KWB / 8) * 128);
          const uint32_t a0 = wa + 8 * ks, ah = a0 + KWB / 2, al = a0 + KWB;
          const uint32_t acc = (g | ks) ? 1u : 0u;
          mma_ts(tmem + FW_D0, a0, bx[0], ID, acc);  // L0 = W0 X0
          mma_ts(tmem + FW_DR, a0, bx[1], ID, acc);  // rest: W0 X1 + Wh X0 + W0 X2 + Wh X1 + Wl X0
          mma_ts(tmem + FW_DR, ah, bx[0], ID, 1u);
          mma_ts(tmem + FW_DR, a0, bx[2], ID, 1u);
          mma_ts(tmem + FW_DR, ah, bx[1], ID, 1u);
          mma_ts(tmem + FW_DR, al, bx[0], ID, 1u);
        }
        tc::commit(&wfree[s]);
        tc::commit(&xfree[sx]);
      }
      if (ok) tc::commit(&dfull);
      tc::commit(&drain);
      if (!tc::mbar_wait(&drain, 0, kDrainLimit)) s_bad = 1;
    }
    __syncwarp();
  } else if (warp < 9) {
    // ------------------------------------------------ w~ into tensor memory (lane = chain), epilogue.
    // Two warps per 32-lane group of tensor memory (warp % 4 picks the group): warp hf = 0
    // cuts TOAs 0-15 of a stage, hf = 1 TOAs 16-31, into columns 8 hf .. 8 hf + 7 of each piece.
    const int qwp = warp & 3, hf = (warp - 1) >> 2, n = 32 * qwp + lane;
    const uint32_t lanef = (uint32_t)(32 * qwp) << 16;
    const bool valid = n < nvalid;
    const int ew = valid ? exp_up(wmx[(size_t)u * B + b0 + n]) : 0;
    const float wsc = pow2f(12 - ew);  // |w~| < 2^ew: scaled below 2^12
    bool ok = true;
    for (int g = 0; g < nst; ++g) {
      const int s = g % NSB, sx = g % NSM;
      if (!(ok = __all_sync(0xffffffffu, wait(&wland[sx], (g / NSM) & 1)))) break;
      // row n of the swizzled stage: 16-byte chunk j at chunk j ^ (n % 8)
      const unsigned char* row = wsm + sx * FW_WSB + n * 128;
      uint32_t p0[8], ph[8], pl[8];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int j = 4 * hf + jj;
        const float4 v = *reinterpret_cast<const float4*>(row + 16 * (j ^ (n & 7)));
        const float vv[4] = {v.x, v.y, v.z, v.w};
        float a0[4], ah[4], al[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split_w(vv[e] * wsc, a0[e], ah[e], al[e]);
        p0[2 * jj] = h2(a0[0], a0[1]);
        p0[2 * jj + 1] = h2(a0[2], a0[3]);
        ph[2 * jj] = h2(ah[0], ah[1]);
        ph[2 * jj + 1] = h2(ah[2], ah[3]);
        pl[2 * jj] = h2(al[0], al[1]);
        pl[2 * jj + 1] = h2(al[2], al[3]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&wread[sx]);  // the staged rows may be refilled
      if (g >= NSB && !(ok = __all_sync(0xffffffffu, wait(&wfree[s], ((g / NSB) - 1) & 1)))) break;
      const uint32_t col = tmem + lanef + FW_WB + s * FW_WST + 8 * hf;
      st8(col, p0);
      st8(col + KWB / 2, ph);
      st8(col + KWB, pl);
      wait_st();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&wfull[s]);
    }
    // ghat rows of this unit and column chunk: undo 2^(12 - ew) and 2^(14 - c_q); the two
    // warps of a lane group take alternate 16-column blocks
    const int* ce = m.x16_cexp + (size_t)I * m.x16_kxm + q0;
    if (ok && __all_sync(0xffffffffu, wait(&dfull, 0))) {
      tc::fence_after();
      for (int c0 = 16 * hf; c0 < NQ; c0 += 32) {
        uint32_t l0[16], lr[16];
        ld16(tmem + lanef + FW_D0 + c0, l0);
        ld16(tmem + lanef + FW_DR + c0, lr);
        if (valid) {
          float* dst = gpart + ((size_t)u * B + b0 + n) * m.Qs + q0;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int q = c0 + j;
            if (q < qw) dst[q] = __fadd_rn(__uint_as_float(l0[j]), __uint_as_float(lr[j])) * pow2f(ew + ce[q] - 26);
          }
        }
      }
    }
  } else if (lane == 0) {
    // ------------------------------------------------ TMA: w~ rows and stored basis rows per stage
    const int tau0 = (start - m.toa_off[I]) / TTA, nkc = kx_of(m, I) / KCB;
    const int blk0 = (int)(m.x16_off[I] / XBW) + q0 / KCB;
    int g = 0;
    for (; g < nst; ++g) {
      const int s = g % NSM;
      if (g >= NSM && !(wait(&wread[s], ((g / NSM) - 1) & 1) && wait(&xfree[s], ((g / NSM) - 1) & 1))) break;
      const int toa = g * KWB, tau = tau0 + toa / TTA, tsub = toa % TTA;
      mbar_expect_tx(&wland[s], FW_WSB);
      for (int h = 0; h < KWB / 32; ++h)
        if (PTA_ALIGNED(m.chk, start + toa + 32 * h, 4, kChkTmaX) &&
            PTA_IN(m.chk, start + toa + 32 * h + 31, m.ntoa_pad, kChkTmaRange) &&
            PTA_IN(m.chk, start + toa + 32 * h - m.toa_off[I], m.n_pad[I], kChkUnit))
          tma_2d(wsm + s * FW_WSB + h * FW_WHB, &tw, start + toa + 32 * h, b0, &wland[s]);
      mbar_expect_tx(&xfull[s], FW_XST);
      if (PTA_ALIGNED(m.chk, 8 * tsub, 8, kChkTmaX) && PTA_IN(m.chk, 8 * tsub + 255, 8 * TTA, kChkTmaRange) &&
          PTA_IN(m.chk, tau * nkc + q0 / KCB, m.n_pad[I] / TTA * nkc, kChkResBasis))
        tma_4d(smem + s * FW_XST, &tx, 8 * tsub, 0, blk0 + tau * nkc, 0, &xfull[s]);
    }
    // no copy in flight into this CTA's shared memory at exit (bounded waits)
    for (int h = max(0, g - NSM); h < g; ++h) {
      tc::mbar_wait(&wland[h % NSM], (h / NSM) & 1, kDrainLimit);
      tc::mbar_wait(&xfull[h % NSM], (h / NSM) & 1, kDrainLimit);
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

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link)
using EncodeTiled = PFN_cuTensorMapEncodeTiled_v12000;
EncodeTiled encode_tiled() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}

template <int NC>
size_t res_smem(const DevModel& m) {
  (void)m;
  return (size_t)RES_NXS * RES_KB * (RES_XSB + 2 * 4 * NC * 16) + 4 * NC * (sizeof(double) + sizeof(float)) +
         NC * sizeof(float);
}

// chains per CTA of k_f16_res: 64 when the coefficient block fits in shared memory
int res_nc(const DevModel& m) { return res_smem<64>(m) <= 227 * 1024 ? 64 : 32; }

template <int NC>
cudaError_t launch_f16_nc(const DevModel& m, const Scratch& s, int B, cudaStream_t st, cudaEvent_t* kev) {
  const int nCB = (B + NC - 1) / NC;
  k_f16_pack<NC><<<dim3(m.npsr, nCB), PACK_THREADS, sizeof(int) * m.x16_kxm, st>>>(m, s.a64, s.c16, s.yexp, B, nCB);
  const size_t sm = res_smem<NC>(m);
  if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(k_f16_res<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  float* w = m.cw ? s.cwwt : s.wres;
  if (kev) cudaEventRecord(kev[0], st);
  k_f16_res<NC><<<dim3(nCB, m.n_units), RES_THREADS, sm, st>>>(m, s.c16, s.yexp, w, s.wmx, s.c2part, s.stat,
                                                              m.cw ? s.cwsig : nullptr, B, nCB);
  if (kev) cudaEventRecord(kev[1], st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_f16_ftw, cudaFuncAttributeMaxDynamicSharedMemorySize, FW_SMEM);
  if (e != cudaSuccess) return e;
  EncodeTiled enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap tw, tx;
  {  // [B][ntoa_pad]: box 32 TOAs x 128 chains, 128-byte swizzle
    const cuuint64_t dim[2] = {(cuuint64_t)m.ntoa_pad, (cuuint64_t)B};
    const cuuint64_t stride[1] = {(cuuint64_t)m.ntoa_pad * 4};
    const cuuint32_t box[2] = {32, 128}, es[2] = {1, 1};
    if (enc(&tw, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, w, dim, stride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {
    const cuuint64_t dim[4] = {8 * TTA, 2, (cuuint64_t)m.x16_blocks, 4};
    const cuuint64_t stride[3] = {2048, (cuuint64_t)RES_XSB, 4096};
    const cuuint32_t box[4] = {8 * KWB, 2, QWB / KCB, 3}, es[4] = {1, 1, 1, 1};
    if (enc(&tx, CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, const_cast<uint32_t*>(m.x16), dim, stride, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  if (kev) cudaEventRecord(kev[2], st);
  k_f16_ftw<<<dim3((m.P + QWB - 1) / QWB, (B + 127) / 128, m.n_units), FW_THREADS, FW_SMEM, st>>>(m, tw, tx, s.wmx,
                                                                                                  s.gpart, s.stat, B);
  if (kev) cudaEventRecord(kev[3], st);
  return cudaGetLastError();
}

}  // namespace

// The exact levels need at most 512 basis columns per pulsar (2 K 2^14 <= 2^24 quanta),
// the timing-model projection at most 128 columns (its shared-memory cache) and the
// coefficient block of 32 chains in shared memory beside the basis stages.
bool f16_supported(const DevModel& m) {
  const int kxm = round_up_hd(m.P + (m.cw ? m.m_max : 0), KCA);
  DevModel t = m;
  t.x16_kxm = kxm;
  return m.P + (m.cw ? m.m_max : 0) <= 512 && m.m_max <= 128 && res_smem<32>(t) <= 227 * 1024;
}

size_t f16_pack_bytes(const DevModel& m, int cap) {
  DevModel t = m;
  t.x16_kxm = round_up_hd(m.P + (m.cw ? m.m_max : 0), KCA);
  const int nc = res_nc(t), nCB = (cap + nc - 1) / nc;
  return (size_t)m.npsr * nCB * 4 * t.x16_kxm * nc * 2;
}

// The stored basis, built once per model: per-pulsar word offsets, column maxima
// (pass 1), column exponents and the pieces (pass 2).  Sets m.x16, m.x16_off,
// m.x16_cexp and m.x16_kxm; the device allocations are appended to `allocs`.
cudaError_t build_f16_basis(DevModel& m, const std::vector<int>& n_pad, const std::vector<int>& mI,
                            std::vector<void*>& allocs) {
  int kxm = KCA;
  std::vector<long long> off(m.npsr);
  long long words = 0;
  for (int I = 0; I < m.npsr; ++I) {
    const int kx = kx_cols(m.P, mI[I], m.cw);
    kxm = std::max(kxm, kx);
    off[I] = words;
    words += (long long)(n_pad[I] / TTA) * (kx / KCB) * XBW;
  }
  uint32_t* img = nullptr;
  long long* doff = nullptr;
  int* cexp = nullptr;
  unsigned long long* cmax = nullptr;
  cudaError_t e = cudaMalloc(&img, sizeof(uint32_t) * std::max<long long>(words, 4));
  if (e == cudaSuccess) allocs.push_back(img);
  if (e == cudaSuccess && (e = cudaMalloc(&doff, sizeof(long long) * m.npsr)) == cudaSuccess) allocs.push_back(doff);
  if (e == cudaSuccess && (e = cudaMalloc(&cexp, sizeof(int) * (size_t)m.npsr * kxm)) == cudaSuccess)
    allocs.push_back(cexp);
  if (e == cudaSuccess) e = cudaMalloc(&cmax, sizeof(unsigned long long) * (size_t)m.npsr * kxm);
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(doff, off.data(), sizeof(long long) * m.npsr, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(cmax, 0, sizeof(unsigned long long) * (size_t)m.npsr * kxm);
  if (e == cudaSuccess) e = cudaMemset(cexp, 0, sizeof(int) * (size_t)m.npsr * kxm);
  if (e == cudaSuccess) {
    m.x16_off = doff;
    m.x16_kxm = kxm;
    const dim3 grid(m.n_units, kxm / KCA);
    k_f16_colmax<<<grid, 128>>>(m, cmax, kxm);
    k_f16_image<<<grid, 128>>>(m, cmax, kxm, img, cexp);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  cudaFree(cmax);
  if (e != cudaSuccess) return e;
  m.x16 = img;
  m.x16_cexp = cexp;
  m.x16_blocks = words / XBW;
  return cudaSuccess;
}

cudaError_t launch_toa_f16(const DevModel& m, const Scratch& s, int B, cudaStream_t st, cudaEvent_t* kev) {
  if (!f16_supported(m) || !m.x16 || !s.c16 || !s.yexp || !s.wmx || (!m.cw && !s.wres)) return cudaErrorInvalidValue;
  return res_nc(m) == 64 ? launch_f16_nc<64>(m, s, B, st, kev) : launch_f16_nc<32>(m, s, B, st, kev);
}

}  // namespace pta
