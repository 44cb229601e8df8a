// TOA contractions on the tcgen05 tensor cores (kind::tf32, FP32 accumulation in
// tensor memory), the same quantities as k_toa_simt:
//   y  = [F | M | F~_lo] coef          (GEMM1, per 128-TOA tile)
//   r~ = dt'' - y,  w~ = N^-1 r~,  chi2 += r~ . w~
//   ghat += F^T w~                     (GEMM2, accumulated over the unit's tiles)
// 3-term split TF32 (x = hi + lo, products hi*hi + hi*lo + lo*hi) reaches FP32-level
// accuracy; the single-term variant is kept for reporting.
//
// One CTA (256 threads) per (work unit, block of 64 chains).  Every operand is
// K-major in shared memory, no swizzle: core matrices of 8 rows x 16 bytes.
//   GEMM1: A = basis chunk [128 TOAs x 32 columns], generated (Fourier columns from
//          the 64-bit phase) or loaded (timing-model and projected low-frequency
//          columns); B = coefficient chunk [64 chains x 32 columns].
//   GEMM2: A = F^T chunk [128 basis rows x 32 TOAs], regenerated in transposed
//          order; B = W [64 chains x 128 TOAs] written by the epilogue.
// Two 48 KB stages alternate between operand generation (all threads) and MMA
// (one elected thread); tcgen05.commit arrives on the stage's mbarrier when the
// MMAs that read it have finished.  Tensor memory: D1 (64 columns) and one
// 64-column accumulator per 128-row tile of ghat.
#include "pta_internal.cuh"
#include "tc_ptx.cuh"

namespace pta {
namespace {

constexpr int kTcThreads = 256;
constexpr int TT = 128;                   // TOAs per tile
constexpr int NCH = 64;                   // chains per CTA
constexpr int KC = 32;                    // basis columns per GEMM1 chunk
constexpr int TC2 = 32;                   // TOAs per GEMM2 chunk
constexpr int XCH = TT * KC * 4;          // 16 KB
constexpr int CCH = NCH * KC * 4;         // 8 KB
constexpr int FCH = 128 * TC2 * 4;        // 16 KB
constexpr int STAGE = 2 * XCH + 2 * CCH;  // 48 KB
constexpr int W_LBO = 144;                // padded core stride along TOAs (conflict-free stores)
constexpr int W_SBO = (TT / 4) * W_LBO;   // 4608
constexpr int WCOPY = (NCH / 8) * W_SBO;  // 36864
constexpr int SMEM_TC = 2 * STAGE + 2 * WCOPY;
constexpr uint32_t kWaitLimit = 20000000u;
constexpr uint32_t IDESC = tc::idesc_tf32(128, 64);

static_assert(2 * FCH <= STAGE, "GEMM2 chunk must fit in a stage");

// byte offset of element (row r, column k) of a K-major operand whose rows hold
// 32 columns (8 core matrices of 4 columns): lbo = 128, sbo = 1024
__device__ __forceinline__ int off32(int r, int k) { return (r >> 3) * 1024 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4; }

__device__ __forceinline__ void st4(unsigned char* base, int off, float4 v) {
  *reinterpret_cast<float4*>(base + off) = v;
}
__device__ __forceinline__ void split4(const float (&v)[4], float4& hi, float4& lo) {
  float h, l;
  tc::split_tf32(v[0], h, l);
  hi.x = h;
  lo.x = l;
  tc::split_tf32(v[1], h, l);
  hi.y = h;
  lo.y = l;
  tc::split_tf32(v[2], h, l);
  hi.z = h;
  lo.z = l;
  tc::split_tf32(v[3], h, l);
  hi.w = h;
  lo.w = l;
}

template <int TERMS>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_toa_tc(DevModel m, const float* __restrict__ a32, float* __restrict__ gpart, double* __restrict__ c2part,
             int32_t* __restrict__ stat, int B) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ float dts[TT], nis[TT];
  __shared__ double c2red[4][NCH];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_bad;
  unsigned char* stage[2] = {smem, smem + STAGE};
  unsigned char* Whi = smem + 2 * STAGE;
  unsigned char* Wlo = Whi + WCOPY;

  const int u = blockIdx.x, b0 = blockIdx.y * NCH, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int I = m.unit_psr[u], start = m.unit_start[u], len = m.unit_len[u];
  const int P = m.P, na = m.na, nd = m.nd, mI = m.m[I], NL = m.NL;
  const int KA = P + mI + NL, KC1 = (KA + KC - 1) / KC, nMT = (P + 127) / 128;
  const int ncols = nMT <= 3 ? 256 : 512;
  const float* Mg = m.M32 + m.m_off[I] + (long long)(start - m.toa_off[I]) * mI;
  const float* Lg = m.Flo + m.flo_off[I] + (long long)(start - m.toa_off[I]) * NL;
  const float* arows = a32 + ((size_t)I * B + b0) * m.PM;
  const int nvalid = min(NCH, B - b0);

  if (warp == 0) tc::tmem_alloc(&tmem_base, ncols);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    s_bad = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  uint32_t cnt[2] = {0, 0};  // commits issued to each stage's mbarrier
  int cur = 0;               // next stage to fill
  double c2acc = 0.0;
  bool d2_init[8] = {false, false, false, false, false, false, false, false};
  bool bad = false;

  // wait until stage s can be overwritten (its last MMA batch has completed)
  auto stage_free = [&](int s) {
    if (cnt[s] > 0 && !tc::mbar_wait(&mbar[s], (cnt[s] - 1) & 1, kWaitLimit)) s_bad = 1;
  };

  for (int t0 = 0; t0 < len && !bad; t0 += TT) {
    const int ta = start + t0;  // absolute TOA index of the tile
    if (tid < TT) {
      dts[tid] = m.dt[ta + tid];
      nis[tid] = m.ninv[ta + tid];
    }
    // ---------------- GEMM1: y[t][n] = sum_q X[t][q] C[q][n]
    for (int kc = 0; kc < KC1; ++kc) {
      const int s = cur;
      stage_free(s);
      unsigned char* Xh = stage[s];
      unsigned char* Xl = Xh + XCH;
      unsigned char* Ch = Xl + XCH;
      unsigned char* Cl = Ch + CCH;
      {  // basis chunk: thread (TOA t, half h) produces 16 columns
        const int t = tid & (TT - 1), h = tid >> 7;
        const int q0 = kc * KC + h * 16;
        const uint64_t U = m.phase[ta + t];
        const float wch = m.chrom[ta + t];
        float v[16];
#pragma unroll
        for (int e = 0; e < 16; e += 2) {
          const int q = q0 + e;
          if (q < P) {
            const bool dm = q >= 2 * na;
            const int k = dm ? (q - 2 * na) / 2 + 1 : q / 2 + 1;
            float sn, cs;
            sincos_turns64(U * (uint64_t)k, &sn, &cs);
            const float wt = dm ? wch : 1.0f;
            v[e] = sn * wt;
            v[e + 1] = cs * wt;
          } else {
#pragma unroll
            for (int f = 0; f < 2; ++f) {
              const int qq = q + f - P;
              v[e + f] = qq < mI ? Mg[(long long)(t0 + t) * mI + qq]
                                 : (qq < mI + NL ? Lg[(long long)(t0 + t) * NL + (qq - mI)] : 0.f);
            }
          }
        }
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const float w4[4] = {v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]};
          float4 hi, lo;
          split4(w4, hi, lo);
          const int off = off32(t, h * 16 + 4 * g);
          st4(Xh, off, hi);
          st4(Xl, off, lo);
        }
      }
      for (int e = tid; e < NCH * (KC / 4); e += kTcThreads) {  // coefficient chunk
        const int n = e % NCH, g = e / NCH;
        float4 cv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n < nvalid) cv = *reinterpret_cast<const float4*>(arows + (size_t)n * m.PM + kc * KC + 4 * g);
        const float w4[4] = {cv.x, cv.y, cv.z, cv.w};
        float4 hi, lo;
        split4(w4, hi, lo);
        const int off = off32(n, 4 * g);
        st4(Ch, off, hi);
        st4(Cl, off, lo);
      }
      tc::fence_async_smem();
      __syncthreads();
      if (s_bad) {
        bad = true;
        break;
      }
      if (tid == 0) {
        tc::fence_after();
        const uint32_t xh = tc::smem_u32(Xh), xl = tc::smem_u32(Xl), ch = tc::smem_u32(Ch), cl = tc::smem_u32(Cl);
#pragma unroll
        for (int ks = 0; ks < KC / 8; ++ks) {
          const uint32_t o = ks * 256;
          const uint32_t acc0 = (kc > 0 || ks > 0) ? 1u : 0u;
          tc::mma_tf32(tmem, tc::desc(xh + o, 128, 1024), tc::desc(ch + o, 128, 1024), IDESC, acc0);
          if (TERMS == 3) {
            tc::mma_tf32(tmem, tc::desc(xh + o, 128, 1024), tc::desc(cl + o, 128, 1024), IDESC, 1u);
            tc::mma_tf32(tmem, tc::desc(xl + o, 128, 1024), tc::desc(ch + o, 128, 1024), IDESC, 1u);
          }
        }
        tc::commit(&mbar[s]);
      }
      cnt[s] += 1;
      cur ^= 1;
    }
    if (bad) break;
    // ---------------- epilogue: wait for GEMM1, projected residual, W, chi2
    {
      const int sl = cur ^ 1;  // stage of the last GEMM1 batch
      if (!tc::mbar_wait(&mbar[sl], (cnt[sl] - 1) & 1, kWaitLimit)) s_bad = 1;
      tc::fence_after();
      const int lanebase = 32 * (warp & 3), colbase = 32 * (warp >> 2);
      uint32_t r[32];
      tc::ld32(tmem + ((uint32_t)lanebase << 16) + colbase, r);
      const int t = lanebase + lane;
      const float dtv = dts[t], ni = nis[t];
      float q[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float rr = dtv - __uint_as_float(r[i]);
        const float ww = rr * ni;
        q[i] = rr * ww;
        float hi, lo;
        tc::split_tf32(ww, hi, lo);
        const int n = colbase + i;
        const int off = (n >> 3) * W_SBO + (t >> 2) * W_LBO + (n & 7) * 16 + (t & 3) * 4;
        *reinterpret_cast<float*>(Whi + off) = hi;
        *reinterpret_cast<float*>(Wlo + off) = lo;
      }
      // reduce q over the warp's 32 TOAs: lane l ends with the sum for chain colbase + l
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        const bool upper = lane & o;
#pragma unroll
        for (int i = 0; i < o; ++i) {
          const float send = upper ? q[i] : q[i + o];
          const float recv = __shfl_xor_sync(0xffffffffu, send, o);
          q[i] = (upper ? q[i + o] : q[i]) + recv;
        }
      }
      c2acc += (double)q[0];
      tc::fence_async_smem();
      tc::fence_before();
      __syncthreads();
      if (s_bad) {
        bad = true;
        break;
      }
    }
    // ---------------- GEMM2: ghat[p][n] += sum_t F^T[p][t] W[t][n]
    for (int c = 0; c < TT / TC2 && !bad; ++c) {
      for (int j = 0; j < nMT; ++j) {
        const int s = cur;
        stage_free(s);
        unsigned char* Fh = stage[s];
        unsigned char* Fl = Fh + FCH;
        for (int e = tid; e < 64 * (TC2 / 4); e += kTcThreads) {
          const int rp = e % 64, tq = e / 64;     // row pair (2 basis rows), TOA quad
          const int p = 128 * j + 2 * rp;
          const int tl = c * TC2 + 4 * tq;        // tile-local TOA of the quad
          float sv[4], cv[4];
          if (p < P) {
            const bool dm = p >= 2 * na;
            const int k = dm ? (p - 2 * na) / 2 + 1 : p / 2 + 1;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              float sn, cs;
              sincos_turns64(m.phase[ta + tl + i] * (uint64_t)k, &sn, &cs);
              const float wt = dm ? m.chrom[ta + tl + i] : 1.0f;
              sv[i] = sn * wt;
              cv[i] = cs * wt;
            }
          } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) sv[i] = cv[i] = 0.f;
          }
          float4 hi, lo;
          split4(sv, hi, lo);
          st4(Fh, off32(2 * rp, 4 * tq), hi);
          st4(Fl, off32(2 * rp, 4 * tq), lo);
          split4(cv, hi, lo);
          st4(Fh, off32(2 * rp + 1, 4 * tq), hi);
          st4(Fl, off32(2 * rp + 1, 4 * tq), lo);
        }
        tc::fence_async_smem();
        __syncthreads();
        if (s_bad) {
          bad = true;
          break;
        }
        if (tid == 0) {
          tc::fence_after();
          const uint32_t fh = tc::smem_u32(Fh), fl = tc::smem_u32(Fl);
          const uint32_t wh = tc::smem_u32(Whi), wl = tc::smem_u32(Wlo);
          const uint32_t dcol = tmem + 64 + 64 * j;
#pragma unroll
          for (int ks = 0; ks < TC2 / 8; ++ks) {
            const uint32_t oa = ks * 256, ob = (8 * c + 2 * ks) * W_LBO;
            const uint32_t acc0 = d2_init[j] ? 1u : 0u;
            d2_init[j] = true;
            tc::mma_tf32(dcol, tc::desc(fh + oa, 128, 1024), tc::desc(wh + ob, W_LBO, W_SBO), IDESC, acc0);
            if (TERMS == 3) {
              tc::mma_tf32(dcol, tc::desc(fh + oa, 128, 1024), tc::desc(wl + ob, W_LBO, W_SBO), IDESC, 1u);
              tc::mma_tf32(dcol, tc::desc(fl + oa, 128, 1024), tc::desc(wh + ob, W_LBO, W_SBO), IDESC, 1u);
            }
          }
          tc::commit(&mbar[s]);
        }
        cnt[s] += 1;
        cur ^= 1;
      }
    }
  }
  // ---------------- drain and write the unit's partial sums
  {
    const int sl = cur ^ 1;
    if (cnt[sl] > 0 && !tc::mbar_wait(&mbar[sl], (cnt[sl] - 1) & 1, kWaitLimit)) s_bad = 1;
    const int so = cur;
    if (cnt[so] > 0 && !tc::mbar_wait(&mbar[so], (cnt[so] - 1) & 1, kWaitLimit)) s_bad = 1;
  }
  tc::fence_after();
  __syncthreads();
  bad = bad || s_bad;
  if (!bad) {
    const int lanebase = 32 * (warp & 3), colbase = 32 * (warp >> 2);
    for (int j = 0; j < nMT; ++j) {
      uint32_t r[32];
      tc::ld32(tmem + ((uint32_t)lanebase << 16) + 64 + 64 * j + colbase, r);
      const int row = 128 * j + lanebase + lane;
      if (row < P) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int n = colbase + i;
          if (n < nvalid) gpart[((size_t)u * B + b0 + n) * m.Qs + row] = __uint_as_float(r[i]);
        }
      }
    }
    c2red[warp & 3][colbase + lane] = c2acc;
  }
  tc::fence_before();
  __syncthreads();
  if (!bad && tid < NCH && tid < nvalid)
    c2part[(size_t)u * B + b0 + tid] = ((c2red[0][tid] + c2red[1][tid]) + c2red[2][tid]) + c2red[3][tid];
  if (bad && tid < nvalid) atomicOr(&stat[b0 + tid], 4);
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

}  // namespace

cudaError_t launch_toa_tc(const DevModel& m, const Scratch& s, int B, int terms, cudaStream_t st) {
  if ((m.P + 127) / 128 > 7 || m.PM % KC != 0) return cudaErrorInvalidValue;
  dim3 grid(m.n_units, (B + NCH - 1) / NCH);
  cudaError_t e;
  if (terms == 3) {
    e = cudaFuncSetAttribute(k_toa_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_TC);
    if (e != cudaSuccess) return e;
    k_toa_tc<3><<<grid, kTcThreads, SMEM_TC, st>>>(m, s.a32, s.gpart, s.c2part, s.stat, B);
  } else {
    e = cudaFuncSetAttribute(k_toa_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_TC);
    if (e != cudaSuccess) return e;
    k_toa_tc<1><<<grid, kTcThreads, SMEM_TC, st>>>(m, s.a32, s.gpart, s.c2part, s.stat, B);
  }
  return cudaGetLastError();
}

}  // namespace pta
