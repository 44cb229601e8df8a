// TOA-domain part of the evaluation: the timing-model-marginalised likelihood of
// Eq. (raw_det_posterior) with N~^-1 of Eq. (Gmatrix_proj) in its projected form,
//   c  = (M^T N^-1 M)^-1 M^T N^-1 (dt - F a)          (FP64, per pulsar and chain)
//   r~ = dt - F a - M c,   w~ = N^-1 r~ = N~^-1 (dt - F a)
//   chi2 = r~ . w~,        ghat = F^T w~ = d logp / d a
// The projection is applied before the TOA-length sums, so neither chi2 nor ghat
// is a small difference of large terms (the unprojected residual can be orders
// of magnitude above the noise where F a carries timing-model-like power).
//
// Work unit = (pulsar, chunk of <= 2048 TOAs) x block of chains; each unit writes
// its partial sums to its own slot and the FP64 reduction sums them in a fixed
// order, so results do not depend on scheduling.
//
// FP32 variant: the Fourier basis of Eq. (Fourier_series) and its DM copy weighted
// by (nu_ref/nu)^2 are generated in shared memory from a 64-bit fixed-point phase
// k * U_i mod 2^64 (exact argument reduction); with the timing-model rows they
// form one transposed tile X^T[q][t] used by both contractions.
// FP64 variant (plain path): stored FP64 basis, one CTA per (unit, chain).
#include <algorithm>

#include "dwarith.cuh"
#include "pta_internal.cuh"

namespace pta {
namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// Timing-model prologue, one CTA (128 threads) per (pulsar, chain).
// With the reference coefficients a_ref (the projected reference residual dt''
// satisfies M^T N^-1 dt'' = 0) and da = a - a_ref, the projected residual is
//   r~ = dt'' - F da - M c,  c = -(M^T N^-1 M)^-1 H^T da,  H = F^T N^-1 M.
// c is applied as an FP64 matrix-vector product with the stored (M^T N^-1 M)^-1.
// FP64 path: c from the full H in FP64; row = [da, c].
// FP32 path: the lowest-frequency columns (nla achromatic, nld DM bins) use the
// stored projected basis F~_lo = F_lo - M K^-1 H_lo^T, so c only carries the other
// columns: c_hi = -K^-1 H_hi^T da_hi.  H_hi^T da_hi is a compensated FP32 dot
// product (error-free FMA products and sums, Ogita-Rump-Oishi "Dot2") on hi/lo
// splits of H and da; the K solve is FP64.  Row = [da with zeros on the low
// columns, c_hi, da_lo] matching the tile rows [F, M, F~_lo].
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool is_low_col(const DevModel& m, int p) {
  return p < 2 * m.nla || (p >= 2 * m.na && p < 2 * m.na + 2 * m.nld);
}
__device__ __forceinline__ int low_col(const DevModel& m, int q) {
  return q < 2 * m.nla ? q : 2 * m.na + (q - 2 * m.nla);
}

__global__ void __launch_bounds__(128)
    k_tm_prologue(DevModel m, double* __restrict__ a64, float* __restrict__ a32, const double* __restrict__ cwbs,
                  int B, int fp64) {  // fp64: 0 FP32 packed rows, 1 FP64 path, 2 exact-split path
  extern __shared__ double smp[];
  const int I = blockIdx.x, b = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int P = m.P, mI = m.m[I];
  double* da = smp;             // [P]
  double* part = da + P;        // [4][mI]
  double* cv = part + 4 * mI;   // [mI]
  float* dah = reinterpret_cast<float*>(cv + mI);  // [P] hi part of da (0 on low columns)
  float* dal = dah + P;                            // [P] lo part
  double* row = a64 + ((size_t)I * B + b) * m.PM;
  const double* ar = m.aref + (size_t)I * P;
  for (int p = tid; p < P; p += 128) {
    const double v = row[p] - ar[p];
    da[p] = v;
    const bool lo = is_low_col(m, p);
    const float h = lo ? 0.f : (float)v;
    dah[p] = h;
    dal[p] = lo ? 0.f : (float)(v - (double)h);
  }
  __syncthreads();
  for (int j0 = 0; j0 < mI; j0 += 32) {
    const int j = j0 + lane;
    if (j < mI && fp64 == 2) {
      part[warp * mI + j] = 0.0;  // projected basis: c carries only the signal's projection
    } else if (j < mI) {
      if (fp64) {
        const double* H = m.H + m.h_off[I];
        double s = 0.0;
        for (int p = warp; p < P; p += 4) s = fma(H[(size_t)p * mI + j], da[p], s);
        part[warp * mI + j] = s;
      } else {
        const float* Hh = m.Hhi + m.h_off[I];
        const float* Hl = m.Hlo + m.h_off[I];
        float s = 0.f, comp = 0.f;
        for (int p = warp; p < P; p += 4) {
          const float xh = dah[p], xl = dal[p];
          const float hh = Hh[(size_t)p * mI + j], hl = Hl[(size_t)p * mI + j];
          const float pr = hh * xh;
          const float pe = fmaf(hh, xh, -pr);          // exact product error
          const float t = s + pr;
          const float z = t - s;
          const float se = (s - (t - z)) + (pr - z);   // exact sum error
          s = t;
          comp += se + pe + fmaf(hh, xl, hl * xh);
        }
        part[warp * mI + j] = (double)s + (double)comp;
      }
    }
  }
  __syncthreads();
  // c = -(M^T N^-1 M)^-1 hv, hv = H^T da: FP64 matvec with the stored inverse
  double* hv = part;  // in place: hv[j] = sum of the four warp partials of column j
  for (int j = tid; j < mI; j += 128) {
    double v = ((part[j] + part[mI + j]) + part[2 * mI + j]) + part[3 * mI + j];
    if (cwbs)  // deterministic signal: c also absorbs M^T N^-1 s
      for (int q = 0; q < m.nunit[I]; ++q) v += cwbs[((size_t)(m.unit0[I] + q) * B + b) * m.m_max + j];
    hv[j] = v;
  }
  __syncthreads();
  {
    const double* Ki = m.Kinv + m.lk_off[I];
    for (int i = tid; i < mI; i += 128) {
      double s = 0.0;
      for (int j = 0; j < mI; ++j) s = fma(Ki[i * mI + j], hv[j], s);
      cv[i] = -s;
    }
  }
  __syncthreads();
  if (fp64 == 1) {
    for (int p = tid; p < P; p += 128) row[p] = da[p];
    for (int j = tid; j < mI; j += 128) row[P + j] = cv[j];
  } else if (fp64 == 2) {
    // exact-split tensor-core path (fully projected basis): a stays in place, c_s follows
    for (int j = tid; j < mI; j += 128) row[P + j] = cv[j];
  } else {
    // FP32 packed row [da (low columns zero) | c | da of the low columns | 0]
    float* r32 = a32 + ((size_t)I * B + b) * m.PM;
    for (int q = tid; q < m.PM; q += 128) {
      float v = 0.f;
      if (q < P)
        v = is_low_col(m, q) ? 0.f : (float)da[q];
      else if (q < P + mI)
        v = (float)cv[q - P];
      else if (q < P + mI + m.NL)
        v = (float)da[low_col(m, q - P - mI)];
      r32[q] = v;
    }
  }
}

template <int BC, int TT, int QPT>
struct SimtCfg {
  static constexpr int CG = BC / 4;            // chain groups of 4
  static constexpr int RG = kThreads / CG;     // row groups (GEMM1) == q lanes (GEMM2)
  static constexpr int RPT = TT / RG;          // TOA rows per thread in GEMM1
  static constexpr int QPAD = RG * QPT;        // rows of ghat covered by GEMM2
  static constexpr int XS = TT + 4;            // X^T row stride (floats)
  static constexpr int AS = BC + 4;            // A row stride
  static constexpr int WS = BC + 4;            // W row stride
  static_assert(RPT >= 1 && RG * RPT == TT, "tile shape");
};

// Basis-tile rows.  PF = 0: [F (P) | M (m_I) | F~_lo (NL) | zero], PM coefficient rows.
// PF = 1: [F (P) | zero up to QPAD | M | F~_lo]: F^T w never reads the M / F~_lo rows,
// so those rows can be refilled for the next tile while it runs.
template <int BC, int TT, int QPT, int PF>
int simt_xrows(const DevModel& m) {
  using C = SimtCfg<BC, TT, QPT>;
  if (PF) return C::QPAD + m.m_max + m.NL;
  return C::QPAD > m.PM ? C::QPAD : m.PM;
}
template <int BC, int TT, int QPT, int PF>
int simt_arows(const DevModel& m) {
  return PF ? simt_xrows<BC, TT, QPT, PF>(m) : m.PM;
}

template <int BC, int TT, int QPT, int PF>
size_t simt_smem(const DevModel& m) {
  using C = SimtCfg<BC, TT, QPT>;
  return sizeof(float) * ((size_t)simt_xrows<BC, TT, QPT, PF>(m) * C::XS +
                          (size_t)simt_arows<BC, TT, QPT, PF>(m) * C::AS + (size_t)TT * C::WS +
                          (size_t)C::RG * BC + 2 * TT);
}

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
// Packed FP32 pairs: one fma.rn.f32x2 does two independent FP32 multiply-adds (same
// rounding as two fmaf), halving the issue slots of the register-blocked products.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2dup(float v) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ void f2unpack(f32x2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 f2fma(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// ORD selects the instruction order of the two register-blocked products:
//   0: F a unrolled by 2 along the coefficient index; F^T w as nested FMAs over the
//      four TOAs of a step (one dependent chain of 4 per accumulator);
//   1: F a unrolled by 4; F^T w with the four TOAs outermost, so every FMA of a
//      TOA is independent of the others (longer register lifetimes, no chains).
// PF = 1 prefetches the next tile while F^T w of the current one runs: its timing-
// model and F~_lo rows by cp.async into the (then unread) rows of the basis tile,
// its phases, weights, residuals and noise weights into registers.
template <int BC, int TT, int QPT, int ORD, int PF>
__global__ void __launch_bounds__(kThreads, 1)
    k_toa_simt(DevModel m, const float* __restrict__ a32, float* __restrict__ gpart, double* __restrict__ c2part,
               int B, int XR, const float* __restrict__ cwsig, float* __restrict__ cwwt, int* __restrict__ queue,
               int nCB) {
  using C = SimtCfg<BC, TT, QPT>;
  extern __shared__ float4 sm4[];
  float* Xs = reinterpret_cast<float*>(sm4);            // [XR][XS]  basis rows (layout above)
  float* As = Xs + XR * C::XS;                          // [AR][AS]  coefficient rows in the same order
  const int AR = PF ? XR : m.PM;
  float* Ws = As + AR * C::AS;                          // [TT][WS]
  float* C2 = Ws + TT * C::WS;                          // [RG][BC]
  float* dts = C2 + C::RG * BC;                         // [TT]
  float* nis = dts + TT;                                // [TT]
  // Work items are (unit, block of BC chains).  queue == nullptr: one item per CTA
  // (blockIdx.x = unit, blockIdx.y = chain block).  Otherwise the launch is
  // persistent: every resident CTA takes items from an atomic counter, units in the
  // order m.unit_order (longest first), until none are left.
  __shared__ int s_item;
  const int tid = threadIdx.x;
  int item = 0;
  if (queue) {
    if (tid == 0) s_item = atomicAdd(queue, 1);
    __syncthreads();
    item = s_item;
  }
  for (;;) {
  if (queue && item >= m.n_units * nCB) break;
  const int u = queue ? m.unit_order[item / nCB] : blockIdx.x;
  const int b0 = (queue ? item % nCB : blockIdx.y) * BC;
  const int I = m.unit_psr[u], start = m.unit_start[u], len = m.unit_len[u];
  const int P = m.P, mI = m.m[I], NL = m.NL, KA = P + mI + NL, na = m.na, nd = m.nd;
  const int kmax = na > nd ? na : nd;
  const float* Mg = m.M32 + m.m_off[I] + (long long)(start - m.toa_off[I]) * mI;
  const float* Lg = m.Flo + m.flo_off[I] + (long long)(start - m.toa_off[I]) * NL;
  const int rowM = PF ? C::QPAD : P;  // first timing-model row of the tile
  for (int e = tid; e < KA * BC; e += kThreads) {
    const int c = e / KA, p = e % KA;
    As[(p < P ? p : rowM + p - P) * C::AS + c] = (b0 + c < B) ? a32[((size_t)I * B + b0 + c) * m.PM + p] : 0.f;
  }
  // PF: prefetched per-TOA data of the next tile, and the first tile's fixed rows
  uint64_t pf_U = 0;
  float pf_w = 0.f, pf_dt = 0.f, pf_ni = 0.f;
  auto prefetch = [&](int t1) {
    const int t = tid % TT;
    pf_U = m.phase[start + t1 + t];
    pf_w = m.chrom[start + t1 + t];
    if (tid < TT) {
      pf_dt = m.dt[start + t1 + tid];
      pf_ni = m.ninv[start + t1 + tid];
    }
    for (int e = tid; e < TT * mI; e += kThreads) {
      const int tt = e / mI, j = e % mI;
      cp_async4(Xs + (rowM + j) * C::XS + tt, Mg + (long long)(t1 + tt) * mI + j);
    }
    for (int e = tid; e < TT * NL; e += kThreads) {
      const int tt = e / NL, j = e % NL;
      cp_async4(Xs + (rowM + mI + j) * C::XS + tt, Lg + (long long)(t1 + tt) * NL + j);
    }
    cp_async_commit();
  };
  if constexpr (PF) {
    for (int e = tid; e < (C::QPAD - P) * TT; e += kThreads) Xs[(P + e / TT) * C::XS + e % TT] = 0.f;
    prefetch(0);
  }
  const int cg = tid % C::CG, rg = tid / C::CG;
  f32x2 acc[QPT][2];  // ghat pairs (chains 4cg, 4cg+1) and (4cg+2, 4cg+3)
#pragma unroll
  for (int i = 0; i < QPT; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = 0ull;
  double c2acc = 0.0;

  for (int t0 = 0; t0 < len; t0 += TT) {
    if constexpr (PF) cp_async_wait_all();
    __syncthreads();  // previous tile fully consumed
    {
      const int t = tid % TT;
      const int lane_k = tid / TT, kstride = kThreads / TT;
      const uint64_t U = PF ? pf_U : m.phase[start + t0 + t];
      const float wch = PF ? pf_w : m.chrom[start + t0 + t];
      uint64_t ph = U * (uint64_t)(lane_k + 1);
      const uint64_t dph = U * (uint64_t)kstride;
      for (int k = lane_k + 1; k <= kmax; k += kstride, ph += dph) {
        float s, c;
        sincos_turns64(ph, &s, &c);
        if (k <= na) {
          Xs[(2 * (k - 1)) * C::XS + t] = s;
          Xs[(2 * (k - 1) + 1) * C::XS + t] = c;
        }
        if (k <= nd) {
          Xs[(2 * na + 2 * (k - 1)) * C::XS + t] = s * wch;
          Xs[(2 * na + 2 * (k - 1) + 1) * C::XS + t] = c * wch;
        }
      }
      if constexpr (PF) {
        if (tid < TT) {
          dts[tid] = pf_dt;
          nis[tid] = pf_ni;
        }
      } else {
        for (int e = tid; e < TT * mI; e += kThreads) {
          const int tt = e / mI, j = e % mI;
          Xs[(P + j) * C::XS + tt] = Mg[(long long)(t0 + tt) * mI + j];
        }
        for (int e = tid; e < TT * NL; e += kThreads) {
          const int tt = e / NL, j = e % NL;
          Xs[(P + mI + j) * C::XS + tt] = Lg[(long long)(t0 + tt) * NL + j];
        }
        for (int e = tid; e < (XR - KA) * TT; e += kThreads) {
          const int q = KA + e / TT, tt = e % TT;
          Xs[q * C::XS + tt] = 0.f;
        }
        if (tid < TT) {
          dts[tid] = m.dt[start + t0 + tid];
          nis[tid] = m.ninv[start + t0 + tid];
        }
      }
    }
    __syncthreads();
    // --- y[t][c] = sum_p [F | M | F~_lo][t][p] coef[p][c]
    f32x2 y2[C::RPT][2];
#pragma unroll
    for (int r = 0; r < C::RPT; ++r) y2[r][0] = y2[r][1] = 0ull;
    const float* xrow = Xs + rg * C::RPT;
    const float* arow = As + 4 * cg;
    auto g1 = [&](int p) {
      const ulonglong2 av = *reinterpret_cast<const ulonglong2*>(arow + p * C::AS);
      float fv[C::RPT];
      if constexpr (C::RPT % 4 == 0) {
#pragma unroll
        for (int r = 0; r < C::RPT; r += 4) {
          const float4 f4 = *reinterpret_cast<const float4*>(xrow + p * C::XS + r);
          fv[r] = f4.x;
          fv[r + 1] = f4.y;
          fv[r + 2] = f4.z;
          fv[r + 3] = f4.w;
        }
      } else {
#pragma unroll
        for (int r = 0; r < C::RPT; ++r) fv[r] = xrow[p * C::XS + r];
      }
#pragma unroll
      for (int r = 0; r < C::RPT; ++r) {
        const f32x2 f = f2dup(fv[r]);
        y2[r][0] = f2fma(f, av.x, y2[r][0]);
        y2[r][1] = f2fma(f, av.y, y2[r][1]);
      }
    };
    if constexpr (PF) {
#pragma unroll(ORD == 0 ? 2 : 4)
      for (int p = 0; p < P; ++p) g1(p);
#pragma unroll(ORD == 0 ? 2 : 4)
      for (int p = rowM; p < rowM + mI + NL; ++p) g1(p);
    } else {
#pragma unroll(ORD == 0 ? 2 : 4)
      for (int p = 0; p < KA; ++p) g1(p);
    }
    float y[C::RPT][4];
#pragma unroll
    for (int r = 0; r < C::RPT; ++r) {
      f2unpack(y2[r][0], y[r][0], y[r][1]);
      f2unpack(y2[r][1], y[r][2], y[r][3]);
    }
    // --- projected residual, whitened residual, chi2 pieces
    float q4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int r = 0; r < C::RPT; ++r) {
      const int t = rg * C::RPT + r;
      const float dtv = dts[t], ni = nis[t];
      float4 wv;
      float* wp = reinterpret_cast<float*>(&wv);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float rr = dtv - y[r][j];
        const int bb = b0 + 4 * cg + j;
        const size_t ci = (size_t)bb * m.ntoa_pad + start + t0 + t;
        if (cwsig && bb < B) rr -= cwsig[ci];  // r~ = dt'' - s - y
        const float ww = rr * ni;
        wp[j] = ww;
        q4[j] = fmaf(rr, ww, q4[j]);
        if (cwwt && bb < B) cwwt[ci] = ww;
      }
      *reinterpret_cast<float4*>(Ws + t * C::WS + 4 * cg) = wv;
    }
    *reinterpret_cast<float4*>(C2 + rg * BC + 4 * cg) = make_float4(q4[0], q4[1], q4[2], q4[3]);
    __syncthreads();
    if (tid < BC) {  // fixed-order chi2 reduction over row groups: thread c owns chain c; FP64, so
                     // the rounding of a 64-term FP32 running sum does not accumulate over tiles
      double s = 0.0;
      for (int g = 0; g < C::RG; ++g) s += (double)C2[g * BC + tid];
      c2acc += s;
    }
    // F a of this tile is done with the timing-model rows: fetch the next tile's
    if constexpr (PF)
      if (t0 + TT < len) prefetch(t0 + TT);
    // --- ghat[q][c] += sum_t F^T[q][t] w~[t][c],  q = rg + RG*i < P; four TOAs per step
    // so each basis row is one 16-byte load
#pragma unroll 1
    for (int t = 0; t < TT; t += 4) {
      ulonglong2 wv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) wv[r] = *reinterpret_cast<const ulonglong2*>(Ws + (t + r) * C::WS + 4 * cg);
      if constexpr (ORD == 0) {
#pragma unroll
        for (int i = 0; i < QPT; ++i) {
          const float4 xv = *reinterpret_cast<const float4*>(Xs + (rg + C::RG * i) * C::XS + t);
          const f32x2 dx = f2dup(xv.x), dy = f2dup(xv.y), dz = f2dup(xv.z), dw = f2dup(xv.w);
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const f32x2 w0 = j ? wv[0].y : wv[0].x, w1 = j ? wv[1].y : wv[1].x;
            const f32x2 w2 = j ? wv[2].y : wv[2].x, w3 = j ? wv[3].y : wv[3].x;
            acc[i][j] = f2fma(dx, w0, f2fma(dy, w1, f2fma(dz, w2, f2fma(dw, w3, acc[i][j]))));
          }
        }
      } else {
        float4 xv[QPT];
#pragma unroll
        for (int i = 0; i < QPT; ++i) xv[i] = *reinterpret_cast<const float4*>(Xs + (rg + C::RG * i) * C::XS + t);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
#pragma unroll
          for (int i = 0; i < QPT; ++i) {
            const float xr = r == 0 ? xv[i].x : (r == 1 ? xv[i].y : (r == 2 ? xv[i].z : xv[i].w));
            const f32x2 d = f2dup(xr);
            acc[i][0] = f2fma(d, wv[r].x, acc[i][0]);
            acc[i][1] = f2fma(d, wv[r].y, acc[i][1]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < QPT; ++i) {
    const int q = rg + C::RG * i;
    if (q < P) {
      float g4[4];
      f2unpack(acc[i][0], g4[0], g4[1]);
      f2unpack(acc[i][1], g4[2], g4[3]);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int b = b0 + 4 * cg + j;
        if (b < B) gpart[((size_t)u * B + b) * m.Qs + q] = g4[j];
      }
    }
  }
  if (tid < BC && b0 + tid < B) c2part[(size_t)u * B + b0 + tid] = c2acc;
  if (!queue) break;
  __syncthreads();  // the item's shared-memory state is no longer read
  if (tid == 0) s_item = atomicAdd(queue, 1);
  __syncthreads();
  item = s_item;
  }
}

// Plain FP64 path.  One CTA of 128 threads per (unit, chain); tile of 128 TOAs,
// thread t owns TOA t for y = F da + M c; F^T w~ columns are warp reductions.
__global__ void __launch_bounds__(128)
    k_toa_fp64(DevModel m, const double* __restrict__ a64, double* __restrict__ gpart, double* __restrict__ c2part,
               int B) {
  extern __shared__ double smd[];
  const int u = blockIdx.x, b = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int I = m.unit_psr[u], start = m.unit_start[u], len = m.unit_len[u];
  const int P = m.P, mI = m.m[I];
  double* as = smd;          // [P + mI]
  double* gacc = as + m.PM;  // [P]
  double* ws = gacc + P;     // [128]
  double* red = ws + 128;    // [4]
  for (int p = tid; p < P + mI; p += 128) as[p] = a64[((size_t)I * B + b) * m.PM + p];
  for (int q = tid; q < P; q += 128) gacc[q] = 0.0;
  double c2 = 0.0;
  const double* F = m.F64 + m.f_off[I];
  const double* Mg = m.M64 + m.m_off[I];
  const int base = start - m.toa_off[I];
  __syncthreads();
  for (int t0 = 0; t0 < len; t0 += 128) {
    const int li = base + t0 + tid;  // TOA index within the pulsar
    double y = 0.0;
    const double* Fr = F + (size_t)li * P;
    for (int p = 0; p < P; ++p) y = fma(Fr[p], as[p], y);
    const double* Mr = Mg + (size_t)li * mI;
    for (int j = 0; j < mI; ++j) y = fma(Mr[j], as[P + j], y);
    const double r = m.dt64[start + t0 + tid] - y;
    const double w = r * m.ninv64[start + t0 + tid];
    ws[tid] = w;
    double q = r * w;
    for (int o = 16; o; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if (lane == 0) red[warp] = q;
    __syncthreads();
    if (tid == 0) c2 += red[0] + red[1] + red[2] + red[3];
    for (int qq = warp; qq < P; qq += 4) {
      double s = 0.0;
      for (int t = lane; t < 128; t += 32) s = fma(F[(size_t)(base + t0 + t) * P + qq], ws[t], s);
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) gacc[qq] += s;
    }
    __syncthreads();
  }
  for (int q = tid; q < P; q += 128) gpart[((size_t)u * B + b) * m.Qs + q] = gacc[q];
  if (tid == 0) c2part[(size_t)u * B + b] = c2;
}

// Reduction over a pulsar's units (fixed order): ghat = F^T N~^-1 r, chi2.  One thread
// per (chain, coefficient) of a pulsar, consecutive threads on consecutive coefficients.
// FP32 partials are summed as double words (exact sums, TwoSum) and reach double with
// one FP64 add; FP64 partials (FP64 mode) are summed in FP64.
__global__ void __launch_bounds__(256)
    k_reduce(DevModel m, const float* __restrict__ gpart, const double* __restrict__ gpart64,
             const double* __restrict__ c2part, double* __restrict__ ghat, double* __restrict__ chi2, int B,
             int fp64) {
  const int I = blockIdx.y, P = m.P, u0 = m.unit0[I], nu = m.nunit[I];
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= B * P) return;
  const int b = r / P, q = r - b * P;
  double s = 0.0;
  if (fp64) {
    for (int j = 0; j < nu; ++j) s += gpart64[((size_t)(u0 + j) * B + b) * m.Qs + q];
  } else {
    float2 acc = make_float2(0.0f, 0.0f);
    for (int j = 0; j < nu; ++j) acc = dw_addf(acc, gpart[((size_t)(u0 + j) * B + b) * m.Qs + q]);
    s = dw2d(acc);
  }
  // tempered likelihood: d logp / d a scales with beta
  ghat[((size_t)I * B + b) * P + q] = m.beta ? m.beta[b] * s : s;
  if (q == 0) {
    double c2 = 0.0;
    for (int j = 0; j < nu; ++j) c2 += c2part[(size_t)(u0 + j) * B + b];
    chi2[(size_t)I * B + b] = c2;
  }
}

template <int BC, int TT, int QPT, int ORD, int PF>
cudaError_t launch_simt(const DevModel& m, const Scratch& s, int B, int ps, cudaStream_t st) {
  const size_t sm = simt_smem<BC, TT, QPT, PF>(m);
  if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
  auto kern = k_toa_simt<BC, TT, QPT, ORD, PF>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int nCB = (B + BC - 1) / BC;
  dim3 grid(m.n_units, nCB);
  int* queue = nullptr;
  if (ps) {  // persistent: as many CTAs as are resident at once
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, sm);
    if (e != cudaSuccess) return e;
    const int resident = std::max(1, per_sm) * m.nsm;
    grid = dim3(std::min(resident, m.n_units * nCB), 1);
    queue = s.queue;
    e = cudaMemsetAsync(queue, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, kThreads, sm, st>>>(m, s.a32, s.gpart, s.c2part, B, simt_xrows<BC, TT, QPT, PF>(m),
                                   m.cw ? s.cwsig : nullptr, m.cw ? s.cwwt : nullptr, queue, nCB);
  return cudaGetLastError();
}

// The tile shapes the autotuner chooses from: chains per CTA (BC), TOAs per tile
// (TT), ghat rows per thread (QPT; 256 / (BC / 4) q lanes x QPT rows must cover P),
// the instruction order (ORD) and next-tile prefetch (PF); ord = ORD + 2 PF.
struct SimtEntry {
  int bc, tt, qpt, ord;  // ord = ORD + 2 PF + 4 persistent
  cudaError_t (*launch)(const DevModel&, const Scratch&, int, int, cudaStream_t);
  size_t (*smem)(const DevModel&);
};
#define SIMT_E(BC, TT, Q, O, F) {BC, TT, Q, O + 2 * F, &launch_simt<BC, TT, Q, O, F>, &simt_smem<BC, TT, Q, F>}
#define SIMT_EP(BC, TT, Q, O, F) {BC, TT, Q, O + 2 * F + 4, &launch_simt<BC, TT, Q, O, F>, &simt_smem<BC, TT, Q, F>}
#define SIMT_Q16P(BC, TT, O, F)                                                                            \
  SIMT_EP(BC, TT, 2, O, F), SIMT_EP(BC, TT, 4, O, F), SIMT_EP(BC, TT, 8, O, F), SIMT_EP(BC, TT, 12, O, F), \
      SIMT_EP(BC, TT, 17, O, F), SIMT_EP(BC, TT, 24, O, F)
#define SIMT_Q16(BC, TT, O, F)                                                                         \
  SIMT_E(BC, TT, 2, O, F), SIMT_E(BC, TT, 4, O, F), SIMT_E(BC, TT, 8, O, F), SIMT_E(BC, TT, 12, O, F), \
      SIMT_E(BC, TT, 17, O, F), SIMT_E(BC, TT, 24, O, F)
#define SIMT_Q32(BC, TT, O, F)                                                                        \
  SIMT_E(BC, TT, 1, O, F), SIMT_E(BC, TT, 2, O, F), SIMT_E(BC, TT, 4, O, F), SIMT_E(BC, TT, 6, O, F), \
      SIMT_E(BC, TT, 9, O, F), SIMT_E(BC, TT, 12, O, F), SIMT_E(BC, TT, 16, O, F), SIMT_E(BC, TT, 20, O, F)
const SimtEntry kSimt[] = {SIMT_Q16(64, 64, 0, 0), SIMT_Q16(64, 64, 1, 0), SIMT_Q16(64, 32, 0, 0),
                           SIMT_Q16(64, 32, 1, 0), SIMT_Q32(32, 64, 0, 0), SIMT_Q32(32, 64, 1, 0),
                           SIMT_Q32(32, 32, 0, 0), SIMT_Q32(32, 32, 1, 0), SIMT_Q16(64, 64, 0, 1),
                           SIMT_Q16(64, 64, 1, 1), SIMT_Q16(64, 32, 0, 1), SIMT_Q16(64, 32, 1, 1),
                           SIMT_Q16P(64, 64, 0, 1), SIMT_Q16P(64, 64, 1, 1), SIMT_Q16P(64, 32, 0, 1),
                           SIMT_Q16P(64, 32, 1, 1)};
constexpr int kNSimt = sizeof(kSimt) / sizeof(kSimt[0]);

int simt_rows(const SimtEntry& e) { return (kThreads / (e.bc / 4)) * e.qpt; }

// usable for this model: ghat rows covered, fits in shared memory, and the
// smallest QPT of its (BC, TT, ORD) family that covers P
bool simt_usable(const DevModel& m, int i) {
  const SimtEntry& e = kSimt[i];
  if (simt_rows(e) < m.P || e.smem(m) > 227 * 1024) return false;
  for (int j = 0; j < kNSimt; ++j) {
    const SimtEntry& f = kSimt[j];
    if (f.bc == e.bc && f.tt == e.tt && f.ord == e.ord && f.qpt < e.qpt && simt_rows(f) >= m.P) return false;
  }
  return true;
}

}  // namespace

int simt_count() { return kNSimt; }
int simt_info(int i, int* bc, int* tt, int* qpt, int* ord) {
  if (i < 0 || i >= kNSimt) return -1;
  *bc = kSimt[i].bc;
  *tt = kSimt[i].tt;
  *qpt = kSimt[i].qpt;
  *ord = kSimt[i].ord;
  return 0;
}
bool simt_valid(const DevModel& m, int i) { return i >= 0 && i < kNSimt && simt_usable(m, i); }

// default before tuning: 64 chains x 64 TOAs, nested order, smallest QPT covering P;
// 32 x 32 when that does not fit
int simt_default(const DevModel& m) {
  for (int pass = 0; pass < 2; ++pass)
    for (int i = 0; i < kNSimt; ++i) {
      const SimtEntry& e = kSimt[i];
      const bool shape = pass == 0 ? (e.bc == 64 && e.tt == 64) : (e.bc == 32 && e.tt == 32);
      if (shape && e.ord == 0 && simt_usable(m, i)) return i;  // nested order, no prefetch
    }
  return -1;
}

cudaError_t launch_toa_fp32_cfg(const DevModel& m, const Scratch& s, int B, int cfg, cudaStream_t st) {
  if (cfg < 0) cfg = simt_default(m);
  if (!simt_valid(m, cfg)) return cudaErrorInvalidValue;
  return kSimt[cfg].launch(m, s, B, (kSimt[cfg].ord & 4) ? 1 : 0, st);
}

namespace {
}  // namespace

cudaError_t launch_tm_prologue(const DevModel& m, const Scratch& s, int B, int fp64, cudaStream_t st) {
  const size_t sm = sizeof(double) * (m.P + 5 * m.m_max) + sizeof(float) * 2 * m.P;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_tm_prologue, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  k_tm_prologue<<<dim3(m.npsr, B), 128, sm, st>>>(m, s.a64, s.a32, m.cw ? s.cwbs : nullptr, B, fp64);
  return cudaGetLastError();
}

cudaError_t launch_toa_fp32(const DevModel& m, const Scratch& s, int B, cudaStream_t st) {
  return launch_toa_fp32_cfg(m, s, B, -1, st);
}

cudaError_t launch_toa_fp64(const DevModel& m, const Scratch& s, int B, cudaStream_t st) {
  const size_t sm = sizeof(double) * (m.PM + m.P + 128 + 4);
  k_toa_fp64<<<dim3(m.n_units, B), 128, sm, st>>>(m, s.a64, s.gpart64, s.c2part, B);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const DevModel& m, const Scratch& s, int B, int fp64, cudaStream_t st) {
  k_reduce<<<dim3((B * m.P + 255) / 256, m.npsr), 256, 0, st>>>(m, s.gpart, s.gpart64, s.c2part, s.ghat, s.chi2, B,
                                                                  fp64);
  return cudaGetLastError();
}

}  // namespace pta
