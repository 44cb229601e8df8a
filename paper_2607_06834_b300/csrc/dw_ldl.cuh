// The double-word LDL^T sweep shared by the dense-bin factorisation (k_chol_forward_dw)
// and the CURN-transform factorisation (k_curn_forward_dw): a symmetric positive
// definite matrix A (scaled so its entries lie in (0, 1]) is overwritten by the pivots D of
// A = L D L^T (L unit lower) on its diagonal and by L^-1 below it, with every operation in
// double-word arithmetic on the FP32 pipes.
//
// Step for columns (j, j+1), whose 2x2 pivot block the previous step factored: pass A
// scales column j, updates column j+1 by it and scales that, for every row below (and
// stages each row's pair (l_ij, l_i,j+1) and each column's unscaled pair as 16-byte
// entries, even and odd indices in separate arrays so that a warp's reads of
// consecutive pairs hit distinct banks), and eliminates row j+1 of L^-1 (staging rows j
// and j+1 of L^-1 per column); pass B applies the rank-2 update in 2x2 tiles, one tile
// per thread and visit, to the trailing triangle and to the rows of L^-1 below, and
// the thread of the trailing triangle's first tile factors the next pivot block.  A
// tile row is one 16-byte load and store (rows start at even elements; a diagonal
// tile's upper entry is the even row's padding).  Two barriers per two columns.
#pragma once
#include "dwarith.cuh"
#include "pta_check.cuh"

namespace pta {

// Packed lower triangle with every row starting at an even element (row i holds i+1
// elements, padded to an even count), so that a pair of entries at an even column is
// one 16-byte access: row i starts at i(i+2)/2 (i even) or (i+1)^2/2 (i odd).
__host__ __device__ __forceinline__ int prow(int i) { return (i & 1) ? (i + 1) * (i + 1) / 2 : i * (i + 2) / 2; }

// v - (p.xy q.xy + p.zw q.zw): one element's rank-2 update from the row's (l_ij, l_i,j+1)
// and the column's two unscaled entries (or L^-1's rows j and j+1).  Both products are
// exact (hi) plus rounded cross terms (lo); the two high parts come off v.x by two
// TwoSums and everything else is summed in the low word before one renormalisation.
__device__ __forceinline__ float2 dw_upd2(float2 v, float4 p, float4 q) {
  const float P0 = __fmul_rn(p.x, q.x), P1 = __fmul_rn(p.z, q.z);
  float E0 = __fmaf_rn(p.x, q.x, -P0), E1 = __fmaf_rn(p.z, q.z, -P1);
  E0 = __fmaf_rn(p.x, q.y, E0);
  E0 = __fmaf_rn(p.y, q.x, E0);
  E1 = __fmaf_rn(p.z, q.w, E1);
  E1 = __fmaf_rn(p.w, q.z, E1);
  const float s1 = __fsub_rn(v.x, P0);  // s1 + e1 = v.x - P0
  const float t1 = __fsub_rn(s1, v.x);
  const float e1 = __fsub_rn(__fsub_rn(v.x, __fsub_rn(s1, t1)), __fadd_rn(P0, t1));
  const float s2 = __fsub_rn(s1, P1);   // s2 + e2 = s1 - P1
  const float t2 = __fsub_rn(s2, s1);
  const float e2 = __fsub_rn(__fsub_rn(s1, __fsub_rn(s2, t2)), __fadd_rn(P1, t2));
  const float lo = __fadd_rn(__fadd_rn(e1, e2), __fsub_rn(v.y, __fadd_rn(E0, E1)));
  return dw_renorm(s2, lo);
}
__device__ __forceinline__ void dw_upd2x2(float4& v, float4 p, float4 q0, float4 q1) {
  const float2 a = dw_upd2(make_float2(v.x, v.y), p, q0), b = dw_upd2(make_float2(v.z, v.w), p, q1);
  v = make_float4(a.x, a.y, b.x, b.y);
}

// packed lower index e -> (row, column) by a float square root (e < 2^22)
__device__ __forceinline__ void tri_decode_f(int e, int& i, int& j) {
  int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  if (r * (r + 1) / 2 > e) --r;
  else if ((r + 1) * (r + 2) / 2 <= e) ++r;
  i = r;
  j = e - r * (r + 1) / 2;
}

// Factor a 2x2 pivot block (a00, a10, a11) of the sweep (or the single pivot a00 when two
// is false): the pivots d0, d1 go to the triangle's diagonal (its (j+1, j) entry becomes
// L^-1's in the next pass A), and r0 = 1/d0, r1 = 1/d1, the unscaled a10, l10 and the
// pivots' square roots at true scale (sqrt(d) usc) to pv for the step that uses them;
// with Lg the step's entries of L D^(1/2) on and next to the diagonal are emitted.  A
// pivot that is not positive marks the factorisation bad and continues with 1.  nT, nL:
// the triangle's and Lg's element counts for the check build's index checks (record chk).
__device__ __forceinline__ void dw_pivot_pair(float2 a00, float2 a10, float2 a11, bool two, float2* T, int j,
                                               float2* pv, int* s_bad, float2* Lg, float usc, int nT = 0,
                                               int nL = 0, long long* chk = nullptr) {
  int bad = !(a00.x > 0.0f);
  if (bad) a00 = make_float2(1.0f, 0.0f);
  const float2 r0 = dw_recip(a00);
  float2 sq0 = dw_sqrt(a00);
  sq0 = make_float2(sq0.x * usc, sq0.y * usc);
  if (PTA_IN(chk, prow(j) + j, nT, kChkSweepT)) T[prow(j) + j] = a00;
  const int tj = j * (j + 1) / 2;
  if (Lg && PTA_IN(chk, tj + j, nL, kChkSweepLg)) Lg[tj + j] = sq0;
  if (two) {
    const float2 l10 = dw_mul(a10, r0);
    float2 d1 = dw_fms(a11, l10, a10);
    if (!(d1.x > 0.0f)) {
      bad = 1;
      d1 = make_float2(1.0f, 0.0f);
    }
    float2 sq1 = dw_sqrt(d1);
    sq1 = make_float2(sq1.x * usc, sq1.y * usc);
    if (PTA_IN(chk, prow(j + 1) + j + 1, nT, kChkSweepT)) T[prow(j + 1) + j + 1] = d1;
    if (Lg && PTA_IN(chk, tj + 2 * j + 2, nL, kChkSweepLg)) {
      Lg[tj + 2 * j + 1] = dw_mul(l10, sq0);  // (j+1, j)
      Lg[tj + 2 * j + 2] = sq1;           // (j+1, j+1)
    }
    pv[0] = r0;
    pv[1] = dw_recip(d1);
    pv[2] = a10;
    pv[3] = l10;
    pv[4] = sq0;
    pv[5] = sq1;
  }
  if (bad) *s_bad = 1;
}

// The sweep on an order-np matrix: T holds A on entry (padded packed lower, rows at
// prow(i), every even row's padding zero) and on exit D on the diagonal and L^-1 (unit
// lower, its diagonal implied) below it.  Column j of L is consumed by its step: pass A
// stages the pair (l_ij, l_i,j+1) and leaves zeros in its place, which pass B's
// eliminations of the rows below turn into L^-1's entries (X_{i,c} -= l_ij X_jc +
// l_i,j+1 X_j+1,c for c <= j+1, with X_jj = X_j+1,j+1 = 1 and X_j,j+1 = 0).  With Lg the
// entries of L D^(1/2) (double words, plain packing, true scale: sqrt(d) usc, usc =
// 2^(E/2) for A scaled by 2^-E) are written to global memory as the steps produce them.
// stage: 6 (np/2 + 1) float4 of shared memory; pv: 6 float2 of shared memory; s_bad: shared
// flag set when a pivot is not positive (the sweep goes on with 1).  trimap:
// packed-lower index -> (row << 8) | column for the ((np-1)/2 + 1) ((np-1)/2 + 2) / 2 tiles
// of the largest trailing triangle, or nullptr to decode by a square root.  Called by every
// thread of the block after a barrier that follows the fill of T; returns after a barrier.
// chk: the check build's index-check record (bounds: prow(np) triangle elements, nh staging
// entries per array, np (np + 1) / 2 elements of Lg).
__device__ __forceinline__ void dw_ldl_sweep(int np, float2* T, float4* stage, float2* pv, int* s_bad,
                                           const unsigned short* trimap, float2* Lg, float usc,
                                           long long* chk = nullptr) {
  const int tid = threadIdx.x, nt = blockDim.x, nh = np / 2 + 1;
  const int nTri = prow(np), nL = np * (np + 1) / 2;
  float4* plE = stage;     // [nh] (l_ij, l_i,j+1) of rows j+2+e, e even (index e/2)
  float4* plO = plE + nh;  // e odd
  float4* uuE = plO + nh;  // [nh] unscaled (u_j, u_j+1) of columns j+2+f, f even
  float4* uuO = uuE + nh;  // f odd
  float4* xrE = uuO + nh;  // [nh] (X_jc, X_j+1,c), c even
  float4* xrO = xrE + nh;  // c odd
  if (tid == 0)
    dw_pivot_pair(T[0], np > 1 ? T[2] : T[0], np > 1 ? T[3] : T[0], np > 1, T, 0, pv, s_bad, Lg, usc, nTri, nL, chk);
  __syncthreads();
  for (int j = 0; j + 1 < np; j += 2) {
    const float2 r0 = pv[0], r1 = pv[1], a10 = pv[2], l10 = pv[3], sq0 = pv[4], sq1 = pv[5];
    const int rj = prow(j), rj1 = prow(j + 1), s2 = np - j - 2;
    // pass A
    for (int e = tid; e < s2 + j + 2; e += nt) {
      if (e < s2) {
        const int i = j + 2 + e;
        float4* ap = reinterpret_cast<float4*>(T + prow(i) + j);
        const bool ok = PTA_IN(chk, prow(i) + j + 1, nTri, kChkSweepT) && PTA_IN(chk, e >> 1, nh, kChkSweepStage);
        const float4 a = ok ? *ap : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const float2 a0 = make_float2(a.x, a.y);
        const float2 l0 = dw_mul(a0, r0);
        const float2 w = dw_fms(make_float2(a.z, a.w), l0, a10);
        const float2 l1 = dw_mul(w, r1);
        const float4 pl = make_float4(l0.x, l0.y, l1.x, l1.y);
        if (ok) {
          *ap = make_float4(0.0f, 0.0f, 0.0f, 0.0f);  // L^-1's entries (i, j), (i, j+1) start at 0
          if (Lg && PTA_IN(chk, i * (i + 1) / 2 + j + 1, nL, kChkSweepLg)) {
            const int ti = i * (i + 1) / 2 + j;
            Lg[ti] = dw_mul(l0, sq0);
            Lg[ti + 1] = dw_mul(l1, sq1);
          }
          (e & 1 ? plO : plE)[e >> 1] = pl;
          (e & 1 ? uuO : uuE)[e >> 1] = make_float4(a0.x, a0.y, w.x, w.y);
        }
      } else {
        const int c = e - s2;  // 0 .. j+1: row j+1 of L^-1 and the staged rows j, j+1
        float2 xj = make_float2(0.0f, 0.0f), x1 = make_float2(1.0f, 0.0f);
        if (!PTA_IN(chk, rj1 + c, nTri, kChkSweepT) || !PTA_IN(chk, c >> 1, nh, kChkSweepStage)) continue;
        if (c < j) {
          xj = T[rj + c];
          x1 = dw_fms(T[rj1 + c], l10, xj);
          T[rj1 + c] = x1;
        } else if (c == j) {  // X_jj = 1, X_j+1,j = -l_j+1,j (the triangle holds d_j and A there)
          xj = make_float2(1.0f, 0.0f);
          x1 = dw_neg(l10);
          T[rj1 + c] = x1;
        }
        (c & 1 ? xrO : xrE)[c >> 1] = make_float4(xj.x, xj.y, x1.x, x1.y);
      }
    }
    if (tid == 0 && (s2 & 1)) plO[s2 >> 1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);  // the odd row's partner
    __syncthreads();
    // pass B: 2x2 tiles; nT row pairs (the last one short when s2 is odd), W = (j+2)/2
    // column pairs of L^-1 (tile rows i0 are even: row i0 starts at i0(i0+2)/2 and row
    // i0+1 at (i0+2)^2/2)
    const int nT = (s2 + 1) >> 1, cntT = nT * (nT + 1) / 2, W = (j + 2) >> 1, cnt = cntT + nT * W;
    const float rw = __fdividef(1.0f, (float)W);  // the quotient below is corrected by +-1
    for (int t = tid; t < cnt; t += nt) {
      if (t < cntT) {
        int I, L;
        if (trimap) {
          const unsigned tm = trimap[t];
          I = tm >> 8;
          L = tm & 255;
        } else {
          tri_decode_f(t, I, L);
        }
        const int i0 = j + 2 + 2 * I, c0 = j + 2 + 2 * L;
        if (!PTA_IN(chk, I, nh, kChkSweepStage) || !PTA_IN(chk, L, nh, kChkSweepStage) ||
            !PTA_IN(chk, (2 * I + 1 < s2 ? (i0 + 2) * (i0 + 2) / 2 : i0 * (i0 + 2) / 2) + c0 + 1, nTri, kChkSweepT))
          continue;
        const float4 p0 = plE[I], p1 = plO[I], q0 = uuE[L], q1 = uuO[L];
        float4* r0p = reinterpret_cast<float4*>(T + i0 * (i0 + 2) / 2 + c0);
        float4 v0 = *r0p;
        dw_upd2x2(v0, p0, q0, q1);  // on a diagonal tile the second entry is the padding
        *r0p = v0;
        const bool row1 = 2 * I + 1 < s2;
        float4 v1 = v0;
        if (row1) {
          float4* r1p = reinterpret_cast<float4*>(T + (i0 + 2) * (i0 + 2) / 2 + c0);
          v1 = *r1p;
          dw_upd2x2(v1, p1, q0, q1);
          *r1p = v1;
        }
        if (t == 0)
          dw_pivot_pair(make_float2(v0.x, v0.y), make_float2(v1.x, v1.y), make_float2(v1.z, v1.w), row1, T, j + 2,
                         pv, s_bad, Lg, usc, nTri, nL, chk);
      } else {
        const int e = t - cntT;
        int q = (int)(((float)e + 0.5f) * rw);
        q -= (q * W > e);
        q += ((q + 1) * W <= e);
        const int cc = e - q * W, i0 = j + 2 + 2 * q, c0 = 2 * cc;
        if (!PTA_IN(chk, q, nh, kChkSweepStage) || !PTA_IN(chk, cc, nh, kChkSweepStage) ||
            !PTA_IN(chk, (2 * q + 1 < s2 ? (i0 + 2) * (i0 + 2) / 2 : i0 * (i0 + 2) / 2) + c0 + 1, nTri, kChkSweepT))
          continue;
        const float4 p0 = plE[q], p1 = plO[q], q0 = xrE[cc], q1 = xrO[cc];
        float4* r0p = reinterpret_cast<float4*>(T + i0 * (i0 + 2) / 2 + c0);
        float4 v0 = *r0p;
        dw_upd2x2(v0, p0, q0, q1);
        *r0p = v0;
        if (2 * q + 1 < s2) {
          float4* r1p = reinterpret_cast<float4*>(T + (i0 + 2) * (i0 + 2) / 2 + c0);
          float4 v1 = *r1p;
          dw_upd2x2(v1, p1, q0, q1);
          *r1p = v1;
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace pta
