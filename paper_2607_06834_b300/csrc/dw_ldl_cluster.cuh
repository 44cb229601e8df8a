// The double-word LDL^T sweep of dw_ldl.cuh for a matrix whose triangle is larger than one
// CTA's shared memory: the C CTAs of a thread-block cluster hold it together, row pair r
// (rows 2r and 2r+1) in the shared memory of CTA r mod C, and each step sends what it stages
// (the unscaled column pair, rows j and j+1 of L^-1, the next pivot block's entries) to every
// CTA of the cluster through distributed shared memory.  A row pair r carries r + 1 tiles of
// pass B in every step it takes part in (I + 1 in the trailing triangle, I = r - (j+2)/2, and
// (j+2)/2 column pairs of L^-1), so interleaving the row pairs splits each step's work evenly.
// Every element sees the same operations in the same order as in dw_ldl_sweep; a cluster
// barrier (release / acquire, which also orders the remote stores) separates pass A from pass
// B, and a barrier of the CTA ends each step.
#pragma once
#include <stdint.h>

#include "dw_ldl.cuh"
#include "pta_check.cuh"

namespace pta {

__device__ __forceinline__ int cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return (int)r;
}
// every thread of every CTA of the cluster; orders shared-memory accesses across the cluster
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// the shared::cluster address of the object at p in CTA q's shared memory
__device__ __forceinline__ uint32_t cl_map(const void* p, int q) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t d;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(q));
  return d;
}
__device__ __forceinline__ void cl_st4(uint32_t a, float4 v) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}
__device__ __forceinline__ float2 cl_ld2(uint32_t a) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ double cl_ldd(uint32_t a) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
  return v;
}
// a 16-byte entry of the staging, written at the same offset in every CTA of the cluster
template <int C>
__device__ __forceinline__ void cl_bcast4(float4* p, float4 v) {
#pragma unroll
  for (int q = 0; q < C; ++q) cl_st4(cl_map(p, q), v);
}

// Offset (float2 units) of row i in the shared memory of the CTA that holds it (rank
// (i/2) mod C): that CTA's row pairs k, k+C, k+2C, ... lie one after another, pair r taking
// 4 (r + 1) elements (row 2r padded to 2r + 2 as in prow, row 2r + 1 holding 2r + 2), so the
// m-th starts at sum_{m' < m} 4 (k + C m' + 1) = 4 m (k + 1) + 2 C m (m - 1).
template <int C>
__host__ __device__ __forceinline__ int crow(int i) {
  const int r = i >> 1, k = r % C, mm = r / C;
  return 4 * mm * (k + 1) + 2 * C * mm * (mm - 1) + ((i & 1) ? 2 * (r + 1) : 0);
}
// number of row pairs, and float2 elements, that rank k holds of an order-np triangle
template <int C>
__host__ __device__ __forceinline__ int cpairs(int np, int k) {
  const int npairs = (np + 1) >> 1;
  return npairs > k ? (npairs - k + C - 1) / C : 0;
}
template <int C>
__host__ __device__ __forceinline__ int cpart(int np, int k) {
  const int M = cpairs<C>(np, k);
  return 4 * M * (k + 1) + 2 * C * M * (M - 1);
}

// float4 entries of a CTA's staging area: (l_ij, l_i,j+1) of its rows (plE, plO), then two sets
// (alternate steps) of what other CTAs write into it: the unscaled column pair (uuE, uuO),
// rows j and j+1 of L^-1 (xrE, xrO), and the next pivot block's rows before their last update
// with their (l_ij, l_i,j+1) (4 entries)
__host__ __device__ __forceinline__ int cstage_f4(int np) { return 10 * (np / 2 + 1) + 8; }

// The factorisation of a 2x2 pivot block (a00, a10, a11), or of the single pivot a00 when two
// is false, as dw_pivot_pair does it: the pivots d0, d1 (1 in place of one that is not
// positive, with bad set) and the step's (1/d0, 1/d1) and (a10, l10).
__device__ __forceinline__ void dwc_pivot(float2 a00, float2 a10, float2 a11, bool two, float2& d0, float2& d1,
                                          float4& ra, float4& rb, int& bad) {
  bad = !(a00.x > 0.0f);
  d0 = bad ? make_float2(1.0f, 0.0f) : a00;
  const float2 r0 = dw_recip(d0);
  float2 r1 = make_float2(0.0f, 0.0f), l10 = r1;
  d1 = r1;
  if (two) {
    l10 = dw_mul(a10, r0);
    d1 = dw_fms(a11, l10, a10);
    if (!(d1.x > 0.0f)) {
      bad = 1;
      d1 = make_float2(1.0f, 0.0f);
    }
    r1 = dw_recip(d1);
  }
  ra = make_float4(r0.x, r0.y, r1.x, r1.y);
  rb = make_float4(a10.x, a10.y, l10.x, l10.y);
}

// The sweep of dw_ldl_sweep on an order-np matrix held by the cluster: T is this CTA's part
// (rows at crow<C>(i), even rows' padding zero on entry), stage cstage_f4(np) float4 and pv
// 4 float2 (16-byte aligned) of shared memory at the same offsets in every CTA, s_bad this
// CTA's flag for a pivot that is not positive.  On exit T holds D on the diagonal and L^-1
// below it for this CTA's rows.  One cluster barrier per step, between pass A and pass B: the
// CTA holding rows j+2 and j+3 sends, in pass A, their pivot-block entries before the step's
// update, and every CTA updates and factors that block itself in pass B (the same operations
// as the owner's tile (0, 0), so the same bits), so pass B ends with a CTA barrier; the
// staging that other CTAs write alternates between two sets, so a CTA that runs a step ahead
// never overwrites what a slower one still reads.  Called by every thread of every CTA of the
// cluster after the fill of T (it begins with a cluster barrier); returns after a barrier of
// its own CTA.  chk: the check build's index-check record (bounds: cpart<C>(np, k) elements of
// T, nh entries per staging array).
template <int C>
__device__ __forceinline__ void dwc_ldl_sweep(int np, float2* T, float4* stage, float2* pv, int* s_bad,
                                              long long* chk = nullptr) {
  const int tid = threadIdx.x, nt = blockDim.x, nh = np / 2 + 1, k = cl_rank(), npairs = (np + 1) >> 1;
  const int nPart = cpart<C>(np, k);
  float4* plE = stage;     // [nh] (l_ij, l_i,j+1) of this CTA's rows j+2+e, e even (index e/2)
  float4* plO = plE + nh;  // e odd
  float4* pv4 = reinterpret_cast<float4*>(pv);
  cl_sync();  // every CTA has started and filled its rows
  if (k == 0 && tid == 0) {
    float2 d0, d1;
    float4 ra, rb;
    int bad;
    dwc_pivot(T[0], np > 1 ? T[2] : T[0], np > 1 ? T[3] : T[0], np > 1, d0, d1, ra, rb, bad);
    T[0] = d0;
    if (np > 1) T[3] = d1;
    if (bad) *s_bad = 1;
    cl_bcast4<C>(pv4, ra);
    cl_bcast4<C>(pv4 + 1, rb);
  }
  cl_sync();
  for (int j = 0; j + 1 < np; j += 2) {
    const float2 r0 = pv[0], r1 = pv[1], a10 = pv[2], l10 = pv[3];
    float4* uuE = plO + nh + ((j >> 1) & 1) * (4 * nh + 4);  // this step's set: [nh] unscaled (u_j, u_j+1) of columns j+2+f, f even
    float4* uuO = uuE + nh;                                  // f odd
    float4* xrE = uuO + nh;                                  // [nh] (X_jc, X_j+1,c), c even
    float4* xrO = xrE + nh;                                  // c odd
    float4* pb = xrO + nh;  // rows j+2, j+3 of the next pivot block before the update, then their l pairs
    const int s2 = np - j - 2, R0 = (j + 2) >> 1;
    int d = (k - R0) % C;
    if (d < 0) d += C;
    const int rf = R0 + d;                                      // this CTA's first trailing row pair
    const int nr = rf < npairs ? (npairs - 1 - rf) / C + 1 : 0;  // and how many it holds
    const bool xown = ((j >> 1) % C) == k;                      // rows j and j+1 are here
    // pass A: this CTA's trailing rows, then (where rows j, j+1 are) row j+1 of L^-1
    const int nA = 2 * nr + (xown ? j + 2 : 0);
    for (int t = tid; t < nA; t += nt) {
      if (t < 2 * nr) {
        const int i = 2 * (rf + C * (t >> 1)) + (t & 1);
        if (i < np && PTA_IN(chk, crow<C>(i) + j + 3, nPart, kChkClusterT) &&
            PTA_IN(chk, (i - j - 2) >> 1, nh, kChkClusterStage)) {
          const int e = i - j - 2;
          float4* ap = reinterpret_cast<float4*>(T + crow<C>(i) + j);
          const float4 a = *ap;
          const float2 a0 = make_float2(a.x, a.y);
          const float2 l0 = dw_mul(a0, r0);
          const float2 w = dw_fms(make_float2(a.z, a.w), l0, a10);
          const float2 l1 = dw_mul(w, r1);
          const float4 pl = make_float4(l0.x, l0.y, l1.x, l1.y);
          *ap = make_float4(0.0f, 0.0f, 0.0f, 0.0f);  // L^-1's entries (i, j), (i, j+1) start at 0
          (e & 1 ? plO : plE)[e >> 1] = pl;
          cl_bcast4<C>((e & 1 ? uuO : uuE) + (e >> 1), make_float4(a0.x, a0.y, w.x, w.y));
          if (e < 2) {  // rows j+2, j+3: the next pivot block
            cl_bcast4<C>(pb + e, *reinterpret_cast<const float4*>(T + crow<C>(i) + j + 2));
            cl_bcast4<C>(pb + 2 + e, pl);
          }
        }
      } else {
        const int c = t - 2 * nr;  // 0 .. j+1
        const int rj = crow<C>(j), rj1 = crow<C>(j + 1);
        if (!PTA_IN(chk, rj1 + c, nPart, kChkClusterT) || !PTA_IN(chk, c >> 1, nh, kChkClusterStage)) continue;
        float2 xj = make_float2(0.0f, 0.0f), x1 = make_float2(1.0f, 0.0f);
        if (c < j) {
          xj = T[rj + c];
          x1 = dw_fms(T[rj1 + c], l10, xj);
          T[rj1 + c] = x1;
        } else if (c == j) {  // X_jj = 1, X_j+1,j = -l_j+1,j
          xj = make_float2(1.0f, 0.0f);
          x1 = dw_neg(l10);
          T[rj1 + c] = x1;
        }
        cl_bcast4<C>((c & 1 ? xrO : xrE) + (c >> 1), make_float4(xj.x, xj.y, x1.x, x1.y));
      }
    }
    if (tid == 0 && (s2 & 1) && (npairs - 1) % C == k) {  // the odd last row's missing partner
      plO[s2 >> 1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      cl_bcast4<C>(uuO + (s2 >> 1), make_float4(0.0f, 0.0f, 0.0f, 0.0f));
      if (s2 == 1) cl_bcast4<C>(pb + 3, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
    }
    cl_sync();
    // pass B: row pair rf + C u carries n0 + C u tiles (n0 = rf + 1), the first S(u) = n0 u +
    // C u (u - 1) / 2 tiles belong to the pairs before it; the trailing tiles of a pair come
    // first, then its L^-1 tiles.
    const int n0 = rf + 1, cnt = nr * n0 + C * nr * (nr - 1) / 2;
    const float bq = (float)n0 - 0.5f * (float)C;
    for (int t = tid; t < cnt; t += nt) {
      int u = (int)((sqrtf(bq * bq + 2.0f * (float)C * (float)t) - bq) * (1.0f / (float)C));
      if (n0 * u + C * u * (u - 1) / 2 > t) --u;
      else if (n0 * (u + 1) + C * (u + 1) * u / 2 <= t) ++u;
      const int s = t - (n0 * u + C * u * (u - 1) / 2);
      const int r = rf + C * u, I = r - R0, i0 = 2 * r;
      const int b0 = crow<C>(i0), b1 = b0 + 2 * (r + 1);
      const bool row1 = i0 + 1 < np;
      if (!PTA_IN(chk, I, nh, kChkClusterStage) || !PTA_IN(chk, s <= I ? s : s - I - 1, nh, kChkClusterStage) ||
          !PTA_IN(chk, (row1 ? b1 : b0) + (s <= I ? j + 2 + 2 * s : 2 * (s - I - 1)) + 1, nPart, kChkClusterT))
        continue;
      const float4 p0 = plE[I], p1 = plO[I];
      float4 q0, q1;
      int c0;
      if (s <= I) {  // trailing tile (I, s)
        c0 = j + 2 + 2 * s;
        q0 = uuE[s];
        q1 = uuO[s];
      } else {  // L^-1 tile: columns 2 cc, 2 cc + 1
        const int cc = s - I - 1;
        c0 = 2 * cc;
        q0 = xrE[cc];
        q1 = xrO[cc];
      }
      float4* r0p = reinterpret_cast<float4*>(T + b0 + c0);
      float4 v0 = *r0p;
      dw_upd2x2(v0, p0, q0, q1);  // on a diagonal tile the second entry is the padding
      *r0p = v0;
      float4 v1 = v0;
      if (row1) {
        float4* r1p = reinterpret_cast<float4*>(T + b1 + c0);
        v1 = *r1p;
        dw_upd2x2(v1, p1, q0, q1);
        *r1p = v1;
      }
      if (s == 0 && I == 0) {  // the owner keeps the next pivots on its diagonal
        float2 d0, d1;
        float4 ra, rb;
        int bad;
        dwc_pivot(make_float2(v0.x, v0.y), make_float2(v1.x, v1.y), make_float2(v1.z, v1.w), row1, d0, d1, ra, rb,
                  bad);
        T[b0 + j + 2] = d0;
        if (row1) T[b1 + j + 3] = d1;
        if (bad) *s_bad = 1;
      }
    }
    if (tid == nt - 1 && s2 > 0) {  // every CTA: the next pivot block, updated and factored as in tile (0, 0)
      const bool two = s2 > 1;
      float4 v0 = pb[0], v1;
      dw_upd2x2(v0, pb[2], uuE[0], uuO[0]);
      v1 = v0;
      if (two) {
        v1 = pb[1];
        dw_upd2x2(v1, pb[3], uuE[0], uuO[0]);
      }
      float2 d0, d1;
      float4 ra, rb;
      int bad;
      dwc_pivot(make_float2(v0.x, v0.y), make_float2(v1.x, v1.y), make_float2(v1.z, v1.w), two, d0, d1, ra, rb, bad);
      pv4[0] = ra;
      pv4[1] = rb;
    }
    __syncthreads();
  }
}

}  // namespace pta
