// CURN-posterior standardizing transform (Eq. PTA_standard_transform_curn; with a
// per-chain beta, the tempered transform T_beta of App. "The standardizing transform
// for tempered likelihoods"), FP64.  Per (pulsar I, chain b):
//   A = beta G~ + diag(1 / phi_C),  G~ = F^T N~^-1 F,
//   phi_C,p = rho_k + kappa_Ik on the two achromatic columns of bin k, kappa^DM_Ik on
//   the DM columns (the prior covariance without inter-pulsar correlations);
//   A = U U^T with U upper triangular and W = U^-1, so that L_CURN = W^T is the lower
//   Cholesky factor of Sigma_CURN = A^-1;
//   a = ahat + W^T z, ahat = beta W^T W g (g = F^T N~^-1 dt), log det L_CURN = sum log W_pp.
// The density (Eq. standardized_stochastic_posterior) is the likelihood times the
// Hellings-Downs prior N(a; 0, phi) times det L_CURN; the prior term is evaluated per
// frequency bin with the factors of Phi_k from the prior stage.
//
// Reversed order.  With p' = P-1-p the upper factor U becomes a lower one:
// A' = J A J = L' D L'^T (LDL^T, L' unit lower) and Y' = D^-1/2 L'^-1 = J W J.  The
// factorisation and the inverse share one packed lower triangle: in the LDL^T sweep
// column j of L' is consumed by step j, and the inverse's column j (-l_ij) takes its
// place, so at every step the triangle holds the trailing part of A' and the finished
// rows of L'^-1.  P^3/3 FP64 multiply-adds per (pulsar, chain), the same count as a
// Cholesky factorisation plus a triangular inverse.  The triangle lives in shared
// memory when it fits, else in the per-(pulsar, chain) slot of the global inverse
// buffer (L2-resident for the CTAs in flight).
//
// Gradient.  With gbar = d logp / d a = beta F^T N~^-1 r - phi^-1 a (likelihood and HD
// prior), d logp / d z = W gbar, and for the diagonal d_p = 1 / phi_C,p of A
//   d logp / d d_p = -(A^-1 gbar)_p ahat_p
//                    - sum_{i<j<=p} W_ip z_i s_j W_jp - 1/2 sum_i W_ip^2 (z_i s_i + 1),
// s = W gbar (from dahat = -A^-1 dA ahat, dW^T = -W^T Psi(W dA W^T)^T with Psi the
// upper triangle and half the diagonal, and d log det L_CURN = -1/2 tr(A^-1 dA)): the
// columns of W give every p in O(P^2).
#include <algorithm>
#include <cmath>

#include "dw_ldl.cuh"
#include "dw_ldl_cluster.cuh"
#include "dwarith.cuh"
#include "pta_internal.cuh"

namespace pta {
namespace {

constexpr int kCT = 128;  // threads per (pulsar, chain) CTA

__device__ __forceinline__ int trl(int i, int j) { return i * (i + 1) / 2 + j; }

// packed lower index e -> (row, column), e < 2^23
__device__ __forceinline__ void tri_decode(int e, int& i, int& j) {
  int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  if (r * (r + 1) / 2 > e) --r;
  else if ((r + 1) * (r + 2) / 2 <= e) ++r;
  i = r;
  j = e - r * (r + 1) / 2;
}

// position in x of the z entry of coefficient p of pulsar I (prior-whitened layout)
__device__ __forceinline__ int zidx(const DevModel& m, int I, int p) {
  if (p < 2 * m.na) return m.z_ach + p * m.npsr + I;
  const int q = p - 2 * m.na;
  return m.z_dm + (I * m.nd + (q >> 1)) * 2 + (q & 1);
}

// phi_CURN of coefficient p of pulsar I for chain b
__device__ __forceinline__ double phic(const DevModel& m, const double* sk, const double* skd,
                                       const double* srho, int b, int I, int p) {
  if (p < 2 * m.na) {
    const int k = p >> 1;
    const double r = srho[(size_t)b * m.na + k], q = sk[((size_t)b * m.npsr + I) * m.na + k];
    return fma(r, r, q * q);
  }
  const double q = skd[((size_t)b * m.npsr + I) * m.nd + ((p - 2 * m.na) >> 1)];
  return q * q;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];  // fixed order
  return s;
}

// ---------------------------------------------------------------------------
// Forward: factor, inverse, a = ahat + W^T z, ahat, log det L_CURN.  Grid (npsr, B).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kCT)
    k_curn_forward(DevModel m, const float* __restrict__ x, const double* __restrict__ sk,
                   const double* __restrict__ skd, const double* __restrict__ srho, double* a64, double* Wg,
                   double* ahat, double* ld, int32_t* stat, const double* __restrict__ g0, int B, int in_smem) {
  extern __shared__ double sm[];
  __shared__ int s_bad;
  __shared__ double red[kCT / 32];
  const int I = blockIdx.x, b = blockIdx.y, tid = threadIdx.x, P = m.P;
  const int ntri = P * (P + 1) / 2;
  const size_t o = (size_t)I * B + b;
  double* Wslot = Wg + o * ntri;
  double* T = in_smem ? sm : Wslot;
  double* d = in_smem ? sm + ntri : sm;  // pivots d_j, then d_j^-1/2
  double* rd = d + P;                     // diagonal prior precision, then 1/d_j
  double* u = rd + P;                     // unscaled column j
  double* lc = u + P;                     // l_ij of column j
  double* gp = lc + P;                    // g, reversed
  double* zp = gp + P;                    // z, reversed
  double* up = zp + P;                    // Y' g'
  double* tp = up + P;                    // beta Y' g' + z'
  const double bt = m.beta ? m.beta[b] : 1.0;
  const double gsc = g0 ? 1.0 : bt;  // factor of Y'^T Y' g in the mean
  const float* xb = x + (size_t)b * m.d;
  const double* G = m.Grev + (size_t)I * ntri;
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int i = tid; i < P; i += kCT) {
    const int p = P - 1 - i;
    const double ph = phic(m, sk, skd, srho, b, I, p);
    double dv = 1.0;
    if (ph > 0.0 && ph < INFINITY)
      dv = 1.0 / ph;
    else
      s_bad = 1;
    rd[i] = dv;
    // g = F^T N~^-1 dt, or with the deterministic signal the already beta-scaled
    // beta F^T N~^-1 (dt - h) = g0 + beta G~ a_ref (Eq. decenter_det_PTA)
    gp[i] = g0 ? fma(bt, m.ga[(size_t)I * P + p], g0[o * P + p]) : m.gt[(size_t)I * P + p];
    zp[i] = (double)xb[zidx(m, I, p)];
  }
  __syncthreads();
  for (int e = tid; e < ntri; e += kCT) {
    int i, j;
    tri_decode(e, i, j);
    const double v = bt * G[e];
    T[e] = (i == j) ? v + rd[i] : v;
  }
  __syncthreads();
  if (tid == 0) {
    double dd = T[0];
    if (!(dd > 0.0)) {
      s_bad = 1;
      dd = 1.0;
    }
    d[0] = dd;
    rd[0] = recip64(dd);
  }
  __syncthreads();
  for (int j = 0; j < P; ++j) {
    const double r = rd[j];
    const int s = P - 1 - j;
    for (int e = tid; e < s; e += kCT) {
      const int i = j + 1 + e;
      const double v = T[trl(i, j)];
      const double l = v * r;
      u[i] = v;
      lc[i] = l;
      T[trl(i, j)] = -l;  // column j of L'^-1
    }
    __syncthreads();
    // trailing triangle (rank-1 update) and the rows of L'^-1 below j (columns < j)
    const int cntA = s * (s + 1) / 2, w = j, cnt = cntA + s * w;
    const float rw = w > 0 ? 1.0f / (float)w : 0.0f;
    for (int idx = tid; idx < cnt; idx += kCT) {
      if (idx < cntA) {
        int ii, ll;
        tri_decode(idx, ii, ll);
        const int i = j + 1 + ii, l = j + 1 + ll;
        const double v = fma(-lc[i], u[l], T[trl(i, l)]);
        if (idx == 0) {  // (j+1, j+1) receives its last update: the next pivot
          double dd = v;
          if (!(dd > 0.0)) {
            s_bad = 1;
            dd = 1.0;
          }
          T[trl(i, l)] = dd;
          d[j + 1] = dd;
          rd[j + 1] = recip64(dd);
        } else {
          T[trl(i, l)] = v;
        }
      } else {
        const int e = idx - cntA;
        int q = (int)(((float)e + 0.5f) * rw);
        q -= (q * w > e);
        q += ((q + 1) * w <= e);
        const int i = j + 1 + q, c = e - q * w;
        T[trl(i, c)] = fma(-lc[i], T[trl(j, c)], T[trl(i, c)]);
      }
    }
    __syncthreads();
  }
  for (int i = tid; i < P; i += kCT) d[i] = rsqrt64(d[i]);
  __syncthreads();
  // Y' = D^-1/2 L'^-1 (unit diagonal implied in the sweep)
  for (int e = tid; e < ntri; e += kCT) {
    int i, j;
    tri_decode(e, i, j);
    T[e] = (i == j) ? d[i] : T[e] * d[i];
  }
  __syncthreads();
  for (int i = tid; i < P; i += kCT) {
    const double* row = T + trl(i, 0);
    double sacc = 0.0;
    for (int c = 0; c <= i; ++c) sacc = fma(row[c], gp[c], sacc);
    up[i] = sacc;
    tp[i] = fma(gsc, sacc, zp[i]);
  }
  __syncthreads();
  for (int c = tid; c < P; c += kCT) {
    double sa = 0.0, sh = 0.0;
    for (int i = c; i < P; ++i) {
      const double y = T[trl(i, c)];
      sa = fma(y, tp[i], sa);
      sh = fma(y, up[i], sh);
    }
    const int p = P - 1 - c;
    a64[o * m.PM + p] = sa;
    ahat[o * P + p] = gsc * sh;
  }
  double acc = 0.0;
  for (int i = tid; i < P; i += kCT) acc += log(d[i]);
  acc = block_sum(acc, red);
  if (tid == 0) {
    ld[o] = acc;
    if (s_bad) atomicOr(&stat[b], 2);
  }
  if (in_smem)
    for (int e = tid; e < ntri; e += kCT) Wslot[e] = T[e];
}

// ---------------------------------------------------------------------------
// The forward of k_curn_forward with the factorisation in double-word arithmetic on the
// FP32 pipes (dw_ldl_sweep, one triangle, on A' scaled by 2^-E, E even, from its largest
// diagonal entry), the inverse's scaling, both triangular products and the transform in double
// words; outputs as k_curn_forward except Y', which the W slot holds as float pairs for
// k_curn_adjoint_dw (log det L_CURN in FP64).  Used outside FP64 mode when the two
// triangles fit in shared memory.
// ---------------------------------------------------------------------------
constexpr int kCTdw = 128;

__global__ void __launch_bounds__(kCTdw)
    k_curn_forward_dw(DevModel m, const float* __restrict__ x, const double* __restrict__ sk,
                      const double* __restrict__ skd, const double* __restrict__ srho, double* a64, double* Wg,
                      double* ahat, double* ld, int32_t* stat, const double* __restrict__ g0, int B) {
  extern __shared__ float4 smq[];
  __shared__ float2 pv[6];
  __shared__ int s_bad;
  __shared__ double red[kCTdw / 32];
  const int I = blockIdx.x, b = blockIdx.y, tid = threadIdx.x, nt = blockDim.x, P = m.P;
  const int ntri = P * (P + 1) / 2, nh = P / 2 + 1;
  float2* A = reinterpret_cast<float2*>(smq + 6 * nh);  // after the sweep's staging: one padded packed triangle
  float2* X = A;                                        // L'^-1 replaces L' in it
  const size_t o = (size_t)I * B + b;
  const double bt = m.beta ? m.beta[b] : 1.0;
  const double gsc = g0 ? 1.0 : bt;  // factor of Y'^T Y' g in the mean
  const float2 btw = d2dw_bits(bt), gscw = d2dw_bits(gsc);
  const float* xb = x + (size_t)b * m.d;
  const float2* G = m.Grev_dw + (size_t)I * ntri;
  float2* rdw = reinterpret_cast<float2*>(smq);  // [P] 1 / phi_C of reversed coefficient i (staging, free until the sweep)
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int i = tid; i < P; i += nt) {
    const double ph = phic(m, sk, skd, srho, b, I, P - 1 - i);
    float2 r = make_float2(1.0f, 0.0f);
    if (ph > 0.0 && ph < INFINITY)
      r = dw_recip(d2dw_bits(ph));
    else
      s_bad = 1;
    rdw[i] = r;
  }
  __syncthreads();
  // scale 2^-E, E even, from the largest diagonal entry (every warp computes it)
  float dmax = 0.0f;
  for (int i = tid & 31; i < P; i += 32) dmax = fmaxf(dmax, dw_add(dw_mul(btw, G[i * (i + 3) / 2]), rdw[i]).x);
  for (int off = 16; off; off >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
  int E = 0;
  if (dmax > 0.0f && dmax < INFINITY) frexpf(dmax, &E);
  E += E & 1;
  const float sc = __int_as_float((127 - E) << 23);  // 2^-E (E within the float exponent range here)
  for (int e = tid; e < ntri; e += nt) {
    int i, j;
    tri_decode_f(e, i, j);
    float2 v = dw_mul(btw, G[e]);
    if (i == j) v = dw_add(v, rdw[i]);
    const int q = prow(i) + j;
    A[q] = make_float2(v.x * sc, v.y * sc);
    if (i == j && !(i & 1)) A[q + 1] = make_float2(0.0f, 0.0f);
  }
  __syncthreads();
  dw_ldl_sweep(P, A, smq, pv, &s_bad, nullptr, nullptr, 1.0f, m.chk);
  // 1 / sqrt(d_i) at the true scale, g and z in reversed order (the staging area is free)
  float2* rqw = reinterpret_cast<float2*>(smq);  // [P]
  float2* gpw = rqw + P;                          // [P] g'
  float2* zpw = gpw + P;                          // [P] z'
  float2* upw = zpw + P;                          // [P] Y' g'
  float2* tpw = upw + P;                          // [P] gsc Y' g' + z'
  const float usc = __int_as_float((127 - E / 2) << 23);  // 2^(-E/2)
  for (int i = tid; i < P; i += nt) {
    const int p = P - 1 - i;
    const float2 r = dw_recip(dw_sqrt(A[prow(i) + i]));
    rqw[i] = make_float2(r.x * usc, r.y * usc);
    gpw[i] = d2dw_bits(g0 ? fma(bt, m.ga[(size_t)I * P + p], g0[o * P + p]) : m.gt[(size_t)I * P + p]);
    zpw[i] = make_float2(xb[zidx(m, I, p)], 0.0f);
  }
  __syncthreads();
  // Y' = D^-1/2 L'^-1, in place of L'^-1
  for (int e = tid; e < ntri; e += nt) {
    int i, j;
    tri_decode_f(e, i, j);
    const int q = prow(i) + j;
    X[q] = (i == j) ? rqw[i] : dw_mul(X[q], rqw[i]);
  }
  __syncthreads();
  for (int i = tid; i < P; i += nt) {
    const float2* row = X + prow(i);
    float2 acc = make_float2(0.0f, 0.0f);
    for (int c = 0; c <= i; ++c) acc = dw_fms(acc, row[c], dw_neg(gpw[c]));
    upw[i] = acc;
    tpw[i] = dw_add(dw_mul(gscw, acc), zpw[i]);
  }
  __syncthreads();
  for (int c = tid; c < P; c += nt) {
    float2 sa = make_float2(0.0f, 0.0f), sh = sa;
    for (int i = c; i < P; ++i) {
      const float2 y = X[prow(i) + c];
      sa = dw_fms(sa, y, dw_neg(tpw[i]));
      sh = dw_fms(sh, y, dw_neg(upw[i]));
    }
    const int p = P - 1 - c;
    a64[o * m.PM + p] = dw2d(sa);
    ahat[o * P + p] = dw2d(dw_mul(gscw, sh));
  }
  double acc = 0.0;  // log det L_CURN = sum_i log Y'_ii
  for (int i = tid; i < P; i += nt) acc += log(dw2d(rqw[i]));
  acc = block_sum(acc, red);
  if (tid == 0) {
    ld[o] = acc;
    if (s_bad) atomicOr(&stat[b], 2);
  }
  float2* Wslot = reinterpret_cast<float2*>(Wg) + o * ntri;  // Y' as float pairs, for k_curn_adjoint_dw
  for (int e = tid; e < ntri; e += nt) {
    int i, j;
    tri_decode_f(e, i, j);
    Wslot[e] = X[prow(i) + j];
  }
}

// ---------------------------------------------------------------------------
// k_curn_forward_dw for P whose triangle exceeds one CTA's shared memory: a cluster of C
// CTAs per (pulsar, chain) holds A' by interleaved row pairs (dwc_ldl_sweep); every row
// operation after the sweep runs where the row is, the column sums of the transform are
// formed per CTA over its rows and added across the cluster in rank order, and each CTA
// writes its rows of Y' to the W slot.  Grid (npsr C, B), cluster (C, 1, 1), NT threads
// (at most 64 registers: one 1024-thread CTA, or two 512-thread CTAs, per SM).
// ---------------------------------------------------------------------------
template <int C, int NT>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(NT, 1024 / NT)
    k_curn_forward_dwc(DevModel m, const float* __restrict__ x, const double* __restrict__ sk,
                       const double* __restrict__ skd, const double* __restrict__ srho, double* a64, double* Wg,
                       double* ahat, double* ld, int32_t* stat, const double* __restrict__ g0, int B) {
  extern __shared__ float4 smq[];
  __shared__ __align__(16) float2 pv[4];
  __shared__ int s_bad;
  __shared__ double red[NT / 32];
  __shared__ double s_ld;
  const int k = cl_rank(), I = blockIdx.x / C, b = blockIdx.y, tid = threadIdx.x, nt = blockDim.x, P = m.P;
  const int lane = tid & 31, wp = tid >> 5, nw = nt >> 5;
  const int nrow = 2 * cpairs<C>(P, k);  // this CTA's rows 2 (k + C m) + h, m < nrow / 2, h = 0, 1
  float2* part = reinterpret_cast<float2*>(smq + cstage_f4(P));  // [2P] column sums over this CTA's rows
  float2* T = part + 2 * P;                                 // this CTA's row pairs of A', then of L'^-1
  const size_t o = (size_t)I * B + b;
  const double bt = m.beta ? m.beta[b] : 1.0;
  const double gsc = g0 ? 1.0 : bt;
  const float2 btw = d2dw_bits(bt), gscw = d2dw_bits(gsc);
  const float* xb = x + (size_t)b * m.d;
  const float2* G = m.Grev_dw + (size_t)I * (P * (P + 1) / 2);
  float2* rdw = reinterpret_cast<float2*>(smq);  // [P] 1 / phi_C of reversed coefficient i
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int i = tid; i < P; i += nt) {
    const double ph = phic(m, sk, skd, srho, b, I, P - 1 - i);
    float2 r = make_float2(1.0f, 0.0f);
    if (ph > 0.0 && ph < INFINITY)
      r = dw_recip(d2dw_bits(ph));
    else
      s_bad = 1;
    rdw[i] = r;
  }
  __syncthreads();
  float dmax = 0.0f;  // the same 2^-E in every CTA of the cluster
  for (int i = lane; i < P; i += 32) dmax = fmaxf(dmax, dw_add(dw_mul(btw, G[i * (i + 3) / 2]), rdw[i]).x);
  for (int off = 16; off; off >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
  int E = 0;
  if (dmax > 0.0f && dmax < INFINITY) frexpf(dmax, &E);
  E += E & 1;
  const float sc = __int_as_float((127 - E) << 23);
  for (int rr = wp; rr < nrow; rr += nw) {  // a warp per row
    const int i = 2 * (k + C * (rr >> 1)) + (rr & 1);
    if (i >= P || !PTA_IN(m.chk, crow<C>(i) + i + ((i & 1) ? 0 : 1), cpart<C>(P, k), kChkClusterT)) continue;
    float2* row = T + crow<C>(i);
    const float2* Gi = G + i * (i + 1) / 2;
    for (int c = lane; c <= i; c += 32) {
      float2 v = dw_mul(btw, Gi[c]);
      if (c == i) v = dw_add(v, rdw[i]);
      row[c] = make_float2(v.x * sc, v.y * sc);
    }
    if (!(i & 1) && lane == 0) row[i + 1] = make_float2(0.0f, 0.0f);
  }
  dwc_ldl_sweep<C>(P, T, smq, pv, &s_bad, m.chk);
  float2* rqw = reinterpret_cast<float2*>(smq);  // [P] (this CTA's rows)
  float2* gpw = rqw + P;
  float2* zpw = gpw + P;
  float2* upw = zpw + P;  // (this CTA's rows)
  float2* tpw = upw + P;  // (this CTA's rows)
  const float usc = __int_as_float((127 - E / 2) << 23);
  for (int i = tid; i < P; i += nt) {
    const int p = P - 1 - i;
    if ((i >> 1) % C == k) {
      const float2 r = dw_recip(dw_sqrt(T[crow<C>(i) + i]));
      rqw[i] = make_float2(r.x * usc, r.y * usc);
    }
    gpw[i] = d2dw_bits(g0 ? fma(bt, m.ga[(size_t)I * P + p], g0[o * P + p]) : m.gt[(size_t)I * P + p]);
    zpw[i] = make_float2(xb[zidx(m, I, p)], 0.0f);
  }
  __syncthreads();
  for (int rr = wp; rr < nrow; rr += nw) {  // Y' = D^-1/2 L'^-1
    const int i = 2 * (k + C * (rr >> 1)) + (rr & 1);
    if (i >= P) continue;
    float2* row = T + crow<C>(i);
    const float2 ri = rqw[i];
    for (int c = lane; c <= i; c += 32) row[c] = (c == i) ? ri : dw_mul(row[c], ri);
  }
  __syncthreads();
  for (int rr = tid; rr < nrow; rr += nt) {
    const int i = 2 * (k + C * (rr >> 1)) + (rr & 1);
    if (i >= P) continue;
    const float2* row = T + crow<C>(i);
    float2 acc = make_float2(0.0f, 0.0f);
    for (int c = 0; c <= i; ++c) acc = dw_fms(acc, row[c], dw_neg(gpw[c]));
    upw[i] = acc;
    tpw[i] = dw_add(dw_mul(gscw, acc), zpw[i]);
  }
  __syncthreads();
  for (int c = tid; c < P; c += nt) {  // this CTA's rows i >= c, in increasing order
    float2 sa = make_float2(0.0f, 0.0f), sh = sa;
    int r = c >> 1;
    int d = (k - r) % C;
    if (d < 0) d += C;
    for (r += d; 2 * r < P; r += C) {
      const int b0 = crow<C>(2 * r);
      if (2 * r >= c) {
        const float2 y = T[b0 + c];
        sa = dw_fms(sa, y, dw_neg(tpw[2 * r]));
        sh = dw_fms(sh, y, dw_neg(upw[2 * r]));
      }
      if (2 * r + 1 < P) {
        const float2 y = T[b0 + 2 * (r + 1) + c];
        sa = dw_fms(sa, y, dw_neg(tpw[2 * r + 1]));
        sh = dw_fms(sh, y, dw_neg(upw[2 * r + 1]));
      }
    }
    part[c] = sa;
    part[P + c] = sh;
  }
  double acc = 0.0;
  for (int i = tid; i < P; i += nt)
    if ((i >> 1) % C == k) acc += log(dw2d(rqw[i]));
  acc = block_sum(acc, red);
  if (tid == 0) {
    s_ld = acc;
    if (s_bad) atomicOr(&stat[b], 2);
  }
  float2* Wslot = reinterpret_cast<float2*>(Wg) + o * (P * (P + 1) / 2);
  for (int rr = wp; rr < nrow; rr += nw) {
    const int i = 2 * (k + C * (rr >> 1)) + (rr & 1);
    if (i >= P) continue;
    const float2* row = T + crow<C>(i);
    if (!PTA_IN(m.chk, i * (i + 1) / 2 + i, P * (P + 1) / 2, kChkWslot)) continue;
    for (int c = lane; c <= i; c += 32) Wslot[i * (i + 1) / 2 + c] = row[c];
  }
  cl_sync();  // every CTA's column sums and log det part are in place
  for (int c = k + C * tid; c < P; c += C * nt) {
    float2 sa = make_float2(0.0f, 0.0f), sh = sa;
    for (int q = 0; q < C; ++q) {
      sa = dw_add(sa, cl_ld2(cl_map(part + c, q)));
      sh = dw_add(sh, cl_ld2(cl_map(part + P + c, q)));
    }
    const int p = P - 1 - c;
    a64[o * m.PM + p] = dw2d(sa);
    ahat[o * P + p] = dw2d(dw_mul(gscw, sh));
  }
  if (k == 0 && tid == 0) {
    double s = 0.0;
    for (int q = 0; q < C; ++q) s += cl_ldd(cl_map(&s_ld, q));
    ld[o] = s;
  }
  cl_sync();  // no CTA leaves while another reads its shared memory
}

// ---------------------------------------------------------------------------
// HD prior at the transformed coefficients, per (achromatic bin or DM block, chain):
// v = Phi_k^-1 a (stored for the gradient), the term -1/2 a^T Phi_k^-1 a - log det Phi_k
// over both columns, and its derivatives at fixed a:
//   kappa_I d/dkappa_I = kappa_I (1/2 sum_c v_cI^2 - (Phi_k^-1)_II),
//   rho d/drho = 1/2 sum_c a_c . v_c - N_p - sum_I kappa_I d/dkappa_I (scaling identity).
// Dense bins use L_k^-1 from the prior stage, GWB-only bins chol(Gamma)^-1 / sqrt(rho),
// diagonal bins 1 / kappa.  Grid (na + 1, B).
// ---------------------------------------------------------------------------
template <bool DWL>  // dense-bin inverse factors as double-word float pairs (k_chol_forward_dw)
__global__ void __launch_bounds__(kCT)
    k_curn_whiten(DevModel m, const double* __restrict__ a64, const double* __restrict__ Lipk,
                  const double* __restrict__ sk, const double* __restrict__ skd, const double* __restrict__ srho,
                  double* vbuf, double* qout, double* dlnk, double* dlnkd, double* dlnr, int B) {
  extern __shared__ double sm[];
  __shared__ double red[kCT / 32];
  const int kb = blockIdx.x, b = blockIdx.y, tid = threadIdx.x, np = m.npsr, P = m.P;
  double q = 0.0;  // this thread's part of the prior term
  if (kb == m.na) {  // DM block: Phi = kappa^DM per (pulsar, bin)
    for (int r = tid; r < np * m.nd; r += kCT) {
      const int I = r / m.nd, k = r % m.nd;
      const double s = skd[((size_t)b * np + I) * m.nd + k], kap = s * s, ik = 1.0 / kap;
      const size_t o = (size_t)I * B + b;
      const int p = 2 * m.na + 2 * k;
      const double a0 = a64[o * m.PM + p], a1 = a64[o * m.PM + p + 1];
      vbuf[o * P + p] = a0 * ik;
      vbuf[o * P + p + 1] = a1 * ik;
      const double qq = fma(a0, a0, a1 * a1) * ik;
      q += -0.5 * qq - log(kap);
      dlnkd[((size_t)b * np + I) * m.nd + k] = 0.5 * qq - 1.0;
    }
    q = block_sum(q, red);
    if (tid == 0) qout[(size_t)b * (m.na + 1) + kb] = q;
    return;
  }
  const int k = kb;
  if (k >= m.n_chol + m.n_gwbonly) {  // red noise only: Phi = diag(kappa)
    for (int I = tid; I < np; I += kCT) {
      const double s = sk[((size_t)b * np + I) * m.na + k], kap = s * s, ik = 1.0 / kap;
      const size_t o = (size_t)I * B + b;
      const double a0 = a64[o * m.PM + 2 * k], a1 = a64[o * m.PM + 2 * k + 1];
      vbuf[o * P + 2 * k] = a0 * ik;
      vbuf[o * P + 2 * k + 1] = a1 * ik;
      const double qq = fma(a0, a0, a1 * a1) * ik;
      q += -0.5 * qq - log(kap);
      dlnk[((size_t)b * np + I) * m.na + k] = 0.5 * qq - 1.0;
    }
    q = block_sum(q, red);
    if (tid == 0) {
      qout[(size_t)b * (m.na + 1) + kb] = q;
      dlnr[(size_t)b * m.na + k] = 0.0;
    }
    return;
  }
  // correlated bins: X = L_k^-1 packed (dense) or chol(Gamma)^-1 / sqrt(rho) (GWB only)
  const bool dense = k < m.n_chol;
  const int ntri = np * (np + 1) / 2;
  double* X = sm;
  double* a = X + ntri;   // [2][np]
  double* zq = a + 2 * np; // [2][np] X a
  const double sr = srho[(size_t)b * m.na + k];
  if (dense) {
    const double* Xg = Lipk + ((size_t)b * m.n_chol + k) * ntri;
    for (int e = tid; e < ntri; e += kCT) X[e] = DWL ? dw2d(reinterpret_cast<const float2*>(Xg)[e]) : Xg[e];
  } else {
    const double isr = 1.0 / sr;
    for (int e = tid; e < ntri; e += kCT) {
      int i, j;
      tri_decode(e, i, j);
      X[e] = m.LGammaInv[i * np + j] * isr;
    }
  }
  for (int e = tid; e < 2 * np; e += kCT) {
    const int c = e / np, I = e % np;
    a[e] = a64[((size_t)I * B + b) * m.PM + 2 * k + c];
  }
  __syncthreads();
  for (int e = tid; e < 2 * np; e += kCT) {
    const int c = e / np, I = e % np;
    const double* row = X + trl(I, 0);
    const double* ac = a + c * np;
    double s = 0.0;
    for (int J = 0; J <= I; ++J) s = fma(row[J], ac[J], s);
    zq[e] = s;
    q -= 0.5 * s * s;
  }
  __syncthreads();
  double part = 0.0;  // 1/2 sum_c a_c . v_c - kappa d/dkappa, this thread's pulsars
  for (int J = tid; J < np; J += kCT) {
    double v0 = 0.0, v1 = 0.0, dg = 0.0;
    for (int I = J; I < np; ++I) {
      const double xij = X[trl(I, J)];
      v0 = fma(xij, zq[I], v0);
      v1 = fma(xij, zq[np + I], v1);
      dg = fma(xij, xij, dg);
    }
    const size_t o = (size_t)J * B + b;
    vbuf[o * P + 2 * k] = v0;
    vbuf[o * P + 2 * k + 1] = v1;
    q += 2.0 * log(X[trl(J, J)]);  // -log det Phi_k = 2 sum log (L_k^-1)_JJ
    const double s = sk[((size_t)b * np + J) * m.na + k], kap = s * s;
    const double dk = kap * (0.5 * fma(v0, v0, v1 * v1) - dg);
    dlnk[((size_t)b * np + J) * m.na + k] = dk;
    part += 0.5 * fma(a[J], v0, a[np + J] * v1) - dk;
  }
  q = block_sum(q, red);
  part = block_sum(part, red);
  if (tid == 0) {
    qout[(size_t)b * (m.na + 1) + kb] = q;
    dlnr[(size_t)b * m.na + k] = part - (double)np;
  }
}

// ---------------------------------------------------------------------------
// Gradient through the transform.  Grid (npsr, B).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kCT)
    k_curn_adjoint(DevModel m, const float* __restrict__ x, const double* __restrict__ ghat,
                   const double* __restrict__ Wg, const double* __restrict__ vbuf, const double* __restrict__ ahat,
                   const double* __restrict__ sk, const double* __restrict__ skd, const double* __restrict__ srho,
                   float* grad, double* dlnk, double* dlnkd, double* dlnrc, double* v2, int B, int in_smem) {
  extern __shared__ double sm[];
  const int I = blockIdx.x, b = blockIdx.y, tid = threadIdx.x, P = m.P, np = m.npsr;
  const int ntri = P * (P + 1) / 2;
  const size_t o = (size_t)I * B + b;
  const double* Yg = Wg + o * ntri;
  double* Ys = sm;
  double* gb = in_smem ? sm + ntri : sm;  // gbar, reversed
  double* zp = gb + P;                     // z, reversed
  double* sp = zp + P;                     // s' = Y' gbar'
  double* ah = sp + P;                     // ahat, reversed
  double* pd = ah + P;                     // phi_C d logp / d phi_C, coefficient order
  const double* Y = in_smem ? Ys : Yg;
  if (in_smem)
    for (int e = tid; e < ntri; e += kCT) Ys[e] = Yg[e];
  const float* xb = x + (size_t)b * m.d;
  for (int i = tid; i < P; i += kCT) {
    const int p = P - 1 - i;
    gb[i] = ghat[o * P + p] - vbuf[o * P + p];
    zp[i] = (double)xb[zidx(m, I, p)];
    ah[i] = ahat[o * P + p];
  }
  __syncthreads();
  float* gout = grad + (size_t)b * m.d;
  for (int i = tid; i < P; i += kCT) {
    const double* row = Y + trl(i, 0);
    double s = 0.0;
    for (int c = 0; c <= i; ++c) s = fma(row[c], gb[c], s);
    sp[i] = s;
    gout[zidx(m, I, P - 1 - i)] = (float)s;  // d logp / d z = W gbar
  }
  __syncthreads();
  for (int c = tid; c < P; c += kCT) {
    double h = 0.0, R = 0.0, Tc = 0.0, Dg = 0.0;
    for (int i = P - 1; i >= c; --i) {
      const double y = Y[trl(i, c)];
      const double ys = y * sp[i];
      h += ys;                               // (A^-1 gbar)'_c
      Tc = fma(ys, R, Tc);                   // sum over rows below of y z' times y s'
      R = fma(y, zp[i], R);
      Dg = fma(y * y, fma(zp[i], sp[i], 1.0), Dg);
    }
    const double ab = -h * ah[c] - Tc - 0.5 * Dg;  // d logp / d d_p
    const int p = P - 1 - c;
    if (v2) v2[o * P + p] = h;  // A^-1 gbar, for the CW gradient through the mean
    pd[p] = -ab / phic(m, sk, skd, srho, b, I, p);  // phi d/dphi = -d_p d/dd_p
  }
  __syncthreads();
  for (int k = tid; k < m.na; k += kCT) {
    const double S = pd[2 * k] + pd[2 * k + 1];
    const double r = srho[(size_t)b * m.na + k], q = sk[((size_t)b * np + I) * m.na + k];
    const double rho = r * r, kap = q * q, iphi = 1.0 / (rho + kap);
    dlnrc[((size_t)b * np + I) * m.na + k] = S * rho * iphi;
    dlnk[((size_t)b * np + I) * m.na + k] += S * kap * iphi;
  }
  for (int k = tid; k < m.nd; k += kCT)
    dlnkd[((size_t)b * np + I) * m.nd + k] += pd[2 * m.na + 2 * k] + pd[2 * m.na + 2 * k + 1];
}

// The gradient of k_curn_adjoint from the double-word Y' of k_curn_forward_dw, in
// double words.  The column walk of each p (from the last row up) is cut into nseg
// segments taken by different threads: segment q returns its sums h_q = sum y s', Dg_q,
// R_q = sum y z' and T_q (the walk's cross term with R started at zero), and the walk is
// T = sum_q (T_q + h_q R_above), R_above the R of the segments above q.
__global__ void __launch_bounds__(kCTdw)
    k_curn_adjoint_dw(DevModel m, const float* __restrict__ x, const double* __restrict__ ghat,
                      const float2* __restrict__ Wg, const double* __restrict__ vbuf, const double* __restrict__ ahat,
                      const double* __restrict__ sk, const double* __restrict__ skd, const double* __restrict__ srho,
                      float* grad, double* dlnk, double* dlnkd, double* dlnrc, double* v2, int B, int ysm) {
  extern __shared__ float2 smw[];
  const int I = blockIdx.x, b = blockIdx.y, tid = threadIdx.x, nt = blockDim.x, P = m.P, np = m.npsr;
  const int ntri = P * (P + 1) / 2, nseg = max(1, min(4, nt / P));
  const size_t o = (size_t)I * B + b;
  float2* Ys = smw;                    // [ntri] Y', plain packing (ysm), else read from the W slot
  float2* gb = Ys + (ysm ? ntri : 0);  // [P] gbar', reversed
  float2* zp = gb + P;                 // [P] z'
  float2* sp = zp + P;                 // [P] s' = Y' gbar'
  float2* seg = sp + P;                // [nseg][P][4] (h, T, R, Dg) per segment and column
  double* pd = reinterpret_cast<double*>(seg + 4 * nseg * P);  // [P] phi_C d logp / d phi_C
  const float2* Yg = Wg + o * ntri;
  if (ysm)
    for (int e = tid; e < ntri; e += nt) Ys[e] = Yg[e];
  const float2* Y = ysm ? Ys : Yg;
  const float* xb = x + (size_t)b * m.d;
  for (int i = tid; i < P; i += nt) {
    const int p = P - 1 - i;
    gb[i] = d2dw_bits(ghat[o * P + p] - vbuf[o * P + p]);
    zp[i] = make_float2(xb[zidx(m, I, p)], 0.0f);
  }
  __syncthreads();
  float* gout = grad + (size_t)b * m.d;
  for (int i = tid; i < P; i += nt) {
    const float2* row = Y + trl(i, 0);
    float2 s = make_float2(0.0f, 0.0f);
    for (int c = 0; c <= i; ++c) s = dw_fms(s, row[c], dw_neg(gb[c]));
    sp[i] = s;
    gout[zidx(m, I, P - 1 - i)] = __fadd_rn(s.x, s.y);  // d logp / d z = W gbar
  }
  __syncthreads();
  for (int r = tid; r < nseg * P; r += nt) {
    const int c = r % P, q = r / P, len = P - c;
    const int hi = P - len * q / nseg, lo = P - len * (q + 1) / nseg;  // rows [lo, hi), walked downward
    float2 h = make_float2(0.0f, 0.0f), R = h, T = h, Dg = h;
    for (int i = hi - 1; i >= lo; --i) {
      const float2 y = Y[trl(i, c)];
      const float2 ys = dw_mul(y, sp[i]);
      h = dw_add(h, ys);
      T = dw_fms(T, ys, dw_neg(R));
      R = dw_fms(R, y, dw_neg(zp[i]));
      Dg = dw_fms(Dg, dw_mul(y, y), dw_neg(dw_fms(make_float2(1.0f, 0.0f), zp[i], dw_neg(sp[i]))));
    }
    float2* sg = seg + 4 * r;
    sg[0] = h;
    sg[1] = T;
    sg[2] = R;
    sg[3] = Dg;
  }
  __syncthreads();
  for (int c = tid; c < P; c += nt) {
    float2 h = make_float2(0.0f, 0.0f), T = h, R = h, Dg = h;
    for (int q = 0; q < nseg; ++q) {  // top segment first
      const float2* sg = seg + 4 * (q * P + c);
      T = dw_add(T, dw_fms(sg[1], sg[0], dw_neg(R)));
      h = dw_add(h, sg[0]);
      R = dw_add(R, sg[2]);
      Dg = dw_add(Dg, sg[3]);
    }
    const int p = P - 1 - c;
    const double hd = dw2d(h);
    const double ab = -hd * ahat[o * P + p] - dw2d(T) - 0.5 * dw2d(Dg);  // d logp / d d_p
    if (v2) v2[o * P + p] = hd;  // A^-1 gbar, for the CW gradient through the mean
    pd[p] = -ab / phic(m, sk, skd, srho, b, I, p);  // phi d/dphi = -d_p d/dd_p
  }
  __syncthreads();
  for (int k = tid; k < m.na; k += nt) {
    const double S = pd[2 * k] + pd[2 * k + 1];
    const double r = srho[(size_t)b * m.na + k], q = sk[((size_t)b * np + I) * m.na + k];
    const double rho = r * r, kap = q * q, iphi = 1.0 / (rho + kap);
    dlnrc[((size_t)b * np + I) * m.na + k] = S * rho * iphi;
    dlnk[((size_t)b * np + I) * m.na + k] += S * kap * iphi;
  }
  for (int k = tid; k < m.nd; k += nt)
    dlnkd[((size_t)b * np + I) * m.nd + k] += pd[2 * m.na + 2 * k] + pd[2 * m.na + 2 * k + 1];
}

// Auxiliary passes of the deterministic-signal transform: a = a_ref - v per (pulsar,
// chain), and the difference of two per-TOA weight arrays.
__global__ void k_set_a(DevModel m, double* a64, const double* __restrict__ v, int B) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)m.npsr * B * m.P) return;
  const int p = (int)(i % m.P);
  const size_t o = i / m.P;           // I * B + b
  const int I = (int)(o / B);
  const double a = m.aref[(size_t)I * m.P + p];
  a64[o * m.PM + p] = v ? a - v[i] : a;
}

__global__ void k_sub(float* out, const float* __restrict__ w, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] -= w[i];
}

size_t fwd_smem(const DevModel& m, bool tri) {
  const size_t P = m.P;
  return ((tri ? P * (P + 1) / 2 : 0) + 8 * P) * sizeof(double);
}
size_t adj_smem(const DevModel& m, bool tri) {
  const size_t P = m.P;
  return ((tri ? P * (P + 1) / 2 : 0) + 5 * P) * sizeof(double);
}
constexpr size_t kCurnSmemMax = 200 * 1024;

}  // namespace

size_t curn_w_doubles(const DevModel& m) { return (size_t)m.P * (m.P + 1) / 2; }

// shared memory of k_curn_forward_dw and of k_curn_forward_dwc<C> (its largest part of the
// triangle); which CURN forward runs: 0 the FP64 kernel (FP64 mode, PTA_CHOL_FP64, or no
// cluster of at most 8 CTAs holds the triangle), 1 the double-word kernel with the triangle
// in one CTA, C > 1 the double-word kernel over a cluster of C CTAs
static size_t curn_fwd_smem_dw(const DevModel& m) {
  return 6 * (size_t)(m.P / 2 + 1) * sizeof(float4) + (size_t)prow(m.P) * sizeof(float2);
}
template <int C>
static size_t curn_fwd_smem_dwc(const DevModel& m) {
  int mx = 0;
  for (int k = 0; k < C; ++k) mx = std::max(mx, cpart<C>(m.P, k));
  return (size_t)cstage_f4(m.P) * sizeof(float4) + 2 * (size_t)m.P * sizeof(float2) + (size_t)mx * sizeof(float2);
}
constexpr size_t kDwSmemMax = 226 * 1024;  // of the 227 KB a CTA may opt into, 1 KB for static shared memory
static int curn_dw_mode(const DevModel& m, int fp64) {
  if (fp64 || m.chol64) return 0;
  if (curn_fwd_smem_dw(m) <= kDwSmemMax) return 1;
  if (curn_fwd_smem_dwc<2>(m) <= kDwSmemMax) return 2;
  if (curn_fwd_smem_dwc<4>(m) <= kDwSmemMax) return 4;
  if (curn_fwd_smem_dwc<8>(m) <= kDwSmemMax) return 8;
  return 0;
}

template <int C>
static cudaError_t launch_fwd_dwc(const DevModel& m, const Scratch& s, int B, const float* x, cudaStream_t st) {
  constexpr int NT = C == 2 ? 1024 : 512;
  const size_t sm = curn_fwd_smem_dwc<C>(m);
  cudaError_t e =
      cudaFuncSetAttribute(k_curn_forward_dwc<C, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_curn_forward_dwc<C, NT><<<dim3(m.npsr * C, B), NT, sm, st>>>(m, x, s.sk, s.skd, s.srho, s.a64, s.curnW,
                                                               s.curnAhat, s.curnLd, s.stat,
                                                               m.cw ? s.curnG0 : nullptr, B);
  return cudaGetLastError();
}

cudaError_t launch_curn_forward(const DevModel& m, const Scratch& s, int B, const float* x, int fp64,
                                cudaStream_t st) {
  const int mode = curn_dw_mode(m, fp64);
  cudaError_t e = cudaSuccess;
  if (mode == 1) {
    const size_t smdw = curn_fwd_smem_dw(m);
    e = cudaFuncSetAttribute(k_curn_forward_dw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smdw);
    if (e != cudaSuccess) return e;
    k_curn_forward_dw<<<dim3(m.npsr, B), kCTdw, smdw, st>>>(m, x, s.sk, s.skd, s.srho, s.a64, s.curnW, s.curnAhat,
                                                            s.curnLd, s.stat, m.cw ? s.curnG0 : nullptr, B);
  } else if (mode > 1) {
    e = mode == 2 ? launch_fwd_dwc<2>(m, s, B, x, st)
                  : (mode == 4 ? launch_fwd_dwc<4>(m, s, B, x, st) : launch_fwd_dwc<8>(m, s, B, x, st));
    if (e != cudaSuccess) return e;
  } else {
    const bool tri = fwd_smem(m, true) <= kCurnSmemMax;
    const size_t sm = fwd_smem(m, tri);
    e = cudaFuncSetAttribute(k_curn_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_curn_forward<<<dim3(m.npsr, B), kCT, sm, st>>>(m, x, s.sk, s.skd, s.srho, s.a64, s.curnW, s.curnAhat,
                                                      s.curnLd, s.stat, m.cw ? s.curnG0 : nullptr, B, tri ? 1 : 0);
  }
  const size_t ws = ((size_t)m.npsr * (m.npsr + 1) / 2 + 4 * m.npsr) * sizeof(double);
  const bool dwl = chol_uses_dw(m, fp64);
  e = dwl ? cudaFuncSetAttribute(k_curn_whiten<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ws)
          : cudaFuncSetAttribute(k_curn_whiten<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ws);
  if (e != cudaSuccess) return e;
  (dwl ? k_curn_whiten<true> : k_curn_whiten<false>)<<<dim3(m.na + 1, B), kCT, ws, st>>>(
      m, s.a64, s.Lipk, s.sk, s.skd, s.srho, s.curnV, s.curnQ, s.dlnk, s.dlnkd, s.dlnr, B);
  return cudaGetLastError();
}

cudaError_t launch_curn_adjoint(const DevModel& m, const Scratch& s, int B, const float* x, float* grad, int fp64,
                                cudaStream_t st) {
  if (curn_dw_mode(m, fp64)) {  // Y' in shared memory while it fits, else read from the W slot
    const size_t P = m.P, nseg = std::max<size_t>(1, std::min<size_t>(4, kCTdw / P));
    const size_t rest = (3 * P + 4 * nseg * P) * sizeof(float2) + P * sizeof(double);
    const bool ysm = P * (P + 1) / 2 * sizeof(float2) + rest <= kDwSmemMax;
    const size_t sm = (ysm ? P * (P + 1) / 2 * sizeof(float2) : 0) + rest;
    cudaError_t e = cudaFuncSetAttribute(k_curn_adjoint_dw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_curn_adjoint_dw<<<dim3(m.npsr, B), kCTdw, sm, st>>>(
        m, x, s.ghat, reinterpret_cast<const float2*>(s.curnW), s.curnV, s.curnAhat, s.sk, s.skd, s.srho, grad,
        s.dlnk, s.dlnkd, s.dlnrc, m.cw ? s.curnV2 : nullptr, B, ysm ? 1 : 0);
    return cudaGetLastError();
  }
  const bool tri = adj_smem(m, true) <= kCurnSmemMax;
  const size_t sm = adj_smem(m, tri);
  cudaError_t e = cudaFuncSetAttribute(k_curn_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_curn_adjoint<<<dim3(m.npsr, B), kCT, sm, st>>>(m, x, s.ghat, s.curnW, s.curnV, s.curnAhat, s.sk, s.skd, s.srho,
                                                    grad, s.dlnk, s.dlnkd, s.dlnrc, m.cw ? s.curnV2 : nullptr, B,
                                                    tri ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_curn_set_a(const DevModel& m, const Scratch& s, int B, const double* v, cudaStream_t st) {
  const size_t n = (size_t)m.npsr * B * m.P;
  k_set_a<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m, s.a64, v, B);
  return cudaGetLastError();
}

cudaError_t launch_sub(float* out, const float* w, size_t n, cudaStream_t st) {
  k_sub<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, w, n);
  return cudaGetLastError();
}

}  // namespace pta
