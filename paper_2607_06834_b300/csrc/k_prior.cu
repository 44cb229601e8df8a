// Prior side of the evaluation: spectra (Eq. power_law), the per-frequency
// prior covariance Phi_k = rho_k Gamma + diag(kappa_.k) (Eq. prior_cov, Gamma of
// Eq. HD), its Cholesky factor, inverse and log-det, the standardizing transform
// a = L z (Eq. standardizing_transform with mu = 0), the adjoint of that transform
// and the final per-chain sum.
//
// FP64 issue is the scarce resource on this part (about 1/64 of the FP32 rate).  In
// FP64 mode the dense-bin kernel keeps every FP64 warp instruction full: the triangular
// updates walk a flat index over the active triangle / rectangle (decoded from a
// table, no per-element square roots), the factorisation and the inverse advance in
// one sweep with two barriers per column, and the per-column pivot work is one
// Newton-refined reciprocal (LDL^T form; the square roots come at the end, all
// pivots at once).  In the other modes the dense-bin sweep and its adjoint run in
// double-word arithmetic on the FP32 pipes (k_chol_forward_dw, k_chol_adjoint_dw);
// spectra, pivots' square roots and every sum stay FP64.
#include <cmath>

#include "dw_ldl.cuh"
#include "dwarith.cuh"
#include "pta_internal.cuh"

namespace pta {
namespace {

__device__ __forceinline__ int tri(int i, int j) { return i * (i + 1) / 2 + j; }

// ---------------------------------------------------------------------------
// Spectra: sqrt(kappa_Ik) (red noise, k < n_rn; 0 up to na), sqrt(kappa^DM_Ik),
// sqrt(rho_k) (k < n_gwb), one thread per value: exp(ln_pl / 2) (Eq. power_law) or
// 10^((theta + 18) / 2) for a free spectrum.  DW (outside FP64 mode): the argument is
// formed and exponentiated in double-word arithmetic on the FP32 pipes (relative
// error ~1e-13, from the argument's ~2^-48 |terms|), so a value costs one FP64 add
// instead of an FP64 exponential; FP64 mode keeps the FP64 exponential.
// ---------------------------------------------------------------------------
template <bool DW>
__device__ __forceinline__ double half_pl(const DevModel& m, float lnA, float ga, int k) {  // exp(ln_pl/2)
  if (!DW) return exp(0.5 * ln_pl(m.ln_rho0, m.ln_Tfyr, lnA, ga, m.lnk[k]));
  constexpr float2 kLn10 = {0x1.26bb1cp+1f, -0x1.12aabap-25f};
  const float2 arg = dw_add(dw_add(dw_mulf(kLn10, lnA), m.hr0), dw_neg(dw_mulf(m.lkT[k], __fmul_rn(0.5f, ga))));
  return dw_exp_d(arg);
}
template <bool DW>
__device__ __forceinline__ double half_free(float theta) {  // 10^((theta + 18) / 2)
  if (!DW) return exp(0.5 * kLn10 * ((double)theta + 18.0));
  constexpr float2 kHalfLn10 = {0x1.26bb1cp+0f, -0x1.12aabap-26f};
  return dw_exp_d(dw_mul(kHalfLn10, dw_addf(make_float2(theta, 0.0f), 18.0f)));
}

// a = sqrt(kappa) z for a diagonal bin's two coefficients (Eq. standardizing_transform
// with a diagonal Phi_k): an FP64 product, or in double words with one FP64 add each
template <bool DW>
__device__ __forceinline__ void diag_a(double s, float z0, float z1, double* a) {
  if (DW) {
    const float2 sw = d2dw_bits(s);
    *reinterpret_cast<double2*>(a) = make_double2(dw2d(dw_mulf(sw, z0)), dw2d(dw_mulf(sw, z1)));
  } else {
    a[0] = s * z0;
    a[1] = s * z1;
  }
}

// With the transform applied here to the diagonal bins (red-noise-only achromatic bins and
// every DM bin), the value is used where it is made; the dense and GWB-only bins take
// theirs in k_chol_forward(_dw) and k_gwbonly_forward.  a64 is nullptr under the CURN
// transform (a comes from k_curn_forward).
template <bool DW>
__global__ void k_spectra(DevModel m, const float* __restrict__ x, double* sk, double* skd, double* srho,
                          double* a64, int B) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
  const int np = m.npsr, nach = np * m.na, ndm = np * m.nd;
  if (r >= nach + ndm + m.na) return;
  const float* xb = x + (size_t)b * m.d;
  double v = 0.0;
  if (r < nach) {
    const int I = r / m.na, k = r % m.na;
    if (k < m.n_rn)  // free spectrum: kappa = 10^theta s^2 = 10^(theta + 18) ns^2
      v = m.rn_free ? half_free<DW>(xb[m.th_rn + m.n_rn * I + k])
                    : half_pl<DW>(m, xb[m.th_rn + 2 * I], xb[m.th_rn + 2 * I + 1], k + 1);
    sk[(size_t)b * nach + r] = v;
    if (a64 && k >= m.n_chol + m.n_gwbonly && k < m.n_rn)
      diag_a<DW>(v, xb[m.z_ach + (2 * k) * np + I], xb[m.z_ach + (2 * k + 1) * np + I],
                 a64 + ((size_t)I * B + b) * m.PM + 2 * k);
  } else if (r < nach + ndm) {
    const int q = r - nach, I = q / m.nd, k = q % m.nd;
    v = half_pl<DW>(m, xb[m.th_dm + 2 * I], xb[m.th_dm + 2 * I + 1], k + 1);
    skd[(size_t)b * ndm + q] = v;
    if (a64) {
      const int zo = m.z_dm + (I * m.nd + k) * 2;
      diag_a<DW>(v, xb[zo], xb[zo + 1], a64 + ((size_t)I * B + b) * m.PM + 2 * m.na + 2 * k);
    }
  } else {
    const int k = r - nach - ndm;
    if (k < m.n_gwb)
      v = m.gwb_free ? half_free<DW>(xb[m.th_gwb + k]) : half_pl<DW>(m, xb[m.th_gwb], xb[m.th_gwb + 1], k + 1);
    srho[(size_t)b * m.na + k] = v;
  }
}

// ---------------------------------------------------------------------------
// Dense bins k < n_chol: Phi_k = rho_k Gamma + diag(kappa_.k).  One CTA per
// (bin, chain).  The sweep is the LDL^T form of the Cholesky factorisation
// (Phi = L D L^T, L unit lower): column j is scaled by 1/d_j (the pivot's
// reciprocal from recip64, taken by the thread that finishes the pivot), the
// trailing triangle takes the rank-1 update with the unscaled column, and the rows
// of X = L^-1 below j take the same elimination step.  No square root or division
// sits on the column-to-column path; sqrt(d) for all pivots at once at the end
// gives the Cholesky factor L D^(1/2), its inverse D^(-1/2) X and the transform.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512)
    k_chol_forward(DevModel m, const float* __restrict__ x, const double* __restrict__ sk,
                   const double* __restrict__ srho, double* a64, double* Lpk, double* Lipk, int32_t* stat) {
  extern __shared__ double sm[];
  const int np = m.npsr, ntri = np * (np + 1) / 2;
  double* A = sm;              // packed lower: becomes L (unit, below the diagonal) and D (diagonal)
  double* X = sm + ntri;       // packed lower: becomes L^-1 (unit lower)
  double* zs = X + ntri;       // [2][np]
  double* rd = zs + 2 * np;    // [np] 1 / d_j, then 1 / sqrt(d_j)
  double* u = rd + np;         // [np] unscaled column j, then sqrt(d_j)
  __shared__ int s_bad;
  const int k = blockIdx.x, b = blockIdx.y, tid = threadIdx.x, nt = blockDim.x;
  const float* xb = x + (size_t)b * m.d;
  const double sr = srho[(size_t)b * m.na + k];
  const double rho = sr * sr;
  const double* skb = sk + (size_t)b * np * m.na + k;
  if (tid == 0) s_bad = 0;
  for (int idx = tid; idx < ntri; idx += nt) {
    const unsigned t = m.trimap[idx];
    const int i = t >> 8, j = t & 255;
    double v = rho * m.Gamma[i * np + j];
    if (i == j) {
      const double s = skb[(size_t)i * m.na];
      v = fma(s, s, v);
    }
    A[idx] = v;
    X[idx] = (i == j) ? 1.0 : 0.0;
  }
  for (int i = tid; i < 2 * np; i += nt) zs[i] = (double)xb[m.z_ach + (2 * k) * np + i];
  __syncthreads();
  if (tid == 0) {
    double d = A[0];
    if (!(d > 0.0)) {
      s_bad = 1;
      d = 1.0;
      A[0] = d;
    }
    rd[0] = recip64(d);
  }
  __syncthreads();
  for (int j = 0; j < np; ++j) {
    const double r = rd[j];
    const int s = np - j - 1;
    for (int e = tid; e < s; e += nt) {
      const int i = j + 1 + e;
      const double v = A[tri(i, j)];
      u[i] = v;
      A[tri(i, j)] = v * r;  // l_ij
    }
    __syncthreads();
    const int cntA = s * (s + 1) / 2, w = j + 1, cnt = cntA + s * w;
    const float rw = 1.0f / (float)w;
    for (int idx = tid; idx < cnt; idx += nt) {
      if (idx < cntA) {
        const unsigned t = m.trimap[idx];
        const int i = (t >> 8) + j + 1, l = (t & 255) + j + 1;
        const double v = fma(-A[tri(i, j)], u[l], A[tri(i, l)]);
        if (idx == 0) {  // element (j+1, j+1) receives its last update: the next pivot d_{j+1}
          double d = v;
          if (!(d > 0.0)) {
            s_bad = 1;
            d = 1.0;
          }
          A[tri(i, l)] = d;
          rd[j + 1] = recip64(d);
        } else {
          A[tri(i, l)] = v;
        }
      } else {
        const int e = idx - cntA;
        int q = (int)(((float)e + 0.5f) * rw);
        q -= (q * w > e);
        q += ((q + 1) * w <= e);
        const int i = j + 1 + q, c = e - q * w;
        X[tri(i, c)] = fma(-A[tri(i, j)], X[tri(j, c)], X[tri(i, c)]);
      }
    }
    __syncthreads();
  }
  if (s_bad && tid == 0) atomicOr(&stat[b], 2);
  // sqrt(d_j) and 1/sqrt(d_j) for all pivots at once
  for (int j = tid; j < np; j += nt) {
    const double y = rsqrt64(A[tri(j, j)]);
    u[j] = A[tri(j, j)] * y;
    rd[j] = y;
  }
  __syncthreads();
  // a_{I,k,c} = sum_J (L D^(1/2))[I][J] z_{J,k,c} = sum_{J<=I} L[I][J] sqrt(d_J) z_{J,k,c}
  for (int I = tid; I < np; I += nt) {
    double s0 = u[I] * zs[I], s1 = u[I] * zs[np + I];
    for (int J = 0; J < I; ++J) {
      const double l = A[tri(I, J)] * u[J];
      s0 = fma(l, zs[J], s0);
      s1 = fma(l, zs[np + J], s1);
    }
    const size_t o = ((size_t)I * gridDim.y + b) * m.PM + 2 * k;
    a64[o] = s0;
    a64[o + 1] = s1;
  }
  // Cholesky factor L D^(1/2) and its inverse D^(-1/2) L^-1 for the adjoint
  double* Lg = Lpk + ((size_t)b * m.n_chol + k) * ntri;
  double* Xg = Lipk + ((size_t)b * m.n_chol + k) * ntri;
  for (int idx = tid; idx < ntri; idx += nt) {
    const unsigned t = m.trimap[idx];
    const int i = t >> 8, j = t & 255;
    Lg[idx] = (i == j) ? u[j] : A[idx] * u[j];
    Xg[idx] = (i == j) ? rd[i] : X[idx] * rd[i];
  }
}

// The dense-bin factorisation of k_chol_forward with the sweep in double-word
// arithmetic (dw_ldl_sweep, two columns per step, 2x2 tiles).  Phi_k is scaled by 2^-E
// (E from its largest diagonal entry, so every entry and pivot lies in (0, 1]) before
// the sweep, which leaves the unit factor and its inverse unchanged and scales the
// pivots by 2^-E; the pivots return to double and their true scale before the square
// roots.  Outputs: a64 as k_chol_forward; L D^(1/2) and D^(-1/2) L^-1 packed lower (plain
// packing) in the same slots as k_chol_forward's, as double-word float pairs (read by
// k_chol_adjoint_dw and, under the CURN transform, by k_curn_whiten).
__global__ void __launch_bounds__(512, 4)  // 32 registers: 8 CTAs of 256 threads per SM at 67 pulsars
    k_chol_forward_dw(DevModel m, const float* __restrict__ x, const double* __restrict__ sk,
                      const double* __restrict__ srho, double* a64, float2* Lpk, float2* Lipk, int32_t* stat) {
  extern __shared__ float4 smq[];
  const int np = m.npsr, ntri = np * (np + 1) / 2, nh = np / 2 + 1;
  float2* T = reinterpret_cast<float2*>(smq + 6 * nh);  // after the sweep's staging: one padded packed triangle
  __shared__ float2 pv[6];                              // the step's pivot block (dw_pivot_pair)
  __shared__ int s_bad;
  const int k = blockIdx.x, b = blockIdx.y, tid = threadIdx.x, nt = blockDim.x;
  const float* xb = x + (size_t)b * m.d;
  const double sr = srho[(size_t)b * m.na + k];
  const double rho = sr * sr;
  const double* skb = sk + (size_t)b * np * m.na + k;
  // scale 2^-E, E even, from the largest diagonal entry (every warp computes it; no barrier)
  double dmax = 0.0;
  for (int i = tid & 31; i < np; i += 32) {
    const double s = skb[(size_t)i * m.na];
    dmax = fmax(dmax, fma(s, s, rho * m.Gamma[i * np + i]));
  }
  for (int o = 16; o; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  int E = 0;
  if (dmax > 0.0 && isfinite(dmax)) frexp(dmax, &E);
  E += E & 1;
  const float2 rhow = d2dw_bits(ldexp(rho, -E));
  if (tid == 0) s_bad = 0;
  for (int idx = tid; idx < ntri; idx += nt) {
    const unsigned t = m.trimap[idx];
    const int i = t >> 8, j = t & 255, o = prow(i) + j;
    float2 v = dw_mul(rhow, m.Gamma_dw[idx]);
    if (i == j) {
      const double s = skb[(size_t)i * m.na];
      v = dw_add(v, d2dw_bits(ldexp(s * s, -E)));
      if (!(i & 1)) T[o + 1] = make_float2(0.0f, 0.0f);  // an even row's padding
    }
    T[o] = v;
  }
  __syncthreads();
  float2* Lg = Lpk + ((size_t)b * m.n_chol + k) * ntri;
  float2* Xg = Lipk + ((size_t)b * m.n_chol + k) * ntri;
  const float usc = __int_as_float((127 + E / 2) << 23);  // 2^(E/2): sqrt of the true pivots
  dw_ldl_sweep(np, T, smq, pv, &s_bad, m.trimap, Lg, usc, m.chk);
  if (s_bad && tid == 0) atomicOr(&stat[b], 2);
  // 1/sqrt(d_j) at true scale and z (the staging area is free now)
  float2* rqw = reinterpret_cast<float2*>(smq);  // [np]
  float* zs = reinterpret_cast<float*>(rqw + np);  // [2][np]
  for (int j = tid; j < np; j += nt) {
    const float2 sq = dw_sqrt(T[prow(j) + j]);
    rqw[j] = dw_recip(make_float2(sq.x * usc, sq.y * usc));
  }
  for (int i = tid; i < 2 * np; i += nt) zs[i] = xb[m.z_ach + (2 * k) * np + i];
  __syncthreads();
  // D^(-1/2) L^-1 for the adjoint (L D^(1/2) went out during the sweep)
  for (int idx = tid; idx < ntri; idx += nt) {
    const unsigned t = m.trimap[idx];
    const int i = t >> 8, j = t & 255;
    Xg[idx] = (i == j) ? rqw[i] : dw_mul(T[prow(i) + j], rqw[i]);
  }
  // a_{I,k,c} = sum_{J<=I} (L D^(1/2))[I][J] z_{J,k,c}, from the rows this block wrote
  for (int i = tid; i < 2 * np; i += nt) {
    const int c = i / np, I = i % np;
    const float2* row = Lg + I * (I + 1) / 2;
    const float* zc = zs + c * np;
    float2 acc = make_float2(0.0f, 0.0f);
    for (int J = 0; J <= I; ++J) acc = dw_fms(acc, row[J], make_float2(-zc[J], 0.0f));
    a64[((size_t)I * gridDim.y + b) * m.PM + 2 * k + c] = dw2d(acc);
  }
}

// Adjoint of k_chol_forward_dw's transform (the formulas of k_chol_adjoint below) in
// double-word arithmetic, from its double-word factors.  The walk over a >= I behind
// kappa_I d logp / d kappa_I is cut into nseg segments taken by different threads:
// segment q returns its own sum with prefixes started at zero (loc), its prefix totals
// P_c = sum u_a z_ca and the sums V_c = sum gt_ca u_a, and the walk is
// sum_q loc_q + sum_c (P_c of the segments before q) V_cq.

__global__ void __launch_bounds__(512)
    k_chol_adjoint_dw(DevModel m, const float* __restrict__ x, const double* __restrict__ ghat,
                      const float2* __restrict__ Lpk, const float2* __restrict__ Lipk, const double* __restrict__ sk,
                      float* grad, double* dlnk, double* dlnr, int B) {
  extern __shared__ float2 smw[];
  const int np = m.npsr, ntri = np * (np + 1) / 2, nt = blockDim.x;
  const int nseg = max(1, min(4, nt / np));
  float2* Ls = smw;
  float2* Xs = smw + max(ntri, 5 * nseg * np + np);
  float2* gs = Xs + ntri;   // [2][np] ghat
  float2* gt = gs + 2 * np; // [2][np] L^T ghat
  // once gt no longer needs L, its slot holds the partial walks: (loc, V0, V1) per
  // segment, the prefix totals P_c, and kappa d logp / d kappa
  float2* seg = Ls;                                            // [nseg][np][3]
  double* segp = reinterpret_cast<double*>(Ls + 3 * nseg * np);  // [nseg][np][2]
  double* red = segp + 2 * nseg * np;                          // [np]
  const int k = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
  const float* xb = x + (size_t)b * m.d;
  const float* zb = xb + m.z_ach + (2 * k) * np;  // [2][np]
  const float2* Lg = Lpk + ((size_t)b * m.n_chol + k) * ntri;
  const float2* Xg = Lipk + ((size_t)b * m.n_chol + k) * ntri;
  for (int idx = tid; idx < ntri; idx += nt) {
    Ls[idx] = Lg[idx];
    Xs[idx] = Xg[idx];
  }
  for (int i = tid; i < 2 * np; i += nt) {
    const int c = i / np, I = i % np;
    gs[i] = d2dw_bits(ghat[((size_t)I * B + b) * m.P + 2 * k + c]);
  }
  __syncthreads();
  for (int i = tid; i < 2 * np; i += nt) {
    const int c = i / np, J = i % np;
    const float2* gc = gs + c * np;
    float2 s = make_float2(0.0f, 0.0f);
    for (int I = J; I < np; ++I) s = dw_fms(s, Ls[tri(I, J)], dw_neg(gc[I]));
    gt[i] = s;
    grad[(size_t)b * m.d + m.z_ach + (2 * k) * np + i] = __fadd_rn(__fsub_rn(s.x, zb[i]), s.y);
  }
  __syncthreads();
  for (int r = tid; r < nseg * np; r += nt) {
    const int I = r % np, q = r / np, len = np - I;
    const int a0 = I + len * q / nseg, a1 = I + len * (q + 1) / nseg;
    float2 p0 = make_float2(0.0f, 0.0f), p1 = p0, v0 = p0, v1 = p0, acc = p0;
    for (int a = a0; a < a1; ++a) {
      const float2 u = Xs[tri(a, I)];
      const float2 g0 = dw_mul(gt[a], u), g1 = dw_mul(gt[np + a], u);
      const float2 w0 = dw_mulf(u, zb[a]), w1 = dw_mulf(u, zb[np + a]);
      const float2 h0 = dw_add(p0, make_float2(0.5f * w0.x, 0.5f * w0.y));
      const float2 h1 = dw_add(p1, make_float2(0.5f * w1.x, 0.5f * w1.y));
      acc = dw_fms(acc, g0, dw_neg(h0));
      acc = dw_fms(acc, g1, dw_neg(h1));
      p0 = dw_add(p0, w0);
      p1 = dw_add(p1, w1);
      v0 = dw_add(v0, g0);
      v1 = dw_add(v1, g1);
    }
    float2* sg = seg + 3 * r;
    sg[0] = acc;
    sg[1] = v0;
    sg[2] = v1;
    segp[2 * r] = dw2d(p0);
    segp[2 * r + 1] = dw2d(p1);
  }
  __syncthreads();
  for (int I = tid; I < np; I += nt) {
    double acc = 0.0, p0 = 0.0, p1 = 0.0;
    for (int q = 0; q < nseg; ++q) {
      const int r = q * np + I;
      const float2* sg = seg + 3 * r;
      acc += dw2d(sg[0]) + p0 * dw2d(sg[1]) + p1 * dw2d(sg[2]);
      p0 += segp[2 * r];
      p1 += segp[2 * r + 1];
    }
    const double s = sk[((size_t)b * np + I) * m.na + k];
    const double v = s * s * acc;
    red[I] = v;
    dlnk[((size_t)b * np + I) * m.na + k] = v;
  }
  __syncthreads();
  if (tid < 32) {
    double s = 0.0;
    for (int i = tid; i < np; i += 32)
      s += 0.5 * (dw2d(gt[i]) * (double)zb[i] + dw2d(gt[np + i]) * (double)zb[np + i]) - red[i];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (tid == 0) dlnr[(size_t)b * m.na + k] = s;
  }
}

// Adjoint of a = L z for the dense bins.  With ghat = d logp / d a and
// gt = L^T ghat:  d logp / d z = gt - z (the -z from -|z|^2/2);
// kappa_I d logp/d kappa_I = kappa_I sum_c sum_{a>=I} gt_a u_a (sum_{I<=b<a} u_b z_b + u_a z_a / 2)
// with u = column I of L^-1 (from dL = L tril_half(L^-1 dPhi L^-T), dPhi = e_I e_I^T); and
// rho d logp / d rho = 1/2 sum_c gt.z - sum_I kappa_I d logp/d kappa_I (scaling identity:
// Phi -> s Phi gives a -> sqrt(s) a).
__global__ void __launch_bounds__(512)
    k_chol_adjoint(DevModel m, const float* __restrict__ x, const double* __restrict__ ghat,
                   const double* __restrict__ Lpk, const double* __restrict__ Lipk, const double* __restrict__ sk,
                   float* grad, double* dlnk, double* dlnr, int B) {
  extern __shared__ double sm[];
  const int np = m.npsr, ntri = np * (np + 1) / 2;
  double* Ls = sm;
  double* Xs = sm + ntri;
  double* zs = Xs + ntri;     // [2][np]
  double* gs = zs + 2 * np;   // [2][np] ghat
  double* gt = gs + 2 * np;   // [2][np]
  double* red = gt + 2 * np;  // [np] kappa dlogp/dkappa
  const int k = blockIdx.x, b = blockIdx.y, tid = threadIdx.x, nt = blockDim.x;
  const float* xb = x + (size_t)b * m.d;
  const double* Lg = Lpk + ((size_t)b * m.n_chol + k) * ntri;
  const double* Xg = Lipk + ((size_t)b * m.n_chol + k) * ntri;
  for (int idx = tid; idx < ntri; idx += nt) {
    Ls[idx] = Lg[idx];
    Xs[idx] = Xg[idx];
  }
  for (int i = tid; i < 2 * np; i += nt) {
    const int c = i / np, I = i % np;
    zs[i] = (double)xb[m.z_ach + (2 * k) * np + i];
    gs[i] = ghat[((size_t)I * B + b) * m.P + 2 * k + c];
  }
  __syncthreads();
  for (int i = tid; i < 2 * np; i += nt) {
    const int c = i / np, J = i % np;
    double s = 0.0;
    for (int I = J; I < np; ++I) s = fma(Ls[tri(I, J)], gs[c * np + I], s);
    gt[i] = s;
    grad[(size_t)b * m.d + m.z_ach + (2 * k) * np + i] = (float)(s - zs[i]);
  }
  __syncthreads();
  // kappa_I d logp/d kappa_I, one thread per I (each walk is a short dependent FP64 chain;
  // spreading it over a warp with prefix scans costs several times the FP64 operations)
  for (int I = tid; I < np; I += nt) {
    double p0 = 0.0, p1 = 0.0, acc = 0.0;
    for (int a = I; a < np; ++a) {
      const double u = Xs[tri(a, I)];
      const double h0 = fma(0.5 * u, zs[a], p0), h1 = fma(0.5 * u, zs[np + a], p1);
      acc = fma(gt[a] * u, h0, acc);
      acc = fma(gt[np + a] * u, h1, acc);
      p0 = fma(u, zs[a], p0);
      p1 = fma(u, zs[np + a], p1);
    }
    const double s = sk[((size_t)b * np + I) * m.na + k];
    const double v = s * s * acc;
    red[I] = v;
    dlnk[((size_t)b * np + I) * m.na + k] = v;
  }
  __syncthreads();
  if (tid < 32) {
    double s = 0.0;
    for (int i = tid; i < np; i += 32) s += 0.5 * (gt[i] * zs[i] + gt[np + i] * zs[np + i]) - red[i];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (tid == 0) dlnr[(size_t)b * m.na + k] = s;
  }
}

// ---------------------------------------------------------------------------
// GWB-only bins (no intrinsic red noise): Phi_k = rho_k Gamma, L_k = sqrt(rho_k) chol(Gamma).
// ---------------------------------------------------------------------------
__global__ void k_gwbonly_forward(DevModel m, const float* __restrict__ x, const double* __restrict__ srho,
                                  double* a64) {
  const int k = m.n_chol + blockIdx.x, b = blockIdx.y, np = m.npsr;
  const float* xb = x + (size_t)b * m.d;
  const double sr = srho[(size_t)b * m.na + k];
  for (int I = threadIdx.x; I < np; I += blockDim.x) {
    double s0 = 0.0, s1 = 0.0;
    for (int J = 0; J <= I; ++J) {
      const double l = m.LGamma[I * np + J];
      s0 = fma(l, (double)xb[m.z_ach + (2 * k) * np + J], s0);
      s1 = fma(l, (double)xb[m.z_ach + (2 * k + 1) * np + J], s1);
    }
    const size_t o = ((size_t)I * gridDim.y + b) * m.PM + 2 * k;
    a64[o] = sr * s0;
    a64[o + 1] = sr * s1;
  }
}

__global__ void k_gwbonly_adjoint(DevModel m, const float* __restrict__ x, const double* __restrict__ ghat,
                                  const double* __restrict__ srho, float* grad, double* dlnr, int B) {
  const int k = m.n_chol + blockIdx.x, b = blockIdx.y, np = m.npsr;
  const float* xb = x + (size_t)b * m.d;
  const double sr = srho[(size_t)b * m.na + k];
  double part = 0.0;
  for (int i = threadIdx.x; i < 2 * np; i += blockDim.x) {
    const int c = i / np, J = i % np;
    double s = 0.0;
    for (int I = J; I < np; ++I) s = fma(m.LGamma[I * np + J], ghat[((size_t)I * B + b) * m.P + 2 * k + c], s);
    s *= sr;
    const double z = (double)xb[m.z_ach + (2 * k) * np + i];
    grad[(size_t)b * m.d + m.z_ach + (2 * k) * np + i] = (float)(s - z);
    part += 0.5 * s * z;
  }
  __shared__ double red[32];
  for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    dlnr[(size_t)b * m.na + k] = s;
  }
}

// ---------------------------------------------------------------------------
// Diagonal bins: red-noise-only achromatic bins (n_gwb <= k < n_rn) and DM bins.
// a = sqrt(kappa) z; d logp/d z = sqrt(kappa) ghat - z;
// kappa d logp / d kappa = 1/2 sqrt(kappa) sum_c ghat_c z_c.
// One thread per (chain, pulsar, bin).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void diag_index(const DevModel& m, int r, int& I, int& k, bool& dm) {
  const int nrn_only = m.na - m.n_chol - m.n_gwbonly;  // achromatic diagonal bins
  const int per = nrn_only + m.nd;
  I = r / per;
  const int q = r % per;
  dm = q >= nrn_only;
  k = dm ? q - nrn_only : m.n_chol + m.n_gwbonly + q;
}

// Adjoint of the diagonal bins' transform (their forward is in k_spectra).  DW:
// double-word products (outside FP64 mode), whose only FP64 operation is the final add
// of each double output; the float gradient needs none.  A DM bin's two coefficients,
// z's and gradient entries are adjacent: one paired access each.
template <bool DW>
__global__ void k_diag_adjoint(DevModel m, const float* __restrict__ x, const double* __restrict__ ghat,
                               const double* __restrict__ sk, const double* __restrict__ skd, float* grad,
                               double* dlnk, double* dlnkd, int B, int per_chain) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
  if (r >= per_chain) return;
  int I, k;
  bool dm;
  diag_index(m, r, I, k, dm);
  const float* xb = x + (size_t)b * m.d;
  float* gb = grad + (size_t)b * m.d;
  const double s = dm ? skd[((size_t)b * m.npsr + I) * m.nd + k] : sk[((size_t)b * m.npsr + I) * m.na + k];
  const int z0i = dm ? m.z_dm + (I * m.nd + k) * 2 : m.z_ach + (2 * k) * m.npsr + I;
  const int z1i = dm ? z0i + 1 : z0i + m.npsr;
  const bool pair = dm && !(reinterpret_cast<uintptr_t>(xb + z0i) & 7);  // xb and gb rows share the offset
  const size_t o = ((size_t)I * B + b) * m.P + (dm ? 2 * m.na : 0) + 2 * k;
  const double2 g = *reinterpret_cast<const double2*>(ghat + o);
  float z0, z1;
  if (pair) {
    const float2 zz = *reinterpret_cast<const float2*>(xb + z0i);
    z0 = zz.x;
    z1 = zz.y;
  } else {
    z0 = xb[z0i];
    z1 = xb[z1i];
  }
  float gr0, gr1;
  double v;
  if (DW) {
    const float2 sw = d2dw_bits(s), g0 = dw_mul(sw, d2dw_bits(g.x)), g1 = dw_mul(sw, d2dw_bits(g.y));
    const float2 d0 = dw_addf(g0, -z0), d1 = dw_addf(g1, -z1);
    gr0 = __fadd_rn(d0.x, d0.y);
    gr1 = __fadd_rn(d1.x, d1.y);
    const float2 q = dw_add(dw_mulf(g0, z0), dw_mulf(g1, z1));  // s (g0 z0 + g1 z1)
    v = 0.5 * dw2d(q);
  } else {
    gr0 = (float)(s * g.x - z0);
    gr1 = (float)(s * g.y - z1);
    v = 0.5 * s * (g.x * z0 + g.y * z1);
  }
  if (pair) {
    *reinterpret_cast<float2*>(gb + z0i) = make_float2(gr0, gr1);
  } else {
    gb[z0i] = gr0;
    gb[z1i] = gr1;
  }
  if (dm)
    dlnkd[((size_t)b * m.npsr + I) * m.nd + k] = v;
  else
    dlnk[((size_t)b * m.npsr + I) * m.na + k] = v;
}

// ---------------------------------------------------------------------------
// Final per-chain assembly: logp = -1/2 sum_I chi2_I - 1/2 |z|^2 (FP64), prior box,
// status, and the hyper-parameter gradient by the chain rule through the power law:
// d/d log10A = 2 ln10 sum_k kappa_k dlogp/dkappa_k, d/d gamma = -sum_k ln(f_k/f_yr) (...).
// ---------------------------------------------------------------------------
template <bool DW>
__global__ void k_final(DevModel m, const float* __restrict__ x, const double* __restrict__ chi2,
                        const double* __restrict__ dlnk, const double* __restrict__ dlnkd,
                        const double* __restrict__ dlnr, const int32_t* __restrict__ stat,
                        const double* __restrict__ cwg, const double* __restrict__ curnQ,
                        const double* __restrict__ curnLd, const double* __restrict__ dlnrc, double* logp,
                        float* grad, int32_t* status, int B) {
  const int b = blockIdx.x, tid = threadIdx.x, nt = blockDim.x, np = m.npsr;
  const float* xb = x + (size_t)b * m.d;
  __shared__ double red[32];
  __shared__ int s_flag;
  if (tid == 0) s_flag = stat[b];
  __syncthreads();
  double acc = 0.0;
  if (m.curn) {  // CURN transform: HD prior terms per bin and log det L_CURN per pulsar
    for (int j = tid; j <= m.na; j += nt) acc += curnQ[(size_t)b * (m.na + 1) + j];
    for (int I = tid; I < np; I += nt) acc += curnLd[(size_t)I * B + b];
  } else if (!DW) {
    for (int j = tid; j < m.d_z; j += nt) acc = fma((double)xb[j], (double)xb[j], acc);
    acc *= -0.5;
  } else {  // -|z|^2 / 2: exact squares summed as double words, one FP64 add per thread;
            // four independent loads per step keep the loop off the load latency
    float2 zz = make_float2(0.0f, 0.0f);
    int j = tid;
    for (; j + 3 * nt < m.d_z; j += 4 * nt) {
      const float z0 = xb[j], z1 = xb[j + nt], z2 = xb[j + 2 * nt], z3 = xb[j + 3 * nt];
      const float p0 = __fmul_rn(z0, z0), p1 = __fmul_rn(z1, z1), p2 = __fmul_rn(z2, z2), p3 = __fmul_rn(z3, z3);
      const float2 s01 = dw_add(make_float2(p0, __fmaf_rn(z0, z0, -p0)), make_float2(p1, __fmaf_rn(z1, z1, -p1)));
      const float2 s23 = dw_add(make_float2(p2, __fmaf_rn(z2, z2, -p2)), make_float2(p3, __fmaf_rn(z3, z3, -p3)));
      zz = dw_add(zz, dw_add(s01, s23));
    }
    for (; j < m.d_z; j += nt) {
      const float z = xb[j], p = __fmul_rn(z, z);
      zz = dw_add(zz, make_float2(p, __fmaf_rn(z, z, -p)));
    }
    acc = -0.5 * dw2d(zz);
  }
  const double bt = m.beta ? m.beta[b] : 1.0;  // tempered likelihood: beta chi2
  for (int I = tid; I < np; I += nt) acc -= 0.5 * bt * chi2[(size_t)I * B + b];
  int outside = 0;
  for (int I = tid; I < np; I += nt) {
    if (m.rn_free) {
      for (int k = 0; k < m.n_rn; ++k) {
        const float v = xb[m.th_rn + m.n_rn * I + k];
        outside |= !(v > kFreeLo && v < kFreeHi);
      }
    } else {
      const float la = xb[m.th_rn + 2 * I], ga = xb[m.th_rn + 2 * I + 1];
      outside |= !(la > m.la_lo && la < m.la_hi && ga > m.g_lo && ga < m.g_hi);
    }
    if (m.nd) {
      const float ld = xb[m.th_dm + 2 * I], gd = xb[m.th_dm + 2 * I + 1];
      outside |= !(ld > m.la_lo && ld < m.la_hi && gd > m.g_lo && gd < m.g_hi);
    }
  }
  if (tid == 0) {
    if (m.gwb_free) {
      for (int k = 0; k < m.n_gwb; ++k) outside |= !(xb[m.th_gwb + k] > kFreeLo && xb[m.th_gwb + k] < kFreeHi);
    } else {
      const float la = xb[m.th_gwb], ga = xb[m.th_gwb + 1];
      outside |= !(la > m.la_lo && la < m.la_hi && ga > m.g_lo && ga < m.g_hi);
    }
  }
  if (m.cw) {
    // CW prior: box on the 8 binary parameters, pulsar phases in (0, 2 pi), distances
    // > 0 with a Gaussian of width dist_sigma around each pulsar's nominal distance
    const float* th = xb + m.th_cw;
    if (tid < 8) outside |= !(th[tid] > m.cw_lo[tid] && th[tid] < m.cw_hi[tid]);
    for (int I = tid; I < np; I += nt) {
      const double L = th[8 + 2 * I], ph = th[9 + 2 * I];
      outside |= !(L > 0.0 && ph > 0.0 && ph < 2.0 * kPi);
      const double dz = (L - m.dist[I]) / m.dist_sigma;
      acc -= 0.5 * dz * dz;
    }
  }
  if (outside) atomicOr(&s_flag, 1);
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((tid & 31) == 0) red[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < (nt >> 5); ++w) s += red[w];
    int fl = s_flag;
    if (!isfinite(s) && fl == 0) fl = 3;
    if (fl) {
      if (fl & 1) fl = 1;
      else if (fl & 2) fl = 2;
      s = -INFINITY;
    }
    logp[b] = s;
    if (status) status[b] = fl;
    s_flag = fl;
  }
  __syncthreads();
  if (!grad) return;
  float* gb = grad + (size_t)b * m.d;
  if (s_flag) {
    for (int j = tid; j < m.d; j += nt) gb[j] = 0.f;
    return;
  }
  // noise hyper-parameters: one warp per pulsar, lanes over the bins, shuffle sums
  const int lane = tid & 31, nwarp = nt >> 5;
  if (DW) {  // sums as double words: the FP64 pipe's latency is what this loop would wait on
    constexpr float2 kLn10w = {0x1.26bb1cp+1f, -0x1.12aabap-25f};
    auto wsum = [&](float2 v) {
      for (int o = 16; o; o >>= 1)
        v = dw_add(v, make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)));
      return v;
    };
    auto tof = [](float2 v) { return __fadd_rn(v.x, v.y); };
    for (int I = tid >> 5; I < np; I += nwarp) {
      float2 s1 = make_float2(0.0f, 0.0f), s2 = s1, d1 = s1, d2 = s1;
      for (int k = lane; k < m.n_rn; k += 32) {
        const float2 v = d2dw_bits(dlnk[((size_t)b * np + I) * m.na + k]);  // kappa d logp / d kappa
        if (m.rn_free) gb[m.th_rn + m.n_rn * I + k] = tof(dw_mul(kLn10w, v));  // d kappa / d theta = ln10 kappa
        s1 = dw_add(s1, v);
        s2 = dw_fms(s2, m.lkT[k + 1], v);
      }
      for (int k = lane; k < m.nd; k += 32) {
        const float2 v = d2dw_bits(dlnkd[((size_t)b * np + I) * m.nd + k]);
        d1 = dw_add(d1, v);
        d2 = dw_fms(d2, m.lkT[k + 1], v);
      }
      s1 = wsum(s1);
      s2 = wsum(s2);
      d1 = wsum(d1);
      d2 = wsum(d2);
      if (lane == 0) {
        if (!m.rn_free) {  // power-law chain rule
          gb[m.th_rn + 2 * I] = 2.0f * tof(dw_mul(kLn10w, s1));
          gb[m.th_rn + 2 * I + 1] = tof(s2);
        }
        if (m.nd) {
          gb[m.th_dm + 2 * I] = 2.0f * tof(dw_mul(kLn10w, d1));
          gb[m.th_dm + 2 * I + 1] = tof(d2);
        }
      }
    }
  }
  for (int I = tid >> 5; !DW && I < np; I += nwarp) {
    double s1 = 0.0, s2 = 0.0;
    for (int k = lane; k < m.n_rn; k += 32) {
      const double v = dlnk[((size_t)b * np + I) * m.na + k];  // kappa d logp / d kappa
      if (m.rn_free) gb[m.th_rn + m.n_rn * I + k] = (float)(kLn10 * v);  // d kappa / d theta = ln10 kappa
      s1 += v;
      s2 -= (m.lnk[k + 1] - m.ln_Tfyr) * v;
    }
    double d1 = 0.0, d2 = 0.0;
    for (int k = lane; k < m.nd; k += 32) {
      const double v = dlnkd[((size_t)b * np + I) * m.nd + k];
      d1 += v;
      d2 -= (m.lnk[k + 1] - m.ln_Tfyr) * v;
    }
    for (int o = 16; o; o >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      d1 += __shfl_xor_sync(0xffffffffu, d1, o);
      d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    }
    if (lane == 0) {
      if (!m.rn_free) {  // power-law chain rule
        gb[m.th_rn + 2 * I] = (float)(2.0 * kLn10 * s1);
        gb[m.th_rn + 2 * I + 1] = (float)s2;
      }
      if (m.nd) {
        gb[m.th_dm + 2 * I] = (float)(2.0 * kLn10 * d1);
        gb[m.th_dm + 2 * I + 1] = (float)d2;
      }
    }
  }
  if (tid < 32) {  // GWB hyper-parameters: lanes over the bins
    double s1 = 0.0, s2 = 0.0;
    for (int k = tid; k < m.n_gwb; k += 32) {
      double v = dlnr[(size_t)b * m.na + k];  // rho d logp / d rho
      if (m.curn)  // the transform's part, per pulsar, summed in a fixed order
        for (int I = 0; I < np; ++I) v += dlnrc[((size_t)b * np + I) * m.na + k];
      if (m.gwb_free) gb[m.th_gwb + k] = (float)(kLn10 * v);
      s1 += v;
      s2 -= (m.lnk[k + 1] - m.ln_Tfyr) * v;
    }
    for (int o = 16; o; o >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (!m.gwb_free && tid == 0) {
      gb[m.th_gwb] = (float)(2.0 * kLn10 * s1);
      gb[m.th_gwb + 1] = (float)s2;
    }
  }
  if (m.cw) {
    const float* th = xb + m.th_cw;
    const double* gc = cwg + (size_t)b * np * 10;
    if (tid < 8) {
      double s = 0.0;
      for (int I = 0; I < np; ++I) s += gc[I * 10 + tid];
      gb[m.th_cw + tid] = (float)(bt * s);
    }
    for (int I = tid; I < np; I += nt) {
      const double L = th[8 + 2 * I];
      gb[m.th_cw + 8 + 2 * I] = (float)(bt * gc[I * 10 + 8] - (L - m.dist[I]) / (m.dist_sigma * m.dist_sigma));
      gb[m.th_cw + 9 + 2 * I] = (float)(bt * gc[I * 10 + 9]);
    }
  }
}

}  // namespace

// Threads per CTA of the dense-bin kernels: their two packed triangles allow 5 CTAs per SM
// at 67 pulsars (8 warps each), but only one at 150 (181 KB), where few warps would leave
// the FP64 latency exposed: 16 warps per CTA there.
static int chol_threads(const DevModel& m) { return m.npsr >= 96 ? 512 : 256; }
static int chol_threads_dw(const DevModel& m) { return m.npsr >= 96 ? 512 : 256; }

static size_t chol_smem(const DevModel& m) {
  const size_t np = m.npsr, ntri = np * (np + 1) / 2;
  return (2 * ntri + 4 * np) * sizeof(double);
}
// The double-word sweep and adjoint run everywhere but in FP64 mode and when
// pta_set_cholesky asked for the FP64 sweep.
static bool chol_dw(const DevModel& m, int fp64) { return !fp64 && !m.chol64; }

static size_t adj_smem_dw(const DevModel& m) {
  const size_t np = m.npsr, ntri = np * (np + 1) / 2;
  const size_t nseg = std::max<size_t>(1, std::min<size_t>(4, chol_threads(m) / np));
  return (std::max(ntri, 5 * nseg * np + np) + ntri + 4 * np) * 8;
}
static size_t chol_smem_dw(const DevModel& m) {
  const size_t np = m.npsr, nh = np / 2 + 1;
  return 6 * nh * sizeof(float4) + (size_t)prow((int)np) * sizeof(float2);
}
static size_t adj_smem(const DevModel& m) {
  const size_t np = m.npsr, ntri = np * (np + 1) / 2;
  return (2 * ntri + 7 * np) * sizeof(double);
}

bool chol_uses_dw(const DevModel& m, int fp64) { return chol_dw(m, fp64); }

int count_prior_forward(const DevModel& m) {
  if (m.curn) return 1 + (m.n_chol > 0) + 2;  // spectra, Phi_k factors, CURN transform, HD prior
  return 1 + (m.n_chol > 0) + (m.n_gwbonly > 0);  // the diagonal bins' a comes with the spectra
}
int count_prior_adjoint(const DevModel& m) {
  if (m.curn) return 1;
  return (m.n_chol > 0) + (m.n_gwbonly > 0) + (m.npsr * ((m.na - m.n_chol - m.n_gwbonly) + m.nd) > 0);
}

cudaError_t launch_prior_forward(const DevModel& m, const Scratch& s, int B, const float* x, int fp64,
                                 cudaStream_t st, cudaEvent_t* kev) {
  const int nspec = m.npsr * (m.na + m.nd) + m.na;
  double* ad = m.curn ? nullptr : s.a64;  // the diagonal bins' a, written with their spectra
  if (fp64)
    k_spectra<false><<<dim3((nspec + 127) / 128, B), 128, 0, st>>>(m, x, s.sk, s.skd, s.srho, ad, B);
  else
    k_spectra<true><<<dim3((nspec + 127) / 128, B), 128, 0, st>>>(m, x, s.sk, s.skd, s.srho, ad, B);
  if (m.n_chol > 0) {
    const bool dw = chol_dw(m, fp64);
    const size_t sm = dw ? chol_smem_dw(m) : chol_smem(m);
    cudaError_t e = dw ? cudaFuncSetAttribute(k_chol_forward_dw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)
                       : cudaFuncSetAttribute(k_chol_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (kev) cudaEventRecord(kev[0], st);
    if (dw)
      k_chol_forward_dw<<<dim3(m.n_chol, B), chol_threads_dw(m), sm, st>>>(
          m, x, s.sk, s.srho, s.a64, reinterpret_cast<float2*>(s.Lpk), reinterpret_cast<float2*>(s.Lipk), s.stat);
    else
      k_chol_forward<<<dim3(m.n_chol, B), chol_threads(m), sm, st>>>(m, x, s.sk, s.srho, s.a64, s.Lpk, s.Lipk,
                                                                      s.stat);
    if (kev) cudaEventRecord(kev[1], st);
  }
  if (m.curn) return cudaGetLastError();  // a comes from the CURN transform (launch_curn_forward)
  if (m.n_gwbonly > 0) k_gwbonly_forward<<<dim3(m.n_gwbonly, B), 128, 0, st>>>(m, x, s.srho, s.a64);
  return cudaGetLastError();
}

cudaError_t launch_prior_adjoint(const DevModel& m, const Scratch& s, int B, const float* x, float* grad, int fp64,
                                 cudaStream_t st) {
  if (m.n_chol > 0) {
    const bool dw = chol_dw(m, fp64);
    const size_t sm = dw ? adj_smem_dw(m) : adj_smem(m);
    cudaError_t e = dw ? cudaFuncSetAttribute(k_chol_adjoint_dw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)
                       : cudaFuncSetAttribute(k_chol_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (dw)
      k_chol_adjoint_dw<<<dim3(m.n_chol, B), chol_threads(m), sm, st>>>(
          m, x, s.ghat, reinterpret_cast<const float2*>(s.Lpk), reinterpret_cast<const float2*>(s.Lipk), s.sk, grad,
          s.dlnk, s.dlnr, B);
    else
      k_chol_adjoint<<<dim3(m.n_chol, B), chol_threads(m), sm, st>>>(m, x, s.ghat, s.Lpk, s.Lipk, s.sk, grad, s.dlnk,
                                                                      s.dlnr, B);
  }
  if (m.n_gwbonly > 0)
    k_gwbonly_adjoint<<<dim3(m.n_gwbonly, B), 128, 0, st>>>(m, x, s.ghat, s.srho, grad, s.dlnr, B);
  const int per = m.npsr * ((m.na - m.n_chol - m.n_gwbonly) + m.nd);
  if (per > 0) {
    if (fp64)
      k_diag_adjoint<false><<<dim3((per + 127) / 128, B), 128, 0, st>>>(m, x, s.ghat, s.sk, s.skd, grad, s.dlnk,
                                                                      s.dlnkd, B, per);
    else
      k_diag_adjoint<true><<<dim3((per + 127) / 128, B), 128, 0, st>>>(m, x, s.ghat, s.sk, s.skd, grad, s.dlnk,
                                                                     s.dlnkd, B, per);
  }
  return cudaGetLastError();
}

cudaError_t launch_final(const DevModel& m, const Scratch& s, int B, const float* x, double* logp, float* grad,
                         int32_t* status, int fp64, cudaStream_t st) {
  (fp64 ? k_final<false> : k_final<true>)<<<B, 512, 0, st>>>(m, x, s.chi2, s.dlnk, s.dlnkd, s.dlnr, s.stat, s.cwg, s.curnQ, s.curnLd, s.dlnrc, logp,
                             grad, status, B);
  return cudaGetLastError();
}

}  // namespace pta
