// Deterministic continuous-wave signal h(theta) of a circular super-massive black
// hole binary (Sec. "Deterministic signals and continuous waves"; phase and
// frequency evolution of Eqs. phase_evolve and CW_evolve; antenna pattern,
// polarisation amplitudes and pulsar term of the circular-binary model of Ellis,
// Siemens & Creighton 2012), its timing-model projection and its gradient.
//
// For each (chain, pulsar) the signal is the pulsar term minus the Earth term,
//   s(t) = sum_T sigma_T alpha0_T (1 - kappa_T t)^(1/8) [A_s sin 2ph_T + A_c cos 2ph_T],
//   ph_T(t) = Phi_T + omega_T t (1 + corr(kappa_T t)),  corr(x) = (1-(1-x)^(5/8))/((5/8)x) - 1,
// with T in {Earth (sigma = -1), pulsar (sigma = +1)}; the pulsar term uses
// omega_P = omega_0 (1 + kappa_E L_f)^(-3/8), kappa_P = kappa_E / (1 + kappa_E L_f),
// L_f = L (1 + Omega . p), and its phase at t = 0 is the free parameter Phi_I.
// The ten per-(chain, pulsar) constants c = (omega_E, kappa_E, Phi_E, alpha0_E,
// omega_P, kappa_P, Phi_P, alpha0_P, A_s, A_c) and their Jacobian with respect to
// (log10 Mc, log10 f, log10 h, cos iota, psi, cos theta, phi, Phi0, L_I, Phi_I) come
// from an FP64 forward-mode (dual-number) evaluation.
//
// Precision: the linear phase omega_T t (up to ~1e2 rad) is formed exactly in
// 64-bit fixed-point turns from the TOA's 64-bit phase fraction; only the small
// chirp correction omega_T t corr(x) is FP32 (binomial series of corr for
// x <= 0.3, the closed form in FP64 above that).
#include <cmath>

#include "pta_internal.cuh"

namespace pta {
namespace {

constexpr int NP = 10;  // parameters per (chain, pulsar): 8 global + L_I + Phi_I

struct Dual {
  double v;
  double d[NP];
};
__device__ __forceinline__ Dual dconst(double v) {
  Dual r;
  r.v = v;
#pragma unroll
  for (int i = 0; i < NP; ++i) r.d[i] = 0.0;
  return r;
}
__device__ __forceinline__ Dual dvar(double v, int i) {
  Dual r = dconst(v);
  r.d[i] = 1.0;
  return r;
}
__device__ __forceinline__ Dual operator+(const Dual& a, const Dual& b) {
  Dual r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < NP; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
__device__ __forceinline__ Dual operator-(const Dual& a, const Dual& b) {
  Dual r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < NP; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
__device__ __forceinline__ Dual operator*(const Dual& a, const Dual& b) {
  Dual r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < NP; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
__device__ __forceinline__ Dual operator*(double s, const Dual& a) {
  Dual r;
  r.v = s * a.v;
#pragma unroll
  for (int i = 0; i < NP; ++i) r.d[i] = s * a.d[i];
  return r;
}
__device__ __forceinline__ Dual operator+(double s, const Dual& a) {
  Dual r = a;
  r.v += s;
  return r;
}
// f(a) with f'(a) given
__device__ __forceinline__ Dual dmap(const Dual& a, double f, double fp) {
  Dual r;
  r.v = f;
#pragma unroll
  for (int i = 0; i < NP; ++i) r.d[i] = fp * a.d[i];
  return r;
}
__device__ __forceinline__ Dual operator/(const Dual& a, const Dual& b) { return a * dmap(b, 1.0 / b.v, -1.0 / (b.v * b.v)); }
__device__ __forceinline__ Dual dsin(const Dual& a) { return dmap(a, sin(a.v), cos(a.v)); }
__device__ __forceinline__ Dual dcos(const Dual& a) { return dmap(a, cos(a.v), -sin(a.v)); }
__device__ __forceinline__ Dual dsqrt(const Dual& a) {
  const double s = sqrt(a.v);
  return dmap(a, s, 0.5 / s);
}
__device__ __forceinline__ Dual dpow(const Dual& a, double e) {
  const double p = pow(a.v, e);
  return dmap(a, p, e * p / a.v);
}
__device__ __forceinline__ Dual dexp10(const Dual& a) {
  const double p = exp10(a.v);
  return dmap(a, p, kLn10 * p);
}

// Per-(chain, pulsar) CW constants for the TOA kernels (FP32 where the TOA kernels
// compute in FP32, fixed-point turns for the phases) and the FP64 Jacobian.
struct CwConst {
  unsigned long long w_int[2], w_frac[2], phi_fix[2];  // 2 omega_T T/(2 pi) as 64.64 turns; Phi_T/pi
  float omega[2], kappa[2], alpha0[2];                 // per term (0 Earth, 1 pulsar)
  float As, Ac, T;
};

__device__ __forceinline__ void to_fixed_turns(double turns, unsigned long long& whole, unsigned long long& frac) {
  const double w = floor(turns);
  whole = (unsigned long long)(long long)w;
  const double f = turns - w;  // [0, 1)
  const double hi = floor(f * 4294967296.0);
  const double lo = floor((f * 4294967296.0 - hi) * 4294967296.0);
  frac = ((unsigned long long)hi << 32) + (unsigned long long)lo;
}

__global__ void k_cw_prep(DevModel m, const float* __restrict__ x, CwConst* __restrict__ cc,
                          double* __restrict__ jac, int B) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= B * m.npsr) return;
  const int b = r / m.npsr, I = r % m.npsr;
  const float* th = x + (size_t)b * m.d + m.th_cw;
  Dual p[NP];
#pragma unroll
  for (int i = 0; i < 8; ++i) p[i] = dvar((double)th[i], i);
  p[8] = dvar((double)th[8 + 2 * I], 8);
  p[9] = dvar((double)th[9 + 2 * I], 9);
  const Dual Mc = kTsunS * dexp10(p[0]);
  const Dual w0 = kPi * dexp10(p[1]);
  const Dual h = dexp10(p[2]);
  const Dual& ci = p[3];
  const Dual& psi = p[4];
  const Dual& ct = p[5];
  const Dual& phi = p[6];
  const double px = m.pos[3 * I], py = m.pos[3 * I + 1], pz = m.pos[3 * I + 2];
  const Dual st = dsqrt(1.0 + (-1.0) * (ct * ct));
  const Dual cph = dcos(phi), sph = dsin(phi);
  // propagation direction Omega = -(st cos phi, st sin phi, cos theta); basis m, n
  const Dual op = (-px) * (st * cph) + (-py) * (st * sph) + (-pz) * ct;
  const Dual mp = px * sph + (-py) * cph;
  const Dual np_ = (-px) * (ct * cph) + (-py) * (ct * sph) + pz * st;
  const Dual den = 1.0 + op;
  const Dual Fp = 0.5 * (mp * mp - np_ * np_) / den;
  const Dual Fx = (mp * np_) / den;
  const Dual kE = (256.0 / 5.0) * (dpow(Mc, 5.0 / 3.0) * dpow(w0, 8.0 / 3.0));
  const Dual Lf = (kKpcS * p[8]) * den;
  const Dual q = 1.0 + kE * Lf;
  const Dual wP = w0 * dpow(q, -3.0 / 8.0);
  const Dual kP = kE / q;
  const Dual w023 = dpow(w0, 2.0 / 3.0);
  const Dual a0E = (0.5e9) * (h / w0);  // ns
  const Dual a0P = (0.5e9) * (h / (w023 * dpow(wP, 1.0 / 3.0)));
  const Dual c2 = dcos(2.0 * psi), s2 = dsin(2.0 * psi);
  const Dual As = (-1.0) * ((1.0 + ci * ci) * (Fp * c2 + Fx * s2));
  const Dual Ac = 2.0 * (ci * (Fx * c2 - Fp * s2));
  const Dual* c[NP] = {&w0, &kE, &p[7], &a0E, &wP, &kP, &p[9], &a0P, &As, &Ac};
  double* J = jac + (size_t)r * NP * NP;
  for (int a = 0; a < NP; ++a)
#pragma unroll
    for (int j = 0; j < NP; ++j) J[a * NP + j] = c[a]->d[j];
  CwConst out;
  const double T = m.T;
  const double om[2] = {w0.v, wP.v}, ka[2] = {kE.v, kP.v}, ph[2] = {p[7].v, p[9].v}, al[2] = {a0E.v, a0P.v};
  for (int tt = 0; tt < 2; ++tt) {
    to_fixed_turns(om[tt] * T / kPi, out.w_int[tt], out.w_frac[tt]);  // 2 omega t / (2 pi) per unit span
    unsigned long long wh, fr;
    to_fixed_turns(ph[tt] / kPi, wh, fr);
    out.phi_fix[tt] = fr;
    out.omega[tt] = (float)om[tt];
    out.kappa[tt] = (float)ka[tt];
    out.alpha0[tt] = (float)al[tt];
  }
  out.As = (float)As.v;
  out.Ac = (float)Ac.v;
  out.T = (float)T;
  cc[r] = out;
}

// corr(x) and corr'(x) of the chirp phase; the binomial series (coefficients
// c_1 = 3/16, c_{n+1} = c_n (n + 1 - 5/8)/(n + 2)) below x = 0.3, closed form above.
__device__ __forceinline__ void chirp_corr(float x, float& corr, float& dcorr) {
  if (x <= 0.3f) {
    float cn[15];
    cn[0] = 0.1875f;
#pragma unroll
    for (int n = 1; n < 15; ++n) cn[n] = cn[n - 1] * ((float)n + 0.375f) / ((float)n + 2.0f);
    float s = cn[14], ds = 15.0f * cn[14];
#pragma unroll
    for (int n = 13; n >= 0; --n) {
      s = fmaf(s, x, cn[n]);
      ds = fmaf(ds, x, (float)(n + 1) * cn[n]);
    }
    corr = s * x;
    dcorr = ds;
  } else {  // late inspiral (rare): closed form in FP64
    const double xd = x, l = log1p(-xd);
    const double g = -expm1(0.625 * l);  // 1 - (1 - x)^(5/8)
    corr = (float)(g / (0.625 * xd) - 1.0);
    const double gp = 0.625 * exp(-0.375 * l);  // g'(x)
    dcorr = (float)((gp * xd - g) / (0.625 * xd * xd));
  }
}

// One term of the signal at one TOA: value and partials with respect to
// (omega, kappa, Phi, alpha0, A_s, A_c).
struct TermEval {
  float val, d_om, d_ka, d_ph, d_a0, d_as, d_ac;
};

__device__ __forceinline__ TermEval cw_term(const CwConst& k, int T, uint64_t U, float t) {
  const float x = k.kappa[T] * t;
  float corr, dcorr;
  chirp_corr(x, corr, dcorr);
  // phase of 2 ph in fixed-point turns: exact linear part + Phi + FP32 correction
  const uint64_t lin = k.w_int[T] * U + __umul64hi(k.w_frac[T], U);
  float ct = k.omega[T] * t * corr * 0.31830988618f;  // omega t corr / pi  (turns of 2 ph)
  ct -= rintf(ct);
  const uint64_t cfix = (uint64_t)(long long)__float2ll_rn(ct * 1.8446744e19f);
  float s2, c2;
  sincos_turns64(lin + k.phi_fix[T] + cfix, &s2, &c2);
  const float u = 1.0f - x;
  const float amp = k.alpha0[T] * expf(0.125f * log1pf(-x));
  const float pol = k.As * s2 + k.Ac * c2;
  TermEval e;
  e.val = amp * pol;
  const float dph = 2.0f * amp * (k.As * c2 - k.Ac * s2);  // d val / d ph
  e.d_ph = dph;
  e.d_om = dph * t * (1.0f + corr);
  e.d_ka = dph * k.omega[T] * t * t * dcorr - pol * amp * t / (8.0f * u);
  e.d_a0 = pol * (amp / k.alpha0[T]);
  e.d_as = amp * s2;
  e.d_ac = amp * c2;
  return e;
}

__device__ __forceinline__ float toa_time(const DevModel& m, uint64_t U) {
  return (float)(unsigned)(U >> 32) * (float)(m.T * 2.3283064365386963e-10);
}

// s at every TOA for one chain (CTA per (unit, chain), thread per TOA), stored
// chain-major [B][ntoa_pad], and bs = M^T N^-1 s per (unit, chain) (FP32 per-thread
// sums, FP64 fixed-order block sum).
__global__ void __launch_bounds__(128)
    k_cw_signal(DevModel m, const CwConst* __restrict__ cc, float* __restrict__ sig, double* __restrict__ bspart,
                int B, long long ntot) {
  extern __shared__ float accs[];  // [m_I][128]
  const int u = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
  const int I = m.unit_psr[u], start = m.unit_start[u], len = m.unit_len[u], mI = m.m[I];
  const CwConst k = cc[(size_t)b * m.npsr + I];
  const float* Mg = m.M32 + m.m_off[I] + (long long)(start - m.toa_off[I]) * mI;
  for (int j = 0; j < mI; ++j) accs[j * 128 + tid] = 0.f;
  for (int t0 = 0; t0 < len; t0 += 128) {
    const int ia = start + t0 + tid;
    const uint64_t U = m.phase[ia];
    const float t = toa_time(m, U);
    const TermEval e = cw_term(k, 0, U, t), p = cw_term(k, 1, U, t);
    const float s = p.val - e.val;
    const float ni = m.ninv[ia];
    sig[(size_t)b * ntot + ia] = ni > 0.f ? s : 0.f;
    const float sn = s * ni;
    for (int j = 0; j < mI; ++j) accs[j * 128 + tid] = fmaf(Mg[(long long)(t0 + tid) * mI + j], sn, accs[j * 128 + tid]);
  }
  __syncthreads();
  for (int j = tid; j < mI; j += 128) {
    double acc = 0.0;
    for (int i = 0; i < 128; ++i) acc += (double)accs[j * 128 + i];
    bspart[((size_t)u * B + b) * m.m_max + j] = acc;
  }
}

// sum_i w~_i ds_i/dc for the ten constants (CTA per (unit, chain), thread per TOA).
__global__ void __launch_bounds__(128)
    k_cw_grad(DevModel m, const CwConst* __restrict__ cc, const float* __restrict__ wt, double* __restrict__ gpart,
              int B, long long ntot) {
  __shared__ float red[NP][128];
  const int u = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
  const int I = m.unit_psr[u], start = m.unit_start[u], len = m.unit_len[u];
  const CwConst k = cc[(size_t)b * m.npsr + I];
  float g[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) g[i] = 0.f;
  for (int t0 = 0; t0 < len; t0 += 128) {
    const int ia = start + t0 + tid;
    const float w = wt[(size_t)b * ntot + ia];
    const uint64_t U = m.phase[ia];
    const float t = toa_time(m, U);
    const TermEval e = cw_term(k, 0, U, t), p = cw_term(k, 1, U, t);
    // s = pulsar - Earth
    g[0] = fmaf(-w, e.d_om, g[0]);
    g[1] = fmaf(-w, e.d_ka, g[1]);
    g[2] = fmaf(-w, e.d_ph, g[2]);
    g[3] = fmaf(-w, e.d_a0, g[3]);
    g[4] = fmaf(w, p.d_om, g[4]);
    g[5] = fmaf(w, p.d_ka, g[5]);
    g[6] = fmaf(w, p.d_ph, g[6]);
    g[7] = fmaf(w, p.d_a0, g[7]);
    g[8] = fmaf(w, p.d_as - e.d_as, g[8]);
    g[9] = fmaf(w, p.d_ac - e.d_ac, g[9]);
  }
#pragma unroll
  for (int i = 0; i < NP; ++i) red[i][tid] = g[i];
  __syncthreads();
  if (tid < NP) {
    double acc = 0.0;
    for (int i = 0; i < 128; ++i) acc += (double)red[tid][i];
    gpart[((size_t)u * B + b) * NP + tid] = acc;
  }
}

// Per (chain, pulsar): reduce the unit partials, apply the Jacobian; the result
// d logp / d theta (10 numbers: 8 global contributions + L_I + Phi_I) is summed over
// pulsars for the global ones in k_final.
__global__ void k_cw_apply(DevModel m, const double* __restrict__ gpart, const double* __restrict__ jac,
                           double* __restrict__ gcw, int B) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= B * m.npsr) return;
  const int b = r / m.npsr, I = r % m.npsr;
  double G[NP];
  for (int a = 0; a < NP; ++a) G[a] = 0.0;
  for (int j = 0; j < m.nunit[I]; ++j) {
    const double* gp = gpart + ((size_t)(m.unit0[I] + j) * B + b) * NP;
    for (int a = 0; a < NP; ++a) G[a] += gp[a];
  }
  const double* J = jac + (size_t)r * NP * NP;
  for (int j = 0; j < NP; ++j) {
    double s = 0.0;
    for (int a = 0; a < NP; ++a) s = fma(G[a], J[a * NP + j], s);
    gcw[(size_t)r * NP + j] = s;
  }
}

}  // namespace

size_t cw_const_bytes() { return sizeof(CwConst); }

cudaError_t launch_cw_forward(const DevModel& m, const Scratch& s, int B, const float* x, cudaStream_t st) {
  const int n = B * m.npsr;
  k_cw_prep<<<(n + 63) / 64, 64, 0, st>>>(m, x, reinterpret_cast<CwConst*>(s.cwc), s.cwjac, B);
  const size_t sm = sizeof(float) * 128 * std::max(1, m.m_max);
  cudaError_t e = cudaFuncSetAttribute(k_cw_signal, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_cw_signal<<<dim3(m.n_units, B), 128, sm, st>>>(m, reinterpret_cast<const CwConst*>(s.cwc), s.cwsig, s.cwbs, B,
                                                   m.ntoa_pad);
  return cudaGetLastError();
}

cudaError_t launch_cw_gradient(const DevModel& m, const Scratch& s, int B, cudaStream_t st) {
  k_cw_grad<<<dim3(m.n_units, B), 128, 0, st>>>(m, reinterpret_cast<const CwConst*>(s.cwc), s.cwwt, s.cwgp, B,
                                                m.ntoa_pad);
  const int n = B * m.npsr;
  k_cw_apply<<<(n + 127) / 128, 128, 0, st>>>(m, s.cwgp, s.cwjac, s.cwg, B);
  return cudaGetLastError();
}

}  // namespace pta
