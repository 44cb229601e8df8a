// Fixed-length HMC transitions (App. "Hamiltonian Monte Carlo": Eqs. Hamiltonian,
// Hamilton's_eq, Gaussian_momentum, HMC_acceptance) for a batch of chains.  The
// leapfrog loop and the accept step run as one CUDA graph per (B, n_leapfrog),
// captured on first use and replayed afterwards.  The graph only touches
// context-owned buffers; the caller's state is copied in and out around it.
//
// Bounded coordinates.  Every coordinate with a finite prior box [lo, hi] (the noise
// and GWB hyper-parameters, the CW box parameters and pulsar phases) moves during a
// trajectory in u = logit((x - lo) / (hi - lo)), x = lo + (hi - lo) sigmoid(u), with the
// target's log-Jacobian sum log((hi - lo) s (1 - s)) added to the Hamiltonian, so a
// trajectory never leaves the prior support (the unconstrained reparameterisation of a
// box-bounded parameter).  The caller's state, logp and gradient stay in x.
//
// Random numbers: Philox4x32-10 (Salmon et al., SC'11) with counter
// (block j, chain, iteration lo, iteration hi) and key (seed lo, seed hi); each
// block gives two Box-Muller pairs.  The Metropolis uniform uses block index
// 0xFFFFFFFF.
#include <cmath>

#include "pta_internal.cuh"

int pta_eval_internal(pta_ctx* c, int B, const float* x, double* logp, float* grad, int32_t* status,
                      cudaStream_t st);
int pta_prepare_internal(pta_ctx* c, int B);
int pta_ensure_bounds(pta_ctx* c);
int pta_check_result(pta_ctx* c, cudaStream_t st);

namespace pta {
namespace {

struct Philox {
  uint32_t c[4];
};

__device__ __forceinline__ Philox philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                           uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  Philox o;
  o.c[0] = c0;
  o.c[1] = c1;
  o.c[2] = c2;
  o.c[3] = c3;
  return o;
}

__device__ __forceinline__ float u01f(uint32_t w) { return fmaf((float)w, 2.3283064365386963e-10f, 1.1641532e-10f); }

__global__ void k_set_ctr(uint64_t* ctr, uint64_t seed, uint64_t it) {
  ctr[0] = seed;
  ctr[1] = it;
}

// p = n / sqrt(inv_mass), n ~ N(0, 1) from Philox block j of this chain
__global__ void k_momentum(const uint64_t* ctr, const float* imass, float* p, int D, int B) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
  if (4 * j >= D) return;
  const uint64_t seed = ctr[0], it = ctr[1];
  const Philox r = philox10((uint32_t)j, (uint32_t)b, (uint32_t)it, (uint32_t)(it >> 32), (uint32_t)seed,
                            (uint32_t)(seed >> 32));
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const float ua = u01f(r.c[2 * q]), ub = u01f(r.c[2 * q + 1]);
    const float rad = sqrtf(-2.0f * logf(ua));
    float s, c;
    sincospif(2.0f * ub, &s, &c);
    const float v[2] = {rad * c, rad * s};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int idx = 4 * j + 2 * q + e;
      if (idx < D) p[(size_t)b * D + idx] = v[e] * rsqrtf(imass[idx]);
    }
  }
}

__device__ __forceinline__ bool bounded(double lo, double hi) { return isfinite(lo) && isfinite(hi); }

// log sigmoid(u), stable for either sign
__device__ __forceinline__ double log_sig(double u) { return u >= 0.0 ? -log1p(exp(-u)) : u - log1p(exp(u)); }

// x = lo + (hi - lo) sigmoid(u) as a float strictly inside (lo, hi)
__device__ __forceinline__ float u_to_x(double u, double lo, double hi) {
  const double sg = 1.0 / (1.0 + exp(-u));
  float xf = (float)fma(hi - lo, sg, lo);
  for (int t = 0; t < 4 && (double)xf <= lo; ++t) xf = nextafterf(xf, INFINITY);
  for (int t = 0; t < 4 && (double)xf >= hi; ++t) xf = nextafterf(xf, -INFINITY);
  return xf;
}

// d/du of logp(x(u)) + log J(u) from g = d logp / dx
__device__ __forceinline__ float grad_u(float g, float u, double lo, double hi) {
  const double sg = 1.0 / (1.0 + exp(-(double)u));
  return (float)fma((double)g * (hi - lo), sg * (1.0 - sg), 1.0 - 2.0 * sg);
}

// Start of a trajectory: u from x (bounded coordinates), and K0 - log J(u0) per chain
// (FP64 accumulation, fixed order), the kinetic energy 1/2 p^T M^-1 p minus the
// log-Jacobian, so that H0 = -logp0 + kin0.
__global__ void k_start(const float* x0, const float* p, const float* imass, const double* lo, const double* hi,
                        float* us, double* kin, int D) {
  const int b = blockIdx.x;
  double s = 0.0;
  for (int j = threadIdx.x; j < D; j += blockDim.x) {
    const double v = p[(size_t)b * D + j];
    s += 0.5 * v * v * imass[j];
    const double xv = x0[(size_t)b * D + j];
    if (bounded(lo[j], hi[j])) {
      const double t = (xv - lo[j]) / (hi[j] - lo[j]);
      const double u = log(t) - log1p(-t);
      us[(size_t)b * D + j] = (float)u;
      s -= log(hi[j] - lo[j]) + log(t) + log1p(-t);
    } else {
      us[(size_t)b * D + j] = (float)xv;
    }
  }
  __shared__ double red[32];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    kin[b] = t;
  }
}

// half kick + drift in u:  p += eps/2 g_u;  u += eps M^-1 p;  x = x(u) for the evaluation
__global__ void k_kick_drift(float* us, float* x, float* p, const float* g, const float* step, const float* imass,
                             const double* lo, const double* hi, int D, int B) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)B * D) return;
  const int b = (int)(i / D), j = (int)(i % D);
  const float e = step[b];
  const bool bd = bounded(lo[j], hi[j]);
  const float gu = bd ? grad_u(g[i], us[i], lo[j], hi[j]) : g[i];
  const float pv = fmaf(0.5f * e, gu, p[i]);
  p[i] = pv;
  const float u = fmaf(e * imass[j], pv, us[i]);
  us[i] = u;
  x[i] = bd ? u_to_x(u, lo[j], hi[j]) : u;
}

__global__ void k_kick(float* p, const float* g, const float* us, const float* step, const double* lo,
                       const double* hi, int D, int B) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)B * D) return;
  const int j = (int)(i % D);
  const float gu = bounded(lo[j], hi[j]) ? grad_u(g[i], us[i], lo[j], hi[j]) : g[i];
  p[i] = fmaf(0.5f * step[i / D], gu, p[i]);
}

// Metropolis accept: H = -logp - log J(u) + K; accept if log u < H0 - H1 (finite H1 only).
__global__ void k_accept(const uint64_t* ctr, const double* lp0, const double* kin0, const double* lp1,
                         const float* p, const float* imass, const float* us, const double* lo, const double* hi,
                         float* x0, float* g0, double* lp0w, const float* x1, const float* g1, int32_t* accepted,
                         int D) {
  const int b = blockIdx.x;
  __shared__ double red[32];
  __shared__ int s_acc;
  double s = 0.0;
  for (int j = threadIdx.x; j < D; j += blockDim.x) {
    const double v = p[(size_t)b * D + j];
    s += 0.5 * v * v * imass[j];
    if (bounded(lo[j], hi[j])) {
      const double u = us[(size_t)b * D + j];
      s -= log(hi[j] - lo[j]) + log_sig(u) + log_sig(-u);
    }
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double k1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) k1 += red[w];
    const uint64_t seed = ctr[0], it = ctr[1];
    const Philox r = philox10(0xFFFFFFFFu, (uint32_t)b, (uint32_t)it, (uint32_t)(it >> 32), (uint32_t)seed,
                              (uint32_t)(seed >> 32));
    const double u = ((double)r.c[0] + 0.5) * 0x1.0p-32;
    const double H0 = -lp0[b] + kin0[b], H1 = -lp1[b] + k1;
    const int acc = isfinite(H1) && (log(u) < H0 - H1);
    s_acc = acc;
    accepted[b] = acc;
    if (acc) lp0w[b] = lp1[b];
  }
  __syncthreads();
  if (s_acc)
    for (int j = threadIdx.x; j < D; j += blockDim.x) {
      x0[(size_t)b * D + j] = x1[(size_t)b * D + j];
      g0[(size_t)b * D + j] = g1[(size_t)b * D + j];
    }
}

__global__ void k_fill(float* v, float val, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = val;
}

}  // namespace
}  // namespace pta

using namespace pta;

static int hmc_record(pta_ctx* c, int B, int L, cudaStream_t st) {
  const Scratch& s = c->sc;
  const int D = c->dm.d;
  const size_t n = (size_t)B * D;
  const unsigned nb = (unsigned)((n + 255) / 256);
  const double *lo = c->hmc_lo, *hi = c->hmc_hi;
  k_momentum<<<dim3((unsigned)(((D + 3) / 4 + 127) / 128), B), 128, 0, st>>>(s.hmc_ctr, s.imass, s.p, D, B);
  k_start<<<B, 256, 0, st>>>(s.x0, s.p, s.imass, lo, hi, s.us, s.kin0, D);
  cudaMemcpyAsync(s.gs, s.g0, n * sizeof(float), cudaMemcpyDeviceToDevice, st);
  for (int l = 0; l < L; ++l) {
    k_kick_drift<<<nb, 256, 0, st>>>(s.us, s.xs, s.p, s.gs, s.step, s.imass, lo, hi, D, B);
    int rc = pta_eval_internal(c, B, s.xs, s.lps, s.gs, nullptr, st);
    if (rc != PTA_OK) return rc;
    k_kick<<<nb, 256, 0, st>>>(s.p, s.gs, s.us, s.step, lo, hi, D, B);
  }
  k_accept<<<B, 256, 0, st>>>(s.hmc_ctr, s.lp0, s.kin0, s.lps, s.p, s.imass, s.us, lo, hi, s.x0, s.g0, s.lp0,
                              s.xs, s.gs, s.acc, D);
  return cudaGetLastError() == cudaSuccess ? PTA_OK : PTA_ECUDA;
}

extern "C" int pta_hmc_trajectory(pta_ctx* c, int B, float* x, double* logp, float* grad, const float* step,
                                  const float* inv_mass, int L, uint64_t seed, uint64_t iteration,
                                  int32_t* accepted, void* stream) {
  if (!c) return PTA_EINVAL;
  if (B < 0 || L < 1 || L > 100000 || (B > 0 && (!x || !logp || !grad || !step || !accepted))) {
    c->err = "hmc_trajectory: bad arguments";
    return PTA_EINVAL;
  }
  if (B == 0) return PTA_OK;
  if (c->dm.cw && c->precision != PTA_PREC_FP32 && c->precision != PTA_PREC_F16SPLIT) {
    c->err = "the continuous-wave model runs on the FP32 and exact-split paths (PTA_PREC_FP32, PTA_PREC_F16SPLIT)";
    return PTA_EINVAL;
  }
  int rc = pta_prepare_internal(c, B);
  if (rc == PTA_OK) rc = pta_ensure_bounds(c);
  if (rc != PTA_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const Scratch& s = c->sc;
  const int D = c->dm.d;
  const size_t n = (size_t)B * D;
  cudaError_t e = cudaSuccess;
  if (inv_mass)
    e = cudaMemcpyAsync(s.imass, inv_mass, D * sizeof(float), cudaMemcpyDeviceToDevice, st);
  else
    k_fill<<<(D + 255) / 256, 256, 0, st>>>(s.imass, 1.0f, D);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s.step, step, B * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s.x0, x, n * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s.g0, grad, n * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s.lp0, logp, B * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) {
    c->err = std::string("hmc copy-in: ") + cudaGetErrorString(e);
    return PTA_ECUDA;
  }
  k_set_ctr<<<1, 1, 0, st>>>(s.hmc_ctr, seed, iteration);
  cudaGraphExec_t exec = nullptr;
  for (auto& g : c->graphs)
    if (g.B == B && g.L == L) exec = g.exec;
  if (!exec) {
    // warm the launch attributes outside capture, then record the graph on a private stream
    if (!c->cap_stream) cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    cudaStreamSynchronize(st);
    rc = pta_eval_internal(c, B, s.x0, s.lps, s.gs, nullptr, c->cap_stream);
    if (rc != PTA_OK) return rc;
    cudaStreamSynchronize(c->cap_stream);
    cudaGraph_t graph;
    e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      c->err = std::string("graph capture: ") + cudaGetErrorString(e);
      return PTA_ECUDA;
    }
    rc = hmc_record(c, B, L, c->cap_stream);
    e = cudaStreamEndCapture(c->cap_stream, &graph);
    if (rc != PTA_OK || e != cudaSuccess) {
      c->err = std::string("graph capture: ") + cudaGetErrorString(e);
      return PTA_ECUDA;
    }
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      c->err = std::string("graph instantiate: ") + cudaGetErrorString(e);
      return PTA_ECUDA;
    }
    c->graphs.push_back({B, L, exec});
  }
  e = cudaGraphLaunch(exec, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(x, s.x0, n * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(grad, s.g0, n * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(logp, s.lp0, B * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(accepted, s.acc, B * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) {
    c->err = std::string("hmc launch: ") + cudaGetErrorString(e);
    return PTA_ECUDA;
  }
  return pta_check_result(c, st);
}
