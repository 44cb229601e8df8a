// Gram form of the timing-model-marginalised likelihood (Eq. posterior_implemented):
// with the per-pulsar matrices G~ = F^T N~^-1 F, g'' = F^T N^-1 dt'' and the constant
// c'' = dt''^T N^-1 dt'' stored at finalize (dt'' the projected reference residual of
// the reference fit a_ref), every evaluation needs only
//   da = a - a_ref,   v = G~ da,
//   chi2 = c'' - 2 da . g'' + da . v,   ghat = d logp / d a = g'' - v,
// per (pulsar, chain): P^2 multiply-adds instead of the 2 N (2P + m) of the TOA pass.
// The deterministic signal enters at the TOA level and is not supported here.
//
// Precision: at the 67-pulsar size da . g'' and da . G~ da are ~1e5, so FP32 rounding of
// G~ or da alone would cost ~1e-2 nats.  G~ and da are split into FP32 hi/lo pairs and
// each row of v is an Ogita-Rump-Oishi Dot2 (error-free products and sums) over the
// terms hi*hi with hi*lo + lo*hi added to the compensation: about FP64 accuracy at
// FP32 speed.  da . g'', da . v, chi2 and ghat are FP64.
#include "pta_internal.cuh"

namespace pta {
namespace {

constexpr int kGThreads = 256;

// stride of a per-chain row in shared memory: >= P, multiple of 4, = 4 (mod 32), so
// that the 16-byte loads of 8 consecutive chains hit disjoint banks
__host__ __device__ inline int gram_stride(int P) {
  int s = (P + 3) & ~3;
  while ((s & 31) != 4) s += 4;
  return s;
}

// one term of a compensated dot product (Ogita, Rump & Oishi 2005, Dot2) on hi/lo
// operands: s + c accumulates (a + al)(x + xl) to about twice the working precision
__device__ __forceinline__ void dot2_step(float a, float al, float x, float xl, float& s, float& c) {
  const float pr = a * x;
  const float pe = fmaf(a, x, -pr);            // exact product error
  const float t = s + pr;
  const float z = t - s;
  const float se = (s - (t - z)) + (pr - z);   // exact sum error
  s = t;
  c += se + pe + fmaf(a, xl, al * x);
}

template <int BC>
__global__ void __launch_bounds__(kGThreads)
    k_gram(DevModel m, const double* __restrict__ a64, double* __restrict__ ghat, double* __restrict__ chi2, int B) {
  extern __shared__ float4 smg4[];
  const int I = blockIdx.x, b0 = blockIdx.y * BC, tid = threadIdx.x;
  const int P = m.P, P4 = (P + 3) & ~3, SP = gram_stride(P);
  float* dh = reinterpret_cast<float*>(smg4);  // [BC][SP]  da, FP32 head
  float* dl = dh + BC * SP;                     // [BC][SP]  da, FP32 tail
  double* red = reinterpret_cast<double*>(dl + BC * SP);  // [2][kGThreads / BC][BC]
  const double* aref = m.aref + (size_t)I * P;
  for (int e = tid; e < BC * SP; e += kGThreads) {
    const int c = e / SP, p = e % SP, b = b0 + c;
    double d = 0.0;
    if (b < B && p < P) d = a64[((size_t)I * B + b) * m.PM + p] - aref[p];
    const float h = (float)d;
    dh[e] = h;
    dl[e] = (float)(d - (double)h);
  }
  __syncthreads();
  // v = G~ da, one row per warp-iteration: the row's loads are warp-uniform broadcasts
  constexpr int NR = kGThreads / BC;  // row groups
  const int c = tid % BC, rg = tid / BC;
  const float* Gh = m.Gth + (size_t)I * P * P4;
  const float* Gl = m.Gtl + (size_t)I * P * P4;
  const float4* xh4 = reinterpret_cast<const float4*>(dh + c * SP);
  const float4* xl4 = reinterpret_cast<const float4*>(dl + c * SP);
  double t2 = 0.0;  // da . v for this thread's rows
  double* gout = ghat + ((size_t)I * B + b0 + c) * P;
  const double bt = (m.beta && b0 + c < B) ? m.beta[b0 + c] : 1.0;  // tempered likelihood
  const double* g2 = m.g2 + (size_t)I * P;
  for (int r = rg; r < P; r += NR) {
    const float4* gh4 = reinterpret_cast<const float4*>(Gh + (size_t)r * P4);
    const float4* gl4 = reinterpret_cast<const float4*>(Gl + (size_t)r * P4);
    float s = 0.f, cmp = 0.f;
    for (int q = 0; q < P4 / 4; ++q) {
      const float4 a = __ldg(gh4 + q), al = __ldg(gl4 + q), x = xh4[q], xl = xl4[q];
      dot2_step(a.x, al.x, x.x, xl.x, s, cmp);
      dot2_step(a.y, al.y, x.y, xl.y, s, cmp);
      dot2_step(a.z, al.z, x.z, xl.z, s, cmp);
      dot2_step(a.w, al.w, x.w, xl.w, s, cmp);
    }
    const double v = (double)s + (double)cmp;
    if (b0 + c < B) gout[r] = bt * (g2[r] - v);
    t2 = fma((double)dh[c * SP + r] + (double)dl[c * SP + r], v, t2);
  }
  // da . g'' over this thread's share of the coefficients
  double t1 = 0.0;
  for (int p = rg; p < P; p += NR) t1 = fma((double)dh[c * SP + p] + (double)dl[c * SP + p], g2[p], t1);
  red[rg * BC + c] = t1;
  red[NR * BC + rg * BC + c] = t2;
  __syncthreads();
  if (tid < BC && b0 + tid < B) {
    double s1 = 0.0, s2 = 0.0;
    for (int g = 0; g < NR; ++g) {  // fixed order
      s1 += red[g * BC + tid];
      s2 += red[NR * BC + g * BC + tid];
    }
    chi2[(size_t)I * B + b0 + tid] = m.c2[I] - 2.0 * s1 + s2;
  }
}

template <int BC>
size_t gram_smem(const DevModel& m) {
  return sizeof(float) * 2 * (size_t)BC * gram_stride(m.P) + sizeof(double) * 2 * kGThreads;
}

template <int BC>
cudaError_t launch_gram_bc(const DevModel& m, const Scratch& s, int B, cudaStream_t st) {
  const size_t sm = gram_smem<BC>(m);
  cudaError_t e = cudaFuncSetAttribute(k_gram<BC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_gram<BC><<<dim3(m.npsr, (B + BC - 1) / BC), kGThreads, sm, st>>>(m, s.a64, s.ghat, s.chi2, B);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gram(const DevModel& m, const Scratch& s, int B, cudaStream_t st) {
  if (m.cw) return cudaErrorInvalidValue;
  if (gram_smem<32>(m) <= 200 * 1024) return launch_gram_bc<32>(m, s, B, st);
  if (gram_smem<16>(m) <= 200 * 1024) return launch_gram_bc<16>(m, s, B, st);
  if (gram_smem<8>(m) <= 200 * 1024) return launch_gram_bc<8>(m, s, B, st);
  return cudaErrorInvalidValue;
}

}  // namespace pta
