// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ptahmc.h"
#include "pta_check.cuh"

namespace pta {


constexpr double kYearS = 365.25 * 86400.0;
constexpr double kFyr = 1.0 / kYearS;
constexpr double kLn10 = 2.302585092994045684;
constexpr double kPi = 3.141592653589793238;
constexpr double kTsunS = 4.925490947641267e-06;  // G Msun / c^3
constexpr double kKpcS = 1.0292712503e11;         // 1 kpc / c
constexpr int kTile = 128;       // TOAs per pulsar are padded to a multiple of this
constexpr int kChunk = 2048;     // TOAs per work unit of the TOA kernels
// The per-frequency Cholesky and its adjoint hold two packed N_p x N_p triangles
// and 7 N_p vectors in FP64 shared memory: (N_p (N_p + 1) + 7 N_p) x 8 B <= 227 KB.
constexpr int kMaxPsr = 166;
constexpr int kLowBins = 4;  // lowest frequencies whose basis columns are projected off the timing model
constexpr double kFreeLo = -20.0, kFreeHi = -5.0;  // free-spectrum prior box, log10 (s^2) (Sec. Priors)

// Everything a kernel needs about the model and the resident data.  Passed by
// value; all pointers are device pointers owned by the context.
struct DevModel {
  int npsr, na, nd, n_gwb, n_rn, P, Qs, PM, d_z, d, cw;   // PM: coefficient row stride
  int nla, nld, NL;  // projected low-frequency columns: achromatic k <= nla, DM k <= nld; NL = 2 (nla + nld)
  int z_ach, z_dm, th_rn, th_dm, th_gwb, th_cw;
  int n_chol;      // bins k < n_chol: Phi_k = rho_k Gamma + diag(kappa_.k), full Cholesky
  int n_gwbonly;   // bins n_chol <= k < n_chol + n_gwbonly: Phi_k = rho_k Gamma
  int n_units, m_max;
  long long ntoa_pad;           // padded TOA count (row length of per-chain TOA arrays)
  double cw_lo[8], cw_hi[8];    // CW prior box; pulsar phase in (0, 2 pi), distance > 0
  double dist_sigma;            // pulsar-distance prior width [kpc]
  double T, ln_Tfyr, ln_rho0;   // T [s], ln(T f_yr), power-law normalisation (see ln_pl)
  double la_lo, la_hi, g_lo, g_hi;
  // per TOA (padded; padding rows have ninv = 0)
  const uint64_t* phase;        // round(2^64 (t - t0)/T)
  const float* chrom;           // (nu_ref/nu)^2
  const float* dt;              // reference-projected residual dt'' [ns] (see finalize)
  const float* ninv;            // 1/N_ii [1/ns^2]
  const float* M32;             // per pulsar [n_pad x m_I] row-major, normalised columns
  const double* dt64;
  const double* ninv64;
  const double* chrom64;
  const double* F64;            // per pulsar [n_pad x P] (FP64 path only, built on first use)
  const unsigned char* xmlo;    // BF16 tensor-core path: fixed basis columns per 64-TOA tile (built on first use)
  // Gram form (Eq. posterior_implemented) with the reference fit: per pulsar
  // G~ = F^T N~^-1 F [P x P] as FP32 hi/lo, g'' = F^T N^-1 dt'' [P], c'' = dt''^T N^-1 dt''
  int gwb_free, rn_free;        // free spectral models (one log10 variance per bin)
  int nthr;                     // red-noise parameters per pulsar (2, or n_rn when free)
  const double* beta;           // per-chain inverse temperature (App. "tempered likelihoods"); nullptr: 1
  int inject;                   // test hook (pta_debug_inject): 1 = the BF16 kernel withholds one MMA completion
  long long* chk;               // index-check record of the check build (site, value, limit); unused otherwise
  const float* Gth;
  const float* Gtl;
  const double* g2;
  const double* c2;
  const double* M64;            // per pulsar [n_pad x m_I]
  // per pulsar
  const int* toa_off;           // start of the pulsar in the padded TOA arrays
  const int* n_pad;
  const int* m;
  const long long* m_off;       // element offset of the pulsar's M block
  const long long* f_off;       // element offset of the pulsar's F64 block
  const int* unit0;             // first work unit of the pulsar
  const int* nunit;
  const int* lk_off;            // offset of chol(M^T N^-1 M) (m x m, row-major FP64)
  const double* LK;
  const double* Kinv;           // (M^T N^-1 M)^-1, same offsets as LK
  const int* h_off;             // offset of F^T N^-1 M (P x m row-major FP64)
  const double* H;
  const float* Hhi;             // H split into FP32 hi + lo parts (same layout as H)
  const float* Hlo;
  const double* aref;           // [npsr][P] reference coefficients (numerical conditioning)
  const float* Flo;             // per pulsar [n_pad x NL] projected low-frequency basis
  const long long* flo_off;
  const double* pos;            // [npsr][3]
  const double* dist;           // [npsr]
  // per unit
  const int* unit_psr;
  const int* unit_start;        // absolute padded TOA index
  const int* unit_len;          // multiple of 64
  const int* unit_order;        // units by decreasing length (persistent TOA launches)
  int nsm;                      // streaming multiprocessors of the device
  // global
  const double* lnk;            // ln k, k = 0..max(na, nd) (entry 0 unused)
  const float2* lkT;            // ln k - ln(T f_yr) as float pairs, k = 0..max(na, nd)
  int chol64;                   // 1: FP64 dense-bin Cholesky even outside FP64 mode (pta_set_cholesky)
  float2 hr0;                   // ln_rho0 / 2 as a float pair
  const unsigned short* trimap; // packed-lower index -> (row << 8) | col, for npsr <= 256
  const double* Gamma;          // [npsr x npsr]
  const float2* Gamma_dw;       // Gamma packed lower (trimap order) as double-word float pairs
  const double* LGamma;         // chol(Gamma), lower, [npsr x npsr]
  const double* LGammaInv;      // chol(Gamma)^-1, lower, [npsr x npsr]
  // CURN-posterior transform (Eq. PTA_standard_transform_curn), when curn = 1
  int curn;
  const double* Grev;           // per pulsar G~ = F^T N~^-1 F, packed lower in reversed order
                                // (element (i', l') = G~[P-1-i'][P-1-l']), P (P + 1) / 2 each
  const float2* Grev_dw;        // the same as double-word float pairs
  const double* gt;             // [npsr][P] F^T N~^-1 dt (FP64)
  const double* ga;             // [npsr][P] G~ a_ref (mean with the deterministic signal)
  // exact-split fp16 tensor-core path (PTA_PREC_F16SPLIT)
  const double* KiH;            // (M^T N^-1 M)^-1 H^T per pulsar [m_I x P] FP64, offsets h_off
  // exact-split fp16 tensor-core path: the stored basis pieces (built on first use)
  const uint32_t* x16;          // pieces; pulsar I's start at word x16_off[I]
  const long long* x16_off;
  const int* x16_cexp;          // [npsr][x16_kxm] column exponents c_q: |column q| < 2^c_q
  int x16_kxm;                  // stored columns per pulsar, largest (row length of x16_cexp)
  long long x16_blocks;         // stored 16 KB blocks in all
};

// Scratch sized for a batch of up to `cap` chains.
struct Scratch {
  int cap = 0;
  float* a32 = nullptr;        // [npsr][cap][PM]  (a, then timing-model offsets c)
  unsigned char* a16 = nullptr; // BF16 hi/lo coefficient chunks in the tensor-core layout
  double* a64 = nullptr;       // [npsr][cap][PM]
  double* Lpk = nullptr;       // [cap][n_chol][np(np+1)/2]; double-word float pairs outside FP64 mode
  double* Lipk = nullptr;      // same, inverse factor
  float* gpart = nullptr;      // [units][cap][Qs]
  double* gpart64 = nullptr;   // [units][cap][Qs] (FP64 path)
  double* c2part = nullptr;    // [units][cap]
  double* ghat = nullptr;      // [npsr][cap][P]
  double* chi2 = nullptr;      // [npsr][cap]
  double* dlnk = nullptr;      // [cap][npsr][na]  kappa dlogp/dkappa (achromatic)
  double* dlnkd = nullptr;     // [cap][npsr][nd]  same for DM
  double* dlnr = nullptr;      // [cap][na]        rho dlogp/drho
  int32_t* stat = nullptr;     // [cap]
  double* sk = nullptr;        // [cap][npsr][na]  sqrt(kappa) intrinsic red noise (0 above n_rn)
  double* skd = nullptr;       // [cap][npsr][nd]  sqrt(kappa) DM
  double* srho = nullptr;      // [cap][na]        sqrt(rho) GWB (0 above n_gwb)
  // continuous-wave signal (only when the model has it)
  unsigned char* cwc = nullptr; // [cap][npsr] per-(chain, pulsar) constants
  double* cwjac = nullptr;     // [cap][npsr][10][10]
  float* cwsig = nullptr;      // [cap][ntoa_pad] signal s
  double* cwbs = nullptr;      // [units][cap][m_max] M^T N^-1 s partials
  float* cwwt = nullptr;       // [cap][ntoa_pad] whitened projected residual w~
  double* cwgp = nullptr;      // [units][cap][10]
  double* cwg = nullptr;       // [cap][npsr][10] d logp / d theta contributions
  // HMC state
  float* x0 = nullptr;         // [cap][d]
  float* g0 = nullptr;
  float* p = nullptr;
  double* lp0 = nullptr;
  float* xs = nullptr;         // working state (x, evaluated)
  float* us = nullptr;         // working state with bounded coordinates in u = logit((x - lo)/(hi - lo))
  float* gs = nullptr;
  double* lps = nullptr;
  float* step = nullptr;       // [cap]
  float* imass = nullptr;      // [d]
  double* kin0 = nullptr;      // [cap]
  uint64_t* hmc_ctr = nullptr; // [2] seed, iteration
  int32_t* acc = nullptr;      // [cap] accept flags
  int* queue = nullptr;        // [1] work counter of persistent launches
  // CURN transform (allocated when it is selected)
  double* curnW = nullptr;     // [npsr][cap][P (P + 1) / 2] inverse factor Y' (reversed order)
  double* curnAhat = nullptr;  // [npsr][cap][P] ahat
  double* curnV = nullptr;     // [npsr][cap][P] phi^-1 a (HD prior)
  double* curnLd = nullptr;    // [npsr][cap] log det L_CURN
  double* curnQ = nullptr;     // [cap][na + 1] HD-prior terms per achromatic bin and the DM block
  double* dlnrc = nullptr;     // [cap][npsr][na] rho d logp / d rho through the transform, per pulsar
  // CURN transform with the deterministic signal (Eq. decenter_det_PTA)
  double* curnG0 = nullptr;    // [npsr][cap][P] beta F^T N~^-1 (dt'' - s) from the pass at a = a_ref
  double* curnV2 = nullptr;    // [npsr][cap][P] A^-1 gbar (CW gradient through the mean)
  float* cwwt2 = nullptr;      // [cap][ntoa_pad] N~^-1 F A^-1 gbar at every TOA
  double* chi2b = nullptr;     // [npsr][cap] chi2 of the auxiliary passes (unused)
  float* zeros = nullptr;      // [ntoa_pad] zero residual for the auxiliary pass
  // exact-split fp16 tensor-core path (allocated when it is selected)
  unsigned char* c16 = nullptr; // [npsr][chain blocks] 4 fp16 pieces of the scaled coefficients
  int* yexp = nullptr;          // [npsr][cap] exponent of F a per chain
  float* wres = nullptr;        // [cap][ntoa_pad] whitened projected residual w~
  float* wmx = nullptr;         // [units][cap] max |w~| of the unit
};

// Kernel launchers (defined in the .cu files).
cudaError_t launch_prior_forward(const DevModel& m, const Scratch& s, int B, const float* x,
                                 int fp64, cudaStream_t st, cudaEvent_t* kev = nullptr);  // kev: 2 events around k_chol_forward
cudaError_t launch_toa_fp32(const DevModel& m, const Scratch& s, int B, cudaStream_t st);
// SIMT tile-shape table (autotuner): entry count, shape of entry i, whether entry i
// can run this model, the default entry, and a launch with a chosen entry (-1: default)
int simt_count();
int simt_info(int i, int* bc, int* tt, int* qpt, int* ord);
bool simt_valid(const DevModel& m, int i);
int simt_default(const DevModel& m);
cudaError_t launch_toa_fp32_cfg(const DevModel& m, const Scratch& s, int B, int cfg, cudaStream_t st);
cudaError_t launch_toa_fp64(const DevModel& m, const Scratch& s, int B, cudaStream_t st);
cudaError_t launch_toa_tc(const DevModel& m, const Scratch& s, int B, int terms, cudaStream_t st);
bool bf16_supported(const DevModel& m);
size_t bf16_pack_bytes(const DevModel& m, int cap);
size_t bf16_xmlo_bytes(const DevModel& m);
cudaError_t build_bf16_xmlo(const DevModel& m, unsigned char* out, cudaStream_t st);
cudaError_t launch_toa_bf16(const DevModel& m, const Scratch& s, int B, cudaStream_t st);
cudaError_t launch_gram(const DevModel& m, const Scratch& s, int B, cudaStream_t st);
bool f16_supported(const DevModel& m);
size_t f16_pack_bytes(const DevModel& m, int cap);
cudaError_t build_f16_basis(DevModel& m, const std::vector<int>& n_pad, const std::vector<int>& mI,
                            std::vector<void*>& allocs);
// kev (optional): 4 events recorded around k_f16_res and k_f16_ftw
cudaError_t launch_toa_f16(const DevModel& m, const Scratch& s, int B, cudaStream_t st, cudaEvent_t* kev = nullptr);
size_t cw_const_bytes();
cudaError_t launch_cw_forward(const DevModel& m, const Scratch& s, int B, const float* x, cudaStream_t st);
cudaError_t launch_cw_gradient(const DevModel& m, const Scratch& s, int B, cudaStream_t st);
cudaError_t launch_tm_prologue(const DevModel& m, const Scratch& s, int B, int fp64, cudaStream_t st);
cudaError_t launch_reduce(const DevModel& m, const Scratch& s, int B, int fp64, cudaStream_t st);
cudaError_t launch_prior_adjoint(const DevModel& m, const Scratch& s, int B, const float* x,
                                 float* grad, int fp64, cudaStream_t st);
int count_prior_forward(const DevModel& m);
size_t curn_w_doubles(const DevModel& m);  // P (P + 1) / 2
cudaError_t launch_curn_forward(const DevModel& m, const Scratch& s, int B, const float* x, int fp64,
                                cudaStream_t st);
// the dense-bin Cholesky of this evaluation runs in double words (factors as float pairs)
bool chol_uses_dw(const DevModel& m, int fp64);
cudaError_t launch_curn_adjoint(const DevModel& m, const Scratch& s, int B, const float* x, float* grad, int fp64,
                                cudaStream_t st);
// a64 = a_ref - v (v == nullptr: a_ref) for every chain; out -= w elementwise
cudaError_t launch_curn_set_a(const DevModel& m, const Scratch& s, int B, const double* v, cudaStream_t st);
cudaError_t launch_sub(float* out, const float* w, size_t n, cudaStream_t st);
int count_prior_adjoint(const DevModel& m);
cudaError_t launch_final(const DevModel& m, const Scratch& s, int B, const float* x,
                         double* logp, float* grad, int32_t* status, int fp64, cudaStream_t st);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
// log of the power-law spectrum (Eq. power_law) in ns^2 at bin k (f_k = k/T):
// rho_k = A^2 / (12 pi^2 f_yr^3 T) (f_k / f_yr)^(-gamma), so
// ln rho_k = 2 ln10 log10A + ln_rho0 - gamma (ln k - ln(T f_yr))  (argument lnk = ln k),
// ln_rho0 = ln(1e18 / (12 pi^2 f_yr^3 T)) computed on the host in FP64.
__host__ __device__ inline double ln_pl(double ln_rho0, double ln_Tfyr, double log10A, double gamma, double lnk) {
  return 2.0 * kLn10 * log10A + ln_rho0 - gamma * (lnk - ln_Tfyr);
}

// sin and cos of 2 pi * phi / 2^64 for a 64-bit fixed-point phase phi.  The top
// three bits select the octant; the next 32 bits are a fraction of pi/4 (the
// dropped bits are below 2^-32 of pi/4), so the reduced argument |x| <= pi/4 is
// exact to float rounding.  Taylor polynomials (sin to x^9, cos to x^10, truncation
// error below 2e-9) give sin x and cos x; the octant then swaps and negates them:
// angle = oct*pi/4 + x for even octants, (oct+1)*pi/4 - x for odd ones.
__device__ __forceinline__ void sincos_turns64(uint64_t phi, float* s, float* c) {
  const unsigned oct = (unsigned)(phi >> 61);
  uint64_t rem = phi & ((1ull << 61) - 1);
  rem = (oct & 1u) ? (1ull << 61) - rem : rem;
  const float x = (float)(unsigned)(rem >> 29) * 1.8286476e-10f;  // (pi/4) / 2^32
  const float x2 = x * x;
  float sp = fmaf(x2, 2.7557319e-06f, -1.9841270e-04f);
  sp = fmaf(x2, sp, 8.3333333e-03f);
  sp = fmaf(x2, sp, -1.6666667e-01f);
  const float sv = fmaf(x * x2, sp, x);
  float cp = fmaf(x2, -2.7557319e-07f, 2.4801587e-05f);
  cp = fmaf(x2, cp, -1.3888889e-03f);
  cp = fmaf(x2, cp, 4.1666667e-02f);
  cp = fmaf(x2, cp, -0.5f);
  const float cv = fmaf(x2, cp, 1.0f);
  const bool swap = ((oct + 1u) >> 1) & 1u;     // octants 1, 2, 5, 6
  const float s0 = swap ? cv : sv, c0 = swap ? sv : cv;
  *s = (oct >= 4u) ? -s0 : s0;                  // octants 4..7
  *c = (((oct + 2u) >> 2) & 1u) ? -c0 : c0;     // octants 2..5
}

// 1/d in FP64 from an FP32 seed and two Newton steps (r <- r + r (1 - d r)); the
// relative error squares at each step, 2^-24 -> 2^-48 -> FP64 rounding.  Outside the
// FP32 normal range the plain FP64 division is used.
__device__ __forceinline__ double recip64(double d) {
  const float f = (float)d;
  if (!(fabsf(f) >= 1.2e-38f && fabsf(f) <= 3.0e38f)) return 1.0 / d;
  double r = (double)__frcp_rn(f);
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  return fma(r, e, r);
}
// 1/sqrt(d) likewise (y <- y (3/2 - d y^2 / 2)), d > 0
__device__ __forceinline__ double rsqrt64(double d) {
  const float f = (float)d;
  if (!(f >= 1.2e-38f && f <= 3.0e38f)) return 1.0 / sqrt(d);
  double y = (double)rsqrtf(f);
  const double h = 0.5 * d;
  y = y * fma(-h * y, y, 1.5);
  y = y * fma(-h * y, y, 1.5);
  return y * fma(-h * y, y, 1.5);
}

inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

}  // namespace pta

// The context (opaque to C callers).
struct pta_ctx {
  pta_model_desc desc{};
  std::string err;
  bool finalized = false;
  struct HostPsr {
    int n, m, nb;
    std::vector<double> t, nu, dt, sig, efac, equad, M;
    std::vector<int32_t> be;
    double pos[3];
    double dist;
  };
  std::vector<HostPsr> psrs;
  pta::DevModel dm{};
  pta::Scratch sc{};
  std::vector<void*> dev_allocs;   // data buffers freed at destroy
  double logp_const = 0.0;
  double t0 = 0.0;
  long long ntoa = 0;
  int precision = PTA_PREC_FP32;
  double* beta_dev = nullptr;      // pta_set_beta's copy of the inverse temperatures
  int beta_n = 0;                  // chains it covers
  int toa_cfg = -1;                // SIMT tile-shape entry (-1: default), set by the autotuner
  int transform = PTA_TRANSFORM_PRIOR;
  // prior support box per coordinate (HMC moves bounded coordinates in logit space)
  double* hmc_lo = nullptr;
  double* hmc_hi = nullptr;
  bool bounds_dirty = true;
  pta_layout_t lay{};
  // HMC graphs keyed by (B, n_leapfrog)
  struct Graph {
    int B, L;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  cudaStream_t cap_stream = nullptr;
  // stage profiler
  bool prof = false;
  std::vector<cudaEvent_t> prof_ev;   // pairs (start, end) per recorded stage
  std::vector<int> prof_stage;
  double prof_ms[PTA_NSTAGES] = {};
  long long prof_launch[PTA_NSTAGES] = {};
};
