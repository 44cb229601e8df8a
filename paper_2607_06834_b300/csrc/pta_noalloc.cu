// pta_logp_and_grad_noalloc: the batched log posterior + gradient with every
// per-call scratch buffer carved out of one file-scope device array instead of
// context-owned allocations.
//
// Who needs it: callers that must not call cudaMalloc at evaluation time, e.g. a host
// framework that owns all device allocation and forbids allocations outside its own
// allocator, or a long sampler loop that must not pay for, or risk the failure of, an
// allocation in the middle of a run.  The
// context's resident data (uploaded by pta_finalize) is still used as is; only
// the per-call workspace moves here.
//
// The array is kNoallocBytes (32 MiB) and lives on every GPU that loads the
// library until the process exits.  Host code cannot use the array's name as a
// device address (it is a host-side stand-in), so the first call on each device
// asks the runtime for the device address with cudaGetSymbolAddress, with that
// device current, and caches it; make that first call before any stream capture.
// All calls share the array: calls that overlap on the GPU (different streams,
// devices excluded) race on it.  The array keeps the last call's contents; what must
// start at zero (the per-chain status flags, and the work counter of persistent TOA
// launches) is cleared on the caller's stream within every call.
#include <mutex>

#include "pta_internal.cuh"

int pta_check_result(pta_ctx* c, cudaStream_t st);
int pta_eval_scratch(pta_ctx* c, const pta::Scratch& s, int B, const float* x, double* logp, float* grad,
                     int32_t* status, cudaStream_t st, bool profile);

namespace {

constexpr size_t kNoallocBytes = 32ull << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Bytes of per-call workspace for B chains (same buffers as the context scratch,
// without the HMC state; the FP64 partial sums only for the FP64 path).
size_t noalloc_bytes(const pta::DevModel& m, int B, bool fp64) {
  const size_t np = m.npsr, tri = np * (np + 1) / 2;
  size_t s = 0;
  s += align256(np * B * m.PM * sizeof(float));
  s += align256(np * B * m.PM * sizeof(double));
  s += align256((size_t)B * std::max(1, m.n_chol) * tri * sizeof(double)) * 2;
  s += align256((size_t)m.n_units * B * m.Qs * sizeof(float));
  if (fp64) s += align256((size_t)m.n_units * B * m.Qs * sizeof(double));
  s += align256((size_t)m.n_units * B * sizeof(double));
  s += align256(np * B * m.P * sizeof(double));
  s += align256(np * B * sizeof(double));
  s += align256((size_t)B * np * m.na * sizeof(double));
  s += align256((size_t)B * np * std::max(1, m.nd) * sizeof(double));
  s += align256((size_t)B * m.na * sizeof(double));
  s += align256((size_t)B * sizeof(int32_t));
  s += align256((size_t)B * np * m.na * sizeof(double));
  s += align256((size_t)B * np * std::max(1, m.nd) * sizeof(double));
  s += align256((size_t)B * m.na * sizeof(double));
  s += align256(16);  // work counter of persistent launches
  return s;
}

}  // namespace

extern "C" int pta_logp_and_grad_noalloc(pta_ctx* c, int B, const float* x, double* logp, float* grad,
                                         int32_t* status, void* stream) {
  if (!c) return PTA_EINVAL;
  if (B < 0 || (B > 0 && (!x || !logp))) {
    c->err = "logp_and_grad_noalloc: bad arguments";
    return PTA_EINVAL;
  }
  if (!c->finalized) {
    c->err = "context not finalized";
    return PTA_ESTATE;
  }
  if (B == 0) return PTA_OK;
  if (c->dm.cw) {
    c->err = "logp_and_grad_noalloc: the continuous-wave model needs the allocating entry point";
    return PTA_EINVAL;
  }
  if (c->dm.beta && B > c->beta_n) {
    c->err = "logp_and_grad_noalloc: tempered evaluation with more chains than pta_set_beta gave";
    return PTA_EINVAL;
  }
  if (c->dm.curn) {
    c->err = "logp_and_grad_noalloc: the CURN transform keeps per-chain factors that need the allocating entry point";
    return PTA_EINVAL;
  }
  if (c->precision == PTA_PREC_BF16X3 || c->precision == PTA_PREC_F16SPLIT) {
    c->err = "logp_and_grad_noalloc: the BF16 and exact-split tensor-core paths need the allocating entry point";
    return PTA_EINVAL;
  }
  if (c->precision == PTA_PREC_FP64 && !c->dm.F64) {
    c->err = "logp_and_grad_noalloc: the FP64 path needs the stored FP64 basis, which the allocating "
             "entry point builds on its first FP64 call";
    return PTA_ESTATE;
  }
  const bool fp64 = c->precision == PTA_PREC_FP64;
  const size_t need = noalloc_bytes(c->dm, B, fp64);
  if (need > kNoallocBytes) {
    c->err = "logp_and_grad_noalloc: " + std::to_string(B) + " chains need " + std::to_string(need) +
             " bytes of workspace, above the fixed " + std::to_string(kNoallocBytes) + " bytes; use fewer chains";
    return PTA_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    c->err = "logp_and_grad_noalloc: cudaGetDevice failed or device index out of range";
    return PTA_ECUDA;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      e = cudaGetSymbolAddress(&g_addr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_addr[dev] = nullptr;
        c->err = std::string("logp_and_grad_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return PTA_ECUDA;
      }
    }
    base = g_addr[dev];
  }
  const pta::DevModel& m = c->dm;
  const size_t np = m.npsr, tri = np * (np + 1) / 2;
  unsigned char* p = static_cast<unsigned char*>(base);
  auto take = [&](size_t bytes) {
    void* r = p;
    p += align256(bytes);
    return r;
  };
  pta::Scratch s{};
  s.cap = B;
  s.a32 = (float*)take(np * B * m.PM * sizeof(float));
  s.a64 = (double*)take(np * B * m.PM * sizeof(double));
  s.Lpk = (double*)take((size_t)B * std::max(1, m.n_chol) * tri * sizeof(double));
  s.Lipk = (double*)take((size_t)B * std::max(1, m.n_chol) * tri * sizeof(double));
  s.gpart = (float*)take((size_t)m.n_units * B * m.Qs * sizeof(float));
  if (fp64) s.gpart64 = (double*)take((size_t)m.n_units * B * m.Qs * sizeof(double));
  s.c2part = (double*)take((size_t)m.n_units * B * sizeof(double));
  s.ghat = (double*)take(np * B * m.P * sizeof(double));
  s.chi2 = (double*)take(np * B * sizeof(double));
  s.dlnk = (double*)take((size_t)B * np * m.na * sizeof(double));
  s.dlnkd = (double*)take((size_t)B * np * std::max(1, m.nd) * sizeof(double));
  s.dlnr = (double*)take((size_t)B * m.na * sizeof(double));
  s.stat = (int32_t*)take((size_t)B * sizeof(int32_t));
  s.sk = (double*)take((size_t)B * np * m.na * sizeof(double));
  s.skd = (double*)take((size_t)B * np * std::max(1, m.nd) * sizeof(double));
  s.srho = (double*)take((size_t)B * m.na * sizeof(double));
  s.queue = (int*)take(16);
  // Run the same kernel sequence as pta_logp_and_grad on this workspace; the
  // context's own scratch is not touched.
  const int rc = pta_eval_scratch(c, s, B, x, logp, grad, status, (cudaStream_t)stream, false);
  return rc == PTA_OK ? pta_check_result(c, (cudaStream_t)stream) : rc;
}
