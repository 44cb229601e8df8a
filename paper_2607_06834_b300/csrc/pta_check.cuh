// Index checks of the check build (nvcc -DPTA_CHECK, libptahmc_check.so).  PTA_IN(rec, i, n,
// site) is true when 0 <= i < n; otherwise it records the first failure of the launch
// sequence (site, i, n) in the context's device record rec and is false, so the caller skips
// the access (a skipped load reads zero, a skipped bulk copy leaves its mbarrier short and the
// bounded wait reports it).  PTA_ALIGNED(rec, v, a, site) is the same test for v a multiple of a
// (the record holds the remainder).  The host reads the record after each evaluation and
// returns PTA_ECHECK naming the site.  In the release build both macros are the constant true
// and the record goes unused, so the kernels compile as if they were absent.
#pragma once

namespace pta {

// check sites (the record's first word); names in pta_check_site_name
enum CheckSite {
  kChkNone = 0,
  kChkSweepT = 1,      // dw_ldl_sweep: triangle element
  kChkSweepStage = 2,  // dw_ldl_sweep: staging entry
  kChkSweepLg = 3,     // dw_ldl_sweep: L D^1/2 element in global memory
  kChkClusterT = 4,    // dwc_ldl_sweep: this CTA's part of the triangle
  kChkClusterStage = 5,
  kChkUnit = 6,        // a work unit's TOA range inside its pulsar's (unit offsets)
  kChkResBasis = 7,    // k_f16_res: basis block inside the pulsar's stored blocks
  kChkResCoef = 8,     // k_f16_res: coefficient slice inside the packed pieces
  kChkBulkAlign = 9,   // a bulk copy's addresses and size on 16 bytes
  kChkTmaX = 10,       // k_f16_ftw: innermost TMA coordinate on 16 bytes
  kChkTmaRange = 11,   // k_f16_ftw: TMA coordinates inside the tensor
  kChkWslot = 12,      // CURN: inverse factor slot
  kChkCount
};

#ifdef PTA_CHECK
__device__ __forceinline__ bool chk_in(long long* rec, long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  if (rec && atomicCAS(reinterpret_cast<unsigned long long*>(rec), 0ull, (unsigned long long)site) == 0ull) {
    rec[1] = i;
    rec[2] = n;
  }
  return false;
}
#define PTA_IN(rec, i, n, site) ::pta::chk_in((rec), (long long)(i), (long long)(n), (site))
#define PTA_ALIGNED(rec, v, a, site) ::pta::chk_in((rec), (long long)(v) % (long long)(a), 1, (site))
#else
#define PTA_IN(rec, i, n, site) true
#define PTA_ALIGNED(rec, v, a, site) true
#endif

}  // namespace pta
