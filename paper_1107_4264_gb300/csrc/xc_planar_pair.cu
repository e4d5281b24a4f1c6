// xc_planar_pair.cu -- the CTA-pair (tcgen05 cta_group::2) instantiations
// of the planar tensor-core X-engine (xc_planar_kernel.cuh), compiled apart
// from the single-CTA ones so the two build in parallel.
#include "xc_planar_kernel.cuh"

namespace xc {

namespace {

template <bool IS_INT, int DT, int FMT, bool MULTI = false>
const void* pair_kernel_of() {
  return reinterpret_cast<const void*>(planar_pair_kernel<IS_INT, DT, FMT, MULTI>);
}

}  // namespace

const void* planar_pair_select(int in_dtype, int fmt, bool multi) {
  if (in_dtype == 0) {
    if (fmt == kFmtF8) return multi ? nullptr : pair_kernel_of<true, 0, kFmtF8>();
    return multi ? pair_kernel_of<true, 0, kFmtF16, true>() : pair_kernel_of<true, 0, kFmtF16>();
  }
  if (multi) return nullptr;
  if (in_dtype != 1 && in_dtype != 2) return nullptr;
  const bool h = in_dtype == 1;
  switch (fmt) {
    case kFmtF16: return h ? pair_kernel_of<false, 1, kFmtF16>() : pair_kernel_of<false, 2, kFmtF16>();
    case kFmtHiLo: return h ? pair_kernel_of<false, 1, kFmtHiLo>() : pair_kernel_of<false, 2, kFmtHiLo>();
    case kFmtF8: return h ? pair_kernel_of<false, 1, kFmtF8>() : pair_kernel_of<false, 2, kFmtF8>();
    default: return nullptr;
  }
}

}  // namespace xc
