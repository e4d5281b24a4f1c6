// xc_planar_wide.cu -- the 128 x 256 (one CTA, N = 256 MMAs) instantiations
// of the planar tensor-core X-engine (xc_planar_kernel.cuh), compiled apart
// from the other shapes so they build in parallel.
#include "xc_planar_kernel.cuh"

namespace xc {

namespace {

template <bool IS_INT, int DT, int FMT, bool MULTI = false>
const void* wide_kernel_of() {
  return reinterpret_cast<const void*>(planar_wide_kernel<IS_INT, DT, FMT, MULTI>);
}

}  // namespace

const void* planar_wide_select(int in_dtype, int fmt, bool multi) {
  if (in_dtype == 0) {
    if (fmt == kFmtF8) return multi ? nullptr : wide_kernel_of<true, 0, kFmtF8>();
    return multi ? wide_kernel_of<true, 0, kFmtF16, true>() : wide_kernel_of<true, 0, kFmtF16>();
  }
  if (multi) return nullptr;
  if (in_dtype != 1 && in_dtype != 2) return nullptr;
  const bool h = in_dtype == 1;
  switch (fmt) {
    case kFmtF16: return h ? wide_kernel_of<false, 1, kFmtF16>() : wide_kernel_of<false, 2, kFmtF16>();
    // Hi/lo operands keep their running sums in TMEM columns a 128 x 256
    // accumulator fills: no such variant.
    case kFmtHiLo: return nullptr;
    case kFmtF8: return h ? wide_kernel_of<false, 1, kFmtF8>() : wide_kernel_of<false, 2, kFmtF8>();
    default: return nullptr;
  }
}

}  // namespace xc
