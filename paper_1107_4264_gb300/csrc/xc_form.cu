// xc_form.cu -- operand formation for the tensor-core X-engine.
//
// The complex Hermitian rank-T update of Eq. (outer) (Sec. 2.1) is evaluated
// as a real symmetric product G_f = Y_f Y_f^T per channel, where Y_f has one
// row per real input component (r = (s*P + p)*2 + c, c = re/im) and one
// column per time sample.  This kernel writes Y_f in fp16, K-major
// (time fastest), into the workspace [F][R][Tp], zero padding t >= T.
//
// 8-bit input (Sec. 5) is exact in fp16 (|x| <= 128 < 2^11); fp16 input is
// copied; fp32 input is rounded to nearest fp16.
//
// Each block transposes a 64-sample x 128-row tile through shared memory:
// reads are contiguous along the station axis of the corner-turned input
// (Sec. 4.1), writes are contiguous 128-byte rows of the workspace.
#include <cuda_fp16.h>

#include "xc_launch.h"

namespace xc {
namespace {

constexpr int kTT = 64;    // samples per tile (one operand K-block)
constexpr int kTR = 128;   // rows per tile
constexpr int kPitch = kTT + 2;  // halves per shared row (33 words: conflict-free column writes)

template <int DT>
__device__ __forceinline__ __half load_component(const void* in, int64_t idx) {
  if constexpr (DT == 0) {
    return __int2half_rn(static_cast<int>(static_cast<const int8_t*>(in)[idx]));
  } else if constexpr (DT == 1) {
    return static_cast<const __half*>(in)[idx];
  } else {
    return __float2half_rn(static_cast<const float*>(in)[idx]);
  }
}

template <int DT>
__global__ void __launch_bounds__(256) form_operands_kernel(const void* __restrict__ in,
                                                            __half* __restrict__ ws, Geometry g) {
  __shared__ __align__(16) __half tile[kTR * kPitch];
  const int r0 = blockIdx.x * kTR;
  const int t0 = blockIdx.y * kTT;
  const int f = blockIdx.z;
  const int64_t R = g.R;

  // Load: 64 samples x 128 rows; a warp reads 32 consecutive rows of one sample.
#pragma unroll 4
  for (int j = 0; j < (kTT * kTR) / 256; ++j) {
    const int idx = j * 256 + threadIdx.x;
    const int tl = idx / kTR;
    const int rl = idx % kTR;
    const int t = t0 + tl;
    const int r = r0 + rl;
    __half v = __float2half_rn(0.0f);
    if (t < g.T && r < R) v = load_component<DT>(in, (static_cast<int64_t>(t) * g.F + f) * R + r);
    tile[rl * kPitch + tl] = v;
  }
  __syncthreads();

  // Store: 128 rows x 64 samples as 16-byte chunks (8 per row).
#pragma unroll
  for (int j = 0; j < (kTR * kTT / 8) / 256; ++j) {
    const int idx = j * 256 + threadIdx.x;
    const int rl = idx / 8;
    const int ch = idx % 8;
    const int r = r0 + rl;
    if (r < R) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(tile + rl * kPitch + ch * 8);
      uint4 v;
      v.x = src[0];
      v.y = src[1];
      v.z = src[2];
      v.w = src[3];
      __half* dst = ws + (static_cast<int64_t>(f) * R + r) * g.Tp + t0 + ch * 8;
      *reinterpret_cast<uint4*>(dst) = v;
    }
  }
}

}  // namespace

cudaError_t launch_form_operands(const void* in, int in_dtype, void* ws, const Geometry& g,
                                 cudaStream_t s) {
  dim3 grid((g.R + kTR - 1) / kTR, g.Tp / kTT, g.F);
  if (grid.y > 65535u || grid.z > 65535u) return cudaErrorInvalidConfiguration;
  __half* w = static_cast<__half*>(ws);
  switch (in_dtype) {
    case 0: form_operands_kernel<0><<<grid, 256, 0, s>>>(in, w, g); break;
    case 1: form_operands_kernel<1><<<grid, 256, 0, s>>>(in, w, g); break;
    case 2: form_operands_kernel<2><<<grid, 256, 0, s>>>(in, w, g); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace xc
