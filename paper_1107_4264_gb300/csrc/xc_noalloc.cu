// xc_noalloc.cu -- xc_correlate_noalloc: the tensor-core X-engine for callers
// that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: a real-time correlator loop that has
// reserved its memory at start-up and may not add allocations (each one can
// stall the device and fragment a budget sized in advance), an application
// whose memory is entirely held by another allocator, or a plug-in whose host
// forbids allocation from inside its processing callback.  They cannot create
// an xc_handle, because xc_create allocates the operand workspace.  This file
// gives them one call that allocates nothing: its scratch is a file-scope
// static __device__ array, created with the library's device image and kept
// by every GPU that loads the library until the process exits.
//
// The array holds the fp16 operand matrices of a group of channels.  The
// call walks the band in channel groups that fit the array: for each group it
// forms the operands into the array (a channel-offset variant of the
// operand-formation kernel that names the array directly) and runs the
// tensor-core X-engine on them through a TMA descriptor over the array's
// device address.  All work is queued on the caller's stream in order, so a
// group's operands are overwritten only after the previous group's
// X-engine has read them.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "xc.h"
#include "xc_internal.h"
#include "xc_launch.h"

namespace {

// The scratch shared by every call on a device (see XC_NOALLOC_SCRATCH_BYTES).
static __device__ __align__(256) unsigned char g_noalloc_scratch[XC_NOALLOC_SCRATCH_BYTES];
// Fallback status word for callers that pass no status pointer.
static __device__ int g_noalloc_status;

constexpr int kKBlock = 64;
constexpr int kTT = 64;
constexpr int kTR = 128;
constexpr int kPitch = kTT + 2;
constexpr int kMaxDevices = 64;

template <int DT>
__device__ __forceinline__ __half component(const void* in, int64_t idx) {
  if constexpr (DT == 0) {
    return __int2half_rn(static_cast<int>(static_cast<const int8_t*>(in)[idx]));
  } else if constexpr (DT == 1) {
    return static_cast<const __half*>(in)[idx];
  } else {
    return __float2half_rn(static_cast<const float*>(in)[idx]);
  }
}

// Operands of channels f0 .. f0 + gridDim.z - 1 into the static scratch,
// laid out [group channel][R][Tp] fp16, K-major, zero padded for t >= T.
template <int DT>
__global__ void __launch_bounds__(256) form_group_kernel(const void* __restrict__ in,
                                                         xc::Geometry g, int f0) {
  __shared__ __align__(16) __half tile[kTR * kPitch];
  __half* ws = reinterpret_cast<__half*>(g_noalloc_scratch);
  const int r0 = blockIdx.x * kTR;
  const int t0 = blockIdx.y * kTT;
  const int fl = blockIdx.z;
  const int f = f0 + fl;
  const int64_t R = g.R;
#pragma unroll 4
  for (int j = 0; j < (kTT * kTR) / 256; ++j) {
    const int idx = j * 256 + threadIdx.x;
    const int tl = idx / kTR;
    const int rl = idx % kTR;
    const int t = t0 + tl;
    const int r = r0 + rl;
    __half v = __float2half_rn(0.0f);
    if (t < g.T && r < R) v = component<DT>(in, (static_cast<int64_t>(t) * g.F + f) * R + r);
    tile[rl * kPitch + tl] = v;
  }
  __syncthreads();
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
      *reinterpret_cast<uint4*>(ws + (static_cast<int64_t>(fl) * R + r) * g.Tp + t0 + ch * 8) = v;
    }
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Per-device set-up: device addresses of the static arrays, SM count.
struct DeviceSetup {
  bool done = false;
  bool ok = false;
  void* scratch = nullptr;
  int* status = nullptr;
  int num_sms = 0;
  char why[160] = "";
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];
EncodeTiledFn g_encode = nullptr;

const DeviceSetup* setup_device(int dev) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& s = g_setup[dev];
  if (s.done) return &s;
  s.done = true;
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) {
    snprintf(s.why, sizeof(s.why), "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
    return &s;
  }
  if (!(prop.major == 10 && prop.minor == 3)) {
    snprintf(s.why, sizeof(s.why), "device %d is sm_%d%d; this library is built for sm_103a", dev,
             prop.major, prop.minor);
    return &s;
  }
  // In host code the array names are host-side stand-ins; the kernels must be
  // given the device addresses, looked up with this device current.
  e = cudaGetSymbolAddress(&s.scratch, g_noalloc_scratch);
  if (e == cudaSuccess) e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.status), g_noalloc_status);
  if (e != cudaSuccess) {
    snprintf(s.why, sizeof(s.why), "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    return &s;
  }
  if (!g_encode) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<EncodeTiledFn>(p);
  }
  if (!g_encode) {
    snprintf(s.why, sizeof(s.why), "cuTensorMapEncodeTiled unavailable from the driver");
    return &s;
  }
  s.num_sms = prop.multiProcessorCount;
  s.ok = true;
  return &s;
}

}  // namespace

extern "C" xc_status xc_correlate_noalloc(int nstation, int npol, int nfreq, int ntime,
                                          xc_dtype in_dtype, const void* in, void* out,
                                          int* status, void* stream) {
  using xc::record_error;
  if (nstation <= 0 || nfreq <= 0 || ntime <= 0 || (npol != 1 && npol != 2) || !in || !out)
    return record_error(XC_ERR_INVALID_ARG, "bad size, npol or NULL buffer");
  if (in_dtype != XC_CI8 && in_dtype != XC_CF16 && in_dtype != XC_CF32)
    return record_error(XC_ERR_INVALID_ARG, "unknown input dtype %d", static_cast<int>(in_dtype));
  if (in_dtype == XC_CI8 && ntime > XC_CI8_MAX_NTIME)
    return record_error(XC_ERR_OVERFLOW_RISK, "8-bit input with ntime=%d > %d", ntime,
                        XC_CI8_MAX_NTIME);
  if (nfreq > 65535) return record_error(XC_ERR_UNSUPPORTED, "nfreq=%d > 65535", nfreq);
  if ((reinterpret_cast<uintptr_t>(in) & 15u) || (reinterpret_cast<uintptr_t>(out) & 15u))
    return record_error(XC_ERR_ALIGNMENT, "input and output must be 16-byte aligned");
  const int64_t R = 2LL * npol * nstation;
  const int64_t Tp = (static_cast<int64_t>(ntime) + kKBlock - 1) / kKBlock * kKBlock;
  const int64_t per_channel = R * Tp * 2;
  if (per_channel > static_cast<int64_t>(XC_NOALLOC_SCRATCH_BYTES) || Tp / kKBlock > 65535)
    return record_error(XC_ERR_UNSUPPORTED,
                        "one channel needs %lld bytes of operand scratch (2*npol*nstation rows x "
                        "ntime rounded up to 64 x 2 bytes); the static scratch holds %u bytes",
                        static_cast<long long>(per_channel), XC_NOALLOC_SCRATCH_BYTES);
  const int group = static_cast<int>(
      std::min<int64_t>(nfreq, static_cast<int64_t>(XC_NOALLOC_SCRATCH_BYTES) / per_channel));

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return record_error(XC_ERR_NO_DEVICE, "no usable current CUDA device");
  }
  const DeviceSetup* s = setup_device(dev);
  if (!s->ok) return record_error(XC_ERR_NO_DEVICE, "set-up failed: %s", s->why);

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  xc::Geometry g;
  g.N = nstation;
  g.P = npol;
  g.F = nfreq;
  g.T = ntime;
  g.R = static_cast<int>(R);
  g.Tp = static_cast<int>(Tp);
  g.NB = static_cast<int64_t>(nstation) * (nstation + 1) / 2;
  const int64_t out_per_channel = g.NB * npol * npol * 2;  // int32 or fp32 elements

  for (int f0 = 0; f0 < nfreq; f0 += group) {
    const int fc = std::min(group, nfreq - f0);
    dim3 grid(static_cast<unsigned>((R + kTR - 1) / kTR), static_cast<unsigned>(Tp / kTT), fc);
    switch (in_dtype) {
      case XC_CI8: form_group_kernel<0><<<grid, 256, 0, st>>>(in, g, f0); break;
      case XC_CF16: form_group_kernel<1><<<grid, 256, 0, st>>>(in, g, f0); break;
      default: form_group_kernel<2><<<grid, 256, 0, st>>>(in, g, f0); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return record_error(XC_ERR_CUDA, "operand formation: %s", cudaGetErrorString(e));

    // TMA view of this group's operands: {t (Tp), row (R), channel (fc)} fp16.
    CUtensorMap tmap;
    const cuuint64_t dims[3] = {static_cast<cuuint64_t>(Tp), static_cast<cuuint64_t>(R),
                                static_cast<cuuint64_t>(fc)};
    const cuuint64_t strides[2] = {static_cast<cuuint64_t>(Tp) * 2,
                                   static_cast<cuuint64_t>(R) * Tp * 2};
    const cuuint32_t box[3] = {64, 128, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (g_encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, s->scratch, dims, strides, box, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return record_error(XC_ERR_CUDA, "cuTensorMapEncodeTiled failed");

    xc::TcLaunch L;
    L.g = g;
    L.g.F = fc;
    L.out = static_cast<char*>(out) + static_cast<int64_t>(f0) * out_per_channel * 4;
    L.is_int = in_dtype == XC_CI8 ? 1 : 0;
    L.accumulate = 0;
    L.grid = s->num_sms;
    L.timeout_ns = 2000ull * 1000000ull;
    L.status = status ? status : s->status;
    e = xc::launch_tc_xengine(&tmap, L, st);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return record_error(XC_ERR_CUDA, "tensor-core X-engine: %s", cudaGetErrorString(e));
    }
  }
  return record_error(XC_OK, "");
}
