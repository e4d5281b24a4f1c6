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
// The call runs the same tensor-core kernel as xc_correlate with default
// options: the small-array engine for 8-bit input of the sizes it serves
// (it needs no scratch), else the planar engine (same tile shape, same
// operand formation and scaling, same exact chunks for 8-bit input), so its
// visibilities are identical to xc_correlate's.  The planar scratch
// holds, in order: the status word, the ring counters, the per-channel and
// per-(channel, input) maxima of the scale pre-pass, and then as many
// operand-ring channel slots as fit.  All work is queued on the caller's
// stream.
#include <cuda.h>
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

constexpr int kKBlock = 64;
constexpr int kMaxDevices = 64;

// Per-device set-up: the device address of the static array and the SM
// count.  Recorded only once it has succeeded, so a failed attempt (say the
// device image could not be loaded) is retried by the next call.
struct DeviceSetup {
  bool ok = false;
  unsigned char* scratch = nullptr;
  int num_sms = 0;
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];

xc_status setup_device(int dev, DeviceSetup* out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& s = g_setup[dev];
  if (s.ok) {
    *out = s;
    return XC_OK;
  }
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return xc::record_error(XC_ERR_CUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
  }
  if (!(prop.major == 10 && prop.minor == 3))
    return xc::record_error(XC_ERR_NO_DEVICE, "device %d is sm_%d%d; this library is built for sm_103a",
                            dev, prop.major, prop.minor);
  // In host code the array name is a host-side stand-in; kernels must be
  // given the device address, looked up with this device current.  (With
  // lazy module loading this is also when the array is created.)
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return xc::record_error(XC_ERR_CUDA, "cudaGetSymbolAddress of the static scratch: %s",
                            cudaGetErrorString(e));
  }
  s.scratch = static_cast<unsigned char*>(p);
  s.num_sms = prop.multiProcessorCount;
  s.ok = true;
  *out = s;
  return XC_OK;
}

int64_t round256(int64_t x) { return (x + 255) / 256 * 256; }

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
  if (R > (1LL << 30) || Tp / kKBlock > 65535)
    return record_error(XC_ERR_UNSUPPORTED, "problem too large (rows=%lld, ntime=%d)",
                        static_cast<long long>(R), ntime);

  xc::Geometry g;
  g.N = nstation;
  g.P = npol;
  g.F = nfreq;
  g.T = ntime;
  g.R = static_cast<int>(R);
  g.Tp = static_cast<int>(Tp);
  g.NB = static_cast<int64_t>(nstation) * (nstation + 1) / 2;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return record_error(XC_ERR_NO_DEVICE, "no usable current CUDA device");
  }
  DeviceSetup s;
  const xc_status st0 = setup_device(dev, &s);
  if (st0 != XC_OK) return st0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // Small arrays with 8-bit input: the small-array engine, as xc_correlate
  // runs them; it needs no scratch beyond the status word.
  if (in_dtype == XC_CI8 && xc::small_tile_channels(g) > 0) {
    xc::XeLaunch X;
    X.g = g;
    X.in = in;
    X.in_dtype = 0;
    X.out = out;
    X.accumulate = 0;
    X.grid = s.num_sms;
    X.timeout_ns = 2000ull * 1000000ull;
    X.status = status ? status : reinterpret_cast<int*>(s.scratch);
    CUtensorMap in_map;
    const xc_status se = xc::encode_small_map(&in_map, in, g);
    if (se != XC_OK) return se;
    const cudaError_t e = xc::launch_small(&in_map, X, st);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return record_error(XC_ERR_CUDA, "small-array tensor-core X-engine: %s", cudaGetErrorString(e));
    }
    return record_error(XC_OK, "");
  }

  int pack = 1;
  const xc::Geometry pg = xc::planar_geometry(g, &pack);
  const int64_t n = static_cast<int64_t>(pg.N) * pg.P;

  // Scratch plan: status | counters | per-channel max |x| | per-(channel,
  // input) maxima (float input) | ring slots.
  const int64_t off_ctr = 256;
  const int64_t off_amax = off_ctr + round256(2LL * xc::kMaxRingSlots * 4);
  const int64_t off_inamax = off_amax + round256(static_cast<int64_t>(pg.F) * 4);
  const int64_t off_ring =
      off_inamax + (in_dtype == XC_CI8 ? 0 : round256(static_cast<int64_t>(pg.F) * n * 4));
  const int64_t slot_bytes = xc::planar_slot_bytes(pg, XC_PREC_FP16);
  const int64_t room = static_cast<int64_t>(XC_NOALLOC_SCRATCH_BYTES) - off_ring;
  if (room < slot_bytes)
    return record_error(XC_ERR_UNSUPPORTED,
                        "the static scratch (%u bytes) cannot hold one channel's operands (%lld "
                        "bytes: 2*npol*nstation rows x ntime rounded up to 64 x 2 bytes) after its "
                        "%lld bytes of counters and scales",
                        XC_NOALLOC_SCRATCH_BYTES, static_cast<long long>(slot_bytes),
                        static_cast<long long>(off_ring));

  const int slots = static_cast<int>(
      std::min<int64_t>(xc::planar_ring_slots(pg, s.num_sms, XC_PREC_FP16), room / slot_bytes));
  xc::XeLaunch X;
  X.g = pg;
  X.pack = pack;
  X.in = in;
  X.in_dtype = static_cast<int>(in_dtype);
  X.out = out;
  X.accumulate = 0;
  X.ring = s.scratch + off_ring;
  X.ring_slots = slots;
  X.counters = reinterpret_cast<unsigned*>(s.scratch + off_ctr);
  X.amax = reinterpret_cast<unsigned*>(s.scratch + off_amax);
  X.gains = nullptr;
  X.fmt = XC_PREC_FP16;
  X.in_amax = in_dtype == XC_CI8 ? nullptr : reinterpret_cast<unsigned*>(s.scratch + off_inamax);
  X.grid = s.num_sms;
  X.timeout_ns = 2000ull * 1000000ull;
  X.status = status ? status : reinterpret_cast<int*>(s.scratch);

  // The input in TMA boxes when its rows allow it (as xc_correlate does).
  CUtensorMap in_map;
  const CUtensorMap* im = nullptr;
  if (xc::input_map_possible(in_dtype, pg)) {
    const xc_status st = xc::encode_input_map(&in_map, in, pg, in_dtype);
    if (st != XC_OK) return st;
    im = &in_map;
  }
  // Kernel parameter block on the stack: nothing is allocated, host or device.
  xc::PlanarKernel k;
  const CUtensorMap* maps[1] = {im};
  cudaError_t e = xc::planar_prepare(&X, maps, 1, &k, xc::planar_default_shape(pg, XC_PREC_FP16));
  if (e == cudaSuccess && k.grid > 0) e = xc::planar_setup(&X, 1, st);
  if (e == cudaSuccess) e = xc::planar_launch(k, st);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return record_error(XC_ERR_CUDA, "tensor-core X-engine: %s", cudaGetErrorString(e));
  }
  return record_error(XC_OK, "");
}
