// xc_launch.h -- host-side launchers of the engine's kernels (internal).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "xc.h"
#include "xc_internal.h"

namespace xc {

// Operand formation (K-major fp16 workspace [F][R][Tp], zero padded in t and
// beyond R):  int8 / fp16 / fp32 complex input [T][F][N][P][2].
cudaError_t launch_form_operands(const void* in, int in_dtype, void* ws, const Geometry& g,
                                 cudaStream_t s);

// Tensor-core X-engine over the operand workspace described by `tmap`.
struct TcLaunch {
  Geometry g;
  void* out;
  int is_int;      // 1: int32 output with exact drains every 1024 samples
  int accumulate;  // 1: out += V
  int grid;        // persistent CTAs
  unsigned long long timeout_ns;
  int* status;
};
cudaError_t launch_tc_xengine(const CUtensorMap* tmap, const TcLaunch& p, cudaStream_t s);
int tc_smem_bytes();

// Fused persistent tensor-core X-engine: converter warps form the fp16
// operands into a ring of channel slots (`ring`, [ring_slots][R][Tp]) read
// through `tmap` ({Tp, R, ring_slots}, 64 x 128 x 1 boxes, 128B swizzle).
struct XeLaunch {
  Geometry g;
  const void* in;
  int in_dtype;  // 0 int8 (int32 out, exact), 1 fp16, 2 fp32
  void* out;
  int accumulate;
  void* ring;
  int ring_slots;
  unsigned* counters;  // 2 * ring_slots, zeroed by the launcher on `s`
  unsigned* amax;      // [F] per-channel max |x| (planar engine, 8-bit input)
  const void* gains;   // cf32 [N][P] applied to float input (planar engine), or NULL
  // Planar engine, float input:
  int fmt = 0;              // operand format: 0 fp16, 1 split hi/lo fp16, 2 e4m3
  unsigned* in_amax = nullptr;  // [F][N*P] scale pre-pass buffer (NULL: unscaled)
  double* acc64 = nullptr;  // FP64 block sums in the output layout (NULL: off)
  int f64_block = 0;        // samples per fp32 block when acc64 is set (multiple of 64)
  int test_no_publish = 0;  // test hook (XC_OPT_TEST_NO_PUBLISH)
  // Planar engine: g is the virtual geometry of planar_geometry(), with `pack`
  // consecutive real channels in each virtual channel (1: no packing).
  int pack = 1;
  int grid;
  unsigned long long timeout_ns;
  int* status;
};
cudaError_t launch_xengine(const CUtensorMap* tmap, const XeLaunch& p, cudaStream_t s);
// Planar complex form (separate real/imaginary fp16 planes, 4 MMAs per step
// into D_re/D_im).  The ring holds planar_slot_bytes() per channel slot;
// `in_map` (8-bit input with R % 16 == 0, else NULL) is {R, F, T} int8 in
// 128 x 1 x 64 boxes.  shape: kPlanar128 (128 x 128 blocks on single CTAs),
// kPlanarPair (two blocks sharing a column block on a CTA pair, tcgen05
// cta_group::2) or kPlanarWide (two blocks sharing a row block on one CTA,
// N = 256 MMAs).
enum : int { kPlanar128 = 0, kPlanarPair = 1, kPlanarWide = 2 };
cudaError_t launch_planar(const CUtensorMap* in_map, const XeLaunch& p, int shape, cudaStream_t s);
// The default shape for a (virtual) geometry and operand format.
int planar_default_shape(const Geometry& g, int fmt);
constexpr int kMaxRingSlots = 256;
// Samples per converter unit of the planar engine (8-bit input arrives by TMA
// in 128-row x 1 x kPlanarUnitT boxes).
constexpr int kPlanarUnitT = 64;
int planar_ring_slots(const Geometry& g, int grid, int fmt);
// Small arrays (n = N P <= 64 inputs): k consecutive channels, k the largest
// divisor of F with k n <= 128, are correlated as one virtual channel of k N
// stations.  The input [T][F][n] is the same memory as [T][F / k][k n], so
// nothing moves; one 128 x 128 block then holds the k channels' own blocks on
// its diagonal.  Returns that virtual geometry and k (1 for larger arrays).
Geometry planar_geometry(const Geometry& g, int* pack);

// F-engine (xc_fengine.cu): in [n][T F] complex (in_dtype 0 int8, 1 fp16,
// 2 fp32) -> out [T - ntaps + 1][F][n] complex (out_dtype 0 int8
// requantised, 1 fp16, 2 fp32), the DFT of each block of F samples (after the
// polyphase taps [ntaps][F] when taps is not NULL) times `scale`; F a power
// of two in [16, 4096]; taps NULL needs ntaps = 1.
cudaError_t launch_fengine(const void* in, int in_dtype, void* out, int out_dtype, int n, int F,
                           int T, float scale, const float* taps, int ntaps, cudaStream_t s);
int64_t planar_slot_bytes(const Geometry& g, int fmt);

// One planar launch over up to kMaxSub subarrays (same input type and
// format; every subarray with its own ring region, counters and buffers).
// planar_prepare fills the kernel and its parameter block (maps[i]: the
// 8-bit input map of subarray i, or NULL; TMA staging is used only when all
// subarrays have one); planar_setup issues the stream-ordered set-up
// (counter zeroing, float scale pre-pass); planar_launch launches.
constexpr int kMaxSub = 8;
constexpr int kBatchArgBytes = 4096;
struct PlanarKernel {
  alignas(128) unsigned char args[kBatchArgBytes];  // holds the kernel's Batch (128-byte aligned)
  const void* func = nullptr;
  int grid = 0, block = 0, smem = 0;
  int shape = kPlanar128;  // kPlanarPair: clusters of two, fixed in the kernel
};
// The grid is capped at the CTAs (clusters) that can be resident at once.
cudaError_t planar_prepare(const XeLaunch* subs, const CUtensorMap* const* maps, int nsub,
                           PlanarKernel* k, int shape);
cudaError_t planar_setup(const XeLaunch* subs, int nsub, cudaStream_t s);
cudaError_t planar_launch(PlanarKernel& k, cudaStream_t s);
// Same as launch_xengine, on CTA pairs (tcgen05 cta_group::2, 256 x 256 blocks).
cudaError_t launch_xengine_pair(const CUtensorMap* tmap, const XeLaunch& p, cudaStream_t s);
// Ring slots for a geometry (2..16 channels, about 32 MiB).
int xengine_ring_slots(const Geometry& g);

// FP32 CUDA-core X-engine (comparator) directly from the input; `gains`
// (cf32 [N][P], float input only) may be NULL.
cudaError_t launch_fp32_xengine(const void* in, int in_dtype, void* out, const Geometry& g,
                                int accumulate, const void* gains, cudaStream_t s);

// FP32 peak probe (xc_fp32_peak_probe): returns the flops launched, -1 on a
// launch error; `sink` is a device float array of 4 * num_sms elements.
long long launch_ffma_probe(long long iters, float* sink, int num_sms, cudaStream_t s);

// Adjoint of the float forward: H_f = G_f + G_f^H into `h_ws` ([F][n][n]
// cf32), grad_in = conj(g) H_f (g x) (cf32, layout of the input) and
// grad_g = sum conj(x) H_f (g x) (cf32 [n], may be NULL).
cudaError_t launch_adjoint(const void* grad_out, const void* in, const void* gains, void* grad_in,
                           float* grad_g, void* h_ws, const Geometry& g, cudaStream_t s);
// H_f = G_f + G_f^H from grad_out (the first step of both adjoints).
cudaError_t launch_build_h(const void* grad_out, void* h_ws, const Geometry& g, cudaStream_t s);
// Tensor-core adjoint: the same result with H'_f = H_f diag(g) and x split
// into fp16 hi/lo MMA tiles in `tc_ws` (adjoint_tc_workspace_bytes) and a
// tcgen05 GEMM; bounded waits report through `status`.
size_t adjoint_tc_workspace_bytes(const Geometry& g);
cudaError_t launch_adjoint_tc(const void* grad_out, const void* in, const void* gains, void* grad_in,
                              float* grad_g, void* h_ws, void* tc_ws, const Geometry& g,
                              unsigned long long timeout_ns, int* status, cudaStream_t s);

// The planar converters' TMA view of the input [T][F][n] (complex) of a
// (virtual) geometry: 8-bit rows in 128 x 1 x kPlanarUnitT boxes, fp16 as
// 32-bit complex elements in 64 x 1 x 32 boxes, fp32 components in
// 128 x 1 x 16 boxes.  Possible when a row is a multiple of 16 bytes.
bool input_map_possible(xc_dtype dtype, const Geometry& g);
xc_status encode_input_map(CUtensorMap* map, const void* in, const Geometry& g, xc_dtype dtype);

// Small-array engine (xc_small.cu): 8-bit input whose channels have
// W = 2 N P in {16, 32, 64, 128, 256} real rows; fp16 operands, or e4m3
// when XeLaunch::fmt is 2.  small_tile_channels() is
// the number of channels per channel group (128 / W, or 1 for W = 256,
// whose channel spans two 128-row tiles), or 0 when the geometry does not
// qualify.  The input map is {W, F, T} bytes in boxes of W x group x 64.  launch_small() may queue a memset of the output
// before the kernel (when it splits T across CTAs and does not accumulate).
int small_tile_channels(const Geometry& g);
xc_status encode_small_map(CUtensorMap* map, const void* in, const Geometry& g);
cudaError_t launch_small(const CUtensorMap* in_map, const XeLaunch& X, cudaStream_t s);

// Record `s` and a printf-style message as this thread's last error
// (xc_last_error / xc_last_error_message); returns s.
xc_status record_error(xc_status s, const char* fmt, ...);

}  // namespace xc
