// xc_api.cpp -- the C ABI of include/xc.h: handle life cycle, argument
// checks, the TMA descriptor of the operand workspace, kernel dispatch and
// the integrated host->device pipeline of Sec. 5 (Algorithm 1).
#include "xc.h"

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "xc_internal.h"
#include "xc_launch.h"

namespace {

thread_local xc_status t_status = XC_OK;
thread_local char t_msg[512] = "";

xc_status fail(xc_status s, const char* fmt, ...) {
  t_status = s;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_msg, sizeof(t_msg), fmt, ap);
  va_end(ap);
  return s;
}

xc_status succeed() {
  t_status = XC_OK;
  t_msg[0] = '\0';
  return XC_OK;
}

xc_status cuda_fail(cudaError_t e, const char* what) {
  (void)cudaGetLastError();  // clear a sticky launch error for the next call
  if (e == cudaErrorMemoryAllocation) return fail(XC_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(XC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tensor_map_encoder() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

constexpr int kKBlock = 64;  // operand K-block (samples) of the tensor-core engine

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

size_t sample_bytes(xc_dtype d) { return d == XC_CI8 ? 1 : (d == XC_CF16 ? 2 : 4); }

}  // namespace

// Batched handle: every subarray's geometry and its region of the shared
// operand ring, counters and per-channel maxima, the chosen schedule and the
// captured graph (memsets + one persistent launch).
struct BatchSub {
  xc::Geometry g{};
  xc::Geometry pg{};   // planar engine's geometry: `pack` channels per virtual channel
  int pack = 1;
  int slots_unpacked = 0;  // ring depth 1x without channel packing (pack > 1 only)
  size_t in_bytes = 0, out_bytes = 0;
  void* ring = nullptr;
  int slots_base = 0;  // ring depth 1x (xc::planar_ring_slots)
  int max_slots = 0;   // slots the region holds (for the 2x candidate)
  unsigned* counters = nullptr;
  unsigned* amax = nullptr;
};
struct BatchState {
  int nsub = 0;
  BatchSub sub[XC_BATCH_MAX_SUB];
  void* ring_all = nullptr;
  unsigned* ctr_all = nullptr;
  int order[XC_BATCH_MAX_SUB];
  int depth = 1;
  bool packing = true;  // small subarrays' channels packed into one block (see planar_geometry)
  char cache_path[1024] = "";  // xc_batch_set_cache
  int shape = xc::kPlanar128;  // tile shape (xc::kPlanar*), tuned by xc_batch_tune
  int shape_default = xc::kPlanar128;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t knode = nullptr;
  xc::PlanarKernel k;
};

struct xc_handle {
  int device = 0;
  BatchState* batch = nullptr;
  xc::Geometry g{};
  xc_dtype dtype = XC_CI8;
  size_t in_bytes = 0, out_bytes = 0;
  int engine = XC_ENGINE_TENSOR;
  int accumulate = 0;
  unsigned long long timeout_ns = 2000ull * 1000000ull;
  int num_sms = 0;
  // Fused engine: ring of fp16 operand slots [ring_slots][R][Tp] + counters.
  void* ring = nullptr;
  int ring_slots = 0;
  unsigned* counters = nullptr;
  unsigned* chan_amax = nullptr;  // [F] per-channel max |x| (planar engine)
  CUtensorMap ring_tmap;     // interleaved form: {Tp, R, ring_slots}
  int planar_slots = 0;       // planar form: xc::planar_slot_bytes() per slot
  // Planar engine geometry: small arrays pack `pack` consecutive channels into
  // one virtual channel (xc::planar_geometry); pg is that virtual geometry.
  xc::Geometry pg{};
  int pack = 1;
  size_t ring_bytes = 0;
  // Float input on the planar engine: operand precision, scale pre-pass
  // buffer [F][n] and the FP64 block sums (allocated on use).
  int precision = XC_PREC_FP16;
  int fp64_block = 0;
  int tile = XC_TILE_AUTO;  // planar engine tile shape (XC_OPT_TILE)
  int test_no_publish = 0;
  unsigned* in_amax = nullptr;
  double* acc64 = nullptr;
  // Complex gains (float input) and the adjoint's buffers, allocated on use.
  void* gains = nullptr;     // cf32 [n]
  int gains_set = 0;
  void* adj_ws = nullptr;    // cf32 [F][n][n]: H_f = G_f + G_f^H
  void* adj_tc_ws = nullptr; // tensor-core adjoint: fp16 hi/lo operand tiles
  float* grad_g = nullptr;   // cf32 [n]
  // Two-pass engine (allocated when selected): fp16 operands [F][R][Tp].
  void* ws = nullptr;
  CUtensorMap tmap;
  int* d_status = nullptr;
  // Integrated pipeline (allocated on first use).
  void* stage[2] = {nullptr, nullptr};
  cudaStream_t copy_stream = nullptr, d2h_stream = nullptr;
  cudaEvent_t ev_ready[2] = {nullptr, nullptr};
  cudaEvent_t ev_free[2] = {nullptr, nullptr};
  bool free_recorded[2] = {false, false};  // ev_free[b] marks the last read of stage[b]
  cudaEvent_t ev_start = nullptr, ev_computed = nullptr, ev_d2h = nullptr;
  // Kernel timing (XC_OPT_PROFILE): events bracketing each launch.
  int profile = 0;
  struct Timed {
    cudaEvent_t ev[3];
    int nkern;  // 1: main kernel only (FP32 engine); 2: formation + main
  };
  std::vector<Timed> timed;
  size_t timed_used = 0;
  double acc_ms[2] = {0.0, 0.0};
  long long acc_launches[2] = {0, 0};
};

namespace {

xc_status encode_operand_map(CUtensorMap* map, void* base, int64_t R, int64_t Tp, int64_t n);
void batch_drop_graph(BatchState* b);

// Planar tile shape for an XC_TILE_* option value (-1: not available).
int planar_shape(int tile, const xc::Geometry& pg, int fmt) {
  switch (tile) {
    case XC_TILE_128: return xc::kPlanar128;
    case XC_TILE_PAIR: return xc::kPlanarPair;
    case XC_TILE_WIDE: return fmt == XC_PREC_HILO ? -1 : xc::kPlanarWide;
    default: return xc::planar_default_shape(pg, fmt);
  }
}

void release(xc_handle* h) {
  if (!h) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  for (auto& t : h->timed)
    for (int i = 0; i < 3; ++i)
      if (t.ev[i]) {
        cudaEventSynchronize(t.ev[i]);
        cudaEventDestroy(t.ev[i]);
      }
  if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);
  if (h->d2h_stream) cudaStreamSynchronize(h->d2h_stream);
  for (int b = 0; b < 2; ++b) {
    if (h->stage[b]) cudaFree(h->stage[b]);
    if (h->ev_ready[b]) cudaEventDestroy(h->ev_ready[b]);
    if (h->ev_free[b]) cudaEventDestroy(h->ev_free[b]);
  }
  if (h->ev_start) cudaEventDestroy(h->ev_start);
  if (h->ev_computed) cudaEventDestroy(h->ev_computed);
  if (h->ev_d2h) cudaEventDestroy(h->ev_d2h);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  if (h->d2h_stream) cudaStreamDestroy(h->d2h_stream);
  if (h->ws || h->d_status || h->ring || h->batch) cudaDeviceSynchronize();
  if (h->ws) cudaFree(h->ws);
  if (h->gains) cudaFree(h->gains);
  if (h->adj_ws) cudaFree(h->adj_ws);
  if (h->adj_tc_ws) cudaFree(h->adj_tc_ws);
  if (h->grad_g) cudaFree(h->grad_g);
  if (h->ring) cudaFree(h->ring);
  if (h->counters) cudaFree(h->counters);
  if (h->chan_amax) cudaFree(h->chan_amax);
  if (h->in_amax) cudaFree(h->in_amax);
  if (h->acc64) cudaFree(h->acc64);
  if (h->d_status) cudaFree(h->d_status);
  if (BatchState* b = h->batch) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->ring_all) cudaFree(b->ring_all);
    if (b->ctr_all) cudaFree(b->ctr_all);
    delete b;
  }
  cudaSetDevice(cur);
  delete h;
}

// Events for one timed launch (reused from the handle's pool).
xc_handle::Timed* next_timed(xc_handle* h, int nkern) {
  if (h->timed_used == h->timed.size()) {
    xc_handle::Timed t{};
    for (int i = 0; i < 3; ++i)
      if (cudaEventCreate(&t.ev[i]) != cudaSuccess) return nullptr;
    h->timed.push_back(t);
  }
  xc_handle::Timed* t = &h->timed[h->timed_used++];
  t->nkern = nkern;
  return t;
}

// The small-array engine serves XC_ENGINE_TENSOR handles with 8-bit input,
// fp16 or e4m3 operands and 2 N P in {16, 32, 64, 128, 256} (XC_TILE_AUTO or
// XC_TILE_SMALL).
bool use_small_engine(const xc_handle* h, const void* in) {
  return h->dtype == XC_CI8 && (h->precision == XC_PREC_FP16 || h->precision == XC_PREC_FP8) &&
         (h->tile == XC_TILE_AUTO || h->tile == XC_TILE_SMALL) && xc::small_tile_channels(h->g) > 0 &&
         aligned16(in);
}

xc_status launch_one(xc_handle* h, const void* in, void* out, cudaStream_t s) {
  if (h->batch) return fail(XC_ERR_UNSUPPORTED, "batch handle: use xc_batch_correlate");
  cudaError_t e;
  xc_handle::Timed* tm = nullptr;
  if (h->profile) {
    tm = next_timed(h, h->engine == XC_ENGINE_FP32 ? 1 : 2);
    if (!tm) return fail(XC_ERR_CUDA, "profiling event creation failed");
    cudaEventRecord(tm->ev[0], s);
  }
  const void* gains = h->gains_set ? h->gains : nullptr;
  if (gains && h->engine != XC_ENGINE_FP32 && h->engine != XC_ENGINE_TENSOR)
    return fail(XC_ERR_UNSUPPORTED, "gains need the planar tensor-core or the FP32 engine");
  if ((h->precision != XC_PREC_FP16 || h->fp64_block) && h->engine != XC_ENGINE_TENSOR)
    return fail(XC_ERR_UNSUPPORTED, "precision forms and FP64 block sums need XC_ENGINE_TENSOR");
  if (h->engine == XC_ENGINE_FP32) {
    e = xc::launch_fp32_xengine(in, static_cast<int>(h->dtype), out, h->g, h->accumulate, gains, s);
    if (e != cudaSuccess) return cuda_fail(e, "fp32 X-engine launch");
    if (tm) cudaEventRecord(tm->ev[1], s);
    return succeed();
  }
  if (h->engine == XC_ENGINE_TENSOR && use_small_engine(h, in)) {
    // Small arrays, 8-bit input: real-row tiles converted in shared memory.
    xc::XeLaunch X;
    X.g = h->g;
    X.in = in;
    X.in_dtype = 0;
    X.out = out;
    X.accumulate = h->accumulate;
    X.fmt = h->precision;  // fp16 or e4m3 operands
    X.test_no_publish = h->test_no_publish;
    X.grid = h->num_sms;
    X.timeout_ns = h->timeout_ns;
    X.status = h->d_status;
    CUtensorMap in_map;
    if (xc::encode_small_map(&in_map, in, h->g) != XC_OK) return t_status;
    if (tm) tm->nkern = 1;
    e = xc::launch_small(&in_map, X, s);
    if (e != cudaSuccess) return cuda_fail(e, "small-array tensor-core X-engine launch");
    if (tm) cudaEventRecord(tm->ev[1], s);
    return succeed();
  }
  if (h->engine == XC_ENGINE_TENSOR && h->tile == XC_TILE_SMALL)
    return fail(XC_ERR_UNSUPPORTED,
                "XC_TILE_SMALL needs 8-bit input, fp16 or e4m3 operands and 2*nstation*npol in {16, 32, 64, 128, 256}");
  if (h->engine == XC_ENGINE_TENSOR) {
    xc::XeLaunch X;
    X.g = h->pg;
    X.pack = h->pack;
    X.in = in;
    X.in_dtype = static_cast<int>(h->dtype);
    X.out = out;
    X.accumulate = h->accumulate;
    X.ring = h->ring;
    X.ring_slots = h->planar_slots;
    X.counters = h->counters;
    X.amax = h->chan_amax;
    X.gains = gains;
    X.fmt = h->precision;
    X.in_amax = h->in_amax;
    X.acc64 = h->fp64_block ? h->acc64 : nullptr;
    X.f64_block = h->fp64_block;
    X.test_no_publish = h->test_no_publish;
    X.grid = h->num_sms;
    X.timeout_ns = h->timeout_ns;
    X.status = h->d_status;
    // Input in TMA boxes when its rows are 16-byte strided.
    CUtensorMap in_map;
    const CUtensorMap* im = nullptr;
    if (xc::input_map_possible(h->dtype, h->pg)) {
      if (xc::encode_input_map(&in_map, in, h->pg, h->dtype) != XC_OK) return t_status;
      im = &in_map;
    }
    if (tm) tm->nkern = 1;
    const int shape = planar_shape(h->tile, h->pg, X.in_dtype == 0 ? 0 : h->precision);
    if (shape < 0) return fail(XC_ERR_UNSUPPORTED, "hi/lo operands do not run on XC_TILE_WIDE");
    e = xc::launch_planar(im, X, shape, s);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core X-engine launch");
    if (tm) cudaEventRecord(tm->ev[1], s);
    return succeed();
  }
  if (h->engine == XC_ENGINE_TENSOR_PAIR || h->engine == XC_ENGINE_TENSOR_1CTA) {
    xc::XeLaunch X;
    X.g = h->g;
    X.in = in;
    X.in_dtype = static_cast<int>(h->dtype);
    X.out = out;
    X.accumulate = h->accumulate;
    X.ring = h->ring;
    X.ring_slots = h->ring_slots;
    X.counters = h->counters;
    X.amax = nullptr;
    X.gains = nullptr;
    X.grid = h->num_sms;
    X.timeout_ns = h->timeout_ns;
    X.status = h->d_status;
    if (tm) tm->nkern = 1;
    e = h->engine == XC_ENGINE_TENSOR_PAIR ? xc::launch_xengine_pair(&h->ring_tmap, X, s)
                                          : xc::launch_xengine(&h->ring_tmap, X, s);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core X-engine launch");
    if (tm) cudaEventRecord(tm->ev[1], s);
    return succeed();
  }
  e = xc::launch_form_operands(in, static_cast<int>(h->dtype), h->ws, h->g, s);
  if (e != cudaSuccess) return cuda_fail(e, "operand formation launch");
  if (tm) cudaEventRecord(tm->ev[1], s);
  xc::TcLaunch L;
  L.g = h->g;
  L.out = out;
  L.is_int = h->dtype == XC_CI8 ? 1 : 0;
  L.accumulate = h->accumulate;
  L.grid = h->num_sms;
  L.timeout_ns = h->timeout_ns;
  L.status = h->d_status;
  e = xc::launch_tc_xengine(&h->tmap, L, s);
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core X-engine launch");
  if (tm) cudaEventRecord(tm->ev[2], s);
  return succeed();
}

// TMA view of fp16 operands {t (Tp), row (R), channel/slot (n)}, loaded in
// boxes of 64 samples x 128 rows x 1 with 128-byte swizzle.
xc_status encode_operand_map(CUtensorMap* map, void* base, int64_t R, int64_t Tp, int64_t n) {
  EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) return fail(XC_ERR_CUDA, "cuTensorMapEncodeTiled unavailable from the driver");
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>(Tp), static_cast<cuuint64_t>(R),
                              static_cast<cuuint64_t>(n)};
  const cuuint64_t strides[2] = {static_cast<cuuint64_t>(Tp) * 2,
                                 static_cast<cuuint64_t>(R) * Tp * 2};
  const cuuint32_t box[3] = {64, 128, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult cr = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return fail(XC_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(cr));
  return XC_OK;
}

// Full fp16 operand copy for the two-pass engine, allocated on first use.
xc_status ensure_two_pass_workspace(xc_handle* h) {
  if (h->ws) return XC_OK;
  const size_t bytes = static_cast<size_t>(h->g.F) * h->g.R * h->g.Tp * 2;
  cudaError_t e = cudaMalloc(&h->ws, bytes);
  if (e != cudaSuccess) {
    h->ws = nullptr;
    return cuda_fail(e, "two-pass workspace allocation");
  }
  xc_status st = encode_operand_map(&h->tmap, h->ws, h->g.R, h->g.Tp, h->g.F);
  if (st != XC_OK) {
    cudaFree(h->ws);
    h->ws = nullptr;
  }
  return st;
}

}  // namespace

namespace xc {
// Input [T][F][n] (complex) as a 3-D tensor {row elements, F, T} for the
// planar converters' TMA boxes of 8 KiB (zero fill past the row and T):
//   8-bit: {R = 2n bytes}, boxes of 128 x 1 x kPlanarUnitT;
//   fp16:  {n} 32-bit complex elements, boxes of 64 x 1 x 32;
//   fp32:  {2n} fp32 components, boxes of 128 x 1 x 16.
// A row must be a multiple of 16 bytes (TMA global strides).
bool input_map_possible(xc_dtype dtype, const Geometry& g) {
  const int64_t n = static_cast<int64_t>(g.N) * g.P;
  switch (dtype) {
    case XC_CI8: return g.R % 16 == 0;
    case XC_CF16: return n % 4 == 0;
    case XC_CF32: return n % 2 == 0;
  }
  return false;
}

xc_status encode_input_map(CUtensorMap* map, const void* in, const Geometry& g, xc_dtype dtype) {
  EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) return record_error(XC_ERR_CUDA, "cuTensorMapEncodeTiled unavailable from the driver");
  const cuuint64_t n = static_cast<cuuint64_t>(g.N) * g.P;
  cuuint64_t row = 0, esize = 1;
  cuuint32_t box_x = 0, box_t = 0;
  CUtensorMapDataType type = CU_TENSOR_MAP_DATA_TYPE_UINT8;
  if (dtype == XC_CI8) {
    row = static_cast<cuuint64_t>(g.R);
    box_x = 128;
    box_t = static_cast<cuuint32_t>(xc::kPlanarUnitT);
  } else if (dtype == XC_CF16) {
    type = CU_TENSOR_MAP_DATA_TYPE_UINT32;
    esize = 4;
    row = n;
    box_x = 64;
    box_t = 32;
  } else {
    type = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    esize = 4;
    row = 2 * n;
    box_x = 128;
    box_t = 16;
  }
  const cuuint64_t dims[3] = {row, static_cast<cuuint64_t>(g.F), static_cast<cuuint64_t>(g.T)};
  const cuuint64_t strides[2] = {row * esize, row * esize * static_cast<cuuint64_t>(g.F)};
  const cuuint32_t box[3] = {box_x, 1, box_t};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult cr = enc(map, type, 3, const_cast<void*>(in), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS)
    return record_error(XC_ERR_CUDA, "cuTensorMapEncodeTiled (input) failed (%d)", static_cast<int>(cr));
  return XC_OK;
}

// 8-bit input [T][F][W bytes] for the small-array engine: boxes of one
// channel group (128 / W channels) x 64 samples, zero-filled past F and T.
xc_status encode_small_map(CUtensorMap* map, const void* in, const Geometry& g) {
  EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) return record_error(XC_ERR_CUDA, "cuTensorMapEncodeTiled unavailable from the driver");
  const int m = small_tile_channels(g);
  if (m == 0) return record_error(XC_ERR_UNSUPPORTED, "geometry not served by the small-array engine");
  const cuuint64_t W = static_cast<cuuint64_t>(g.R);
  const cuuint64_t dims[3] = {W, static_cast<cuuint64_t>(g.F), static_cast<cuuint64_t>(g.T)};
  const cuuint64_t strides[2] = {W, W * static_cast<cuuint64_t>(g.F)};
  const cuuint32_t box[3] = {static_cast<cuuint32_t>(W), static_cast<cuuint32_t>(m), 64};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult cr = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void*>(in), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS)
    return record_error(XC_ERR_CUDA, "cuTensorMapEncodeTiled (small-array input) failed (%d)",
                        static_cast<int>(cr));
  return XC_OK;
}

xc_status record_error(xc_status s, const char* fmt, ...) {
  t_status = s;
  if (s == XC_OK) {
    t_msg[0] = '\0';
    return s;
  }
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_msg, sizeof(t_msg), fmt, ap);
  va_end(ap);
  return s;
}
}  // namespace xc

extern "C" {

xc_status xc_last_error(void) { return t_status; }

const char* xc_last_error_message(void) { return t_msg; }

const char* xc_status_string(xc_status s) {
  switch (s) {
    case XC_OK: return "XC_OK";
    case XC_ERR_INVALID_ARG: return "XC_ERR_INVALID_ARG";
    case XC_ERR_UNSUPPORTED: return "XC_ERR_UNSUPPORTED";
    case XC_ERR_OVERFLOW_RISK: return "XC_ERR_OVERFLOW_RISK";
    case XC_ERR_ALIGNMENT: return "XC_ERR_ALIGNMENT";
    case XC_ERR_CUDA: return "XC_ERR_CUDA";
    case XC_ERR_TIMEOUT: return "XC_ERR_TIMEOUT";
    case XC_ERR_OOM: return "XC_ERR_OOM";
    case XC_ERR_NO_DEVICE: return "XC_ERR_NO_DEVICE";
  }
  return "XC_ERR_UNKNOWN";
}

const char* xc_version(void) { return "xc 0.2 (sm_103a)"; }

xc_status xc_fp32_peak_probe(long long iterations, void* sink, void* stream, long long* flops) {
  if (iterations <= 0 || !sink || !flops) return fail(XC_ERR_INVALID_ARG, "bad probe arguments");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(XC_ERR_NO_DEVICE, "no usable CUDA device");
  }
  const long long f = xc::launch_ffma_probe(iterations, static_cast<float*>(sink), sms,
                                            static_cast<cudaStream_t>(stream));
  if (f < 0) return cuda_fail(cudaErrorLaunchFailure, "FFMA probe launch");
  *flops = f;
  return succeed();
}

int64_t xc_tri_index(int64_t bx, int64_t by) { return xc::tri_index(bx, by); }

int xc_small_engine_channels(int nstation, int npol) {
  if (nstation <= 0 || (npol != 1 && npol != 2) || nstation > 128) return 0;
  xc::Geometry g{};
  g.N = nstation;
  g.P = npol;
  g.R = 2 * nstation * npol;
  return xc::small_tile_channels(g);
}

int xc_channels_packed(int nstation, int npol, int nfreq) {
  // The sizes xc_create accepts (npol 1 or 2; rows 2 P N within its limit).
  if (nstation <= 0 || nfreq <= 0 || (npol != 1 && npol != 2)) return 0;
  const int64_t R = 2LL * npol * nstation;
  if (R > (1LL << 30)) return 0;
  xc::Geometry g{};
  g.N = nstation;
  g.P = npol;
  g.F = nfreq;
  g.T = 1;
  g.R = static_cast<int>(R);
  g.Tp = 64;
  g.NB = static_cast<int64_t>(nstation) * (nstation + 1) / 2;
  int pack = 1;
  (void)xc::planar_geometry(g, &pack);
  return pack;
}

void xc_tri_coords(int64_t g, int64_t* bx, int64_t* by) {
  int64_t x = 0, y = 0;
  xc::tri_coords(g, &x, &y);
  if (bx) *bx = x;
  if (by) *by = y;
}

size_t xc_input_bytes(const xc_handle* h) { return h ? h->in_bytes : 0; }
size_t xc_output_bytes(const xc_handle* h) { return h ? h->out_bytes : 0; }

xc_handle* xc_create(int nstation, int npol, int nfreq, int ntime, xc_dtype in_dtype) {
  if (nstation <= 0 || nfreq <= 0 || ntime <= 0) {
    fail(XC_ERR_INVALID_ARG, "sizes must be positive (nstation=%d nfreq=%d ntime=%d)", nstation,
         nfreq, ntime);
    return nullptr;
  }
  if (npol != 1 && npol != 2) {
    fail(XC_ERR_INVALID_ARG, "npol must be 1 or 2 (got %d)", npol);
    return nullptr;
  }
  if (in_dtype != XC_CI8 && in_dtype != XC_CF16 && in_dtype != XC_CF32) {
    fail(XC_ERR_INVALID_ARG, "unknown input dtype %d", static_cast<int>(in_dtype));
    return nullptr;
  }
  if (in_dtype == XC_CI8 && ntime > XC_CI8_MAX_NTIME) {
    fail(XC_ERR_OVERFLOW_RISK, "8-bit input with ntime=%d > %d can overflow int32 visibilities",
         ntime, XC_CI8_MAX_NTIME);
    return nullptr;
  }
  if (nfreq > 65535) {
    fail(XC_ERR_UNSUPPORTED, "nfreq=%d > 65535 (split the band across handles)", nfreq);
    return nullptr;
  }
  const int64_t R = 2LL * npol * nstation;
  const int64_t Tp = (static_cast<int64_t>(ntime) + kKBlock - 1) / kKBlock * kKBlock;
  if (R > (1LL << 30) || Tp / kKBlock > 65535) {
    fail(XC_ERR_UNSUPPORTED, "problem too large (rows=%lld, ntime=%d)", static_cast<long long>(R),
         ntime);
    return nullptr;
  }

  int dev = 0, ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    (void)cudaGetLastError();
    fail(XC_ERR_NO_DEVICE, "no CUDA device");
    return nullptr;
  }
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) {
    cuda_fail(e, "cudaGetDeviceProperties");
    return nullptr;
  }
  if (!(prop.major == 10 && prop.minor == 3)) {
    fail(XC_ERR_NO_DEVICE, "device %d is sm_%d%d; this library is built for sm_103a only", dev,
         prop.major, prop.minor);
    return nullptr;
  }

  xc_handle* h = new (std::nothrow) xc_handle();
  if (!h) {
    fail(XC_ERR_OOM, "host allocation failed");
    return nullptr;
  }
  h->device = dev;
  h->dtype = in_dtype;
  h->num_sms = prop.multiProcessorCount;
  h->g.N = nstation;
  h->g.P = npol;
  h->g.F = nfreq;
  h->g.T = ntime;
  h->g.R = static_cast<int>(R);
  h->g.Tp = static_cast<int>(Tp);
  h->g.NB = static_cast<int64_t>(nstation) * (nstation + 1) / 2;
  h->in_bytes = static_cast<size_t>(ntime) * nfreq * nstation * npol * 2 * sample_bytes(in_dtype);
  h->out_bytes = static_cast<size_t>(nfreq) * h->g.NB * npol * npol * 2 * 4;

  e = cudaMalloc(reinterpret_cast<void**>(&h->d_status), sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(int));
  if (e != cudaSuccess) {
    cuda_fail(e, "status word");
    release(h);
    return nullptr;
  }
  h->ring_slots = xc::xengine_ring_slots(h->g);
  h->pg = xc::planar_geometry(h->g, &h->pack);
  h->planar_slots = xc::planar_ring_slots(h->pg, h->num_sms, XC_PREC_FP16);
  const int slots = std::max({h->ring_slots, h->planar_slots, xc::kMaxRingSlots});
  h->ring_bytes = std::max(static_cast<size_t>(h->ring_slots) * R * Tp * 2,
                           static_cast<size_t>(h->planar_slots) *
                               xc::planar_slot_bytes(h->pg, XC_PREC_FP16));
  e = cudaMalloc(&h->ring, h->ring_bytes);
  if (e == cudaSuccess)
    e = cudaMalloc(reinterpret_cast<void**>(&h->counters), 2 * sizeof(unsigned) * slots);
  if (e == cudaSuccess)
    e = cudaMalloc(reinterpret_cast<void**>(&h->chan_amax), sizeof(unsigned) * nfreq);
  if (e == cudaSuccess && in_dtype != XC_CI8)
    e = cudaMalloc(reinterpret_cast<void**>(&h->in_amax),
                   sizeof(unsigned) * static_cast<size_t>(nfreq) * nstation * npol);
  if (e != cudaSuccess) {
    cuda_fail(e, "operand ring allocation");
    release(h);
    return nullptr;
  }
  if (encode_operand_map(&h->ring_tmap, h->ring, R, Tp, h->ring_slots) != XC_OK) {
    release(h);
    return nullptr;
  }
  succeed();
  return h;
}

void xc_destroy(xc_handle* h) {
  release(h);
  succeed();
}

xc_status xc_set_option(xc_handle* h, int key, long long value) {
  if (!h) return fail(XC_ERR_INVALID_ARG, "NULL handle");
  switch (key) {
    case XC_OPT_ENGINE:
      if (h->batch && value != XC_ENGINE_TENSOR)
        return fail(XC_ERR_UNSUPPORTED, "batch handles run the tensor-core engine only");
      if (value != XC_ENGINE_TENSOR && value != XC_ENGINE_FP32 && value != XC_ENGINE_TENSOR_2PASS &&
          value != XC_ENGINE_TENSOR_1CTA && value != XC_ENGINE_TENSOR_PAIR)
        return fail(XC_ERR_INVALID_ARG, "unknown engine %lld", value);
      if (value == XC_ENGINE_TENSOR_2PASS) {
        xc_status st = ensure_two_pass_workspace(h);
        if (st != XC_OK) return st;
      }
      h->engine = static_cast<int>(value);
      return succeed();
    case XC_OPT_ACCUMULATE:
      if (value != 0 && value != 1) return fail(XC_ERR_INVALID_ARG, "ACCUMULATE must be 0 or 1");
      h->accumulate = static_cast<int>(value);
      return succeed();
    case XC_OPT_PROFILE:
      if (value != 0 && value != 1) return fail(XC_ERR_INVALID_ARG, "PROFILE must be 0 or 1");
      h->profile = static_cast<int>(value);
      return succeed();
    case XC_OPT_TIMEOUT_MS:
      if (value <= 0 || value > 3600LL * 1000) return fail(XC_ERR_INVALID_ARG, "bad timeout");
      h->timeout_ns = static_cast<unsigned long long>(value) * 1000000ull;
      return succeed();
    case XC_OPT_PRECISION: {
      if (value != XC_PREC_FP16 && value != XC_PREC_HILO && value != XC_PREC_FP8)
        return fail(XC_ERR_INVALID_ARG, "unknown precision %lld", value);
      if (h->dtype == XC_CI8 && value == XC_PREC_HILO)
        return fail(XC_ERR_UNSUPPORTED, "8-bit input is exact in fp16; hi/lo applies to float input");
      const int fmt = static_cast<int>(value);
      const int slots = xc::planar_ring_slots(h->pg, h->num_sms, fmt);
      const size_t need = static_cast<size_t>(slots) * xc::planar_slot_bytes(h->pg, fmt);
      if (need > h->ring_bytes) {
        // Work already queued may still use the ring.
        cudaError_t e = cudaDeviceSynchronize();
        void* ring = nullptr;
        if (e == cudaSuccess) e = cudaMalloc(&ring, need);
        if (e != cudaSuccess) return cuda_fail(e, "operand ring reallocation");
        xc_status st = encode_operand_map(&h->ring_tmap, ring, h->g.R, h->g.Tp, h->ring_slots);
        if (st != XC_OK) {
          cudaFree(ring);
          return st;
        }
        cudaFree(h->ring);
        h->ring = ring;
        h->ring_bytes = need;
      }
      h->precision = fmt;
      h->planar_slots = slots;
      return succeed();
    }
    case XC_OPT_TILE:
      if (value != XC_TILE_AUTO && value != XC_TILE_128 && value != XC_TILE_PAIR && value != XC_TILE_WIDE &&
          value != XC_TILE_SMALL)
        return fail(XC_ERR_INVALID_ARG, "unknown tile shape %lld", value);
      if (value == XC_TILE_SMALL && h->batch)
        return fail(XC_ERR_UNSUPPORTED, "batched launches run on the planar engine");
      if (h->batch) {
        h->batch->shape = value == XC_TILE_AUTO ? h->batch->shape_default
                                                : planar_shape(static_cast<int>(value), h->pg, 0);
        batch_drop_graph(h->batch);
      }
      h->tile = static_cast<int>(value);
      return succeed();
    case XC_OPT_TEST_NO_PUBLISH:
      if (value != 0 && value != 1) return fail(XC_ERR_INVALID_ARG, "TEST_NO_PUBLISH must be 0 or 1");
      h->test_no_publish = static_cast<int>(value);
      return succeed();
    case XC_OPT_FP64_BLOCK: {
      if (value < 0 || value % 64 != 0 || value > (1LL << 30))
        return fail(XC_ERR_INVALID_ARG, "FP64_BLOCK must be 0 or a positive multiple of 64");
      if (value > 0 && h->dtype == XC_CI8)
        return fail(XC_ERR_UNSUPPORTED, "8-bit input is exact in int32; FP64 block sums apply to float input");
      if (value > 0) {
        // The running sum starts at zero whenever block sums are (re)enabled.
        cudaError_t e = cudaSuccess;
        if (!h->acc64) {
          e = cudaMalloc(reinterpret_cast<void**>(&h->acc64), h->out_bytes * 2);
          if (e != cudaSuccess) h->acc64 = nullptr;
        } else {
          e = cudaDeviceSynchronize();  // queued work may still use the sums
        }
        if (e == cudaSuccess) e = cudaMemset(h->acc64, 0, h->out_bytes * 2);
        if (e != cudaSuccess) return cuda_fail(e, "FP64 block-sum buffer");
      }
      h->fp64_block = static_cast<int>(value);
      return succeed();
    }
    default:
      return fail(XC_ERR_INVALID_ARG, "unknown option key %d", key);
  }
}

xc_status xc_correlate(xc_handle* h, const void* in, void* out, void* stream) {
  if (!h || !in || !out) return fail(XC_ERR_INVALID_ARG, "NULL handle or buffer");
  if (h->batch) return fail(XC_ERR_UNSUPPORTED, "batch handle: use xc_batch_correlate");
  if (!aligned16(in) || !aligned16(out))
    return fail(XC_ERR_ALIGNMENT, "input and output must be 16-byte aligned");
  return launch_one(h, in, out, static_cast<cudaStream_t>(stream));
}

xc_status xc_correlate_backward(xc_handle* h, const void* grad_out, const void* in, void* grad_in,
                                void* stream) {
  if (!h || !grad_out || !in || !grad_in) return fail(XC_ERR_INVALID_ARG, "NULL handle or buffer");
  if (h->dtype != XC_CF32) return fail(XC_ERR_UNSUPPORTED, "backward needs XC_CF32 input");
  if (!aligned16(grad_out) || !aligned16(in) || !aligned16(grad_in))
    return fail(XC_ERR_ALIGNMENT, "buffers must be 16-byte aligned");
  const int64_t n = static_cast<int64_t>(h->g.N) * h->g.P;
  cudaError_t e = cudaSuccess;
  if (!h->adj_ws) e = cudaMalloc(&h->adj_ws, static_cast<size_t>(h->g.F) * n * n * 8);
  if (e == cudaSuccess && !h->grad_g) e = cudaMalloc(reinterpret_cast<void**>(&h->grad_g), 8 * n);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint workspace");
  const void* gains = h->gains_set ? h->gains : nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->engine == XC_ENGINE_FP32) {
    // The FP32 engine's adjoint: complex GEMM on the CUDA cores.
    e = xc::launch_adjoint(grad_out, in, gains, grad_in, h->grad_g, h->adj_ws, h->g, s);
  } else {
    if (!h->adj_tc_ws) {
      e = cudaMalloc(&h->adj_tc_ws, xc::adjoint_tc_workspace_bytes(h->g));
      if (e != cudaSuccess) {
        h->adj_tc_ws = nullptr;
        return cuda_fail(e, "adjoint workspace");
      }
    }
    e = xc::launch_adjoint_tc(grad_out, in, gains, grad_in, h->grad_g, h->adj_ws, h->adj_tc_ws, h->g,
                              h->timeout_ns, h->d_status, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "adjoint launch");
  return succeed();
}

xc_status xc_set_gains(xc_handle* h, const void* gains) {
  if (!h) return fail(XC_ERR_INVALID_ARG, "NULL handle");
  if (!gains) {
    h->gains_set = 0;
    return succeed();
  }
  if (h->dtype == XC_CI8) return fail(XC_ERR_UNSUPPORTED, "gains need float input");
  const size_t bytes = static_cast<size_t>(h->g.N) * h->g.P * 8;
  cudaError_t e = cudaSuccess;
  if (!h->gains) e = cudaMalloc(&h->gains, bytes);
  // Work already queued may still read the previous gains.
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(h->gains, gains, bytes, cudaMemcpyDeviceToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "set gains");
  h->gains_set = 1;
  return succeed();
}

xc_status xc_get_grad_gains(xc_handle* h, void* grad_gains, void* stream) {
  if (!h || !grad_gains) return fail(XC_ERR_INVALID_ARG, "NULL handle or buffer");
  const size_t bytes = static_cast<size_t>(h->g.N) * h->g.P * 8;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = h->grad_g ? cudaMemcpyAsync(grad_gains, h->grad_g, bytes, cudaMemcpyDeviceToDevice, s)
                            : cudaMemsetAsync(grad_gains, 0, bytes, s);
  if (e != cudaSuccess) return cuda_fail(e, "grad gains");
  return succeed();
}

xc_status xc_kernel_times(xc_handle* h, double* ms, long long* launches, int reset) {
  if (!h) return fail(XC_ERR_INVALID_ARG, "NULL handle");
  for (size_t i = 0; i < h->timed_used; ++i) {
    const xc_handle::Timed& t = h->timed[i];
    cudaError_t e = cudaEventSynchronize(t.ev[t.nkern]);
    if (e != cudaSuccess) return cuda_fail(e, "kernel timing");
    float a = 0.f, b = 0.f;
    if (t.nkern == 1) {
      cudaEventElapsedTime(&b, t.ev[0], t.ev[1]);
    } else {
      cudaEventElapsedTime(&a, t.ev[0], t.ev[1]);
      cudaEventElapsedTime(&b, t.ev[1], t.ev[2]);
      h->acc_ms[0] += a;
      h->acc_launches[0] += 1;
    }
    h->acc_ms[1] += b;
    h->acc_launches[1] += 1;
  }
  h->timed_used = 0;
  for (int k = 0; k < 2; ++k) {
    if (ms) ms[k] = h->acc_ms[k];
    if (launches) launches[k] = h->acc_launches[k];
    if (reset) {
      h->acc_ms[k] = 0.0;
      h->acc_launches[k] = 0;
    }
  }
  return succeed();
}

xc_status xc_synchronize(xc_handle* h, void* stream) {
  if (!h) return fail(XC_ERR_INVALID_ARG, "NULL handle");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "synchronize");
  if (st != 0) {
    e = cudaMemsetAsync(h->d_status, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "status reset");
    if (st & xc::kStatusTimeout)
      return fail(XC_ERR_TIMEOUT, "a kernel gave up on a bounded wait (status 0x%x)", st);
    if (st & xc::kStatusRange)
      return fail(XC_ERR_OVERFLOW_RISK,
                  "8-bit input with |x| > 16 on the FP8 tensor path (results are not exact)");
    return fail(XC_ERR_CUDA, "device status 0x%x", st);
  }
  return succeed();
}

xc_status xc_correlate_stream(xc_handle* h, const void* host_in, int n_integrations, void* out,
                              void* host_out, void* stream) {
  if (!h || !host_in || !out) return fail(XC_ERR_INVALID_ARG, "NULL handle or buffer");
  if (n_integrations < 0) return fail(XC_ERR_INVALID_ARG, "n_integrations < 0");
  if (!aligned16(out)) return fail(XC_ERR_ALIGNMENT, "output must be 16-byte aligned");
  if (n_integrations == 0) return succeed();
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (!h->copy_stream) {
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      e = cudaMalloc(&h->stage[b], h->in_bytes);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_ready[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_free[b], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_computed, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_d2h, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->d2h_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "pipeline set-up");
  }
  const char* src = static_cast<const char*>(host_in);
  char* dst = static_cast<char*>(out);
  char* hdst = static_cast<char*>(host_out);
  // Copies out follow the work queued earlier on `stream`.  Copies in wait
  // only until their staging buffer has been read (by this call's
  // correlation of integration i-2, or the last use in an earlier call), so
  // they overlap an earlier call's final copies out.
  e = cudaEventRecord(h->ev_start, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->d2h_stream, h->ev_start, 0);
  for (int i = 0; i < n_integrations && e == cudaSuccess; ++i) {
    const int b = i & 1;
    // H2D of integration i into buffer b once the buffer's previous correlation has read it.
    if (i >= 2 || h->free_recorded[b]) e = cudaStreamWaitEvent(h->copy_stream, h->ev_free[b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->stage[b], src + static_cast<size_t>(i) * h->in_bytes, h->in_bytes,
                          cudaMemcpyHostToDevice, h->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_ready[b], h->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_ready[b], 0);
    if (e != cudaSuccess) break;
    char* o = h->accumulate ? dst : dst + static_cast<size_t>(i) * h->out_bytes;
    xc_status st = launch_one(h, h->stage[b], o, s);
    if (st != XC_OK) return st;
    e = cudaEventRecord(h->ev_free[b], s);
    h->free_recorded[b] = true;
    if (e == cudaSuccess && hdst && (!h->accumulate || i == n_integrations - 1)) {
      e = cudaEventRecord(h->ev_computed, s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(h->d2h_stream, h->ev_computed, 0);
      char* ho = h->accumulate ? hdst : hdst + static_cast<size_t>(i) * h->out_bytes;
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(ho, o, h->out_bytes, cudaMemcpyDeviceToHost, h->d2h_stream);
    }
  }
  // Later work on `stream` is ordered after the copies of this call.
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_d2h, h->d2h_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_d2h, 0);
  if (e != cudaSuccess) return cuda_fail(e, "integrated pipeline");
  return succeed();
}

// -------------------------------------------------------------- F-engine

namespace {

xc_status channelize_impl(const void* in, xc_dtype in_dtype, int nstation, int npol, int nchan,
                          int nblock, const float* taps, int ntaps, float scale, void* out,
                          xc_dtype out_dtype, void* stream) {
  if (!in || !out) return fail(XC_ERR_INVALID_ARG, "NULL buffer");
  if (nstation <= 0 || nblock <= 0 || (npol != 1 && npol != 2))
    return fail(XC_ERR_INVALID_ARG, "bad sizes (nstation=%d npol=%d nblock=%d)", nstation, npol,
                nblock);
  if (in_dtype != XC_CI8 && in_dtype != XC_CF16 && in_dtype != XC_CF32)
    return fail(XC_ERR_INVALID_ARG, "unknown input type %d", static_cast<int>(in_dtype));
  if (out_dtype != XC_CI8 && out_dtype != XC_CF16 && out_dtype != XC_CF32)
    return fail(XC_ERR_INVALID_ARG, "unknown output type %d", static_cast<int>(out_dtype));
  if (ntaps < 1 || ntaps > 64 || ntaps > nblock)
    return fail(XC_ERR_INVALID_ARG, "ntaps=%d: 1 to min(64, nblock=%d)", ntaps, nblock);
  if (nchan < 16 || nchan > 4096 || (nchan & (nchan - 1)) != 0)
    return fail(XC_ERR_UNSUPPORTED, "nchan=%d: powers of two from 16 to 4096 are supported", nchan);
  const int64_t n = static_cast<int64_t>(nstation) * npol;
  if (n > (1LL << 24) || static_cast<int64_t>(nblock) * nchan > (1LL << 36) / n)
    return fail(XC_ERR_UNSUPPORTED, "problem too large");
  // One CTA transforms G consecutive inputs of one block (G = 8192 / nchan,
  // 16384 / nchan for 8-bit output); the input groups form the grid's second
  // dimension (at most 65535).
  const int64_t G = (out_dtype == XC_CI8 ? 16384 : 8192) / nchan;
  if ((n + G - 1) / G > 65535)
    return fail(XC_ERR_UNSUPPORTED, "nstation*npol=%lld above %lld for nchan=%d",
                static_cast<long long>(n), static_cast<long long>(65535 * G), nchan);
  if (!aligned16(in) || !aligned16(out) || (taps && !aligned16(taps)))
    return fail(XC_ERR_ALIGNMENT, "buffers must be 16-byte aligned");
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(XC_ERR_NO_DEVICE, "no usable CUDA device");
  }
  if (!(major == 10 && minor == 3))
    return fail(XC_ERR_NO_DEVICE, "device %d is sm_%d%d; this library is built for sm_103a only", dev,
                major, minor);
  cudaError_t e = xc::launch_fengine(in, static_cast<int>(in_dtype), out, static_cast<int>(out_dtype),
                                     static_cast<int>(n), nchan, nblock, scale, taps, ntaps,
                                     static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "F-engine launch");
  return succeed();
}

}  // namespace

xc_status xc_channelize(const void* in, xc_dtype in_dtype, int nstation, int npol, int nchan,
                        int nblock, float scale, void* out, xc_dtype out_dtype, void* stream) {
  return channelize_impl(in, in_dtype, nstation, npol, nchan, nblock, nullptr, 1, scale, out,
                         out_dtype, stream);
}

xc_status xc_channelize_pfb(const void* in, xc_dtype in_dtype, int nstation, int npol, int nchan,
                            int nblock, const float* taps, int ntaps, float scale, void* out,
                            xc_dtype out_dtype, void* stream) {
  if (!taps) return fail(XC_ERR_INVALID_ARG, "NULL taps");
  return channelize_impl(in, in_dtype, nstation, npol, nchan, nblock, taps, ntaps, scale, out,
                         out_dtype, stream);
}

// ------------------------------------------------------------------ batch

}  // extern "C"

namespace {

// Tuning file lines: "<key>\t<candidate>\t<ms>"; the last line with the key
// wins.  Returns the candidate, or -1 (no file, no line, unreadable).
int cache_lookup_ms(const char* path, const char* key, double* ms) {
  if (!path || !path[0] || !key) return -1;
  FILE* fh = fopen(path, "r");
  if (!fh) return -1;
  const size_t klen = strlen(key);
  char line[2048];
  int found = -1;
  while (fgets(line, sizeof(line), fh)) {
    if (strncmp(line, key, klen) != 0 || line[klen] != '\t') continue;
    int c = -1;
    double m = 0.0;
    if (sscanf(line + klen + 1, "%d\t%lf", &c, &m) >= 1 && c >= 0 && c < XC_BATCH_CANDIDATES) {
      found = c;
      *ms = m;
    }
  }
  fclose(fh);
  return found;
}

// The tuning key of a batch handle (its subarrays in creation order).
void batch_key(const BatchState* b, xc_dtype dtype, char* buf, size_t len) {
  int N[XC_BATCH_MAX_SUB], F[XC_BATCH_MAX_SUB], T[XC_BATCH_MAX_SUB];
  for (int i = 0; i < b->nsub; ++i) {
    N[i] = b->sub[i].g.N;
    F[i] = b->sub[i].g.F;
    T[i] = b->sub[i].g.T;
  }
  if (xc_batch_cache_key(b->nsub, N, F, T, b->sub[0].g.P, dtype, buf, len) < 0) buf[0] = '\0';
}

// Work of subarray i in MMA block-steps: blocks per channel x channels x K-blocks.
double batch_work(const BatchSub& b) {
  const double nib = std::ceil((static_cast<double>(b.pg.N) * b.pg.P) / 128);
  return nib * (nib + 1) / 2 * b.pg.F * (b.pg.Tp / 64);
}

// Candidate c of xc_batch_tune (XC_BATCH_CANDIDATES = 36):
//   c % 3          work-list order: as given, largest first, smallest first;
//   (c / 3) % 2    operand-ring depth: 1x, 2x;
//   (c / 6) % 2    channel packing of small subarrays: on, off;
//   c / 12         tile shape: 128 x 128, CTA pair, 128 x 256.
struct Schedule {
  int order[XC_BATCH_MAX_SUB];
  int depth;
  bool packing;
  int shape;
};

Schedule batch_schedule(const BatchState* b, int c) {
  Schedule sc;
  for (int i = 0; i < b->nsub; ++i) sc.order[i] = i;
  const int kind = c % 3;
  if (kind != 0)
    std::stable_sort(sc.order, sc.order + b->nsub, [&](int x, int y) {
      const double wx = batch_work(b->sub[x]), wy = batch_work(b->sub[y]);
      return kind == 1 ? wx > wy : wx < wy;
    });
  sc.depth = 1 + (c / 3) % 2;
  sc.packing = (c / 6) % 2 == 0;
  sc.shape = c / 12 == 0 ? xc::kPlanar128 : (c / 12 == 1 ? xc::kPlanarPair : xc::kPlanarWide);
  return sc;
}

// The candidate index of a schedule (the inverse of batch_schedule for the
// order kinds it produces).
int batch_candidate(int order_kind, int depth, bool packing, int shape) {
  const int sh = shape == xc::kPlanar128 ? 0 : (shape == xc::kPlanarPair ? 1 : 2);
  return sh * 12 + (packing ? 0 : 6) + (depth - 1) * 3 + order_kind;
}

void batch_drop_graph(BatchState* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->knode = nullptr;
}

// Launch descriptions of the subarrays in work-list order, their input
// maps, and the kernel parameter block in b->k.
xc_status batch_prepare(xc_handle* h, const void* const* in, void* const* out,
                        const int* order, int depth, bool packing, int shape, xc::XeLaunch* L) {
  BatchState* b = h->batch;
  if (!in || !out) return fail(XC_ERR_INVALID_ARG, "NULL pointer array");
  CUtensorMap maps[XC_BATCH_MAX_SUB];
  const CUtensorMap* mp[XC_BATCH_MAX_SUB];
  for (int j = 0; j < b->nsub; ++j) {
    const int i = order[j];
    const BatchSub& s = b->sub[i];
    if (!in[i] || !out[i]) return fail(XC_ERR_INVALID_ARG, "NULL buffer for subarray %d", i);
    if (!aligned16(in[i]) || !aligned16(out[i]))
      return fail(XC_ERR_ALIGNMENT, "subarray %d: buffers must be 16-byte aligned", i);
    xc::XeLaunch& X = L[j];
    X = xc::XeLaunch{};
    const bool packed = packing || s.pack == 1;
    const xc::Geometry& pg = packed ? s.pg : s.g;
    X.g = pg;
    X.pack = packed ? s.pack : 1;
    X.in = in[i];
    X.in_dtype = static_cast<int>(h->dtype);
    X.out = out[i];
    X.accumulate = h->accumulate;
    X.ring = s.ring;
    X.ring_slots = std::min(s.max_slots, (packed ? s.slots_base : s.slots_unpacked) * depth);
    X.counters = s.counters;
    X.amax = s.amax;
    X.gains = nullptr;
    X.grid = h->num_sms;
    X.timeout_ns = h->timeout_ns;
    X.status = h->d_status;
    mp[j] = nullptr;
    if (h->dtype == XC_CI8 && pg.R % 16 == 0) {
      if (xc::encode_input_map(&maps[j], in[i], pg, XC_CI8) != XC_OK) return t_status;
      mp[j] = &maps[j];
    }
  }
  cudaError_t e = xc::planar_prepare(L, mp, b->nsub, &b->k, shape);
  if (e != cudaSuccess) return cuda_fail(e, "batch launch preparation");
  return XC_OK;
}

// Make a schedule the handle's own (later xc_batch_correlate calls capture
// a new graph: ring depths, memset sizes and the kernel may change).
void apply_schedule(BatchState* b, const Schedule& sc) {
  for (int i = 0; i < b->nsub; ++i) b->order[i] = sc.order[i];
  b->depth = sc.depth;
  b->packing = sc.packing;
  b->shape = sc.shape;
  batch_drop_graph(b);
}

}  // namespace

extern "C" {

xc_handle* xc_batch_create(int nsub, const int* nstation, const int* nfreq, const int* ntime,
                           int npol, xc_dtype in_dtype) {
  if (nsub < 1 || nsub > XC_BATCH_MAX_SUB || !nstation || !nfreq || !ntime) {
    fail(XC_ERR_INVALID_ARG, "nsub must be in [1, %d] with size arrays", XC_BATCH_MAX_SUB);
    return nullptr;
  }
  if (in_dtype != XC_CI8) {
    fail(XC_ERR_UNSUPPORTED, "batched correlation takes 8-bit input");
    return nullptr;
  }
  // Validate every subarray as xc_create would (and use the first as the
  // handle's own geometry for its device state).
  xc_handle* h = xc_create(nstation[0], npol, nfreq[0], ntime[0], in_dtype);
  if (!h) return nullptr;
  // The single-geometry operand ring is not used by a batch handle.
  cudaFree(h->ring);
  h->ring = nullptr;
  for (int i = 1; i < nsub; ++i) {
    const int N = nstation[i], F = nfreq[i], T = ntime[i];
    if (N <= 0 || F <= 0 || T <= 0 || F > 65535 || T > XC_CI8_MAX_NTIME ||
        2LL * npol * N > (1LL << 30)) {
      release(h);
      fail(XC_ERR_INVALID_ARG, "subarray %d: bad sizes (nstation=%d nfreq=%d ntime=%d)", i, N, F, T);
      return nullptr;
    }
  }
  BatchState* b = new (std::nothrow) BatchState();
  if (!b) {
    release(h);
    fail(XC_ERR_OOM, "host allocation failed");
    return nullptr;
  }
  h->batch = b;
  b->nsub = nsub;
  size_t ring_total = 0, in_total = 0, out_total = 0;
  std::vector<size_t> ring_off(nsub);
  for (int i = 0; i < nsub; ++i) {
    BatchSub& s = b->sub[i];
    s.g.N = nstation[i];
    s.g.P = npol;
    s.g.F = nfreq[i];
    s.g.T = ntime[i];
    s.g.R = 2 * npol * nstation[i];
    s.g.Tp = (ntime[i] + kKBlock - 1) / kKBlock * kKBlock;
    s.g.NB = static_cast<int64_t>(nstation[i]) * (nstation[i] + 1) / 2;
    s.in_bytes = static_cast<size_t>(ntime[i]) * nfreq[i] * nstation[i] * npol * 2;
    s.out_bytes = static_cast<size_t>(nfreq[i]) * s.g.NB * npol * npol * 2 * 4;
    s.pg = xc::planar_geometry(s.g, &s.pack);
    const int64_t slot_bytes = xc::planar_slot_bytes(s.pg, XC_PREC_FP16);
    s.slots_base = xc::planar_ring_slots(s.pg, h->num_sms, XC_PREC_FP16);
    const int64_t cap2 = std::max<int64_t>(s.slots_base, (512ll << 20) / std::max<int64_t>(slot_bytes, 1));
    s.max_slots = static_cast<int>(std::min<int64_t>(
        {static_cast<int64_t>(xc::kMaxRingSlots), static_cast<int64_t>(s.pg.F), 2ll * s.slots_base, cap2}));
    s.max_slots = std::max(s.max_slots, s.slots_base);
    if (s.pack > 1) {
      // Unpacked, the same channel slot size (one 128-input block) serves
      // pack times as many channels.
      s.slots_unpacked = std::min(s.max_slots, xc::planar_ring_slots(s.g, h->num_sms, XC_PREC_FP16));
    }
    ring_off[i] = ring_total;
    ring_total += static_cast<size_t>(s.max_slots) * slot_bytes;
    in_total += s.in_bytes;
    out_total += s.out_bytes;
  }
  h->in_bytes = in_total;
  h->out_bytes = out_total;
  size_t ctr_words = 0;
  for (int i = 0; i < nsub; ++i) ctr_words += 2 * xc::kMaxRingSlots + b->sub[i].g.F;
  cudaError_t e = cudaMalloc(&b->ring_all, ring_total);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->ctr_all), ctr_words * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cuda_fail(e, "batch allocation");
    release(h);
    return nullptr;
  }
  unsigned* c = b->ctr_all;
  for (int i = 0; i < nsub; ++i) {
    BatchSub& s = b->sub[i];
    s.ring = static_cast<char*>(b->ring_all) + ring_off[i];
    s.counters = c;
    c += 2 * xc::kMaxRingSlots;
    s.amax = c;
    c += s.g.F;
    b->order[i] = i;
  }
  b->depth = 1;
  // The larger shape pays when some subarray has more than one block row.
  for (int i = 0; i < nsub; ++i)
    b->shape_default = std::max(b->shape_default, xc::planar_default_shape(b->sub[i].pg, 0));
  b->shape = b->shape_default;
  succeed();
  return h;
}

xc_status xc_batch_correlate(xc_handle* h, const void* const* in, void* const* out, void* stream) {
  if (!h || !h->batch) return fail(XC_ERR_INVALID_ARG, "not a batch handle");
  BatchState* b = h->batch;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  xc::XeLaunch L[XC_BATCH_MAX_SUB];
  xc_status st = batch_prepare(h, in, out, b->order, b->depth, b->packing, b->shape, L);
  if (st != XC_OK) return st;
  if (b->k.grid <= 0) return succeed();
  cudaError_t e = cudaSuccess;
  if (!b->exec) {
    // Capture set-up + the persistent launch once; later calls only update
    // the kernel node's parameters (new buffers and input maps).
    e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "graph capture");
    cudaError_t e1 = xc::planar_setup(L, b->nsub, b->cap_stream);
    if (e1 == cudaSuccess) e1 = xc::planar_launch(b->k, b->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap_stream, &g);
    if (e1 != cudaSuccess || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(e1 != cudaSuccess ? e1 : e, "graph capture");
    }
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    size_t n = 0;
    if (e == cudaSuccess) e = cudaGraphGetNodes(b->graph, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (e == cudaSuccess && n) e = cudaGraphGetNodes(b->graph, nodes.data(), &n);
    for (size_t i = 0; e == cudaSuccess && i < n; ++i) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
        b->knode = nodes[i];
    }
    if (e == cudaSuccess && !b->knode) e = cudaErrorInvalidValue;
    if (e != cudaSuccess) {
      batch_drop_graph(b);
      return cuda_fail(e, "graph instantiation");
    }
  } else {
    cudaKernelNodeParams kp{};
    void* args[1] = {b->k.args};
    kp.func = const_cast<void*>(b->k.func);
    kp.gridDim = dim3(b->k.grid);
    kp.blockDim = dim3(b->k.block);
    kp.sharedMemBytes = static_cast<unsigned>(b->k.smem);
    kp.kernelParams = args;
    kp.extra = nullptr;
    e = cudaGraphExecKernelNodeSetParams(b->exec, b->knode, &kp);
    if (e != cudaSuccess) return cuda_fail(e, "graph update");
  }
  xc_handle::Timed* tm = nullptr;
  if (h->profile) {
    tm = next_timed(h, 1);
    if (!tm) return fail(XC_ERR_CUDA, "profiling event creation failed");
    cudaEventRecord(tm->ev[0], s);
  }
  e = cudaGraphLaunch(b->exec, s);
  if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  if (tm) cudaEventRecord(tm->ev[1], s);
  return succeed();
}

xc_status xc_batch_tune(xc_handle* h, const void* const* in, void* const* out, void* stream,
                        int reps, double* ms, int* best) {
  if (!h || !h->batch) return fail(XC_ERR_INVALID_ARG, "not a batch handle");
  if (reps < 1 || reps > 1000) return fail(XC_ERR_INVALID_ARG, "reps must be in [1, 1000]");
  BatchState* b = h->batch;
  if (ms)
    for (int c = 0; c < XC_BATCH_CANDIDATES; ++c) ms[c] = -1.0;
  // A tuning file that already holds this batch's choice: no timing.
  char key[512] = "";
  if (b->cache_path[0]) {
    batch_key(b, h->dtype, key, sizeof(key));
    double cms = 0.0;
    const int c = cache_lookup_ms(b->cache_path, key, &cms);
    if (c >= 0 && c < XC_BATCH_CANDIDATES) {
      apply_schedule(b, batch_schedule(b, c));
      if (best) *best = c;
      if (ms) ms[c] = cms;
      return succeed();
    }
  }
  bool any_pack = false;
  for (int i = 0; i < b->nsub; ++i) any_pack = any_pack || b->sub[i].pack > 1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_fail(e, "tuning events");
  double best_ms = 0.0;
  int best_c = -1;
  xc_status st = XC_OK;
  for (int c = 0; c < XC_BATCH_CANDIDATES && st == XC_OK; ++c) {
    const Schedule sc = batch_schedule(b, c);
    if (!sc.packing && !any_pack) continue;  // the same launch as its packed twin
    xc::XeLaunch L[XC_BATCH_MAX_SUB];
    if (batch_prepare(h, in, out, sc.order, sc.depth, sc.packing, sc.shape, L) != XC_OK) {
      if (t_status == XC_ERR_CUDA) continue;  // a shape this device cannot launch: not a candidate
      st = t_status;
      break;
    }
    float t = 0.f;
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
      if (r == 1) e = cudaEventRecord(e0, s);
      if (e == cudaSuccess) e = xc::planar_setup(L, b->nsub, s);
      if (e == cudaSuccess) e = xc::planar_launch(b->k, s);
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "tuning launch");
      break;
    }
    const double m = static_cast<double>(t) / reps;
    if (ms) ms[c] = m;
    if (best_c < 0 || m < best_ms) {
      best_ms = m;
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != XC_OK) return st;
  if (best_c < 0) return fail(XC_ERR_CUDA, "no tuning candidate could be launched");
  // The device status word tells whether any candidate gave up on a wait.
  st = xc_synchronize(h, stream);
  if (st != XC_OK) return st;
  apply_schedule(b, batch_schedule(b, best_c));
  if (best) *best = best_c;
  if (b->cache_path[0]) {
    if (FILE* fh = fopen(b->cache_path, "a")) {
      fprintf(fh, "%s\t%d\t%.6f\n", key, best_c, best_ms);
      fclose(fh);
    }
  }
  return succeed();
}

xc_status xc_batch_set_cache(xc_handle* h, const char* path) {
  if (!h || !h->batch) return fail(XC_ERR_INVALID_ARG, "not a batch handle");
  if (path && strlen(path) >= sizeof(h->batch->cache_path))
    return fail(XC_ERR_INVALID_ARG, "cache path longer than %zu bytes", sizeof(h->batch->cache_path) - 1);
  snprintf(h->batch->cache_path, sizeof(h->batch->cache_path), "%s", path ? path : "");
  return succeed();
}

int xc_batch_cache_key(int nsub, const int* nstation, const int* nfreq, const int* ntime, int npol,
                       xc_dtype in_dtype, char* buf, size_t len) {
  if (nsub < 1 || nsub > XC_BATCH_MAX_SUB || !nstation || !nfreq || !ntime || !buf || len == 0)
    return -1;
  int k = snprintf(buf, len, "%s|npol=%d|dtype=%d|", xc_version(), npol, static_cast<int>(in_dtype));
  for (int i = 0; i < nsub && k >= 0 && static_cast<size_t>(k) < len; ++i)
    k += snprintf(buf + k, len - k, "%s%d:%d:%d", i ? "," : "", nstation[i], nfreq[i], ntime[i]);
  return (k < 0 || static_cast<size_t>(k) >= len) ? -1 : k;
}

int xc_batch_cache_lookup(const char* path, const char* key) {
  double ms = 0.0;
  return cache_lookup_ms(path, key, &ms);
}

}  // extern "C"
