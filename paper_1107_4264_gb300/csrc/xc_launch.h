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

// FP32 CUDA-core X-engine (comparator) directly from the input.
cudaError_t launch_fp32_xengine(const void* in, int in_dtype, void* out, const Geometry& g,
                                int accumulate, cudaStream_t s);

// Record `s` and a printf-style message as this thread's last error
// (xc_last_error / xc_last_error_message); returns s.
xc_status record_error(xc_status s, const char* fmt, ...);

}  // namespace xc
