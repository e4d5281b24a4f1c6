// xc_fp32.cu -- plain FP32 CUDA-core X-engine (the same-GPU comparator).
//
// This is the software-managed-cache design of Sec. 4.4 (kernel 11:
// cooperative loads into shared memory, a register tile per thread,
// double-buffered shared memory with one barrier per step), re-tuned for
// sm_103a: 256 threads per block, a 4 x 4 complex register tile per thread
// (64 FFMA per sample), a 64 x 64 input block per CTA, 32 samples per
// shared-memory stage, triangular block grid of Sec. 4.2.
//
// Every complex multiply-accumulate x_a conj(x_b) is 4 FFMA (8 flops), the
// paper's Eq. (flops) convention.  For 8-bit input the FP32 accumulators are
// exact while every partial sum stays below 2^24: with at most 2 products of
// magnitude <= 2^14 per sample per accumulator, 512 samples are safe, so the
// float accumulators are drained into int32 every 512 samples and the output
// is bit-exact.
#include <cuda_fp16.h>

#include "xc_launch.h"

namespace xc {
namespace {

constexpr int kTile = 64;     // inputs per block side
constexpr int kTK = 32;       // samples per shared-memory stage
constexpr int kDrainStages = 512 / kTK;
constexpr int kThreads = 256;
constexpr int kSmemBytes = 2 /*buf*/ * 2 /*row,col*/ * kTK * kTile * 8;

template <int DT>
__device__ __forceinline__ float2 load_cx(const void* in, int64_t cidx) {
  if constexpr (DT == 0) {
    const char2 v = static_cast<const char2*>(in)[cidx];
    return make_float2(static_cast<float>(v.x), static_cast<float>(v.y));
  } else if constexpr (DT == 1) {
    return __half22float2(static_cast<const __half2*>(in)[cidx]);
  } else {
    return static_cast<const float2*>(in)[cidx];
  }
}

// Fetch 8 consecutive complex inputs (a0 .. a0+7) of sample t into registers.
template <int DT>
__device__ __forceinline__ void fetch8(const void* in, const Geometry& g, int n, int f, int t,
                                       int a0, bool vec, float2 (&v)[8]) {
  if (t >= g.T || a0 >= n) {
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = make_float2(0.f, 0.f);
    return;
  }
  const int64_t base = (static_cast<int64_t>(t) * g.F + f) * n + a0;
  if (vec) {
    if constexpr (DT == 0) {
      const uint4 w = *reinterpret_cast<const uint4*>(static_cast<const char2*>(in) + base);
      const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int b0 = static_cast<int>(static_cast<int8_t>(ws[i] & 0xff));
        const int b1 = static_cast<int>(static_cast<int8_t>((ws[i] >> 8) & 0xff));
        const int b2 = static_cast<int>(static_cast<int8_t>((ws[i] >> 16) & 0xff));
        const int b3 = static_cast<int>(static_cast<int8_t>(ws[i] >> 24));
        v[2 * i] = make_float2(static_cast<float>(b0), static_cast<float>(b1));
        v[2 * i + 1] = make_float2(static_cast<float>(b2), static_cast<float>(b3));
      }
    } else if constexpr (DT == 1) {
      const uint4* src = reinterpret_cast<const uint4*>(static_cast<const __half2*>(in) + base);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint4 w = src[h];
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          __half2 hv;
          *reinterpret_cast<uint32_t*>(&hv) = ws[i];
          v[4 * h + i] = __half22float2(hv);
        }
      }
    } else {
      const float4* src = reinterpret_cast<const float4*>(static_cast<const float2*>(in) + base);
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const float4 w = src[h];
        v[2 * h] = make_float2(w.x, w.y);
        v[2 * h + 1] = make_float2(w.z, w.w);
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i)
      v[i] = (a0 + i < n) ? load_cx<DT>(in, base + i) : make_float2(0.f, 0.f);
  }
}

template <int DT>
__global__ void __launch_bounds__(kThreads, 2)
    fp32_xengine_kernel(const void* __restrict__ in, void* __restrict__ out, Geometry g,
                        int accumulate, int vec, const float2* __restrict__ gains) {
  extern __shared__ __align__(16) float2 sm[];  // [buf][row|col][kTK][kTile]
  const int tx = threadIdx.x & 15;
  const int ty = threadIdx.x >> 4;
  const int f = blockIdx.y;
  int64_t bx64, by64;
  tri_coords(blockIdx.x, &bx64, &by64);
  const int bx = static_cast<int>(bx64), by = static_cast<int>(by64);
  const bool diag = bx == by;
  const int n = g.N * g.P;
  const int row0 = by * kTile, col0 = bx * kTile;

  // Loader role: thread -> (sample lt, 8-input segment seg) of one operand.
  const int lt = threadIdx.x >> 3;
  const int seg = threadIdx.x & 7;

  float2 pre_r[8], pre_c[8];
  // Gains (float input only) y = g x, applied as samples are fetched.
  float2 gr[8], gc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int ar = row0 + seg * 8 + i, ac = col0 + seg * 8 + i;
    gr[i] = (gains && ar < n) ? gains[ar] : make_float2(1.f, 0.f);
    gc[i] = (gains && ac < n) ? gains[ac] : make_float2(1.f, 0.f);
  }
  auto apply = [&](float2 (&v)[8], const float2 (&gv)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
      v[i] = make_float2(gv[i].x * v[i].x - gv[i].y * v[i].y, gv[i].x * v[i].y + gv[i].y * v[i].x);
  };
  auto fetch = [&](int t0) {
    fetch8<DT>(in, g, n, f, t0 + lt, row0 + seg * 8, vec, pre_r);
    if (!diag) fetch8<DT>(in, g, n, f, t0 + lt, col0 + seg * 8, vec, pre_c);
    if (DT != 0 && gains) {
      apply(pre_r, gr);
      if (!diag) apply(pre_c, gc);
    }
  };
  auto stash = [&](int buf) {
    float2* rdst = sm + ((buf * 2 + 0) * kTK + lt) * kTile + seg * 8;
#pragma unroll
    for (int i = 0; i < 8; i += 2)
      *reinterpret_cast<float4*>(rdst + i) = make_float4(pre_r[i].x, pre_r[i].y, pre_r[i + 1].x, pre_r[i + 1].y);
    if (!diag) {
      float2* cdst = sm + ((buf * 2 + 1) * kTK + lt) * kTile + seg * 8;
#pragma unroll
      for (int i = 0; i < 8; i += 2)
        *reinterpret_cast<float4*>(cdst + i) = make_float4(pre_c[i].x, pre_c[i].y, pre_c[i + 1].x, pre_c[i + 1].y);
    }
  };

  // Register tile: rows {2ty, 2ty+1, 32+2ty, 33+2ty}, cols {2tx, 2tx+1, 32+2tx, 33+2tx}.
  float are[4][4], aim[4][4];
  int ire[4][4], iim[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      are[i][j] = aim[i][j] = 0.f;
      ire[i][j] = iim[i][j] = 0;
    }

  const int nstages = (g.T + kTK - 1) / kTK;
  fetch(0);
  stash(0);
  __syncthreads();
  for (int st = 0; st < nstages; ++st) {
    const int buf = st & 1;
    const bool more = st + 1 < nstages;
    if (more) fetch((st + 1) * kTK);
    const float2* rsrc = sm + (buf * 2 + 0) * kTK * kTile;
    const float2* csrc = sm + (buf * 2 + (diag ? 0 : 1)) * kTK * kTile;
#pragma unroll 4
    for (int tt = 0; tt < kTK; ++tt) {
      const float4 ra = *reinterpret_cast<const float4*>(rsrc + tt * kTile + 2 * ty);
      const float4 rb = *reinterpret_cast<const float4*>(rsrc + tt * kTile + 32 + 2 * ty);
      const float4 ca = *reinterpret_cast<const float4*>(csrc + tt * kTile + 2 * tx);
      const float4 cb = *reinterpret_cast<const float4*>(csrc + tt * kTile + 32 + 2 * tx);
      const float xr[4] = {ra.x, ra.z, rb.x, rb.z}, xi[4] = {ra.y, ra.w, rb.y, rb.w};
      const float yr[4] = {ca.x, ca.z, cb.x, cb.z}, yi[4] = {ca.y, ca.w, cb.y, cb.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          // x_i * conj(y_j)
          are[i][j] = fmaf(xr[i], yr[j], are[i][j]);
          are[i][j] = fmaf(xi[i], yi[j], are[i][j]);
          aim[i][j] = fmaf(xi[i], yr[j], aim[i][j]);
          aim[i][j] = fmaf(-xr[i], yi[j], aim[i][j]);
        }
    }
    if (DT == 0 && ((st + 1) % kDrainStages == 0 || !more)) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          ire[i][j] += __float2int_rn(are[i][j]);
          iim[i][j] += __float2int_rn(aim[i][j]);
          are[i][j] = aim[i][j] = 0.f;
        }
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
  }

  // Store the lower station triangle of this block.
  const int P = g.P;
  const int rows[4] = {row0 + 2 * ty, row0 + 2 * ty + 1, row0 + 32 + 2 * ty, row0 + 33 + 2 * ty};
  const int cols[4] = {col0 + 2 * tx, col0 + 2 * tx + 1, col0 + 32 + 2 * tx, col0 + 33 + 2 * tx};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = rows[i];
    const int s1 = a / P, p1 = a - s1 * P;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b = cols[j];
      const int s2 = b / P, p2 = b - s2 * P;
      if (a < n && b < n && s2 <= s1) {
        const int64_t k = static_cast<int64_t>(s1) * (s1 + 1) / 2 + s2;
        const int64_t o = ((static_cast<int64_t>(f) * g.NB + k) * (P * P) + p1 * P + p2) * 2;
        if (DT == 0) {
          int* op = static_cast<int*>(out) + o;
          if (accumulate) {
            op[0] += ire[i][j];
            op[1] += iim[i][j];
          } else {
            *reinterpret_cast<int2*>(op) = make_int2(ire[i][j], iim[i][j]);
          }
        } else {
          float* op = static_cast<float*>(out) + o;
          if (accumulate) {
            op[0] += are[i][j];
            op[1] += aim[i][j];
          } else {
            *reinterpret_cast<float2*>(op) = make_float2(are[i][j], aim[i][j]);
          }
        }
      }
    }
  }
}

}  // namespace

cudaError_t launch_fp32_xengine(const void* in, int in_dtype, void* out, const Geometry& g,
                                int accumulate, const void* gains_v, cudaStream_t s) {
  const float2* gains = static_cast<const float2*>(gains_v);
  const int n = g.N * g.P;
  const int nb = (n + kTile - 1) / kTile;
  const long long ntiles = static_cast<long long>(nb) * (nb + 1) / 2;
  if (ntiles > 0x7fffffffLL || g.F > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid(static_cast<unsigned>(ntiles), g.F);
  const int csize = in_dtype == 0 ? 2 : (in_dtype == 1 ? 4 : 8);
  // 8 consecutive complex samples of one input row start on a 16-byte boundary
  // when the row length n is a multiple of 8 and the base pointer is aligned.
  const int vec = (n % 8 == 0) && (reinterpret_cast<uintptr_t>(in) % 16 == 0) && csize * 8 >= 16;
  cudaError_t e;
  switch (in_dtype) {
    case 0:
      e = cudaFuncSetAttribute(fp32_xengine_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
      if (e != cudaSuccess) return e;
      fp32_xengine_kernel<0><<<grid, kThreads, kSmemBytes, s>>>(in, out, g, accumulate, vec, gains);
      break;
    case 1:
      e = cudaFuncSetAttribute(fp32_xengine_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
      if (e != cudaSuccess) return e;
      fp32_xengine_kernel<1><<<grid, kThreads, kSmemBytes, s>>>(in, out, g, accumulate, vec, gains);
      break;
    case 2:
      e = cudaFuncSetAttribute(fp32_xengine_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
      if (e != cudaSuccess) return e;
      fp32_xengine_kernel<2><<<grid, kThreads, kSmemBytes, s>>>(in, out, g, accumulate, vec, gains);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// FP32 CUDA-core peak probe: every thread runs 8 independent fused
// multiply-add chains (enough to hide the FFMA latency at 16 warps per SM)
// for `iters` rounds, 2 flops per FFMA.  The result is folded into `sink` so
// that no chain can be removed.
__global__ void __launch_bounds__(512) ffma_probe_kernel(long long iters, float* sink) {
  float a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = static_cast<float>(threadIdx.x + i) * 1e-3f;
  const float b = 0.999f, c = 1e-4f;
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = fmaf(a[i], b, c);
    }
  }
  float t = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) t += a[i];
  if (t == 123.456f) sink[blockIdx.x] = t;  // never true for these inputs; keeps the chains live
}

long long launch_ffma_probe(long long iters, float* sink, int num_sms, cudaStream_t s) {
  const int blocks = num_sms * 4;
  ffma_probe_kernel<<<blocks, 512, 0, s>>>(iters, sink);
  if (cudaGetLastError() != cudaSuccess) return -1;
  return 2LL * 8 * 16 * iters * 512 * blocks;
}

}  // namespace xc
