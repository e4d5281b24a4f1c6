// xc_adjoint.cu -- adjoint (backward) of the float X-engine and gain handling.
//
// Forward (Eq. outer of Sec. 2.1 with complex gains g applied to the
// voltages first): V_f[a][b] = sum_t y_a(t) conj(y_b(t)), y = g * x, stored
// on the lower station triangle.  For a real loss L with
// grad_out = dL/dRe V + i dL/dIm V on the stored entries (PyTorch's complex
// convention), G_f is the dense n x n matrix holding grad_out on the stored
// entries and zero elsewhere, and H_f = G_f + G_f^H:
//     grad_y(t) = H_f y(t),   grad_x = conj(g) grad_y,
//     grad_g    = sum_{f,t} conj(x) grad_y.
// (The paper has no adjoint; this is the differentiable form of the engine.)
//
// build_h_kernel scatters grad_out into H_f; adjoint_gemm_kernel computes
// grad_y = H_f Y_f for a 64-input x 64-sample block per CTA with an FP32
// complex register tile (4 x 4 per thread) over 16-input shared-memory
// stages, re-reading x (no forward intermediates are stored), and writes
// grad_x and per-block partial sums of grad_g (atomically added).
#include <cuda_runtime.h>

#include "xc_launch.h"

namespace xc {
namespace {

constexpr int kAT = 64;   // inputs (rows a) per block
constexpr int kTT = 64;   // samples per block
constexpr int kKB = 16;   // inputs b per shared-memory stage

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// H[f][a][b] (complex) from the packed lower-triangle gradient.
__global__ void build_h_kernel(const float2* __restrict__ grad_out, float2* __restrict__ H,
                               Geometry g) {
  const int n = g.N * g.P;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y * blockDim.y + threadIdx.y;
  const int f = blockIdx.z;
  if (a >= n || b >= n) return;
  const int P = g.P;
  const int sa = a / P, pa = a - sa * P;
  const int sb = b / P, pb = b - sb * P;
  const float2* go = grad_out + static_cast<int64_t>(f) * g.NB * P * P;
  float2 h = make_float2(0.f, 0.f);
  if (sa >= sb) {  // G[a][b]
    const float2 v = go[(static_cast<int64_t>(sa) * (sa + 1) / 2 + sb) * P * P + pa * P + pb];
    h.x += v.x;
    h.y += v.y;
  }
  if (sb >= sa) {  // conj(G[b][a])
    const float2 v = go[(static_cast<int64_t>(sb) * (sb + 1) / 2 + sa) * P * P + pb * P + pa];
    h.x += v.x;
    h.y -= v.y;
  }
  H[(static_cast<int64_t>(f) * n + a) * n + b] = h;
}

// grad_y = H Y for rows a0..a0+63, samples t0..t0+63 of channel f.
// Thread (tx, ty): rows a0 + {ty, ty+16, ty+32, ty+48}, samples
// t0 + {tx, tx+16, tx+32, tx+48}.
__global__ void __launch_bounds__(256) adjoint_gemm_kernel(const float2* __restrict__ x,
                                                           const float2* __restrict__ H,
                                                           const float2* __restrict__ gains,
                                                           float2* __restrict__ grad_x,
                                                           float* __restrict__ grad_g, Geometry g) {
  __shared__ float2 Hs[kKB][kAT + 1];  // [b][a]
  __shared__ float2 Ys[kKB][kTT + 1];  // [b][t]
  const int n = g.N * g.P;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int a0 = blockIdx.x * kAT;
  const int t0 = blockIdx.y * kTT;
  const int f = blockIdx.z;
  const float2* Hf = H + static_cast<int64_t>(f) * n * n;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);

  for (int b0 = 0; b0 < n; b0 += kKB) {
    // H tile: 64 rows x 16 columns; Y tile: 16 inputs x 64 samples.
    for (int i = threadIdx.x; i < kKB * kAT; i += 256) {
      const int bb = i % kKB, aa = i / kKB;
      const int a = a0 + aa, b = b0 + bb;
      Hs[bb][aa] = (a < n && b < n) ? Hf[static_cast<int64_t>(a) * n + b] : make_float2(0.f, 0.f);
    }
    for (int i = threadIdx.x; i < kKB * kTT; i += 256) {
      const int bb = i % kKB, tt = i / kKB;
      const int b = b0 + bb, t = t0 + tt;
      float2 y = make_float2(0.f, 0.f);
      if (b < n && t < g.T) {
        y = x[(static_cast<int64_t>(t) * g.F + f) * n + b];
        if (gains) y = cmul(gains[b], y);
      }
      Ys[bb][tt] = y;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kKB; ++k) {
      float2 hv[4], yv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) hv[i] = Hs[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) yv[j] = Ys[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fmaf(hv[i].x, yv[j].x, acc[i][j].x);
          acc[i][j].x = fmaf(-hv[i].y, yv[j].y, acc[i][j].x);
          acc[i][j].y = fmaf(hv[i].x, yv[j].y, acc[i][j].y);
          acc[i][j].y = fmaf(hv[i].y, yv[j].x, acc[i][j].y);
        }
    }
    __syncthreads();
  }

  // grad_x = conj(g) grad_y; grad_g partial = sum_t conj(x) grad_y.
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = a0 + ty + 16 * i;
    const bool row_ok = a < n;
    const float2 ga = (gains && row_ok) ? conjf2(gains[a]) : make_float2(1.f, 0.f);
    float2 gg = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int t = t0 + tx + 16 * j;
      if (row_ok && t < g.T) {
        const int64_t idx = (static_cast<int64_t>(t) * g.F + f) * n + a;
        grad_x[idx] = cmul(ga, acc[i][j]);
        const float2 c = cmul(conjf2(x[idx]), acc[i][j]);
        gg.x += c.x;
        gg.y += c.y;
      }
    }
    // Sum over the 16 threads (tx) sharing row a: 16 consecutive lanes.
    // Every lane takes part, whatever its row.
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      gg.x += __shfl_xor_sync(0xffffffffu, gg.x, o);
      gg.y += __shfl_xor_sync(0xffffffffu, gg.y, o);
    }
    if (row_ok && tx == 0 && grad_g) {
      atomicAdd(grad_g + 2 * a, gg.x);
      atomicAdd(grad_g + 2 * a + 1, gg.y);
    }
  }
}

}  // namespace

cudaError_t launch_build_h(const void* grad_out, void* h_ws, const Geometry& g, cudaStream_t s) {
  const int n = g.N * g.P;
  if (n == 0 || g.F == 0) return cudaSuccess;
  dim3 hb(32, 8);
  dim3 hg((n + 31) / 32, (n + 7) / 8, g.F);
  if (hg.y > 65535u || hg.z > 65535u) return cudaErrorInvalidConfiguration;
  build_h_kernel<<<hg, hb, 0, s>>>(static_cast<const float2*>(grad_out), static_cast<float2*>(h_ws), g);
  return cudaGetLastError();
}

cudaError_t launch_adjoint(const void* grad_out, const void* in, const void* gains, void* grad_in,
                           float* grad_g, void* h_ws, const Geometry& g, cudaStream_t s) {
  const int n = g.N * g.P;
  if (n == 0 || g.F == 0) return cudaSuccess;
  float2* H = static_cast<float2*>(h_ws);
  cudaError_t e = launch_build_h(grad_out, h_ws, g, s);
  if (e != cudaSuccess) return e;
  if (grad_g) {
    e = cudaMemsetAsync(grad_g, 0, sizeof(float) * 2 * n, s);
    if (e != cudaSuccess) return e;
  }
  dim3 gg((n + kAT - 1) / kAT, (g.T + kTT - 1) / kTT, g.F);
  if (gg.y > 65535u || gg.z > 65535u) return cudaErrorInvalidConfiguration;
  adjoint_gemm_kernel<<<gg, 256, 0, s>>>(static_cast<const float2*>(in), H,
                                         static_cast<const float2*>(gains),
                                         static_cast<float2*>(grad_in), grad_g, g);
  return cudaGetLastError();
}

}  // namespace xc
