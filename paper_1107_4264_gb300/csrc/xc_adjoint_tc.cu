// xc_adjoint_tc.cu -- tensor-core adjoint of the float X-engine.
//
// For a real loss L, with grad_out scattered into G_f and H_f = G_f + G_f^H
// (xc_adjoint.cu), the input gradient is grad_x = conj(g) H_f (g x).  The
// gains fold into the matrix: H'_f = H_f diag(g), so per channel
//
//     grad_y[a][t] = sum_b H'[a][b] x[t][b],     grad_x = conj(g_a) grad_y,
//     grad_g[a]   += sum_t conj(x[t][a]) grad_y[a][t],
//
// a complex GEMM with M = a (inputs), N = t (samples), K = b (inputs).  It
// runs on tcgen05 in the planar form of the forward engine:
//     Re = Hr Xr^T - Hi Xi^T,   Im = Hr Xi^T + Hi Xr^T
// (four MMAs per 16-b step, the second with negate-B).  Operands are split
// into fp16 hi + lo parts after a power-of-two scale per channel (from the
// largest component), and each 64-b block runs three steps (hi hi, lo hi,
// hi lo), about 22 significant bits with fp32 accumulation over K = n.
//
// Kernels: amax of H' and of x per channel; operand formation into 16 KiB
// MMA-ready tiles ([8-column chunk][128 rows][8 fp16], the no-swizzle K-major
// layout); the GEMM, a persistent kernel over 128 x 128 (a, t) tiles with a
// bulk-copy producer warp, an MMA warp and four epilogue warps that re-read
// x (nothing from the forward is stored).
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "xc_launch.h"
#include "xc_ptx.cuh"

namespace xc {
namespace {

constexpr int kBlk = 128;  // rows per tile (a or t)
constexpr int kBK = 64;    // K (b) per tile
constexpr int kTile = kBlk * kBK * 2;
constexpr uint32_t kChunkStride = kBlk * 16;
constexpr uint32_t kGroupStride = 8 * 16;
constexpr int kStages = 3;
constexpr int kStageBytes = 4 * kTile;
constexpr int kThreads = 192;  // producer, MMA, 4 epilogue warps
constexpr int kBarOff = kStages * kStageBytes;
constexpr int kNumBars = 2 * kStages + 5;
constexpr int kSmemBytes = kBarOff + kNumBars * 8 + 16 + 1024;
constexpr uint32_t kTmemCols = 512;  // 2 sets x (D_re, D_im)
constexpr uint32_t kIdesc = ptx::idesc_f16_f32(kBlk, kBlk);
constexpr uint32_t kIdescNegB = kIdesc | (1u << 14);

struct AdjGeom {
  Geometry g;
  int n;   // complex inputs N * P
  int na;  // 128-row blocks over a
  int nk;  // 64-column blocks over b (K)
  int nt;  // 128-row blocks over t
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Power-of-two scale exponent: max |v| 2^-e in [2^14, 2^15) (fp16 hi/lo),
// clamped so that products of two scales stay normal floats.
__device__ __forceinline__ int adj_scale_exp(unsigned bits) {
  const int E = static_cast<int>((bits >> 23) & 0xffu);
  if (E == 0) return 0;
  return max(-60, min(60, E - 127 - 14));
}
__device__ __forceinline__ float adj_exp2i(int e) { return __int_as_float((127 + e) << 23); }

// Byte offset of tile (f, plane, hl, row block rb, K block kb) in an operand
// buffer with nrb row blocks per channel.
__device__ __forceinline__ size_t tile_off(int f, int plane, int hl, int rb, int kb, int nrb, int nk) {
  return (((((static_cast<size_t>(f) * 2 + plane) * 2 + hl) * nrb + rb) * nk) + kb) *
         static_cast<size_t>(kTile);
}

// amax[f] = max |component| of H'_f = H_f diag(g).  Block: 8 rows a of one
// channel, threads along b.
__global__ void adj_amax_h(const float2* __restrict__ H, const float2* __restrict__ gains,
                           unsigned* __restrict__ amax, int n) {
  const int f = blockIdx.y;
  float m = 0.f;
  for (int a = blockIdx.x * 8; a < min(n, blockIdx.x * 8 + 8); ++a) {
    const float2* row = H + (static_cast<size_t>(f) * n + a) * n;
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
      float2 v = row[b];
      if (gains) v = cmul(v, gains[b]);
      m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax + f, __float_as_uint(m));
}

// amax[F + f] = max |component| of x over channel f.  Block: 32 samples t of
// one channel, threads along b.
__global__ void adj_amax_x(const float2* __restrict__ x, unsigned* __restrict__ amax, Geometry g,
                           int n) {
  const int f = blockIdx.y;
  float m = 0.f;
  for (int t = blockIdx.x * 32; t < min(g.T, blockIdx.x * 32 + 32); ++t) {
    const float2* row = x + (static_cast<size_t>(t) * g.F + f) * n;
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
      const float2 v = row[b];
      m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax + g.F + f, __float_as_uint(m));
}

// hi + lo fp16 pairs of 8 scaled values: hi[4], lo[4] (two values per word).
__device__ __forceinline__ void split8(const float (&v)[8], uint32_t (&hi)[4], uint32_t (&lo)[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const __half2 h = __floats2half2_rn(v[2 * k], v[2 * k + 1]);
    const __half2 l = __floats2half2_rn(v[2 * k] - __low2float(h), v[2 * k + 1] - __high2float(h));
    hi[k] = *reinterpret_cast<const uint32_t*>(&h);
    lo[k] = *reinterpret_cast<const uint32_t*>(&l);
  }
}

// Write the four 16-byte row chunks (re hi, re lo, im hi, im lo) of row r,
// chunk c of tile (rb, kb) in channel f.
__device__ __forceinline__ void put_chunks(uint8_t* buf, int f, int rb, int kb, int nrb, int nk,
                                           int c, int r, const float (&re)[8], const float (&im)[8]) {
  uint32_t rh[4], rl[4], ih[4], il[4];
  split8(re, rh, rl);
  split8(im, ih, il);
  const size_t o = static_cast<size_t>(c) * kChunkStride + static_cast<size_t>(r) * 16;
  *reinterpret_cast<uint4*>(buf + tile_off(f, 0, 0, rb, kb, nrb, nk) + o) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
  *reinterpret_cast<uint4*>(buf + tile_off(f, 0, 1, rb, kb, nrb, nk) + o) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
  *reinterpret_cast<uint4*>(buf + tile_off(f, 1, 0, rb, kb, nrb, nk) + o) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
  *reinterpret_cast<uint4*>(buf + tile_off(f, 1, 1, rb, kb, nrb, nk) + o) = make_uint4(il[0], il[1], il[2], il[3]);
}

// A operand: H' tiles, rows a (padded to na * 128), K = b (padded to nk * 64).
// One thread per (row a, 8-column chunk); consecutive threads take
// consecutive rows, so a warp writes 512 contiguous bytes per plane.
__global__ void adj_form_h(const float2* __restrict__ H, const float2* __restrict__ gains,
                           const unsigned* __restrict__ amax, uint8_t* __restrict__ At, AdjGeom G) {
  const int f = blockIdx.y;
  const int rows = G.na * kBlk, chunks = G.nk * (kBK / 8);
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * chunks) return;
  const int a = idx % rows, bc = idx / rows;
  const float s = adj_exp2i(-adj_scale_exp(amax[f]));
  float re[8], im[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int b = bc * 8 + j;
    float2 v = make_float2(0.f, 0.f);
    if (a < G.n && b < G.n) {
      v = H[(static_cast<size_t>(f) * G.n + a) * G.n + b];
      if (gains) v = cmul(v, gains[b]);
    }
    re[j] = v.x * s;
    im[j] = v.y * s;
  }
  put_chunks(At, f, a / kBlk, bc / (kBK / 8), G.na, G.nk, bc % (kBK / 8), a % kBlk, re, im);
}

// B operand: x tiles, rows t (padded to nt * 128), K = b.
__global__ void adj_form_x(const float2* __restrict__ x, const unsigned* __restrict__ amax,
                           uint8_t* __restrict__ Bt, AdjGeom G) {
  const int f = blockIdx.y;
  const int rows = G.nt * kBlk, chunks = G.nk * (kBK / 8);
  const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<int64_t>(rows) * chunks) return;
  const int t = static_cast<int>(idx % rows), bc = static_cast<int>(idx / rows);
  const float s = adj_exp2i(-adj_scale_exp(amax[G.g.F + f]));
  float re[8], im[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int b = bc * 8 + j;
    float2 v = make_float2(0.f, 0.f);
    if (t < G.g.T && b < G.n) v = x[(static_cast<size_t>(t) * G.g.F + f) * G.n + b];
    re[j] = v.x * s;
    im[j] = v.y * s;
  }
  put_chunks(Bt, f, t / kBlk, bc / (kBK / 8), G.nt, G.nk, bc % (kBK / 8), t % kBlk, re, im);
}

struct AdjParams {
  AdjGeom G;
  const uint8_t* At;
  const uint8_t* Bt;
  const unsigned* amax;  // [2F]: H' then x
  const float2* x;
  const float2* gains;
  float2* grad_x;
  float* grad_g;
  unsigned long long timeout_ns;
  int* status;
};

// Persistent GEMM: CTA i takes tiles i, i + grid, ... in (channel, t block,
// a block) order with the a block fastest, so the CTAs working at one time
// share their x tiles (and a channel's H' tiles) through L2.  The stage ring
// runs on across tiles and the accumulator is double-buffered in TMEM: the
// epilogue of one tile overlaps the MMAs of the next.
__global__ void __launch_bounds__(kThreads, 1) adj_gemm_tc(const AdjParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  const uint32_t sbase = ptx::smem_u32(smem);
  const uint32_t bar0 = sbase + kBarOff;
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (kStages + s); };
  auto accf_bar = [&](int b) { return bar0 + 8u * (2 * kStages + b); };
  auto acce_bar = [&](int b) { return bar0 + 8u * (2 * kStages + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * kStages + 4);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(smem + kBarOff + kNumBars * 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const AdjGeom& G = P.G;
  const long long ntiles = static_cast<long long>(G.g.F) * G.nt * G.na;
  auto tile_of = [&](long long it, int* f, int* tb, int* ab) {
    *ab = static_cast<int>(it % G.na);
    const long long r = it / G.na;
    *tb = static_cast<int>(r % G.nt);
    *f = static_cast<int>(r / G.nt);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(full_bar(s), 1);
      ptx::mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(accf_bar(b), 1);
      ptx::mbar_init(acce_bar(b), 4);
    }
    ptx::mbar_init(drain_bar, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
    ptx::fence_proxy_async_smem();
  }
  if (warp == 1) {
    ptx::tmem_alloc(ptx::smem_u32(tmem_holder), kTmemCols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  const ptx::WaitCtl wc{P.timeout_ns, P.status, abort_flag};
  const int steps = G.nk * 3;  // (hi, hi), (lo, hi), (hi, lo) per K block

  if (warp == 0) {
    if (lane == 0) {
      int issued_phase[kStages];
      for (int s = 0; s < kStages; ++s) issued_phase[s] = -1;
      bool ok = true;
      long long gst = 0;  // stage-ring position across tiles
      for (long long it = blockIdx.x; ok && it < ntiles; it += gridDim.x) {
        int f, tb, ab;
        tile_of(it, &f, &tb, &ab);
        for (int st = 0; st < steps; ++st, ++gst) {
          const int stage = static_cast<int>(gst % kStages);
          const uint32_t phase = static_cast<uint32_t>(gst / kStages) & 1u;
          if (!ptx::wait_bounded(empty_bar(stage), phase ^ 1u, wc)) {
            ok = false;
            break;
          }
          const int kb = st / 3, j = st % 3;
          const int hla = j == 1 ? 1 : 0, hlb = j == 2 ? 1 : 0;
          const uint32_t dst = sbase + stage * kStageBytes;
          const uint32_t fb = full_bar(stage);
          ptx::mbar_arrive_expect_tx(fb, kStageBytes);
          ptx::bulk_load(dst, P.At + tile_off(f, 0, hla, ab, kb, G.na, G.nk), kTile, fb);
          ptx::bulk_load(dst + kTile, P.At + tile_off(f, 1, hla, ab, kb, G.na, G.nk), kTile, fb);
          ptx::bulk_load(dst + 2 * kTile, P.Bt + tile_off(f, 0, hlb, tb, kb, G.nt, G.nk), kTile, fb);
          ptx::bulk_load(dst + 3 * kTile, P.Bt + tile_off(f, 1, hlb, tb, kb, G.nt, G.nk), kTile, fb);
          issued_phase[stage] = static_cast<int>(phase);
        }
      }
      if (!ok) {
        for (int s = 0; s < kStages; ++s) {
          if (issued_phase[s] < 0) continue;
          const uint64_t t0 = ptx::globaltimer();
          while (!ptx::mbar_try_wait(full_bar(s), static_cast<uint32_t>(issued_phase[s])) &&
                 ptx::globaltimer() - t0 < P.timeout_ns) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true, issued_any = false;
      long long gst = 0;
      uint32_t u = 0;  // tiles done by this CTA
      for (long long it = blockIdx.x; ok && it < ntiles; it += gridDim.x, ++u) {
        const uint32_t ab = u & 1u, ap = (u >> 1) & 1u;
        if (!ptx::wait_bounded(acce_bar(ab), ap ^ 1u, wc)) {
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const uint32_t d_re = tmem + ab * 256, d_im = d_re + 128;
        for (int st = 0; st < steps; ++st, ++gst) {
          const int stage = static_cast<int>(gst % kStages);
          const uint32_t phase = static_cast<uint32_t>(gst / kStages) & 1u;
          if (!ptx::wait_bounded(full_bar(stage), phase, wc)) {
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t ar = sbase + stage * kStageBytes, ai = ar + kTile;
          const uint32_t br = ar + 2 * kTile, bi = ar + 3 * kTile;
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k) {
            const uint32_t acc = (st > 0 || k > 0) ? 1u : 0u;
            const uint32_t ko = k * 2 * kChunkStride;
            const uint64_t dar = ptx::interleave_kmajor_desc(ar + ko, kChunkStride, kGroupStride);
            const uint64_t dai = ptx::interleave_kmajor_desc(ai + ko, kChunkStride, kGroupStride);
            const uint64_t dbr = ptx::interleave_kmajor_desc(br + ko, kChunkStride, kGroupStride);
            const uint64_t dbi = ptx::interleave_kmajor_desc(bi + ko, kChunkStride, kGroupStride);
            ptx::mma_f16_ss(d_re, dar, dbr, kIdesc, acc);      // Re += Hr Xr^T
            ptx::mma_f16_ss(d_re, dai, dbi, kIdescNegB, 1u);   // Re -= Hi Xi^T
            ptx::mma_f16_ss(d_im, dar, dbi, kIdesc, acc);      // Im += Hr Xi^T
            ptx::mma_f16_ss(d_im, dai, dbr, kIdesc, 1u);       // Im += Hi Xr^T
          }
          issued_any = true;
          ptx::mma_commit(empty_bar(stage));
        }
        if (!ok) break;
        ptx::mma_commit(accf_bar(ab));
      }
      if (!ok && issued_any) {
        ptx::mma_commit(drain_bar);
        const uint64_t t0 = ptx::globaltimer();
        while (!ptx::mbar_try_wait(drain_bar, 0) && ptx::globaltimer() - t0 < P.timeout_ns) {
        }
      }
    }
  } else {
    // Epilogue: warp q owns TMEM lanes 32q..32q+31 = rows a of the tile.
    const int q = warp & 3;
    const uint32_t t_lanes = tmem + (static_cast<uint32_t>(q * 32) << 16);
    uint32_t u = 0;
    for (long long it = blockIdx.x; it < ntiles; it += gridDim.x, ++u) {
      int f, tb, abk;
      tile_of(it, &f, &tb, &abk);
      const uint32_t ab = u & 1u, ap = (u >> 1) & 1u;
      const bool got = ptx::wait_bounded(accf_bar(ab), ap, wc);
      if (!__all_sync(0xffffffffu, got)) break;
      ptx::tc_fence_after();
      const int a = abk * kBlk + q * 32 + lane;
      const float sc = adj_exp2i(adj_scale_exp(P.amax[f]) + adj_scale_exp(P.amax[G.g.F + f]));
      const bool row_ok = a < G.n;
      const float2 ga = (P.gains && row_ok) ? P.gains[a] : make_float2(1.f, 0.f);
      const float2 cga = make_float2(ga.x, -ga.y);
      float2 gg = make_float2(0.f, 0.f);
#pragma unroll 1
      for (int piece = 0; piece < kBlk / 32; ++piece) {
        uint32_t vr[32], vi[32];
        ptx::tmem_ld_32x32b_x32(t_lanes + ab * 256 + piece * 32, vr);
        ptx::tmem_ld_32x32b_x32(t_lanes + ab * 256 + 128 + piece * 32, vi);
        ptx::tmem_wait_ld();
        if (piece == kBlk / 32 - 1) {
          ptx::tc_fence_before();
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(acce_bar(ab));
        }
        if (!row_ok) continue;
        // All 32 samples of x first (the compiler may not move these loads
        // above the grad_x stores), then grad_x and the grad_g terms.
        const int t0 = tb * kBlk + piece * 32;
        const size_t step = static_cast<size_t>(G.g.F) * G.n;
        const size_t idx0 = (static_cast<size_t>(t0) * G.g.F + f) * G.n + a;
        float2 xv[32];
#pragma unroll
        for (int j = 0; j < 32; ++j)
          xv[j] = t0 + j < G.g.T ? __ldcs(P.x + idx0 + j * step) : make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (t0 + j >= G.g.T) continue;
          const float2 gy = make_float2(__uint_as_float(vr[j]) * sc, __uint_as_float(vi[j]) * sc);
          __stcs(P.grad_x + idx0 + j * step, cmul(cga, gy));
          gg.x += xv[j].x * gy.x + xv[j].y * gy.y;  // conj(x) gy
          gg.y += xv[j].x * gy.y - xv[j].y * gy.x;
        }
      }
      if (row_ok && P.grad_g) {
        atomicAdd(P.grad_g + 2 * a, gg.x);
        atomicAdd(P.grad_g + 2 * a + 1, gg.y);
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, kTmemCols);
  }
}

AdjGeom adj_geom(const Geometry& g) {
  AdjGeom G;
  G.g = g;
  G.n = g.N * g.P;
  G.na = (G.n + kBlk - 1) / kBlk;
  G.nk = (G.n + kBK - 1) / kBK;
  G.nt = (g.T + kBlk - 1) / kBlk;
  return G;
}

}  // namespace

size_t adjoint_tc_workspace_bytes(const Geometry& g) {
  const AdjGeom G = adj_geom(g);
  const size_t per_rb = static_cast<size_t>(2) * 2 * G.nk * kTile;  // planes x hi/lo x K blocks
  return static_cast<size_t>(g.F) * (G.na + G.nt) * per_rb + 256 + sizeof(unsigned) * 2 * g.F;
}

cudaError_t launch_adjoint_tc(const void* grad_out, const void* in, const void* gains, void* grad_in,
                              float* grad_g, void* h_ws, void* tc_ws, const Geometry& g,
                              unsigned long long timeout_ns, int* status, cudaStream_t s) {
  const AdjGeom G = adj_geom(g);
  if (G.n == 0 || g.F == 0 || g.T == 0) return cudaSuccess;
  cudaError_t e = launch_build_h(grad_out, h_ws, g, s);
  if (e != cudaSuccess) return e;
  uint8_t* At = static_cast<uint8_t*>(tc_ws);
  const size_t per_rb = static_cast<size_t>(2) * 2 * G.nk * kTile;
  uint8_t* Bt = At + static_cast<size_t>(g.F) * G.na * per_rb;
  unsigned* amax = reinterpret_cast<unsigned*>(Bt + static_cast<size_t>(g.F) * G.nt * per_rb);
  const float2* H = static_cast<const float2*>(h_ws);
  const float2* x = static_cast<const float2*>(in);
  const float2* gn = static_cast<const float2*>(gains);
  e = cudaMemsetAsync(amax, 0, sizeof(unsigned) * 2 * g.F, s);
  if (e == cudaSuccess && grad_g) e = cudaMemsetAsync(grad_g, 0, sizeof(float) * 2 * G.n, s);
  if (e != cudaSuccess) return e;
  adj_amax_h<<<dim3((G.n + 7) / 8, g.F), 256, 0, s>>>(H, gn, amax, G.n);
  adj_amax_x<<<dim3((g.T + 31) / 32, g.F), 256, 0, s>>>(x, amax, g, G.n);
  const int rows_a = G.na * kBlk * G.nk * (kBK / 8);
  adj_form_h<<<dim3((rows_a + 255) / 256, g.F), 256, 0, s>>>(H, gn, amax, At, G);
  const int64_t rows_t = static_cast<int64_t>(G.nt) * kBlk * G.nk * (kBK / 8);
  if ((rows_t + 255) / 256 > 0x7fffffff) return cudaErrorInvalidConfiguration;
  adj_form_x<<<dim3(static_cast<unsigned>((rows_t + 255) / 256), g.F), 256, 0, s>>>(x, amax, Bt, G);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(adj_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) return e;
  AdjParams P;
  P.G = G;
  P.At = At;
  P.Bt = Bt;
  P.amax = amax;
  P.x = x;
  P.gains = gn;
  P.grad_x = static_cast<float2*>(grad_in);
  P.grad_g = grad_g;
  P.timeout_ns = timeout_ns;
  P.status = status;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long ntiles = static_cast<long long>(g.F) * G.nt * G.na;
  adj_gemm_tc<<<static_cast<unsigned>(std::min<long long>(ntiles, sms)), kThreads, kSmemBytes, s>>>(P);
  return cudaGetLastError();
}

}  // namespace xc
