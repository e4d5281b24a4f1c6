// xc_xengine.cu -- fused persistent tensor-core X-engine for sm_103a.
//
// One launch per integration does all of Eq. (outer) (Sec. 2.1) for every
// channel: operand formation, the triangular block schedule, the tcgen05
// accumulation and the visibility epilogue.
//
// Operands.  Per channel the complex rank-T update is the real symmetric
// product G_f = Y_f Y_f^T, Y_f having one row per real input component
// (r = (s*P + p)*2 + c) and one column per sample.  Converter warps turn
// each channel's corner-turned input (Sec. 4.1 order) into a K-major fp16
// Y_f once, writing it into a ring of a few channel slots in global memory
// small enough to stay in L2; the 36 (Large-N) tensor-core blocks of the
// channel then read it back through TMA.  Each input element is converted
// once, not once per block that uses it, so conversion costs a few percent of
// the SM's issue slots and none of its shared-memory bandwidth.  The int8 ->
// fp16 widening is exact (|x| <= 128 < 2^11) and the transpose happens in
// registers: a lane loads 4 rows x 16 samples as sixteen 32-bit words and
// byte-permutes them into per-row runs of 8 samples.
//
// Ring protocol (all counters monotonic within a launch, zeroed by the host):
//   ready[slot]: converted units (128 rows x 64 samples) of the channels
//                that occupied `slot`, published in batches of up to 4;
//                channel c = generation c / ring of slot c % ring is
//                complete when ready >= (gen + 1) * units.
//   done[slot]:  blocks whose operands have fully landed in shared memory;
//                a converter may overwrite slot s with channel c once
//                done >= gen(c) * blocks_per_channel.
// Dependencies only point to lower channels (items and units are processed
// in channel order, all CTAs are co-resident), so the ring cannot deadlock;
// every wait is still bounded.
//
// Blocks (Sec. 4.2): 128 x 128 tiles of G_f on or below the diagonal,
// enumerated by g = by(by+1)/2 + bx; tile edges fall on station boundaries.
// Diagonal tiles use one operand slab for both MMA operands and store only
// their lower station triangle (Sec. 4.4).
//
// CTA roles (persistent, one CTA per SM, channel-major items):
//   warp 0      TMA producer (one thread): waits for the channel in the
//               ring, then streams 64-sample K-blocks into a 6-stage ring
//   warp 1      MMA issuer (one thread), owns TMEM (two 128-column fp32
//               accumulators used alternately)
//   warps 2..5  epilogue: TMEM -> registers -> 2x2 complex combine -> store
//   warps 6..9  converters
//
// Exact 8-bit accumulation: a chunk of at most 1024 samples keeps every fp32
// partial sum an integer of magnitude <= 2^24 (exact); each chunk is
// drained, converted to int32 and added into the output (stored for the
// first chunk), so integrations of any length stay bit-exact.
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

#include "xc_convert.cuh"
#include "xc_launch.h"
#include "xc_ptx.cuh"

namespace xc {
namespace {

using namespace conv;

constexpr int kBM = 128;
constexpr int kBN = 128;
constexpr int kBK = 64;
constexpr int kStages = 6;
constexpr int kNumEpiWarps = 4;
constexpr int kThreads = 32 * (2 + kNumEpiWarps + kNumConvWarps);
constexpr int kOperBytes = kBM * kBK * 2;
constexpr int kChunkKB = 16;  // 1024 samples
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kIdesc = ptx::idesc_f16_f32(kBM, kBN);

constexpr int kBarOff = kStages * 2 * kOperBytes;
constexpr int kNumBars = 2 * kStages + 5;
constexpr int kSmemBytes = kBarOff + kNumBars * 8 + 16 + 1024;

// --------------------------------------------------------------- epilogue

// Combine one 32-column piece (8 column stations at P = 2, 16 at P = 1) of
// this thread's G row into visibilities and store them (add when `add`).
template <bool IS_INT>
__device__ __forceinline__ void store_piece(const uint32_t (&r)[32], const XeParams& p, int f,
                                            int bx, int by, int row, int lane, int piece,
                                            bool add) {
  using AccT = typename std::conditional<IS_INT, int, float>::type;
  using OutT = AccT;
  const Geometry& g = p.g;
  OutT* out = static_cast<OutT*>(p.out);
  AccT v[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    if constexpr (IS_INT) {
      v[i] = __float2int_rn(__uint_as_float(r[i]));
    } else {
      v[i] = __uint_as_float(r[i]);
    }
  }
  const int c = lane & 1;
  if (g.P == 2) {
    const int p1 = (row >> 1) & 1;
    const int s1 = by * (kBM / 4) + (row >> 2);
    const bool row_ok = s1 < g.N;
    const int64_t krow = static_cast<int64_t>(f) * g.NB + static_cast<int64_t>(s1) * (s1 + 1) / 2;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const AccT a0 = v[4 * j + 0], a1 = v[4 * j + 1], a2 = v[4 * j + 2], a3 = v[4 * j + 3];
      const AccT v0 = c ? a0 : a2;
      const AccT v1 = c ? a1 : a3;
      const AccT q0 = __shfl_xor_sync(0xffffffffu, v0, 1);
      const AccT q1 = __shfl_xor_sync(0xffffffffu, v1, 1);
      const AccT re = c ? (q0 + a3) : (a0 + q1);
      const AccT im = c ? (a2 - q1) : (q0 - a1);
      const int s2 = bx * (kBN / 4) + piece * 8 + j;
      if (row_ok && s2 <= s1) {
        OutT* o = out + ((krow + s2) * 4 + p1 * 2 + c) * 2;
        if (add) {
          o[0] += re;
          o[1] += im;
        } else if constexpr (IS_INT) {
          *reinterpret_cast<int2*>(o) = make_int2(re, im);
        } else {
          *reinterpret_cast<float2*>(o) = make_float2(re, im);
        }
      }
    }
  } else {
    const int s1 = by * (kBM / 2) + (row >> 1);
    const bool row_ok = s1 < g.N;
    const int64_t krow = static_cast<int64_t>(f) * g.NB + static_cast<int64_t>(s1) * (s1 + 1) / 2;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const AccT a_re = v[2 * j], a_im = v[2 * j + 1];
      const AccT q = __shfl_xor_sync(0xffffffffu, a_im, 1);
      const AccT val = c ? (a_re - q) : (a_re + q);
      const int s2 = bx * (kBN / 2) + piece * 16 + j;
      if (row_ok && s2 <= s1) {
        OutT* o = out + (krow + s2) * 2 + c;
        if (add)
          *o += val;
        else
          *o = val;
      }
    }
  }
}

// ------------------------------------------------------------------ kernel

template <bool IS_INT, int DT>
__global__ void __launch_bounds__(kThreads, 1)
    xengine_kernel(const __grid_constant__ CUtensorMap tmap, const XeParams p) {
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

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(full_bar(s), 1);
      ptx::mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(accf_bar(b), 1);
      ptx::mbar_init(acce_bar(b), kNumEpiWarps);
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

  const ptx::WaitCtl wc{p.timeout_ns, p.status, abort_flag};
  const int nchunks = (p.nkb + p.chunk_kb - 1) / p.chunk_kb;
  const unsigned upc = static_cast<unsigned>(p.units_per_chan);

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      ptx::prefetch_tmap(&tmap);
      int stage = 0;
      uint32_t phase = 0;
      int issued_phase[kStages];
      for (int s = 0; s < kStages; ++s) issued_phase[s] = -1;
      bool ok = true;
      int ready_chan = -1;
      for (long long it = blockIdx.x; ok && it < p.nitems; it += gridDim.x) {
        int f, bx, by;
        item_coords(it, p.ntiles, &f, &bx, &by);
        const int slot = f % p.ring_slots;
        if (f != ready_chan) {
          const unsigned gen = static_cast<unsigned>(f / p.ring_slots);
          if (!wait_counter(p.ready + slot, (gen + 1) * upc, p, abort_flag)) {
            ok = false;
            break;
          }
          fence_proxy_async_global();
          ready_chan = f;
        }
        const bool diag = bx == by;
        for (int kb = 0; kb < p.nkb; ++kb) {
          if (!ptx::wait_bounded(empty_bar(stage), phase ^ 1u, wc)) {
            ok = false;
            break;
          }
          const uint32_t a_dst = sbase + stage * 2 * kOperBytes;
          ptx::mbar_arrive_expect_tx(full_bar(stage), diag ? kOperBytes : 2 * kOperBytes);
          ptx::tma_load_3d(a_dst, &tmap, full_bar(stage), kb * kBK, by * kBM, slot);
          if (!diag)
            ptx::tma_load_3d(a_dst + kOperBytes, &tmap, full_bar(stage), kb * kBK, bx * kBM, slot);
          issued_phase[stage] = static_cast<int>(phase);
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        for (int s = 0; s < kStages; ++s) {
          if (issued_phase[s] < 0) continue;
          const uint64_t t0 = ptx::globaltimer();
          while (!ptx::mbar_try_wait(full_bar(s), static_cast<uint32_t>(issued_phase[s])) &&
                 ptx::globaltimer() - t0 < p.timeout_ns) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t u = 0;
      bool ok = true;
      bool issued_any = false;
      for (long long it = blockIdx.x; ok && it < p.nitems; it += gridDim.x) {
        int f, bx, by;
        item_coords(it, p.ntiles, &f, &bx, &by);
        const bool diag = bx == by;
        for (int ch = 0; ok && ch < nchunks; ++ch) {
          const int kb0 = ch * p.chunk_kb;
          const int kb1 = min(p.nkb, kb0 + p.chunk_kb);
          const uint32_t ab = u & 1u;
          const uint32_t ap = (u >> 1) & 1u;
          if (!ptx::wait_bounded(acce_bar(ab), ap ^ 1u, wc)) {
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t d_tmem = tmem + ab * kBN;
          for (int kb = kb0; kb < kb1; ++kb) {
            if (!ptx::wait_bounded(full_bar(stage), phase, wc)) {
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            const uint32_t a_base = sbase + stage * 2 * kOperBytes;
            const uint32_t b_base = diag ? a_base : a_base + kOperBytes;
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k) {
              ptx::mma_f16_ss(d_tmem, ptx::sw128_kmajor_desc(a_base + k * 32),
                              ptx::sw128_kmajor_desc(b_base + k * 32), kIdesc,
                              (kb > kb0 || k > 0) ? 1u : 0u);
            }
            issued_any = true;
            ptx::mma_commit(empty_bar(stage));
            if (++stage == kStages) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (!ok) break;
          ptx::mma_commit(accf_bar(ab));
          ++u;
        }
        // Every operand K-block of this item has landed: its ring slot has
        // one more block that no longer needs it.
        if (ok) red_release_add(p.done + (f % p.ring_slots), 1u);
      }
      if (!ok && issued_any) {
        ptx::mma_commit(drain_bar);
        const uint64_t t0 = ptx::globaltimer();
        while (!ptx::mbar_try_wait(drain_bar, 0) && ptx::globaltimer() - t0 < p.timeout_ns) {
        }
      }
    }
  } else if (warp < 2 + kNumEpiWarps) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const uint32_t t_row = tmem + (static_cast<uint32_t>(q * 32) << 16);
    uint32_t u = 0;
    bool ok = true;
    for (long long it = blockIdx.x; ok && it < p.nitems; it += gridDim.x) {
      int f, bx, by;
      item_coords(it, p.ntiles, &f, &bx, &by);
      for (int ch = 0; ch < nchunks; ++ch) {
        const uint32_t ab = u & 1u;
        const uint32_t ap = (u >> 1) & 1u;
        const bool got = ptx::wait_bounded(accf_bar(ab), ap, wc);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const bool add = p.accumulate || ch > 0;
#pragma unroll 1
        for (int piece = 0; piece < kBN / 32; ++piece) {
          uint32_t r[32];
          ptx::tmem_ld_32x32b_x32(t_row + ab * kBN + piece * 32, r);
          ptx::tmem_wait_ld();
          if (piece == kBN / 32 - 1) {
            // The accumulator is fully in registers: hand it back to the MMA.
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(acce_bar(ab));
          }
          store_piece<IS_INT>(r, p, f, bx, by, row, lane, piece, add);
        }
        ++u;
      }
    }
  } else {
    // ---------------------------------------------------------- converters
    converter_loop<DT>(p, warp - (2 + kNumEpiWarps), lane, abort_flag);
  }

  // ------------------------------------------------------------- teardown
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, kTmemCols);
  }
}

template <bool IS_INT, int DT>
cudaError_t launch_variant(const CUtensorMap* tmap, const XeParams& p, int grid, cudaStream_t s) {
  auto kern = xengine_kernel<IS_INT, DT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, kSmemBytes, s>>>(*tmap, p);
  return cudaGetLastError();
}

}  // namespace

int xengine_ring_slots(const Geometry& g) {
  const int64_t per = static_cast<int64_t>(g.R) * g.Tp * 2;
  const int64_t target = 32ll << 20;  // keep the ring well inside L2
  int64_t n = target / std::max<int64_t>(per, 1);
  n = std::max<int64_t>(2, std::min<int64_t>(16, n));
  return static_cast<int>(std::min<int64_t>(n, g.F));
}

cudaError_t launch_xengine(const CUtensorMap* tmap, const XeLaunch& L, cudaStream_t s) {
  XeParams p;
  p.g = L.g;
  p.in = L.in;
  p.in_dtype = L.in_dtype;
  p.out = L.out;
  p.accumulate = L.accumulate;
  const int nb = (L.g.R + kBM - 1) / kBM;
  p.ntiles = nb * (nb + 1) / 2;
  p.nitems = static_cast<long long>(p.ntiles) * L.g.F;
  p.nkb = L.g.Tp / kBK;
  p.chunk_kb = L.in_dtype == 0 ? kChunkKB : p.nkb;
  p.ring = static_cast<__half*>(L.ring);
  p.ring_slots = L.ring_slots;
  p.ready = L.counters;
  p.done = L.counters + L.ring_slots;
  p.row_units = (L.g.R + kUnitRows - 1) / kUnitRows;
  p.units_per_chan = p.row_units * (L.g.Tp / kUnitT);
  p.vec4 = (L.g.R % 4 == 0) ? 1 : 0;
  p.timeout_ns = L.timeout_ns;
  p.status = L.status;
  if (p.nitems == 0 || p.nkb == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(L.counters, 0, 2 * sizeof(unsigned) * L.ring_slots, s);
  if (e != cudaSuccess) return e;
  const int grid = static_cast<int>(std::min<long long>(p.nitems, L.grid));
  switch (L.in_dtype) {
    case 0: return launch_variant<true, 0>(tmap, p, grid, s);
    case 1: return launch_variant<false, 1>(tmap, p, grid, s);
    case 2: return launch_variant<false, 2>(tmap, p, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace xc
