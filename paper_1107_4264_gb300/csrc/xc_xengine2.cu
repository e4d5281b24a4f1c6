// xc_xengine2.cu -- fused X-engine on CTA pairs: tcgen05.mma.cta_group::2.
//
// Same computation as xc_xengine.cu (operand formation into the L2 ring,
// lower-triangle blocks of G_f = Y_f Y_f^T, exact 1024-sample chunks for
// 8-bit input, 2x2 complex combine in the epilogue), with a larger block.
//
// Block: 256 x 256 of G_f, computed by the two CTAs of a cluster on two SMs.
// CTA rank k (0 = leader, 1 = peer) stages rows k*128 .. k*128+127 of the
// block's row slab (A half) and of its column slab (B half): 16 KiB each per
// 64-sample K-block.  One thread of the leader issues 256 x 256 x 16 MMAs
// for the pair; each SM's TMEM receives its 128 rows of D (256 fp32
// columns).  Per SM this moves half the operand bytes per flop of a
// 128 x 128 single-CTA block through shared memory and L2.
//
// Diagonal blocks (by == bx): each CTA's A and B halves are the same rows;
// one slab is loaded and used as both operands.  Only the lower station
// triangle is stored; the leader's columns 128..255 of a diagonal block lie
// entirely above the diagonal and are neither read from TMEM nor stored.
//
// Pair hand-offs:
//   full[s]   local TMA completion of stage s (each CTA's producer)
//   pfull[s]  leader only: the peer's relay thread forwards its full[s]
//   empty[s]  both CTAs: the leader's commit, multicast, when the MMAs that
//             read stage s (in both SMs) have completed
//   accf[b]   both CTAs: accumulator b holds a finished chunk (multicast commit)
//   acce[b]   leader only: 8 epilogue warps (4 per CTA) have read accumulator b
// All waits are bounded; a timeout raises the CTA's abort flag and the
// device status word.
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

constexpr int kHalf = 128;  // rows of A and of B staged per CTA
constexpr int kBlk = 256;   // block edge per CTA pair
constexpr int kBK = 64;
constexpr int kStages = 6;
constexpr int kNumEpiWarps = 4;
constexpr int kThreads = 32 * (2 + kNumEpiWarps + kNumConvWarps);
constexpr int kOperBytes = kHalf * kBK * 2;
constexpr int kChunkKB = 16;  // 1024 samples
constexpr uint32_t kTmemCols = 512;  // two 256-column fp32 accumulators
constexpr uint32_t kIdesc = ptx::idesc_f16_f32(kBlk, kBlk);

constexpr int kBarOff = kStages * 2 * kOperBytes;
constexpr int kNumBars = 3 * kStages + 5;
constexpr int kSmemBytes = kBarOff + kNumBars * 8 + 16 + 1024;

// Combine one 32-column piece of this thread's G row into visibilities.
//   s1: station of this thread's row; s2_0: station of the piece's first column.
template <bool IS_INT>
__device__ __forceinline__ void store_piece2(const uint32_t (&r)[32], const XeParams& p, int f,
                                             int s1, int p1, int s2_0, int lane, bool add) {
  using AccT = typename std::conditional<IS_INT, int, float>::type;
  const Geometry& g = p.g;
  AccT* out = static_cast<AccT*>(p.out);
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
  const bool row_ok = s1 < g.N;
  const int64_t krow = static_cast<int64_t>(f) * g.NB + static_cast<int64_t>(s1) * (s1 + 1) / 2;
  if (g.P == 2) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const AccT a0 = v[4 * j + 0], a1 = v[4 * j + 1], a2 = v[4 * j + 2], a3 = v[4 * j + 3];
      const AccT v0 = c ? a0 : a2;
      const AccT v1 = c ? a1 : a3;
      const AccT q0 = __shfl_xor_sync(0xffffffffu, v0, 1);
      const AccT q1 = __shfl_xor_sync(0xffffffffu, v1, 1);
      const AccT re = c ? (q0 + a3) : (a0 + q1);
      const AccT im = c ? (a2 - q1) : (q0 - a1);
      const int s2 = s2_0 + j;
      if (row_ok && s2 <= s1) {
        AccT* o = out + ((krow + s2) * 4 + p1 * 2 + c) * 2;
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
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const AccT a_re = v[2 * j], a_im = v[2 * j + 1];
      const AccT q = __shfl_xor_sync(0xffffffffu, a_im, 1);
      const AccT val = c ? (a_re - q) : (a_re + q);
      const int s2 = s2_0 + j;
      if (row_ok && s2 <= s1) {
        AccT* o = out + (krow + s2) * 2 + c;
        if (add)
          *o += val;
        else
          *o = val;
      }
    }
  }
}

template <bool IS_INT, int DT>
__global__ void __launch_bounds__(kThreads, 1)
    xengine2_kernel(const __grid_constant__ CUtensorMap tmap, const XeParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  const uint32_t sbase = ptx::smem_u32(smem);
  const uint32_t bar0 = sbase + kBarOff;
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto pfull_bar = [&](int s) { return bar0 + 8u * (kStages + s); };
  auto empty_bar = [&](int s) { return bar0 + 8u * (2 * kStages + s); };
  auto accf_bar = [&](int b) { return bar0 + 8u * (3 * kStages + b); };
  auto acce_bar = [&](int b) { return bar0 + 8u * (3 * kStages + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (3 * kStages + 4);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(smem + kBarOff + kNumBars * 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = ptx::cluster_ctarank();
  const bool leader = rank == 0;
  const long long cluster = blockIdx.x >> 1;
  const long long nclusters = gridDim.x >> 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(full_bar(s), 1);
      ptx::mbar_init(pfull_bar(s), 1);
      ptx::mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(accf_bar(b), 1);
      ptx::mbar_init(acce_bar(b), 2 * kNumEpiWarps);
    }
    ptx::mbar_init(drain_bar, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
    ptx::fence_proxy_async_smem();
  }
  if (warp == 1) {
    ptx::tmem_alloc_pair(ptx::smem_u32(tmem_holder), kTmemCols);
    ptx::tmem_relinquish_pair();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::cluster_sync();  // both CTAs' barriers exist before any remote arrive
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  const ptx::WaitCtl wc{p.timeout_ns, p.status, abort_flag};
  const int nchunks = (p.nkb + p.chunk_kb - 1) / p.chunk_kb;
  const unsigned upc = static_cast<unsigned>(p.units_per_chan);
  const int st_per_blk = kBlk / (2 * p.g.P);  // stations per 256-row block
  const int st_per_half = kHalf / (2 * p.g.P);

  if (warp == 0) {
    // ------------------------------------------------------ producer (both)
    if (lane == 0) {
      ptx::prefetch_tmap(&tmap);
      int stage = 0;
      uint32_t phase = 0;
      int issued_phase[kStages];
      for (int s = 0; s < kStages; ++s) issued_phase[s] = -1;
      bool ok = true;
      int ready_chan = -1;
      for (long long it = cluster; ok && it < p.nitems; it += nclusters) {
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
        const int row_a = by * kBlk + static_cast<int>(rank) * kHalf;
        const int row_b = bx * kBlk + static_cast<int>(rank) * kHalf;
        for (int kb = 0; kb < p.nkb; ++kb) {
          if (!ptx::wait_bounded(empty_bar(stage), phase ^ 1u, wc)) {
            ok = false;
            break;
          }
          const uint32_t a_dst = sbase + stage * 2 * kOperBytes;
          ptx::mbar_arrive_expect_tx(full_bar(stage), diag ? kOperBytes : 2 * kOperBytes);
          ptx::tma_load_3d(a_dst, &tmap, full_bar(stage), kb * kBK, row_a, slot);
          if (!diag) ptx::tma_load_3d(a_dst + kOperBytes, &tmap, full_bar(stage), kb * kBK, row_b, slot);
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
    if (lane == 0 && !leader) {
      // ------------------------------------------------------- peer relay
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (long long it = cluster; ok && it < p.nitems; it += nclusters) {
        for (int kb = 0; kb < p.nkb; ++kb) {
          if (!ptx::wait_bounded(full_bar(stage), phase, wc)) {
            ok = false;
            break;
          }
          ptx::mbar_arrive_remote(ptx::mapa_shared(pfull_bar(stage), 0));
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    } else if (lane == 0) {
      // ------------------------------------------------ leader MMA issuer
      int stage = 0;
      uint32_t phase = 0;
      uint32_t u = 0;
      bool ok = true;
      bool issued_any = false;
      for (long long it = cluster; ok && it < p.nitems; it += nclusters) {
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
          const uint32_t d_tmem = tmem + ab * kBlk;
          for (int kb = kb0; kb < kb1; ++kb) {
            if (!ptx::wait_bounded(full_bar(stage), phase, wc) ||
                !ptx::wait_bounded(pfull_bar(stage), phase, wc)) {
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            const uint32_t a_base = sbase + stage * 2 * kOperBytes;
            const uint32_t b_base = diag ? a_base : a_base + kOperBytes;
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k) {
              ptx::mma_f16_ss_pair(d_tmem, ptx::sw128_kmajor_desc(a_base + k * 32),
                                   ptx::sw128_kmajor_desc(b_base + k * 32), kIdesc,
                                   (kb > kb0 || k > 0) ? 1u : 0u);
            }
            issued_any = true;
            ptx::mma_commit_pair_mc(empty_bar(stage), 0x3);
            if (++stage == kStages) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (!ok) break;
          ptx::mma_commit_pair_mc(accf_bar(ab), 0x3);
          ++u;
        }
        // Both CTAs' operand K-blocks of this item have landed.
        if (ok) red_release_add(p.done + (f % p.ring_slots), 1u);
      }
      if (!ok && issued_any) {
        ptx::mma_commit_pair_mc(drain_bar, 0x1);
        const uint64_t t0 = ptx::globaltimer();
        while (!ptx::mbar_try_wait(drain_bar, 0) && ptx::globaltimer() - t0 < p.timeout_ns) {
        }
      }
    }
  } else if (warp < 2 + kNumEpiWarps) {
    // ------------------------------------------------------ epilogue (both)
    const int q = warp & 3;
    const int row = q * 32 + lane;  // row of this CTA's half of the block
    const uint32_t t_row = tmem + (static_cast<uint32_t>(q * 32) << 16);
    const int rpst = 2 * p.g.P;     // G rows per station
    uint32_t u = 0;
    bool ok = true;
    for (long long it = cluster; ok && it < p.nitems; it += nclusters) {
      int f, bx, by;
      item_coords(it, p.ntiles, &f, &bx, &by);
      const int s1_first = by * st_per_blk + static_cast<int>(rank) * st_per_half;
      const int s1 = s1_first + row / rpst;
      const int p1 = (row >> 1) & 1;
      const int s1_hi = min(p.g.N - 1, s1_first + st_per_half - 1);
      const int cols_per_piece_st = 32 / rpst;
      // Pieces 0..last hold columns whose stations can meet the lower triangle.
      int last = -1;
      for (int piece = 0; piece < kBlk / 32; ++piece)
        if (bx * st_per_blk + piece * cols_per_piece_st <= s1_hi) last = piece;
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
        const uint32_t acce_addr = leader ? acce_bar(ab) : ptx::mapa_shared(acce_bar(ab), 0);
        if (last < 0) {
          ptx::tc_fence_before();
          __syncwarp();
          if (lane == 0) {
            if (leader)
              ptx::mbar_arrive(acce_addr);
            else
              ptx::mbar_arrive_remote(acce_addr);
          }
        }
#pragma unroll 1
        for (int piece = 0; piece <= last; ++piece) {
          uint32_t r[32];
          ptx::tmem_ld_32x32b_x32(t_row + ab * kBlk + piece * 32, r);
          ptx::tmem_wait_ld();
          if (piece == last) {
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) {
              if (leader)
                ptx::mbar_arrive(acce_addr);
              else
                ptx::mbar_arrive_remote(acce_addr);
            }
          }
          store_piece2<IS_INT>(r, p, f, s1, p1, bx * st_per_blk + piece * cols_per_piece_st, lane,
                               add);
        }
        ++u;
      }
    }
  } else {
    // ---------------------------------------------------- converters (both)
    converter_loop<DT>(p, warp - (2 + kNumEpiWarps), lane, abort_flag);
  }

  // ------------------------------------------------------------- teardown
  ptx::tc_fence_before();
  __syncthreads();
  ptx::cluster_sync();  // no SM still reads the other's shared memory or TMEM
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc_pair(tmem, kTmemCols);
  }
}

template <bool IS_INT, int DT>
cudaError_t launch_variant(const CUtensorMap* tmap, const XeParams& p, int max_ctas, cudaStream_t s) {
  auto kern = xengine2_kernel<IS_INT, DT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kSmemBytes;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(static_cast<unsigned>(max_ctas & ~1));
  // Every CTA must be resident at once (the operand ring couples them).
  static int resident = -1;
  if (resident < 0) {
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
    if (e != cudaSuccess) return e;
    resident = n;
  }
  long long nclusters = std::min<long long>(resident, max_ctas / 2);
  nclusters = std::min<long long>(nclusters, p.nitems);
  if (nclusters < 1) return cudaErrorInvalidConfiguration;
  cfg.gridDim = dim3(static_cast<unsigned>(2 * nclusters));
  return cudaLaunchKernelEx(&cfg, kern, *tmap, p);
}

}  // namespace

cudaError_t launch_xengine_pair(const CUtensorMap* tmap, const XeLaunch& L, cudaStream_t s) {
  XeParams p;
  p.g = L.g;
  p.in = L.in;
  p.in_dtype = L.in_dtype;
  p.out = L.out;
  p.accumulate = L.accumulate;
  const int nb = (L.g.R + kBlk - 1) / kBlk;
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
  switch (L.in_dtype) {
    case 0: return launch_variant<true, 0>(tmap, p, L.grid, s);
    case 1: return launch_variant<false, 1>(tmap, p, L.grid, s);
    case 2: return launch_variant<false, 2>(tmap, p, L.grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace xc
