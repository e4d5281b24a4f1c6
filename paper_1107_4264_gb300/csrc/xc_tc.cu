// xc_tc.cu -- tensor-core X-engine for sm_103a (tcgen05 + TMEM + TMA).
//
// Per channel f the correlation matrix of Eq. (outer) (Sec. 2.1) is formed
// as the real symmetric product G_f = Y_f Y_f^T of the fp16 operand
// workspace (one row per real input component, r = (s*P + p)*2 + c; one
// column per sample).  The complex visibility of inputs a, b follows from a
// 2x2 block of G:
//     Re V_ab = G[2a][2b] + G[2a+1][2b+1],   Im V_ab = G[2a+1][2b] - G[2a][2b+1].
//
// Work decomposition (Sec. 4.2, re-derived for tensor cores): G_f is tiled
// in 128 x 128 blocks; only blocks on or below the diagonal are computed,
// enumerated with the triangular block map g = by(by+1)/2 + bx.  Tile
// boundaries fall on station boundaries (128 rows = 128/(2P) stations), so
// the block triangle is the station triangle.  Diagonal blocks are computed
// whole and only their lower station triangle is stored (Sec. 4.4); they
// read one operand slab and use it as both MMA operands.
//
// Multi-level tiling (Sec. 2.2 / Sec. 4.1): the accumulator tile lives in
// tensor memory (TMEM), operand K-blocks of 64 samples stream through a
// 6-stage shared-memory ring filled by TMA (the multi-buffer successor of
// the paper's double-buffered shared memory, Sec. 4.4), and only vectors
// (operand rows) ever leave device memory.
//
// CTA roles (persistent, one CTA per SM, work items = (channel, block),
// channel-major so the blocks of a channel run together and share its
// operands through L2):
//   warp 0      TMA producer      (one thread)
//   warp 1      MMA issuer        (one thread; also owns the TMEM allocation)
//   warps 2..5  epilogue          (TMEM -> registers -> visibilities -> HBM)
// Two TMEM accumulators alternate, so the epilogue of one unit overlaps the
// MMAs of the next.
//
// Exact 8-bit path: products of int8 values are exact in fp16 x fp16 -> fp32,
// and every partial sum of an accumulation of at most 1024 samples is an
// integer of magnitude <= 1024 * 128 * 128 = 2^24, hence exact in fp32.  The
// integer engine therefore accumulates 1024-sample chunks in TMEM and drains
// each chunk into int32 registers (one "unit" per chunk).  Float input is
// accumulated in fp32 over the whole integration (one unit per item).
#include <cuda.h>
#include <cuda_fp16.h>

#include "xc_launch.h"
#include "xc_ptx.cuh"

namespace xc {
namespace {

constexpr int kBM = 128;              // tile rows (G rows = operand rows of block by)
constexpr int kBN = 128;              // tile cols (operand rows of block bx)
constexpr int kBK = 64;               // samples per K-block (one 128-byte swizzle atom of fp16)
constexpr int kStages = 6;
constexpr int kThreads = 192;
constexpr int kOperBytes = kBM * kBK * 2;  // 16 KiB per operand per stage
constexpr int kChunkKB = 16;               // 16 x 64 = 1024 samples per exact fp32 chunk
constexpr uint32_t kTmemCols = 256;        // two 128-column fp32 accumulators
constexpr uint32_t kIdesc = ptx::idesc_f16_f32(kBM, kBN);

constexpr int kBarOff = kStages * 2 * kOperBytes;
constexpr int kNumBars = 2 * kStages + 5;
constexpr int kSmemBytes = kBarOff + kNumBars * 8 + 16 + 1024;  // + alignment slack

struct TcParams {
  Geometry g;
  void* out;
  int accumulate;
  int ntiles;       // lower blocks per channel
  long long nitems; // ntiles * F
  int nkb;          // K-blocks per integration (Tp / 64)
  int chunk_kb;     // K-blocks per accumulation unit
  unsigned long long timeout_ns;
  int* status;
};

__device__ __forceinline__ void item_coords(long long it, int ntiles, int* f, int* bx, int* by) {
  *f = static_cast<int>(it / ntiles);
  int64_t x, y;
  tri_coords(it % ntiles, &x, &y);
  *bx = static_cast<int>(x);
  *by = static_cast<int>(y);
}

// Store one finished 128 x 128 block of G as visibilities.
//   acc[j]: G[row][col j] for this thread's row (row = 32*q + lane).
// P = 2: row = 4*s + 2*p1 + c; the thread with c = 0 (re row) and its
// neighbour c = 1 (im row) exchange halves and each writes one pol product
// (p2 = c) {re, im} of every baseline in the block.
// P = 1: row = 2*s + c; thread c writes component c of every baseline.
template <bool IS_INT, typename AccT>
__device__ __forceinline__ void store_block(const AccT (&acc)[kBN], const TcParams& p, int f, int bx,
                                            int by, int row, int lane) {
  const Geometry& g = p.g;
  const int c = lane & 1;
  using OutT = typename std::conditional<IS_INT, int, float>::type;
  OutT* out = static_cast<OutT*>(p.out);
  if (g.P == 2) {
    const int p1 = (row >> 1) & 1;
    const int s1 = by * (kBM / 4) + (row >> 2);
    const bool row_ok = s1 < g.N;
    const int64_t krow = (static_cast<int64_t>(f) * g.NB + static_cast<int64_t>(s1) * (s1 + 1) / 2);
#pragma unroll
    for (int j = 0; j < kBN / 4; ++j) {
      const AccT a0 = acc[4 * j + 0], a1 = acc[4 * j + 1], a2 = acc[4 * j + 2], a3 = acc[4 * j + 3];
      const AccT v0 = c ? a0 : a2;
      const AccT v1 = c ? a1 : a3;
      const AccT r0 = __shfl_xor_sync(0xffffffffu, v0, 1);
      const AccT r1 = __shfl_xor_sync(0xffffffffu, v1, 1);
      const AccT re = c ? (r0 + a3) : (a0 + r1);
      const AccT im = c ? (a2 - r1) : (r0 - a1);
      const int s2 = bx * (kBN / 4) + j;
      if (row_ok && s2 <= s1) {
        OutT* o = out + ((krow + s2) * 4 + p1 * 2 + c) * 2;
        if (p.accumulate) {
          o[0] += re;
          o[1] += im;
        } else {
          if constexpr (IS_INT) {
            *reinterpret_cast<int2*>(o) = make_int2(re, im);
          } else {
            *reinterpret_cast<float2*>(o) = make_float2(re, im);
          }
        }
      }
    }
  } else {
    const int s1 = by * (kBM / 2) + (row >> 1);
    const bool row_ok = s1 < g.N;
    const int64_t krow = (static_cast<int64_t>(f) * g.NB + static_cast<int64_t>(s1) * (s1 + 1) / 2);
#pragma unroll
    for (int j = 0; j < kBN / 2; ++j) {
      const AccT a_re = acc[2 * j + 0], a_im = acc[2 * j + 1];
      const AccT r = __shfl_xor_sync(0xffffffffu, a_im, 1);
      const AccT v = c ? (a_re - r) : (a_re + r);
      const int s2 = bx * (kBN / 2) + j;
      if (row_ok && s2 <= s1) {
        OutT* o = out + (krow + s2) * 2 + c;
        if (p.accumulate) {
          *o += v;
        } else {
          *o = v;
        }
      }
    }
  }
}

template <bool IS_INT>
__global__ void __launch_bounds__(kThreads, 1)
    tc_xengine_kernel(const __grid_constant__ CUtensorMap tmap, const TcParams p) {
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

  const ptx::WaitCtl wc{p.timeout_ns, p.status, abort_flag};
  const int nchunks = (p.nkb + p.chunk_kb - 1) / p.chunk_kb;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      ptx::prefetch_tmap(&tmap);
      int stage = 0;
      uint32_t phase = 0;
      int issued_phase[kStages];
      for (int s = 0; s < kStages; ++s) issued_phase[s] = -1;
      bool ok = true;
      for (long long it = blockIdx.x; ok && it < p.nitems; it += gridDim.x) {
        int f, bx, by;
        item_coords(it, p.ntiles, &f, &bx, &by);
        const bool diag = bx == by;
        for (int kb = 0; kb < p.nkb; ++kb) {
          if (!ptx::wait_bounded(empty_bar(stage), phase ^ 1u, wc)) {
            ok = false;
            break;
          }
          const uint32_t a_dst = sbase + stage * 2 * kOperBytes;
          ptx::mbar_arrive_expect_tx(full_bar(stage), diag ? kOperBytes : 2 * kOperBytes);
          ptx::tma_load_3d(a_dst, &tmap, full_bar(stage), kb * kBK, by * kBM, f);
          if (!diag) ptx::tma_load_3d(a_dst + kOperBytes, &tmap, full_bar(stage), kb * kBK, bx * kBM, f);
          issued_phase[stage] = static_cast<int>(phase);
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        // Let every copy already issued land before the CTA may exit.
        const ptx::WaitCtl drain_wc{p.timeout_ns, p.status, nullptr};
        for (int s = 0; s < kStages; ++s) {
          if (issued_phase[s] < 0) continue;
          const uint64_t t0 = ptx::globaltimer();
          while (!ptx::mbar_try_wait(full_bar(s), static_cast<uint32_t>(issued_phase[s])) &&
                 ptx::globaltimer() - t0 < drain_wc.timeout_ns) {
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
      }
      if (!ok && issued_any) {
        // Wait for the MMAs in flight before TMEM is released.
        ptx::mma_commit(drain_bar);
        const uint64_t t0 = ptx::globaltimer();
        while (!ptx::mbar_try_wait(drain_bar, 0) && ptx::globaltimer() - t0 < p.timeout_ns) {
        }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int row = q * 32 + lane;
    const uint32_t t_row = tmem + (static_cast<uint32_t>(q * 32) << 16);
    uint32_t u = 0;
    bool ok = true;
    for (long long it = blockIdx.x; ok && it < p.nitems; it += gridDim.x) {
      int f, bx, by;
      item_coords(it, p.ntiles, &f, &bx, &by);
      using AccT = typename std::conditional<IS_INT, int, float>::type;
      AccT acc[kBN];
      for (int ch = 0; ch < nchunks; ++ch) {
        const uint32_t ab = u & 1u;
        const uint32_t ap = (u >> 1) & 1u;
        const bool got = ptx::wait_bounded(accf_bar(ab), ap, wc);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        ptx::tc_fence_after();
#pragma unroll
        for (int j = 0; j < kBN / 32; ++j) {
          uint32_t r[32];
          ptx::tmem_ld_32x32b_x32(t_row + ab * kBN + j * 32, r);
          ptx::tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            if constexpr (IS_INT) {
              const int v = __float2int_rn(__uint_as_float(r[i]));
              acc[j * 32 + i] = (ch == 0) ? v : acc[j * 32 + i] + v;
            } else {
              acc[j * 32 + i] = __uint_as_float(r[i]);
            }
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(acce_bar(ab));
        ++u;
      }
      if (!ok) break;
      store_block<IS_INT>(acc, p, f, bx, by, row, lane);
    }
  }

  // ------------------------------------------------------------- teardown
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace

int tc_smem_bytes() { return kSmemBytes; }

cudaError_t launch_tc_xengine(const CUtensorMap* tmap, const TcLaunch& L, cudaStream_t s) {
  TcParams p;
  p.g = L.g;
  p.out = L.out;
  p.accumulate = L.accumulate;
  const int nb = (L.g.R + kBM - 1) / kBM;
  p.ntiles = nb * (nb + 1) / 2;
  p.nitems = static_cast<long long>(p.ntiles) * L.g.F;
  p.nkb = L.g.Tp / kBK;
  p.chunk_kb = L.is_int ? kChunkKB : p.nkb;
  p.timeout_ns = L.timeout_ns;
  p.status = L.status;
  if (p.nitems == 0 || p.nkb == 0) return cudaSuccess;
  const int grid = static_cast<int>(std::min<long long>(p.nitems, L.grid));
  cudaError_t e;
  if (L.is_int) {
    e = cudaFuncSetAttribute(tc_xengine_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmemBytes);
    if (e != cudaSuccess) return e;
    tc_xengine_kernel<true><<<grid, kThreads, kSmemBytes, s>>>(*tmap, p);
  } else {
    e = cudaFuncSetAttribute(tc_xengine_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmemBytes);
    if (e != cudaSuccess) return e;
    tc_xengine_kernel<false><<<grid, kThreads, kSmemBytes, s>>>(*tmap, p);
  }
  return cudaGetLastError();
}

}  // namespace xc
