// xc_small.cu -- tensor-core X-engine for small arrays: 8-bit input with
// W = 2 N P in {16, 32, 64, 128, 256} real rows per channel.
//
// The operation is Eq. (outer) of Sec. 2.1, V_f = sum_t x_f(t) x_f(t)^H per
// channel, lower station triangle only (Sec. 4.2).  Sec. 4.4 computes whole
// diagonal blocks and masks them; Sec. 6.1 raises F to keep a small array
// busy; Sec. 8 leaves small N as future work.  On the planar engine a
// 128 x 128 block holds 128 / n channels of n = N P inputs, and at most
// n / 128 of each MMA pairs inputs of one channel.  This kernel instead
// takes every input as two real rows (re, im: the interleaved order the
// input already has) so that a 128-row operand tile holds m = 128 / (2 n)
// channels at twice that density.  One 128 x 128 MMA per K step (16
// samples; 32 with e4m3 operands), A = B = the tile, gives the real Gram
// matrix G = X X^T of the tile's rows, with channel k's W x W block on the
// diagonal at rows and columns k W .. k W + W - 1.  For inputs a, b with
// real rows (2a, 2a+1), (2b, 2b+1):
//   Re V_ab = G[2a][2b] + G[2a+1][2b+1],  Im V_ab = G[2a+1][2b] - G[2a][2b+1].
// The cross-channel blocks are computed and not read.  (One 128 x W MMA
// per channel would skip them, but a tcgen05.mma costs about as long to
// issue at N = 16 .. 64 as a 128 x 128 one takes to run, so m of them are
// slower than the one full MMA.)  With W = 256 a channel is two tiles
// (inputs 0-63 and 64-127) and two MMAs per step form the lower tile
// blocks: 128 x 128 for G00, 128 x 256 (A = tile 1, B = both tiles) for
// G10 = X1 X0^T and G11 side by side.
//
// No operand ring: a channel's operands are used by one CTA only, so each
// CTA converts its 8-bit input straight into shared-memory operand tiles
// and reads the input once (2 n bytes per channel-sample).  What bounds it
// is that input stream and the shared-memory traffic it shares with the
// conversion and the MMAs' operand reads.
//
// Exactness (Sec. 5's 8-bit input): int8 samples are exact in fp16, their
// products exact in fp32, and a fp32 sum of at most 1024 products of
// magnitude <= 128^2 stays <= 2^24, so each 1024-sample chunk is exact in
// fp32 and chunks add in int32.  With e4m3 operands (opt-in, 4-bit-class
// data) the same holds for |x| <= 16; a larger value sets the range bit of
// the status word.
//
// Roles of a persistent CTA (one per SM, 12 warps; 18 at W = 256):
//   warp 0     TMA producer: [64 samples][m channels][W bytes] int8 boxes;
//   warp 1     TMEM owner and MMA issuer (one thread);
//   warps 2-5  epilogue: TMEM -> V (int32) in the output layout (at
//              W = 256 a second group of four after the converters);
//   warps 6 .. converters: int8 box -> fp16 (or e4m3) tile in the
//              no-swizzle K-major canonical layout, whole stages in turn (a
//              warp pair per stage, one warp per tile, at W = 256).
// Work items are (channel group, segment of T); a CTA takes items in turn.
// When there are too few channel groups to fill the GPU, T is split into
// segments whose results are added to the (pre-zeroed) output with integer
// atomics; integer addition is exact in any order.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "xc.h"
#include "xc_internal.h"
#include "xc_launch.h"
#include "xc_ptx.cuh"

namespace xc {
namespace {

constexpr int kRows = 128;                    // real rows per operand tile
constexpr int kBK = 64;                       // samples per stage
constexpr int kChunk = 1024;                  // samples per exact fp32 chunk
constexpr uint32_t kCore = 128;               // one core matrix: 8 rows x 16 B
constexpr int kConvWarp0 = 6;                 // warps 0 .. 5: producer, MMA, epilogue

// Shapes per channel width W.  W <= 128: kM = 128 / W channels per tile,
// two 128-column accumulator buffers.  W = 256: one channel of two tiles,
// whose three lower 128 x 128 blocks fill 384 TMEM columns (one buffer).
// Converter group gi takes stages gi, gi + kConvGroups, ...; with slot
// counts that are multiples of kConvGroups every input and operand slot
// belongs to one group, which waits on its barriers phase by phase (the two
// warps of a group cannot get a phase apart: a slot's next fill needs both
// of their arrivals).  (A slot shared by two groups lets one of them wait on
// a parity two phases old, which passes too early: mbarrier waits test
// parity, not a phase count.)
template <int W, bool F8>
struct Cfg {
  // Operand tiles: fp16 (8-sample, 16-byte chunks) or, for 4-bit-class
  // 8-bit input, e4m3 (16-sample chunks): [chunk][128 rows][16 B] per stage.
  static constexpr int kTileBytes = kRows * kBK * (F8 ? 1 : 2);   // 16 or 8 KiB
  static constexpr uint32_t kSbo = (kTileBytes / kRows / 16) * kCore;  // between 8-row groups
  static constexpr int kKStep = F8 ? 32 : 16;                     // samples per MMA
  static constexpr int kTiles = W > kRows ? W / kRows : 1;
  static constexpr int kM = W > kRows ? 1 : kRows / W;        // channels per group
  static constexpr int kWt = W > kRows ? kRows : W;           // a channel's rows in one tile
  static constexpr int kBlocks = kTiles * (kTiles + 1) / 2;   // lower tile blocks
  // Converter warps, in groups of kConvPerStage (one warp per tile of a
  // stage); group gi takes stages gi, gi + kConvGroups, ...
  static constexpr int kConvPerStage = kTiles;
  static constexpr int kConvWarps = kTiles == 1 ? 6 : 8;
  static constexpr int kConvGroups = kConvWarps / kConvPerStage;
  // Epilogue warp groups (four warps each, one per TMEM lane quarter): two at
  // W = 256, where the single accumulator's drain holds up the next MMAs.
  static constexpr int kEpiGroups = kTiles == 1 ? 1 : 2;
  static constexpr int kInStages = kTiles == 1 ? 12 : 4;      // int8 boxes in flight
  static constexpr int kOpStages = kTiles == 1 ? 6 : 4;       // operand (tile) slots
  static constexpr int kInBytes = kTiles * kRows * kBK;       // 8 or 16 KiB
  static constexpr int kOpBytes = kTiles * kTileBytes;        // one stage's tiles
  static constexpr int kBufs = kTiles == 1 ? 2 : 1;           // accumulator buffers
  static constexpr int kAccCols = kBlocks * kRows;            // TMEM columns per buffer
  static constexpr uint32_t kTmemCols = kTiles == 1 ? 256 : 512;
  static constexpr int kThreads = 32 * (kConvWarp0 + kConvWarps + 4 * (kEpiGroups - 1));
  static constexpr int kOpOff = 0;
  static constexpr int kInOff = kOpOff + kOpStages * kOpBytes;
  static constexpr int kBarOff = kInOff + kInStages * kInBytes;
  // "Drained" barriers: one per accumulator buffer (W <= 128), or one per
  // tile block of the single accumulator (W = 256), so that the next
  // chunk's MMAs into a block wait only for that block's drain.
  static constexpr int kAcce = kTiles == 1 ? kBufs : kBlocks;
  // in_full, in_empty per input stage; op_full, op_empty per operand stage;
  // accf per accumulator buffer (two reserved); kAcce drained barriers; one
  // drain barrier for the exit.
  static constexpr int kNumBars = 2 * kInStages + 2 * kOpStages + 2 + kAcce + 1;
  static constexpr int kMiscOff = kBarOff + kNumBars * 8;  // TMEM address, abort flag
  static constexpr int kSmemBytes = kMiscOff + 16 + 1024;   // + slack to align the base to 1 KiB
  static_assert(W == 16 || W == 32 || W == 64 || W == 128 || W == 256, "channel widths served");
  static_assert(kInStages % kConvGroups == 0 && kOpStages % kConvGroups == 0,
                "each converter group owns its input and operand slots");
  static_assert(kSmemBytes <= 232448, "shared memory budget");
  static_assert(kBufs * kAccCols <= static_cast<int>(kTmemCols), "TMEM budget");
  // Every epilogue group must load (and then release the accumulator after)
  // at least one 32-column piece of each block.
  static_assert(kEpiGroups <= (kWt >= 32 ? kWt / 32 : 1), "an epilogue group per piece at most");

  __device__ static uint32_t in_full(uint32_t b, int s) { return b + 8u * s; }
  __device__ static uint32_t in_empty(uint32_t b, int s) { return b + 8u * (kInStages + s); }
  __device__ static uint32_t op_full(uint32_t b, int s) { return b + 8u * (2 * kInStages + s); }
  __device__ static uint32_t op_empty(uint32_t b, int s) { return b + 8u * (2 * kInStages + kOpStages + s); }
  __device__ static uint32_t accf(uint32_t b, int ab) { return b + 8u * (2 * kInStages + 2 * kOpStages + ab); }
  __device__ static uint32_t acce(uint32_t b, int i) {
    return b + 8u * (2 * kInStages + 2 * kOpStages + 2 + i);
  }
  __device__ static uint32_t drain(uint32_t b) {
    return b + 8u * (2 * kInStages + 2 * kOpStages + 2 + kAcce);
  }
};

struct SmallParams {
  int P, F, T;
  int ngroups;     // ceil(F / m)
  int nseg;        // segments of T per channel group
  int seg_len;     // samples per segment (a multiple of kChunk)
  int64_t NB;      // baselines N (N + 1) / 2
  int32_t* out;
  int accumulate;  // add into out instead of overwriting it
  int use_red;     // nseg > 1: every chunk is added with atomics (out pre-zeroed)
  int test_no_publish;  // test hook: converted tiles are never marked full
  unsigned long long timeout_ns;
  int* status;
};

// Samples [t0, t1) of work item `it` (channel group it / nseg).
struct Item {
  int g, t0, t1;
};
__device__ __forceinline__ Item item_of(const SmallParams& p, int it) {
  Item x;
  x.g = it / p.nseg;
  const int sg = it % p.nseg;
  x.t0 = sg * p.seg_len;
  x.t1 = min(p.T, x.t0 + p.seg_len);
  return x;
}

// fp16x2 of (byte j of a, byte j of b) as signed 8-bit values: with byte x
// placed under the fp16 pattern 0x6400 (1024) after flipping its sign bit,
// the half is 1152 + x, and subtracting 1152 leaves x exactly.  The selector
// j may differ between lanes.
__device__ __forceinline__ uint32_t i8pair_to_h2(uint32_t a, uint32_t b, uint32_t j) {
  uint32_t d = __byte_perm(a, b, j | ((j + 4u) << 8));
  d = (d & 0x00FF00FFu) ^ 0x64806480u;
  __half2 h = *reinterpret_cast<__half2*>(&d);
  h = __hsub2(h, __half2(__float2half_rn(1152.f), __float2half_rn(1152.f)));
  return *reinterpret_cast<uint32_t*>(&h);
}

// e4m3 bytes of byte j of four consecutive words w[u0 .. u0+3] (four
// samples of one row): the exact fp16 pair conversion above, then one
// fp16x2 -> e4m3x2 conversion per pair (exact for |x| <= 16, saturating).
__device__ __forceinline__ uint32_t i8quad_to_e4m3(const uint32_t (&w)[16], int u0, uint32_t j) {
  const uint32_t h01 = i8pair_to_h2(w[u0], w[u0 + 1], j), h23 = i8pair_to_h2(w[u0 + 2], w[u0 + 3], j);
  __half2_raw r01, r23;
  r01.x = static_cast<unsigned short>(h01 & 0xffffu);
  r01.y = static_cast<unsigned short>(h01 >> 16);
  r23.x = static_cast<unsigned short>(h23 & 0xffffu);
  r23.y = static_cast<unsigned short>(h23 >> 16);
  const uint32_t e01 = __nv_cvt_halfraw2_to_fp8x2(r01, __NV_SATFINITE, __NV_E4M3);
  const uint32_t e23 = __nv_cvt_halfraw2_to_fp8x2(r23, __NV_SATFINITE, __NV_E4M3);
  return (e01 & 0xffffu) | (e23 << 16);
}

__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
               : "memory");
}
__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

// Bounded wait of a whole warp (every lane polls; all give up together).
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, const ptx::WaitCtl& wc) {
  const bool got = ptx::wait_bounded(bar, parity, wc);
  return __all_sync(0xffffffffu, got);
}

// One visibility (int32 re, im; 8-byte aligned): stored (mode 0), read-
// modified-written (mode 1: later chunks of a segment, or accumulate) or
// added with atomics (mode 2: T split into segments).
__device__ __forceinline__ void put_vis(int32_t* dst, int re, int im, int mode) {
  int2* d2 = reinterpret_cast<int2*>(dst);
  if (mode == 0) {
    *d2 = make_int2(re, im);
  } else if (mode == 1) {
    int2 v = *d2;
    v.x += re;
    v.y += im;
    *d2 = v;
  } else {
    atomicAdd(dst, re);
    atomicAdd(dst + 1, im);
  }
}

// W = 2 N P real rows per channel (Cfg holds the shapes); P polarisations
// (a compile-time constant, so the epilogue's station and polarisation
// indices are shifts); F8: e4m3 operands (exact for |x| <= 16; a larger
// value sets the range bit of the status word).
template <int W, int P, bool F8>
__global__ void __launch_bounds__(Cfg<W, F8>::kThreads, 1)
    small_kernel(const __grid_constant__ CUtensorMap in_map, const SmallParams p) {
  static_assert(P == 1 || P == 2, "one or two polarisations");
  using C = Cfg<W, F8>;
  constexpr int kM = C::kM;
  constexpr int kTileBytes = C::kTileBytes;
  constexpr uint32_t kSbo = C::kSbo;
  constexpr int kWt = C::kWt;
  constexpr int kPieces = kWt >= 32 ? kWt / 32 : 1;  // 32-column TMEM loads per block row
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = ptx::smem_u32(smem_raw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  unsigned char* sgen = smem_raw + (sbase - raw);
  const uint32_t bars = sbase + C::kBarOff;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sgen + C::kMiscOff);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sgen + C::kMiscOff + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int items = p.ngroups * p.nseg;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kInStages; ++s) {
      ptx::mbar_init(C::in_full(bars, s), 1);
      ptx::mbar_init(C::in_empty(bars, s), C::kConvPerStage);
    }
    for (int s = 0; s < C::kOpStages; ++s) {
      ptx::mbar_init(C::op_full(bars, s), C::kConvPerStage);
      ptx::mbar_init(C::op_empty(bars, s), 1);
    }
    for (int ab = 0; ab < 2; ++ab) ptx::mbar_init(C::accf(bars, ab), 1);
    for (int i = 0; i < C::kAcce; ++i) ptx::mbar_init(C::acce(bars, i), 4 * C::kEpiGroups);
    ptx::mbar_init(C::drain(bars), 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(ptx::smem_u32(tmem_slot), C::kTmemCols);
    ptx::tmem_relinquish();
  }
  if (warp == 0 && lane == 0) ptx::prefetch_tmap(&in_map);
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const ptx::WaitCtl wc{p.timeout_ns, p.status, abort_flag};

  if (warp == 0) {
    // ---------------------------------------------------------- producer
    if (lane == 0) {
      const uint64_t pol = ptx::l2_policy_evict_first();  // the input streams through once
      int si = 0;
      uint32_t ph = 0;
      long long issued = 0;
      bool ok = true;
      for (int it = blockIdx.x; ok && it < items; it += gridDim.x) {
        const Item x = item_of(p, it);
        for (int t = x.t0; t < x.t1; t += kBK) {
          if (!ptx::wait_bounded(C::in_empty(bars, si), ph ^ 1u, wc)) {
            ok = false;
            break;
          }
          // Past F or T the box is zero-filled; the transaction count is the whole box.
          ptx::mbar_arrive_expect_tx(C::in_full(bars, si), C::kInBytes);
          ptx::tma_load_3d_hint(sbase + C::kInOff + si * C::kInBytes, &in_map, C::in_full(bars, si), 0,
                                x.g * kM, t, pol);
          ++issued;
          if (++si == C::kInStages) {
            si = 0;
            ph ^= 1u;
          }
        }
      }
      // No box may still be landing when the CTA exits (converters that gave
      // up no longer wait for them): wait, bounded, for the last box of every
      // stage.  Issue k used phase k / kInStages of stage k % kInStages.
      for (long long k = max(0LL, issued - C::kInStages); k < issued; ++k) {
        const int s = static_cast<int>(k % C::kInStages);
        const uint32_t par = static_cast<uint32_t>((k / C::kInStages) & 1);
        const uint64_t t0 = ptx::globaltimer();
        while (!ptx::mbar_try_wait(C::in_full(bars, s), par) && ptx::globaltimer() - t0 < p.timeout_ns) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = ptx::idesc_f16_f32(kRows, kRows);
      int so = 0, ab = 0;
      uint32_t oph = 0;
      uint32_t usep = 0;  // bit ab: parity of buffer ab's use count
      bool ok = true;
      for (int it = blockIdx.x; ok && it < items; it += gridDim.x) {
        const Item x = item_of(p, it);
        for (int c0 = x.t0; ok && c0 < x.t1; c0 += kChunk) {
          const int c1 = min(x.t1, c0 + kChunk);
          // The epilogue has read this buffer's previous chunk.  (W = 256:
          // each block's drain is awaited just before the chunk's first
          // MMAs into that block, below.)
          const uint32_t drained = ((usep >> ab) & 1u) ^ 1u;
          if (C::kTiles == 1 && !ptx::wait_bounded(C::acce(bars, ab), drained, wc)) {
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          for (int t = c0; t < c1; t += kBK) {
            if (!ptx::wait_bounded(C::op_full(bars, so), oph, wc)) {
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            const uint32_t stage = sbase + C::kOpOff + so * C::kOpBytes;
            // Row ta of the lower tile triangle: A = tile ta, B = tiles
            // 0 .. ta (contiguous, so one descriptor covers them: N = 128 (ta
            // + 1)), D = blocks (ta, 0) .. (ta, ta), which sit side by side in
            // TMEM; the row's K steps (chunks 2kk, 2kk + 1) in a row.
            // With one tile, A = B = the tile: D holds every channel's block
            // on its diagonal and the epilogue reads only those.
#pragma unroll
            for (int ta = 0; ta < C::kTiles; ++ta) {
              const int blk0 = ta * (ta + 1) / 2;
              if (C::kTiles > 1 && t == c0) {
                for (int b = blk0; b <= blk0 + ta; ++b) {
                  if (!ptx::wait_bounded(C::acce(bars, b), drained, wc)) {
                    ok = false;
                    break;
                  }
                }
                if (!ok) break;
                ptx::tc_fence_after();
              }
              const uint32_t idesc_row = ta == 0 ? idesc : ptx::idesc_f16_f32(kRows, kRows * (ta + 1));
#pragma unroll
              for (int kk = 0; kk < kBK / C::kKStep; ++kk) {
                // K step kk: two 16-byte chunks of every row.
                const uint64_t da =
                    ptx::interleave_kmajor_desc(stage + ta * kTileBytes + kk * 2 * kCore, kCore, kSbo);
                const uint64_t db = ptx::interleave_kmajor_desc(stage + kk * 2 * kCore, kCore, kSbo);
                const uint32_t dcol = tmem + static_cast<uint32_t>(ab * C::kAccCols + blk0 * kRows);
                // (kind::f8f6f4 with e4m3 A and B takes the same descriptor type fields as f16.)
                if constexpr (F8)
                  ptx::mma_f8_ss(dcol, da, db, idesc_row, (t > c0 || kk > 0) ? 1u : 0u);
                else
                  ptx::mma_f16_ss(dcol, da, db, idesc_row, (t > c0 || kk > 0) ? 1u : 0u);
              }
            }
            if (!ok) break;
            ptx::mma_commit(C::op_empty(bars, so));  // the tile may be refilled once read
            if (++so == C::kOpStages) {
              so = 0;
              oph ^= 1u;
            }
          }
          if (!ok) break;
          ptx::mma_commit(C::accf(bars, ab));
          usep ^= 1u << ab;
          ab = (ab + 1) % C::kBufs;
        }
      }
      // Every MMA issued completes before TMEM is freed and the CTA exits.
      ptx::mma_commit(C::drain(bars));
      const uint64_t t0 = ptx::globaltimer();
      while (!ptx::mbar_try_wait(C::drain(bars), 0u) && ptx::globaltimer() - t0 < p.timeout_ns) {
      }
    }
  } else if (warp < kConvWarp0 || warp >= kConvWarp0 + C::kConvWarps) {
    // --------------------------------------------------------- epilogue
    // Warps 2 .. 5 (group 0) and, at W = 256, the warps after the
    // converters (group 1); group eg takes the 32-column pieces pc with
    // pc % kEpiGroups == eg.  Warp w reads TMEM lanes 32 (w % 4) ..: tile
    // row r is TMEM lane r (in every block: block (ta, tb) has the rows of
    // tile ta).
    const int eg = warp < kConvWarp0 ? 0 : 1;
    const int q = warp & 3;
    const int r = 32 * q + lane;
    const int k = r / kWt;          // channel of row r within the tile (W <= 128)
    const int al = (r % kWt) >> 1;  // input of the row within its tile
    const int c = r & 1;            // 0: the row holds re(x_a), 1: im(x_a)
    constexpr int PP = P * P;
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(32 * q) << 16);
    int ab = 0;
    uint32_t usep = 0;  // bit ab: parity of buffer ab's use count
    bool ok = true;
    for (int it = blockIdx.x; ok && it < items; it += gridDim.x) {
      const Item x = item_of(p, it);
      const int ch = x.g * kM + k;
      const bool chan_ok = ch < p.F;
      int32_t* obase = p.out + static_cast<int64_t>(ch) * p.NB * PP * 2;
      for (int c0 = x.t0; c0 < x.t1; c0 += kChunk) {
        if (!warp_wait(C::accf(bars, ab), (usep >> ab) & 1u, wc)) {
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const int mode = p.use_red ? 2 : ((c0 == x.t0 && !p.accumulate) ? 0 : 1);
#pragma unroll 1
        for (int blk = 0; blk < C::kBlocks; ++blk) {
          // Block (ta, tb) of the lower tile triangle (ta >= tb): inputs of
          // tile ta against those of tile tb (64 inputs per tile).
          const int ta = blk == 0 ? 0 : 1, tb = blk == 2 ? 1 : 0;
          const int a = ta * (kRows / 2) + al;  // station a / P, polarisation a % P
          const int s1 = a / P, p1 = a % P;
          // Row s1's records of this channel: baseline s1 (s1 + 1) / 2 + s2,
          // product p1 P + p2, two int32 each.
          int32_t* orow = obase + ((static_cast<int64_t>(s1) * (s1 + 1) / 2) * PP + p1 * P) * 2;
          const bool lower_only = ta == tb;  // diagonal tile blocks keep s2 <= s1
#pragma unroll 1
          for (int pc = eg; pc < kPieces; pc += C::kEpiGroups) {
            uint32_t v[32];
            // Channel k's G columns; with W = 16 the piece holds the warp's two channels.
            const uint32_t col = static_cast<uint32_t>(ab * C::kAccCols + blk * kRows +
                                                       (kWt >= 32 ? k * kWt + 32 * pc : 32 * q));
            ptx::tmem_ld_32x32b_x32(lane_base + col, v);
            ptx::tmem_wait_ld();
            if (pc + C::kEpiGroups >= kPieces && (C::kTiles > 1 || blk == C::kBlocks - 1)) {
              // This warp's last load of the block (W = 256) or of the buffer:
              // the next chunk's MMAs may overwrite it.
              ptx::tc_fence_before();
              __syncwarp();
              if (lane == 0) ptx::mbar_arrive(C::acce(bars, C::kTiles > 1 ? blk : ab));
            }
            constexpr int kJ = kWt >= 32 ? 8 : 4;  // input pairs (2j, 2j + 1) in the piece
            const bool hi = kWt == 16 && lane >= 16;
#pragma unroll
            for (int jj = 0; jj < kJ; ++jj) {
              // Columns 4j .. 4j+3 of the channel block: G[row][2b], G[row][2b+1]
              // for b = 2j (d0, d1) and b = 2j + 1 (d2, d3).
              const float d0 = __uint_as_float(hi ? v[16 + 4 * jj] : v[4 * jj]);
              const float d1 = __uint_as_float(hi ? v[16 + 4 * jj + 1] : v[4 * jj + 1]);
              const float d2 = __uint_as_float(hi ? v[16 + 4 * jj + 2] : v[4 * jj + 2]);
              const float d3 = __uint_as_float(hi ? v[16 + 4 * jj + 3] : v[4 * jj + 3]);
              // This lane produces V(a, b) for b = 2j + c; the partner row (lane ^ 1,
              // same input, other component) sends its two columns for that b.
              const float keep0 = c ? d2 : d0, keep1 = c ? d3 : d1;
              const float send0 = c ? d0 : d2, send1 = c ? d1 : d3;
              const float got0 = __shfl_xor_sync(0xffffffffu, send0, 1);
              const float got1 = __shfl_xor_sync(0xffffffffu, send1, 1);
              const int o0 = __float2int_rn(keep0), o1 = __float2int_rn(keep1);
              const int g0 = __float2int_rn(got0), g1 = __float2int_rn(got1);
              // c = 0: own (rr, ri), partner (ir, ii); c = 1: own (ir, ii), partner (rr, ri).
              const int re = c ? g0 + o1 : o0 + g1;
              const int im = c ? o0 - g1 : g0 - o1;
              const int b = tb * (kRows / 2) + 2 * ((kWt >= 32 ? 8 * pc : 0) + jj) + c;
              const int s2 = b / P, p2 = b % P;
              if (chan_ok && (!lower_only || s2 <= s1)) put_vis(orow + (s2 * PP + p2) * 2, re, im, mode);
            }
          }
        }
        usep ^= 1u << ab;
        ab = (ab + 1) % C::kBufs;
      }
    }
  } else {
    // ------------------------------------------------------- converters
    // The CTA's stages (its items in turn, 64 samples each) are numbered
    // k = 0, 1, ...; converter group gi takes k = gi, gi + kConvGroups, ...
    // (its warps one tile each), so kConvGroups stages are converted at once
    // and each group's latency overlaps the others'.  Stage k uses input slot
    // k % kInStages and operand slot k % kOpStages, in phase k / (slot
    // count).  The box
    // ([64 samples][kTiles x 128 bytes]: byte r of a sample's 128-byte
    // piece t is row r of tile t) becomes the fp16 tiles: lane l reads byte
    // word l (rows 4l .. 4l+3) of each sample and writes one 16-byte
    // core-matrix row per tile row and 8-sample chunk.  Step s writes row
    // 4l + ((s + l / 2) mod 4), so the 8 lanes of each quarter-warp cover
    // the 8 rows of a core matrix, one shared-memory bank group each: the
    // 16-byte stores do not conflict.
    const int cw = warp - kConvWarp0;
    const int cg = cw / C::kConvPerStage;        // converter group: its stages
    const int ctile = cw % C::kConvPerStage;     // this warp's first tile of each stage
    uint32_t jsel[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) jsel[s] = static_cast<uint32_t>((s + (lane >> 1)) & 3);
    // Cursor over the CTA's stages: item `it`, its samples [x.t0, x.t1), stage start t.
    int it = blockIdx.x;
    Item x = item_of(p, it < items ? it : 0);
    int t = x.t0;
    auto advance = [&]() {
      t += kBK;
      if (t >= x.t1) {
        it += gridDim.x;
        if (it < items) {
          x = item_of(p, it);
          t = x.t0;
        }
      }
    };
    for (int s = 0; s < cg && it < items; ++s) advance();
    for (long long k = cg; it < items; k += C::kConvGroups) {
      const int si = static_cast<int>(k % C::kInStages), so = static_cast<int>(k % C::kOpStages);
      const uint32_t iph = static_cast<uint32_t>((k / C::kInStages) & 1);
      const uint32_t oph = static_cast<uint32_t>((k / C::kOpStages) & 1);
      if (!warp_wait(C::in_full(bars, si), iph, wc) || !warp_wait(C::op_empty(bars, so), oph ^ 1u, wc))
        break;
      for (int tl = ctile; tl < C::kTiles; tl += C::kConvPerStage) {
        const uint32_t src = sbase + C::kInOff + si * C::kInBytes + tl * kRows + 4u * lane;
        const uint32_t dst = sbase + C::kOpOff + so * C::kOpBytes + tl * kTileBytes;
        if constexpr (F8) {
          // 16-sample chunks: row j's 16 e4m3 bytes from 16 words.  Bytes
          // with |x| > 16 (not exact in e4m3) set the range bit.
          uint32_t mb = 0;
#pragma unroll 2
          for (int cc = 0; cc < kBK / 16; ++cc) {
            uint32_t w[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              w[u] = lds32(src + static_cast<uint32_t>((16 * cc + u) * C::kTiles * kRows));
              mb = __vmaxu4(mb, __vabs4(w[u]));
            }
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
              const uint32_t j = jsel[qq];
              const uint32_t row = 4u * lane + j;
              sts128(dst + (row >> 3) * kSbo + cc * kCore + (row & 7u) * 16u, i8quad_to_e4m3(w, 0, j),
                     i8quad_to_e4m3(w, 4, j), i8quad_to_e4m3(w, 8, j), i8quad_to_e4m3(w, 12, j));
            }
          }
          if (__vcmpgtu4(mb, 0x10101010u)) atomicOr(p.status, kStatusRange);
        } else {
#pragma unroll 2
          for (int cc = 0; cc < kBK / 8; ++cc) {
            uint32_t w[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
              w[u] = lds32(src + static_cast<uint32_t>((8 * cc + u) * C::kTiles * kRows));
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
              const uint32_t j = jsel[qq];
              const uint32_t row = 4u * lane + j;
              sts128(dst + (row >> 3) * kSbo + cc * kCore + (row & 7u) * 16u, i8pair_to_h2(w[0], w[1], j),
                     i8pair_to_h2(w[2], w[3], j), i8pair_to_h2(w[4], w[5], j), i8pair_to_h2(w[6], w[7], j));
            }
          }
        }
      }
      // The tiles' generic stores before the tensor core's reads; the box's
      // reads are complete (their values were stored).
      ptx::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        ptx::mbar_arrive(C::in_empty(bars, si));
        // (Failure-detection test: without this arrival every MMA wait runs out.)
        if (!p.test_no_publish) ptx::mbar_arrive(C::op_full(bars, so));
      }
      for (int s = 0; s < C::kConvGroups && it < items; ++s) advance();
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, C::kTmemCols);
  }
}

template <int W, int P, bool F8>
cudaError_t launch_wpf(const CUtensorMap* map, const SmallParams& p, int grid, cudaStream_t s) {
  using C = Cfg<W, F8>;
  cudaError_t e =
      cudaFuncSetAttribute(small_kernel<W, P, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
  if (e != cudaSuccess) return e;
  small_kernel<W, P, F8><<<grid, C::kThreads, C::kSmemBytes, s>>>(*map, p);
  return cudaGetLastError();
}

template <int W>
cudaError_t launch_w(const CUtensorMap* map, const SmallParams& p, bool f8, int grid, cudaStream_t s) {
  if (f8) return p.P == 2 ? launch_wpf<W, 2, true>(map, p, grid, s) : launch_wpf<W, 1, true>(map, p, grid, s);
  return p.P == 2 ? launch_wpf<W, 2, false>(map, p, grid, s) : launch_wpf<W, 1, false>(map, p, grid, s);
}

}  // namespace

int small_tile_channels(const Geometry& g) {
  const int W = 2 * g.N * g.P;
  if (W == 256) return 1;
  return (W == 16 || W == 32 || W == 64 || W == 128) ? kRows / W : 0;
}

cudaError_t launch_small(const CUtensorMap* in_map, const XeLaunch& X, cudaStream_t s) {
  const Geometry& g = X.g;
  const int m = small_tile_channels(g);
  if (m == 0 || X.in_dtype != 0 || !in_map) return cudaErrorInvalidValue;
  SmallParams p;
  p.P = g.P;
  p.F = g.F;
  p.T = g.T;
  p.NB = g.NB;
  p.ngroups = (g.F + m - 1) / m;
  // Split T only when the channel groups alone leave SMs idle.
  const int nchunks = (g.T + kChunk - 1) / kChunk;
  int nseg = 1;
  if (p.ngroups < 2 * X.grid) nseg = std::min(nchunks, (2 * X.grid + p.ngroups - 1) / p.ngroups);
  p.seg_len = (nchunks + nseg - 1) / nseg * kChunk;
  p.nseg = (g.T + p.seg_len - 1) / p.seg_len;
  p.out = static_cast<int32_t*>(X.out);
  p.accumulate = X.accumulate;
  p.use_red = p.nseg > 1 ? 1 : 0;
  p.test_no_publish = X.test_no_publish;
  p.timeout_ns = X.timeout_ns;
  p.status = X.status;
  if (p.use_red && !X.accumulate) {
    const size_t bytes = static_cast<size_t>(g.F) * static_cast<size_t>(g.NB) * g.P * g.P * 8;
    const cudaError_t e = cudaMemsetAsync(X.out, 0, bytes, s);
    if (e != cudaSuccess) return e;
  }
  const int items = p.ngroups * p.nseg;
  const int grid = std::max(1, std::min(X.grid, items));
  const bool f8 = X.fmt == 2;  // e4m3 operands (XC_PREC_FP8)
  switch (2 * g.N * g.P) {
    case 16: return launch_w<16>(in_map, p, f8, grid, s);
    case 32: return launch_w<32>(in_map, p, f8, grid, s);
    case 64: return launch_w<64>(in_map, p, f8, grid, s);
    case 128: return launch_w<128>(in_map, p, f8, grid, s);
    default: return launch_w<256>(in_map, p, f8, grid, s);
  }
}

}  // namespace xc
