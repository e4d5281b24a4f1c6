#pragma once
// xc_planar_kernel.cuh -- fused persistent tensor-core X-engine, planar
// complex form: the kernel template, shared by the translation units that
// instantiate its single-CTA (xc_planar.cu) and CTA-pair (xc_planar_pair.cu)
// variants.
//
// Eq. (outer) of Sec. 2.1 per channel f: V_f = sum_t x_f(t) x_f(t)^H over
// n = N*P complex inputs.  With the real and imaginary parts of the inputs
// as separate fp16 operand planes Xr, Xi (n rows x T samples, K-major),
//
//     Re V = Xr Xr^T + Xi Xi^T,      Im V = Xi Xr^T - Xr Xi^T,
//
// so a 128 x 128 block of V (rows a, columns b) is four tcgen05 MMAs per
// 16-sample step into two TMEM accumulators,
//     D_re += Ar Br^T,  D_re += Ai Bi^T,  D_im += Ai Br^T,  D_im += Ar (-Bi)^T,
// the last with the instruction descriptor's negate-B bit.  Four operand
// tiles feed 4 MMAs (half the shared-memory and L2 bytes per MAC of the
// interleaved real form) and every TMEM column is a finished visibility
// component: the epilogue converts and stores, with no lane exchange.
//
// Exact 8-bit input: int8 is exact in fp16, products are exact in fp32, and
// every partial sum of an accumulator is an integer bounded by the sum of
// |products| so far: at most 2 m^2 per sample, m = max |x| of the channel.
// The converters record m per channel; a chunk of S samples with
// 2 m^2 S <= 2^24 is exact in fp32 in any summation order (S >= 512 for any
// int8 data, the whole integration for typical 4-6 bit signal levels).  Each
// chunk is drained into int32 and added into the output (stored for the
// first chunk).  Float input accumulates in fp32 over the whole integration.
//
// Float input (Sec. 5 leaves its precision open): each (channel, input) gets
// a power-of-two scale 2^e from a pre-pass over the integration (max
// component of g x), so y 2^-e spans the operand format's range and the
// epilogue multiplies by 2^(e_a + e_b) exactly.  Three operand formats:
//   FP16   one fp16 plane pair, 4 MMAs per 16 samples;
//   HI/LO  y 2^-e = h + l with h = fp16(.) and l = fp16(. - h); the ring
//          holds H and L tiles and each 64-sample block runs three steps
//          (H H^T, L H^T, H L^T; the l l^T term is dropped), 3x the MMAs;
//   FP8    e4m3 planes (kind::f8f6f4, K = 32), half the operand bytes.
// Optionally (FP64 block sums) the fp32 accumulator is drained every
// T_blk samples into a float64 running sum; the output is its rounding.
//
// Blocks (Sec. 4.2): 128 x 128 blocks of V on or below the block diagonal,
// g = by(by+1)/2 + bx; block edges fall on station boundaries (128 inputs =
// 128/P stations).  Diagonal blocks load one pair of planes for both
// operands and store only their lower station triangle (Sec. 4.4).
//
// Operand formation (Sec. 4.1 input order, Sec. 5 8-bit samples): converter
// warps form each channel's planes once into a ring of channel slots in
// global memory that stays in L2; the blocks of a channel read it back with
// bulk copies.  The ring holds operand tiles exactly as the MMA reads them:
// per (slot, plane, 64-sample K-block, 128-input block) one 16 KiB tile in
// the no-swizzle K-major canonical layout, K inside: [8-input group]
// [8-sample chunk][8 inputs][16 B], so a stage is contiguous tile copies,
// inputs 0..63 and 64..127 of a tile are its two contiguous halves, and the
// 8 x 16 B core matrix that four converter lanes write is one whole line.
// 8-bit input arrives by TMA in 128-row x 64-sample boxes (other types and
// row counts by direct loads); lane l converts inputs l and l + 32 of a
// 64-input half block; each converter warp works through its own stream of
// units.  Ring protocol:
//   ready[slot] counts converted units (128 rows x 64 samples); channel c
//     (generation c / slots of slot c % slots) is complete at
//     ready >= (gen + 1) * units_per_channel;
//   done[slot] counts blocks whose operands have landed in shared memory;
//     slot s may take channel c once done >= gen(c) * blocks_per_channel.
// Dependencies point only to lower channels and all CTAs are co-resident,
// so the ring cannot deadlock; every wait is bounded regardless.
//
// CTA roles (persistent, one CTA per SM, channel-major items):
//   warp 0      producer: 3 stages x (Ar, Ai, Br, Bi) 64-sample tiles (bulk copies)
//   warp 1      MMA issuer; owns TMEM (2 sets x {D_re, D_im} x 128 columns)
//   warps 2..5  epilogue
//   warps 6..9  converters
//
// CTA pairs (PAIR = true, tcgen05 cta_group::2, clusters of two CTAs): one
// item is two 128 x 128 blocks sharing their column block b, computed by one
// 256 x 128 MMA per step over the pair.  CTA k stages the 128 rows of its
// own row block a_k (Ar, Ai tiles) and inputs 64k .. 64k + 63 of block b (the
// k-th halves of the Br, Bi tiles); the leader (rank 0) issues the MMAs, each
// SM's TMEM receives its row block's D_re, D_im.  Per SM the shared-memory
// operand reads per MAC drop by a quarter (A plus half of B per 128 x 128
// product instead of A plus B) and B is staged once for two blocks.
// Pairing (pair_coords): in column block c the blocks of rows c, c+1, ...
// pair off from the diagonal down; the odd one out of a column, (nib-1, c),
// is taken transposed, as rows c times columns nib-1 (its mirror, V[c][nib-1]
// = conj(V[nib-1][c])^T), so the leftovers of all columns share column block
// nib-1 and pair among themselves: ceil(blocks / 2) items per channel, at
// most one CTA of one item idle.  A transposed block is stored as its mirror.
// Hand-offs between the two CTAs:
//   full[s]   local completion of stage s's copies (each CTA)
//   pfull[s]  leader: the peer's relay thread forwards its full[s]
//   empty[s]  both: the leader's commit, multicast, once the MMAs reading
//             stage s in both SMs have completed
//   accf[b]   both: accumulator b holds a finished group (multicast commit)
//   acce[b]   leader: 8 epilogue warps (4 per CTA) have read accumulator b
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "xc_launch.h"
#include "xc_ptx.cuh"

namespace xc {
namespace {

constexpr int kBlk = 128;      // complex inputs per block side
constexpr int kBK = 64;        // samples per stage
constexpr int kNumEpiWarps = 4;
constexpr int kNumConvWarps = 4;
constexpr int kThreads = 32 * (2 + kNumEpiWarps + kNumConvWarps);
constexpr int kTileBytes = kBlk * kBK * 2;  // 16 KiB: one plane tile
constexpr uint32_t kTmemCols = 512;         // 2 sets x (D_re, D_im) x 128
constexpr int kUnitRows = 128;  // converter unit: 128 real rows (64 inputs) x kUnitT samples
constexpr int kUnitT = kPlanarUnitT;
static_assert(kUnitT == 32 || kUnitT == 64, "a unit covers a whole or half 64-sample K-block");
constexpr uint32_t kCoreBytes = 8 * 16;  // one core matrix: 8 inputs x 16 bytes
constexpr int kConvBufBytes = kUnitRows * kUnitT;  // int8 staging per converter warp

// Tile shapes (XC_TILE_*): 128 x 128 blocks on single CTAs; two blocks
// sharing a column block on a CTA pair (256 x 128 MMAs, cta_group::2); two
// blocks sharing a row block on one CTA (128 x 256 MMAs).
enum : int { kShape128 = 0, kShapePair = 1, kShapeWide = 2 };

enum : int { kFmtF16 = 0, kFmtHiLo = 1, kFmtF8 = 2 };

// The stage plan of 8-bit input on e4m3 operands, whose conversion costs the
// most per byte while its MMAs take half the time: half-size stages, and six
// converter warps instead of four (float input keeps the fp16 plan: its
// converters gain nothing from more warps and spill more registers).
template <int FMT, int DT>
constexpr bool f8_int8_plan() {
  return FMT == kFmtF8 && DT == 0;
}
template <int FMT, int DT>
constexpr int conv_warps() {
  return f8_int8_plan<FMT, DT>() ? 6 : kNumConvWarps;
}
template <int FMT, int DT>
constexpr int threads_of() {
  return 32 * (2 + kNumEpiWarps + conv_warps<FMT, DT>());
}

// Shared-memory plan per shape and operand format: stages of (Ar, Ai, Br,
// Bi) tiles; (Ar, Ai, half Br, half Bi) on pairs; (Ar, Ai, Br Br', Bi Bi')
// for 128 x 256; then the converters' staging buffers and the barriers.
// e4m3 tiles are half the size of fp16 ones: for 8-bit input, more stages
// and two more converter warps fit in the same bytes.
template <int SHAPE, int FMT, int DT>
struct Cfg {
  static constexpr bool kF8 = f8_int8_plan<FMT, DT>();
  static constexpr int kStages = kF8 ? (SHAPE == kShapePair ? 7 : (SHAPE == kShapeWide ? 3 : 5))
                                     : (SHAPE == kShapePair ? 4 : (SHAPE == kShapeWide ? 2 : 3));
  static constexpr int kStageBytes =
      (SHAPE == kShapePair ? 3 : (SHAPE == kShapeWide ? 6 : 4)) * (kF8 ? kTileBytes / 2 : kTileBytes);
  static constexpr int kConvOff = kStages * kStageBytes;
  static constexpr int kBarOff = kConvOff + conv_warps<FMT, DT>() * kConvBufBytes;
  // full, empty (and pfull) per stage; accf, acce x 2; drain; one per converter
  static constexpr int kNumBars = (SHAPE == kShapePair ? 3 : 2) * kStages + 5 + conv_warps<FMT, DT>();
  // then the TMEM address, the abort flag and one word per stage (the chunk
  // length of the item whose first step the stage holds)
  static constexpr int kSmemBytes = kBarOff + kNumBars * 8 + 8 + 4 * kStages + 1024;
  static_assert(kSmemBytes <= 232448, "shared memory budget");
};

// Operand formats: tile size (log2 bytes), 16-byte K chunks per tile and
// MMA steps per 64-sample block (ring K-tiles per block: fmt_kt()).
template <int FMT>
struct FmtT {
  static constexpr int kTileShift = FMT == kFmtF8 ? 13 : 14;
  static constexpr int kTile = 1 << kTileShift;
  static constexpr int kChunks = FMT == kFmtF8 ? 4 : 8;
  static constexpr int kSteps = FMT == kFmtHiLo ? 3 : 1;
  // Bytes between 8-input groups of a tile (the descriptor's stride offset);
  // core matrices adjacent in K are kCoreBytes apart (its leading offset).
  static constexpr uint32_t kSbo = kChunks * kCoreBytes;
};

// Byte offset of (input row, 16-byte K chunk) in a tile.
template <int FMT>
__device__ __forceinline__ uint32_t tile_off(int row, int chunk) {
  return static_cast<uint32_t>(row >> 3) * FmtT<FMT>::kSbo + static_cast<uint32_t>(chunk) * kCoreBytes +
         static_cast<uint32_t>(row & 7) * 16u;
}

struct Params {
  Geometry g;
  int n;               // complex inputs per channel = N * P
  const void* in;
  void* out;
  int accumulate;
  int ntiles;          // lower blocks per channel
  int ipc;             // work items per channel: ntiles, or pair items (CTA pairs)
  long long nitems;    // ipc * F
  int nkb;             // Tp / 64
  int is_int;          // 8-bit input: exact chunks from the channel's max |x|
  unsigned* amax;      // [F] max |x| per channel (8-bit input), zeroed by the host
  const float2* gains; // [n] complex gains applied to float input (y = g x), or NULL
  const unsigned* in_amax;  // [F][n] max component of g x (float bits), float input
  double* acc64;       // FP64 block sums: running visibility sums (output layout), or NULL
  int f_chunk_kb;      // float input: K-blocks per fp32 accumulation chunk
  uint8_t* ring;       // tiles [slots][2][nkt][nib][chunks][128][16 B]
  int nkt;             // K-tiles per plane per input block of a slot (nkb or 2 nkb)
  int nib;             // 128-input blocks per channel
  int ring_slots;
  unsigned* ready;
  unsigned* done;
  int row_units;       // 64-input half blocks per channel = 2 * nib
  int units_per_chan;  // row_units * Tp / 64
  int tma_in;          // 8-bit input staged by TMA (else direct loads)
  unsigned long long timeout_ns;
  int* status;
  int test_no_publish;  // test hook: converted units are never published
  // Small arrays: `pack` consecutive channels form one virtual channel of
  // pack * Nr stations (g, n, F above are the virtual geometry; the input
  // [T][F][n] is the same memory as [T][F / pack][pack * n]).  The epilogue
  // keeps only each real channel's own block and stores it at real indices.
  int pack;
  int Nr;              // real stations per channel
  int64_t NBr;         // real baselines per channel
  int gain_n;          // real inputs per channel (gains are indexed a mod gain_n)
};

// One launch over up to kMaxSub subarrays (Sec. 4.2's channel-major raster
// extended across subarrays): items and converter units are numbered
// subarray by subarray; item_base / unit_base are their prefix sums.  Each
// subarray has its own ring region and counters.
struct Batch {
  CUtensorMap maps[kMaxSub];  // 8-bit input of each subarray (read when tma_in)
  Params sub[kMaxSub];
  long long item_base[kMaxSub + 1];
  long long unit_base[kMaxSub + 1];
  int nsub;
};
static_assert(sizeof(Batch) <= kBatchArgBytes && alignof(Batch) <= 128, "batch parameter block");

// Subarray holding global index i, starting the search at cursor s (every
// role walks its items and units in increasing order).  Single-subarray
// launches (MULTI = false) index subarray 0 at compile time.
// End of a prefix-sum table (compile-time index for single launches).
template <bool MULTI>
__device__ __forceinline__ long long table_end(const long long* base, int nsub) {
  if constexpr (!MULTI) {
    return base[1];
  } else {
    return base[nsub];
  }
}

template <bool MULTI>
__device__ __forceinline__ int advance_sub(const long long* base, int nsub, long long i, int s) {
  if constexpr (!MULTI) {
    return 0;
  } else {
    while (s + 1 < nsub && i >= base[s + 1]) ++s;
    return s;
  }
}

// ------------------------------------------------------------ global sync

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __noinline__ bool wait_counter(const unsigned* p, unsigned target, const Params& prm,
                                          volatile int* abort_flag) {
  if (ld_acquire(p) >= target) return true;
  const uint64_t t0 = ptx::globaltimer();
  for (uint32_t it = 1;; ++it) {
    __nanosleep(64);
    if (ld_acquire(p) >= target) return true;
    if ((it & 15u) == 0) {
      if (*abort_flag) return false;
      if (*reinterpret_cast<volatile int*>(prm.status) != 0) {
        *abort_flag = 1;
        return false;
      }
      if (ptx::globaltimer() - t0 > prm.timeout_ns) {
        *abort_flag = 1;
        atomicOr(prm.status, kStatusTimeout);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void item_coords(long long it, int ntiles, int* f, int* bx, int* by) {
  *f = static_cast<int>(it / ntiles);
  int64_t x, y;
  tri_coords(it % ntiles, &x, &y);
  *bx = static_cast<int>(x);
  *by = static_cast<int>(y);
}

// This CTA's share of work item `it` (local to its subarray): channel f,
// row block a and column block b (128 x 256 items: column blocks b and b2,
// b2 = -1 when the item holds one block); idle: the second CTA of a
// one-block pair item.  A block with a column block above its row block
// (b > a) is computed as is and stored as its mirror.
struct Blk {
  int f, a, b, b2;
  bool idle;
};
template <int SHAPE>
__device__ __forceinline__ Blk item_block(const Params& p, long long it, uint32_t rank) {
  Blk k;
  k.b2 = -1;
  k.idle = false;
  if constexpr (SHAPE == kShape128) {
    int bx, by;
    item_coords(it, p.ntiles, &k.f, &bx, &by);
    k.a = by;
    k.b = bx;
    (void)rank;
  } else {
    k.f = static_cast<int>(it / p.ipc);
    int a0, a1, b, single;
    pair_coords(static_cast<int>(it % p.ipc), p.nib, &a0, &a1, &b, &single);
    if constexpr (SHAPE == kShapePair) {
      k.a = rank ? a1 : a0;
      k.b = b;
      k.idle = rank && single;
    } else {
      // The pair schedule transposed: the common block is the row block;
      // the column blocks ascend, so a ragged last block comes second.
      (void)rank;
      k.a = b;
      k.b = single ? a0 : min(a0, a1);
      k.b2 = single ? -1 : max(a0, a1);
    }
  }
  return k;
}

// K-blocks per exact fp32 accumulation chunk for channel f (all K-blocks for
// float input).  Called after the channel is known to be fully converted.
__device__ __forceinline__ int chunk_kblocks(const Params& p, int f) {
  if (!p.is_int) return p.f_chunk_kb;
  const unsigned m = *reinterpret_cast<volatile const unsigned*>(p.amax + f);
  if (m == 0) return p.nkb;
  const unsigned long long per_block = 2ull * m * m * kBK;  // |partial| growth per K-block
  const unsigned long long kb = (1ull << 24) / per_block;
  return static_cast<int>(kb < 1 ? 1 : (kb > static_cast<unsigned long long>(p.nkb) ? p.nkb : kb));
}

// Wait (bounded) until channel f is fully converted into its ring slot.
__device__ __forceinline__ bool channel_ready(const Params& p, int f, volatile int* abort_flag) {
  const unsigned gen = static_cast<unsigned>(f / p.ring_slots);
  return wait_counter(p.ready + f % p.ring_slots, (gen + 1) * static_cast<unsigned>(p.units_per_chan),
                      p, abort_flag);
}

// -------------------------------------------------------------- converter

// fp16x2 of (component j of sample a, component j of sample b), 8-bit input.
__device__ __forceinline__ uint32_t pair_i8(uint32_t a, uint32_t b, uint32_t j) {
  // Byte j of a into byte 0 and byte j of b into byte 2; 0x6400 | (x ^ 0x80)
  // is the fp16 value 1152 + x, so subtracting 1152 gives x exactly.
  uint32_t d = __byte_perm(a, b, j | ((j + 4u) << 8));
  d = (d & 0x00FF00FFu) ^ 0x64806480u;
  __half2 h = *reinterpret_cast<__half2*>(&d);
  h = __hsub2(h, __half2(__float2half_rn(1152.f), __float2half_rn(1152.f)));
  return *reinterpret_cast<uint32_t*>(&h);
}

// Byte address of tile (slot, plane, K-tile kt, ib) in the ring.
template <int FMT>
__device__ __forceinline__ uint8_t* ring_tile(const Params& p, int slot, int plane, int kt, int ib) {
  return p.ring + ((((static_cast<int64_t>(slot) * 2 + plane) * p.nkt + kt) * p.nib + ib)
                   << FmtT<FMT>::kTileShift);
}

// Power-of-two scale exponent e for an input whose largest component is
// `bits` (fp32 bits): max |y| 2^-e lies in [2^14, 2^15) for the fp16 forms
// and in (2^7, 448] for e4m3.  Zero or subnormal maxima are not scaled;
// e is clamped to [-60, 60] so that 2^(e_a + e_b) is a normal float.
template <int FMT>
__device__ __forceinline__ int scale_exp(unsigned bits) {
  const int E = static_cast<int>((bits >> 23) & 0xffu);
  if (E == 0) return 0;
  int e = E - 127 - (FMT == kFmtF8 ? 8 : 14);
  if (FMT == kFmtF8 && (bits & 0x7fffffu) > 0x600000u) ++e;  // 256 (1 + m) > 448
  return max(-60, min(60, e));
}
__device__ __forceinline__ float exp2i(int e) { return __int_as_float((127 + e) << 23); }

// A unit: 64 inputs (half block hb) x kUnitT samples (unit ku along K) of
// channel c, units numbered channel-major with K fastest; it fills 8-sample
// chunks cbase .. cbase + kUnitT/8 - 1 of the tiles of K-block kb.
struct Unit {
  int c, slot, hb, ku, kb, cbase;
};

__device__ __forceinline__ Unit unit_of(const Params& p, long long u) {
  Unit x;
  x.c = static_cast<int>(u / p.units_per_chan);
  const int w = static_cast<int>(u % p.units_per_chan);
  x.slot = x.c % p.ring_slots;
  const int nku = p.nkb * (kBK / kUnitT);
  x.hb = w / nku;
  x.ku = w % nku;
  x.kb = x.ku * kUnitT / kBK;
  x.cbase = (x.ku * kUnitT % kBK) / 8;
  return x;
}

// Before a warp first writes channel c into its slot: the slot's previous
// channel (c - ring_slots) must have been read by all of its blocks.
__device__ __forceinline__ bool claim_slot_warp(const Params& p, int c, int lane,
                                                volatile int* abort_flag) {
  const unsigned gen = static_cast<unsigned>(c / p.ring_slots);
  bool ok = true;
  if (gen > 0 && lane == 0)
    ok = wait_counter(p.done + (c % p.ring_slots), gen * static_cast<unsigned>(p.ipc), p, abort_flag);
  // No proxy fence here: every bulk read of the slot's previous channel has
  // completed (its data sat in shared memory before the MMA thread released
  // done[slot]), so the generic writes that follow cannot reach it.
  return __all_sync(0xffffffffu, ok);
}

// Would a claim of channel c's slot have to wait for the slot's previous
// channel?  (Checked before a warp waits while it holds an unpublished unit.)
__device__ __forceinline__ bool slot_busy(const Params& p, int c, int lane) {
  const unsigned gen = static_cast<unsigned>(c / p.ring_slots);
  bool busy = false;
  if (gen > 0 && lane == 0)
    busy = ld_acquire(p.done + (c % p.ring_slots)) < gen * static_cast<unsigned>(p.ipc);
  return __any_sync(0xffffffffu, busy);
}

// Publish one converted unit: every writing lane orders its generic stores
// before later async-proxy (bulk copy) reads, then one release.
__device__ __forceinline__ void publish_unit(const Params& p, int slot, int lane, unsigned n = 1) {
  if (p.test_no_publish) {  // failure-detection test: every consumer wait runs out
    __syncwarp();
    return;
  }
  fence_proxy_async_global();
  __syncwarp();
  if (lane == 0) red_release_add(p.ready + slot, n);
}

// Converter warps take their units in runs of kUnitRun consecutive units
// (the same channel except at channel ends): one slot claim and one publish
// (fence + release of the whole count) per run instead of per unit.  Warp gw
// of nw takes runs gw, gw + nw, gw + 2 nw, ... of the global unit list.
constexpr int kUnitRun = 2;
__device__ __forceinline__ long long first_unit(long long gw) { return gw * kUnitRun; }
__device__ __forceinline__ long long next_unit(long long u, long long nw) {
  return (u % kUnitRun != kUnitRun - 1) ? u + 1 : u + 1 + (nw - 1) * kUnitRun;
}

// Complex sample (re, im) of input a at sample t, channel c, as fp32.
template <int DT>
__device__ __forceinline__ float2 load_cx(const Params& p, int c, int a, int t) {
  const int64_t idx = (static_cast<int64_t>(t) * p.g.F + c) * p.n + a;
  if constexpr (DT == 0) {
    const char2 v = static_cast<const char2*>(p.in)[idx];
    return make_float2(static_cast<float>(v.x), static_cast<float>(v.y));
  } else if constexpr (DT == 1) {
    return __half22float2(static_cast<const __half2*>(p.in)[idx]);
  } else {
    return static_cast<const float2*>(p.in)[idx];
  }
}

// fp16x2 bits of (a, b).
__device__ __forceinline__ uint32_t h2bits(float a, float b) {
  __half2 q = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&q);
}
// fp16x2 bits of the residuals (a - fp16(a), b - fp16(b)) given h = fp16x2(a, b).
__device__ __forceinline__ uint32_t lo2bits(float a, float b, uint32_t h) {
  const __half2 hh = *reinterpret_cast<const __half2*>(&h);
  return h2bits(a - __low2float(hh), b - __high2float(hh));
}
// Four e4m3 bytes (a, b, c, d), a in the low byte, rounded to nearest with
// saturation to +-448.
__device__ __forceinline__ uint32_t e4m3x4(float a, float b, float c, float d) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
  return (lo & 0xffffu) | (hi << 16);
}

// Direct-load converter (any input type and row count), independent warps:
// lane l loads the complex samples of inputs l and l + 32 of the half block,
// 16 samples (32 loads) in flight at a time, applies the gains and the
// input's power-of-two scale (float input) and writes 16-byte chunks: per
// (input, plane) two fp16 chunks (8 samples each; HI/LO: two more into the
// L tile) or one e4m3 chunk (16 samples).
template <int DT, int FMT, bool MULTI>
__device__ void converter_direct(const Batch& bt, int cw, int lane, volatile int* abort_flag) {
  const long long total = table_end<MULTI>(bt.unit_base, bt.nsub);
  const long long stride = static_cast<long long>(gridDim.x) * conv_warps<FMT, DT>();
  int sb = 0, claimed = -1, claimed_sb = -1;
  for (long long u = static_cast<long long>(blockIdx.x) * conv_warps<FMT, DT>() + cw; u < total; u += stride) {
    sb = advance_sub<MULTI>(bt.unit_base, bt.nsub, u, sb);
    const Params& p = bt.sub[sb];
    const Unit x = unit_of(p, u - bt.unit_base[sb]);
    if (x.c != claimed || sb != claimed_sb) {
      if (!claim_slot_warp(p, x.c, lane, abort_flag)) return;
      claimed = x.c;
      claimed_sb = sb;
    }
    const int ib = x.hb >> 1;
    uint8_t* tre = ring_tile<FMT>(p, x.slot, 0, x.kb, ib);
    uint8_t* tim = ring_tile<FMT>(p, x.slot, 1, x.kb, ib);
    const int a0 = x.hb * 64 + lane, a1 = a0 + 32;
    const int row0 = (x.hb & 1) * 64 + lane;
    // y = g x 2^-e (float input; gains are not defined for 8-bit input).
    float2 g0 = make_float2(1.f, 0.f), g1 = make_float2(1.f, 0.f);
    if (DT != 0) {
      if (p.gains) {
        g0 = a0 < p.n ? p.gains[a0 % p.gain_n] : make_float2(0.f, 0.f);
        g1 = a1 < p.n ? p.gains[a1 % p.gain_n] : make_float2(0.f, 0.f);
      }
      if (p.in_amax) {
        const unsigned* am = p.in_amax + static_cast<int64_t>(x.c) * p.n;
        const float s0 = a0 < p.n ? exp2i(-scale_exp<FMT>(am[a0])) : 0.f;
        const float s1 = a1 < p.n ? exp2i(-scale_exp<FMT>(am[a1])) : 0.f;
        g0 = make_float2(g0.x * s0, g0.y * s0);  // exact: s is a power of two
        g1 = make_float2(g1.x * s1, g1.y * s1);
      }
    }
    const bool apply = DT != 0 && (p.gains || p.in_amax);
    bool unit_over_16 = false;
#pragma unroll 1
    for (int g = 0; g < kUnitT / 16; ++g) {
      float2 v0[16], v1[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int t = x.ku * kUnitT + g * 16 + i;
        v0[i] = (a0 < p.n && t < p.g.T) ? load_cx<DT>(p, x.c, a0, t) : make_float2(0.f, 0.f);
        v1[i] = (a1 < p.n && t < p.g.T) ? load_cx<DT>(p, x.c, a1, t) : make_float2(0.f, 0.f);
      }
      if constexpr (DT == 0 && FMT == kFmtF8) {
#pragma unroll
        for (int i = 0; i < 16; ++i)
          unit_over_16 |= fmaxf(fmaxf(fabsf(v0[i].x), fabsf(v0[i].y)),
                                fmaxf(fabsf(v1[i].x), fabsf(v1[i].y))) > 16.f;
      }
      if (apply) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          v0[i] = make_float2(g0.x * v0[i].x - g0.y * v0[i].y, g0.x * v0[i].y + g0.y * v0[i].x);
          v1[i] = make_float2(g1.x * v1[i].x - g1.y * v1[i].y, g1.x * v1[i].y + g1.y * v1[i].x);
        }
      }
      if constexpr (FMT == kFmtF8) {
        const uint32_t off = tile_off<FMT>(row0, x.cbase / 2 + g);
        const uint32_t off1 = tile_off<FMT>(row0 + 32, x.cbase / 2 + g);
        uint32_t r0[4], i0[4], r1[4], i1[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float2* A = v0 + 4 * k;
          const float2* B = v1 + 4 * k;
          r0[k] = e4m3x4(A[0].x, A[1].x, A[2].x, A[3].x);
          i0[k] = e4m3x4(A[0].y, A[1].y, A[2].y, A[3].y);
          r1[k] = e4m3x4(B[0].x, B[1].x, B[2].x, B[3].x);
          i1[k] = e4m3x4(B[0].y, B[1].y, B[2].y, B[3].y);
        }
        *reinterpret_cast<uint4*>(tre + off) = make_uint4(r0[0], r0[1], r0[2], r0[3]);
        *reinterpret_cast<uint4*>(tim + off) = make_uint4(i0[0], i0[1], i0[2], i0[3]);
        *reinterpret_cast<uint4*>(tre + off1) = make_uint4(r1[0], r1[1], r1[2], r1[3]);
        *reinterpret_cast<uint4*>(tim + off1) = make_uint4(i1[0], i1[1], i1[2], i1[3]);
      } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t off = tile_off<FMT>(row0, x.cbase + 2 * g + h);
          const uint32_t off1 = tile_off<FMT>(row0 + 32, x.cbase + 2 * g + h);
          uint32_t r0[4], i0[4], r1[4], i1[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float2 a = v0[8 * h + 2 * k], b = v0[8 * h + 2 * k + 1];
            const float2 c = v1[8 * h + 2 * k], d = v1[8 * h + 2 * k + 1];
            r0[k] = h2bits(a.x, b.x);
            i0[k] = h2bits(a.y, b.y);
            r1[k] = h2bits(c.x, d.x);
            i1[k] = h2bits(c.y, d.y);
          }
          *reinterpret_cast<uint4*>(tre + off) = make_uint4(r0[0], r0[1], r0[2], r0[3]);
          *reinterpret_cast<uint4*>(tim + off) = make_uint4(i0[0], i0[1], i0[2], i0[3]);
          *reinterpret_cast<uint4*>(tre + off1) = make_uint4(r1[0], r1[1], r1[2], r1[3]);
          *reinterpret_cast<uint4*>(tim + off1) = make_uint4(i1[0], i1[1], i1[2], i1[3]);
          if constexpr (FMT == kFmtHiLo) {
            // Residual tile of the same K-block: K-tile nkb + kb.
            const int64_t lo_off = static_cast<int64_t>(p.nkb) * p.nib << FmtT<FMT>::kTileShift;
            uint32_t l0[4], m0[4], l1[4], m1[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const float2 a = v0[8 * h + 2 * k], b = v0[8 * h + 2 * k + 1];
              const float2 c = v1[8 * h + 2 * k], d = v1[8 * h + 2 * k + 1];
              l0[k] = lo2bits(a.x, b.x, r0[k]);
              m0[k] = lo2bits(a.y, b.y, i0[k]);
              l1[k] = lo2bits(c.x, d.x, r1[k]);
              m1[k] = lo2bits(c.y, d.y, i1[k]);
            }
            *reinterpret_cast<uint4*>(tre + lo_off + off) = make_uint4(l0[0], l0[1], l0[2], l0[3]);
            *reinterpret_cast<uint4*>(tim + lo_off + off) = make_uint4(m0[0], m0[1], m0[2], m0[3]);
            *reinterpret_cast<uint4*>(tre + lo_off + off1) = make_uint4(l1[0], l1[1], l1[2], l1[3]);
            *reinterpret_cast<uint4*>(tim + lo_off + off1) = make_uint4(m1[0], m1[1], m1[2], m1[3]);
          }
        }
      }
    }
    if (DT == 0 && lane == 0) atomicMax(p.amax + x.c, 128u);  // no scan: worst case
    if (DT == 0 && FMT == kFmtF8 && __any_sync(0xffffffffu, unit_over_16) && lane == 0)
      atomicOr(p.status, kStatusRange);  // e4m3 is exact only for |x| <= 16
    publish_unit(p, x.slot, lane);
    if (*abort_flag) return;
  }
}

// Bounded wait for the warp's TMA box still in flight (completing phase
// `phase` of `bar`): a converter that gives up never leaves a copy landing in
// shared memory after it has returned.
__device__ __forceinline__ void drain_tma(uint32_t bar, uint32_t phase, bool pending,
                                          unsigned long long timeout_ns) {
  if (pending) {
    const uint64_t t0 = ptx::globaltimer();
    while (!ptx::mbar_try_wait(bar, phase) && ptx::globaltimer() - t0 < timeout_ns) {
    }
  }
  __syncwarp();
}

// 8-bit converter with TMA-staged input.  Each converter warp is an
// independent worker on its own stream of units (u = global warp id + k *
// warps, channel-major), with an 8 KiB staging buffer ([64 samples][128
// rows] int8 = 64 inputs x {re, im}) that always holds its next unit's box
// in flight while the current one is converted.  A warp claims a slot for
// itself and publishes each unit on its own: no barrier couples the warps.
// A unit is published after the next unit's shared-memory reads, so its
// stores have drained by the time the proxy fence waits for them; a warp
// that would have to wait for a slot publishes first (a consumer of the
// slot's previous channel may need that unit).
template <int FMT, bool MULTI>
__device__ void converter_tma(const Batch& bt, uint32_t buf, uint32_t bar, int cw, int lane,
                              volatile int* abort_flag) {
  static_assert(FMT == kFmtF16 || FMT == kFmtF8, "8-bit input: fp16 or e4m3 operands");
  const long long total = table_end<MULTI>(bt.unit_base, bt.nsub);
  const long long nw = static_cast<long long>(gridDim.x) * conv_warps<FMT, 0>();
  const ptx::WaitCtl wc{bt.sub[0].timeout_ns, bt.sub[0].status, abort_flag};
  int sb_issue = 0;
  bool tma_pending = false;  // a box issued and not yet waited for
  auto issue = [&](long long u) {
    tma_pending = true;
    sb_issue = advance_sub<MULTI>(bt.unit_base, bt.nsub, u, sb_issue);
    const Unit x = unit_of(bt.sub[sb_issue], u - bt.unit_base[sb_issue]);
    if (lane == 0) {
      ptx::mbar_arrive_expect_tx(bar, kConvBufBytes);
      // The input streams through once: first in line for L2 replacement, so
      // the operand ring it is converted into stays resident.
      ptx::tma_load_3d_hint(buf, &bt.maps[sb_issue], bar, x.hb * kUnitRows, x.c, x.ku * kUnitT,
                            ptx::l2_policy_evict_first());
    }
  };
  const uint32_t* src = reinterpret_cast<const uint32_t*>(__cvta_shared_to_generic(static_cast<size_t>(buf)));
  // Lane l converts inputs 2l and 2l + 1 of the half block: word l of each
  // 128-byte sample row holds (re, im) of both.  Per 8-sample chunk and plane
  // the lane writes tile rows 2l and 2l + 1 (32 contiguous bytes), so a warp
  // store covers 1 KiB.
  uint32_t phase = 0;
  int sb = 0, claimed = -1, claimed_sb = -1;
  // Converted units not yet published: their subarray, slot, channel, count.
  const Params* pend = nullptr;
  int pend_slot = 0, pend_c = -1, pend_sb = -1;
  unsigned pend_n = 0;
  long long u = first_unit(static_cast<long long>(blockIdx.x) * conv_warps<FMT, 0>() + cw);
  if (u < total) issue(u);
  for (; u < total; u = next_unit(u, nw)) {
    sb = advance_sub<MULTI>(bt.unit_base, bt.nsub, u, sb);
    const Params& p = bt.sub[sb];
    const Unit x = unit_of(p, u - bt.unit_base[sb]);
    if (x.c != claimed || sb != claimed_sb) {
      if (pend && slot_busy(p, x.c, lane)) {
        publish_unit(*pend, pend_slot, lane, pend_n);
        pend = nullptr;
      }
      if (!claim_slot_warp(p, x.c, lane, abort_flag)) {
        drain_tma(bar, phase, tma_pending, wc.timeout_ns);
        return;
      }
      claimed = x.c;
      claimed_sb = sb;
    }
    const bool got = ptx::wait_bounded(bar, phase, wc);
    if (!__all_sync(0xffffffffu, got)) {
      drain_tma(bar, phase, tma_pending, wc.timeout_ns);
      return;
    }
    tma_pending = false;
    phase ^= 1u;
    // Both inputs' kUnitT samples into registers, then refill the buffer.
    uint32_t w[kUnitT];
#pragma unroll
    for (int t = 0; t < kUnitT; ++t) w[t] = src[t * (kUnitRows / 4) + lane];
    __syncwarp();
    ptx::fence_proxy_async_smem();
    const long long un = next_unit(u, nw);
    if (un < total) issue(un);
    // A finished run (or the units of another channel) is published now: its
    // stores have drained during this unit's shared-memory reads.
    if (pend && (pend_n == kUnitRun || pend_c != x.c || pend_sb != sb)) {
      publish_unit(*pend, pend_slot, lane, pend_n);
      pend = nullptr;
    }
    const int ib = x.hb >> 1;
    uint8_t* tre = ring_tile<FMT>(p, x.slot, 0, x.kb, ib);
    uint8_t* tim = ring_tile<FMT>(p, x.slot, 1, x.kb, ib);
    const int row = (x.hb & 1) * 64 + 2 * lane;  // tile rows 2l and 2l + 1
    // Ring tiles are read back by every block of the channel: keep them in L2.
    const uint64_t pol_last = ptx::l2_policy_evict_last();
    unsigned m = 0;  // max |x| over the unit (zero-filled rows and samples contribute 0)
    if constexpr (FMT == kFmtF16) {
      // max |x| from the converted (exact) fp16 values.
      __half2 mx[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) mx[q] = __float2half2_rn(0.f);
      // Rows 2l and 2l + 1 of one plane: bytes j and j + 2 of the words.
      auto store8 = [&](uint8_t* dst, const uint32_t* W, uint32_t j, __half2& mq) {
        uint32_t v[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          v[k] = pair_i8(W[2 * k], W[2 * k + 1], j);
          v[4 + k] = pair_i8(W[2 * k], W[2 * k + 1], j + 2);
        }
#pragma unroll
        for (int k = 0; k < 8; k += 2)
          mq = __hmax2(mq, __hmax2(__habs2(*reinterpret_cast<const __half2*>(&v[k])),
                                   __habs2(*reinterpret_cast<const __half2*>(&v[k + 1]))));
        ptx::st_global_v8_hint(dst, v, pol_last);
      };
#pragma unroll
      for (int cc = 0; cc < kUnitT / 8; ++cc) {
        const uint32_t off = tile_off<FMT>(row, x.cbase + cc);
        store8(tre + off, w + 8 * cc, 0u, mx[0]);
        store8(tim + off, w + 8 * cc, 1u, mx[1]);
      }
      const __half2 mm = __hmax2(mx[0], mx[1]);
      m = static_cast<unsigned>(fmaxf(__low2float(mm), __high2float(mm)));
    } else {
      // e4m3 operands: exact for |x| <= 16 (a larger value sets the range
      // status bit below).  16-sample chunks; rows 2l and 2l + 1 per store.
      uint32_t mb = 0;  // per-byte |x| maximum
#pragma unroll
      for (int t = 0; t < kUnitT; ++t) mb = __vmaxu4(mb, __vabs4(w[t]));
      m = max(max(mb & 0xffu, (mb >> 8) & 0xffu), max((mb >> 16) & 0xffu, mb >> 24));
      // Component j of four consecutive samples as four e4m3 bytes: the
      // exact fp16 pair conversion of the fp16 path, then one fp16x2 ->
      // e4m3x2 conversion per pair (exact for |x| <= 16).
      auto cvt4 = [](uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, uint32_t j) {
        const uint32_t h01 = pair_i8(w0, w1, j), h23 = pair_i8(w2, w3, j);
        __half2_raw r01, r23;
        r01.x = static_cast<unsigned short>(h01 & 0xffffu);
        r01.y = static_cast<unsigned short>(h01 >> 16);
        r23.x = static_cast<unsigned short>(h23 & 0xffffu);
        r23.y = static_cast<unsigned short>(h23 >> 16);
        const uint32_t e01 = __nv_cvt_halfraw2_to_fp8x2(r01, __NV_SATFINITE, __NV_E4M3);
        const uint32_t e23 = __nv_cvt_halfraw2_to_fp8x2(r23, __NV_SATFINITE, __NV_E4M3);
        return (e01 & 0xffffu) | (e23 << 16);
      };
#pragma unroll
      for (int cc = 0; cc < kUnitT / 16; ++cc) {
        const uint32_t off = tile_off<FMT>(row, x.cbase / 2 + cc);
        const uint32_t* W = w + 16 * cc;
        uint32_t vr[8], vi[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          vr[k] = cvt4(W[4 * k], W[4 * k + 1], W[4 * k + 2], W[4 * k + 3], 0);
          vi[k] = cvt4(W[4 * k], W[4 * k + 1], W[4 * k + 2], W[4 * k + 3], 1);
          vr[4 + k] = cvt4(W[4 * k], W[4 * k + 1], W[4 * k + 2], W[4 * k + 3], 2);
          vi[4 + k] = cvt4(W[4 * k], W[4 * k + 1], W[4 * k + 2], W[4 * k + 3], 3);
        }
        ptx::st_global_v8_hint(tre + off, vr, pol_last);
        ptx::st_global_v8_hint(tim + off, vi, pol_last);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
      atomicMax(p.amax + x.c, m);
      if (FMT == kFmtF8 && m > 16) atomicOr(p.status, kStatusRange);
    }
    if (pend) {
      ++pend_n;
    } else {
      pend = &p;
      pend_slot = x.slot;
      pend_c = x.c;
      pend_sb = sb;
      pend_n = 1;
    }
    if (*abort_flag) {
      drain_tma(bar, phase, tma_pending, wc.timeout_ns);
      return;
    }
  }
  if (pend) publish_unit(*pend, pend_slot, lane, pend_n);
}

// Convert 16 samples of two inputs (v0: input a0, v1: input a1 = a0 + 32;
// gains and scale already applied) into the tiles of one K-block: fp16 (two
// 8-sample chunks from chunk8), hi/lo (the same in the H tiles plus the
// residuals in the L tiles) or e4m3 (one 16-sample chunk).
template <int FMT>
__device__ __forceinline__ void store_group16(const Params& p, uint8_t* tre, uint8_t* tim, int row0,
                                              int chunk8, const float2 (&v0)[16],
                                              const float2 (&v1)[16], uint64_t pol) {
  auto st = [&](uint8_t* dst, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    ptx::st_global_v4_hint(dst, a, b, c, d, pol);
  };
  if constexpr (FMT == kFmtF8) {
    const uint32_t off = tile_off<FMT>(row0, chunk8 / 2);
    const uint32_t off1 = tile_off<FMT>(row0 + 32, chunk8 / 2);
    uint32_t r0[4], i0[4], r1[4], i1[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2* A = v0 + 4 * k;
      const float2* B = v1 + 4 * k;
      r0[k] = e4m3x4(A[0].x, A[1].x, A[2].x, A[3].x);
      i0[k] = e4m3x4(A[0].y, A[1].y, A[2].y, A[3].y);
      r1[k] = e4m3x4(B[0].x, B[1].x, B[2].x, B[3].x);
      i1[k] = e4m3x4(B[0].y, B[1].y, B[2].y, B[3].y);
    }
    st(tre + off, r0[0], r0[1], r0[2], r0[3]);
    st(tim + off, i0[0], i0[1], i0[2], i0[3]);
    st(tre + off1, r1[0], r1[1], r1[2], r1[3]);
    st(tim + off1, i1[0], i1[1], i1[2], i1[3]);
  } else {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t off = tile_off<FMT>(row0, chunk8 + h);
      const uint32_t off1 = tile_off<FMT>(row0 + 32, chunk8 + h);
      uint32_t r0[4], i0[4], r1[4], i1[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 a = v0[8 * h + 2 * k], b = v0[8 * h + 2 * k + 1];
        const float2 c = v1[8 * h + 2 * k], d = v1[8 * h + 2 * k + 1];
        r0[k] = h2bits(a.x, b.x);
        i0[k] = h2bits(a.y, b.y);
        r1[k] = h2bits(c.x, d.x);
        i1[k] = h2bits(c.y, d.y);
      }
      st(tre + off, r0[0], r0[1], r0[2], r0[3]);
      st(tim + off, i0[0], i0[1], i0[2], i0[3]);
      st(tre + off1, r1[0], r1[1], r1[2], r1[3]);
      st(tim + off1, i1[0], i1[1], i1[2], i1[3]);
      if constexpr (FMT == kFmtHiLo) {
        // Residual tile of the same K-block: K-tile nkb + kb.
        const int64_t lo_off = static_cast<int64_t>(p.nkb) * p.nib << FmtT<FMT>::kTileShift;
        uint32_t l0[4], m0[4], l1[4], m1[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float2 a = v0[8 * h + 2 * k], b = v0[8 * h + 2 * k + 1];
          const float2 c = v1[8 * h + 2 * k], d = v1[8 * h + 2 * k + 1];
          l0[k] = lo2bits(a.x, b.x, r0[k]);
          m0[k] = lo2bits(a.y, b.y, i0[k]);
          l1[k] = lo2bits(c.x, d.x, r1[k]);
          m1[k] = lo2bits(c.y, d.y, i1[k]);
        }
        st(tre + lo_off + off, l0[0], l0[1], l0[2], l0[3]);
        st(tim + lo_off + off, m0[0], m0[1], m0[2], m0[3]);
        st(tre + lo_off + off1, l1[0], l1[1], l1[2], l1[3]);
        st(tim + lo_off + off1, m1[0], m1[1], m1[2], m1[3]);
      }
    }
  }
}

// Float converter with TMA-staged input: boxes of 64 inputs x kFBox samples
// (8 KiB: complex fp16, 32 samples, or complex fp32, 16 samples) pass
// through the warp's one staging buffer, kUnitT / kFBox boxes per unit;
// while one box is converted the next (of this unit or of the next) is in
// flight.  Units are taken in runs and published as in converter_tma.
template <int DT, int FMT, bool MULTI>
__device__ void converter_tma_float(const Batch& bt, uint32_t buf, uint32_t bar, int cw, int lane,
                                    volatile int* abort_flag) {
  constexpr int kCx = DT == 1 ? 4 : 8;  // bytes per complex sample
  constexpr int kFBox = kConvBufBytes / (64 * kCx);
  constexpr int kBoxes = kUnitT / kFBox;
  static_assert(kFBox % 16 == 0 && kUnitT % kFBox == 0, "boxes hold whole 16-sample groups");
  const long long total = table_end<MULTI>(bt.unit_base, bt.nsub);
  const long long nw = static_cast<long long>(gridDim.x) * conv_warps<FMT, DT>();
  const ptx::WaitCtl wc{bt.sub[0].timeout_ns, bt.sub[0].status, abort_flag};
  int sb_issue = 0;
  bool tma_pending = false;  // a box issued and not yet waited for
  auto issue = [&](long long u, int j) {
    tma_pending = true;
    sb_issue = advance_sub<MULTI>(bt.unit_base, bt.nsub, u, sb_issue);
    const Unit x = unit_of(bt.sub[sb_issue], u - bt.unit_base[sb_issue]);
    if (lane == 0) {
      ptx::mbar_arrive_expect_tx(bar, kConvBufBytes);
      // Map elements: one complex fp16 (32-bit) or one fp32 component.
      const int ex = DT == 1 ? x.hb * 64 : x.hb * 128;
      ptx::tma_load_3d_hint(buf, &bt.maps[sb_issue], bar, ex, x.c, x.ku * kUnitT + j * kFBox,
                            ptx::l2_policy_evict_first());
    }
  };
  const uint8_t* src = reinterpret_cast<const uint8_t*>(__cvta_shared_to_generic(static_cast<size_t>(buf)));
  const uint64_t pol_last = ptx::l2_policy_evict_last();
  uint32_t phase = 0;
  int sb = 0, claimed = -1, claimed_sb = -1;
  const Params* pend = nullptr;
  int pend_slot = 0, pend_c = -1, pend_sb = -1;
  unsigned pend_n = 0;
  long long u = first_unit(static_cast<long long>(blockIdx.x) * conv_warps<FMT, DT>() + cw);
  if (u < total) issue(u, 0);
  for (; u < total; u = next_unit(u, nw)) {
    sb = advance_sub<MULTI>(bt.unit_base, bt.nsub, u, sb);
    const Params& p = bt.sub[sb];
    const Unit x = unit_of(p, u - bt.unit_base[sb]);
    if (x.c != claimed || sb != claimed_sb) {
      if (pend && slot_busy(p, x.c, lane)) {
        publish_unit(*pend, pend_slot, lane, pend_n);
        pend = nullptr;
      }
      if (!claim_slot_warp(p, x.c, lane, abort_flag)) {
        drain_tma(bar, phase, tma_pending, wc.timeout_ns);
        return;
      }
      claimed = x.c;
      claimed_sb = sb;
    }
    const int ib = x.hb >> 1;
    uint8_t* tre = ring_tile<FMT>(p, x.slot, 0, x.kb, ib);
    uint8_t* tim = ring_tile<FMT>(p, x.slot, 1, x.kb, ib);
    const int a0 = x.hb * 64 + lane, a1 = a0 + 32;
    const int row0 = (x.hb & 1) * 64 + lane;
    // y = g x 2^-e.
    float2 g0 = make_float2(1.f, 0.f), g1 = make_float2(1.f, 0.f);
    if (p.gains) {
      g0 = a0 < p.n ? p.gains[a0 % p.gain_n] : make_float2(0.f, 0.f);
      g1 = a1 < p.n ? p.gains[a1 % p.gain_n] : make_float2(0.f, 0.f);
    }
    if (p.in_amax) {
      const unsigned* am = p.in_amax + static_cast<int64_t>(x.c) * p.n;
      const float s0 = a0 < p.n ? exp2i(-scale_exp<FMT>(am[a0])) : 0.f;
      const float s1 = a1 < p.n ? exp2i(-scale_exp<FMT>(am[a1])) : 0.f;
      g0 = make_float2(g0.x * s0, g0.y * s0);  // exact: s is a power of two
      g1 = make_float2(g1.x * s1, g1.y * s1);
    }
#pragma unroll 1
    for (int j = 0; j < kBoxes; ++j) {
      const bool got = ptx::wait_bounded(bar, phase, wc);
      if (!__all_sync(0xffffffffu, got)) {
        drain_tma(bar, phase, tma_pending, wc.timeout_ns);
        return;
      }
      tma_pending = false;
      phase ^= 1u;
      // Lane l: inputs l and l + 32 of the box's 64, every sample.
      using Raw = typename std::conditional<DT == 1, uint32_t, float2>::type;
      const Raw* box = reinterpret_cast<const Raw*>(src);
      Raw w0[kFBox], w1[kFBox];
#pragma unroll
      for (int t = 0; t < kFBox; ++t) {
        w0[t] = box[t * 64 + lane];
        w1[t] = box[t * 64 + 32 + lane];
      }
      __syncwarp();
      ptx::fence_proxy_async_smem();
      if (j + 1 < kBoxes) {
        issue(u, j + 1);
      } else {
        const long long un = next_unit(u, nw);
        if (un < total) issue(un, 0);
      }
      if (j == 0 && pend && (pend_n == kUnitRun || pend_c != x.c || pend_sb != sb)) {
        publish_unit(*pend, pend_slot, lane, pend_n);
        pend = nullptr;
      }
#pragma unroll
      for (int g16 = 0; g16 < kFBox / 16; ++g16) {
        float2 v0[16], v1[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          float2 c0, c1;
          if constexpr (DT == 1) {
            c0 = __half22float2(*reinterpret_cast<const __half2*>(&w0[16 * g16 + i]));
            c1 = __half22float2(*reinterpret_cast<const __half2*>(&w1[16 * g16 + i]));
          } else {
            c0 = w0[16 * g16 + i];
            c1 = w1[16 * g16 + i];
          }
          v0[i] = make_float2(g0.x * c0.x - g0.y * c0.y, g0.x * c0.y + g0.y * c0.x);
          v1[i] = make_float2(g1.x * c1.x - g1.y * c1.y, g1.x * c1.y + g1.y * c1.x);
        }
        store_group16<FMT>(p, tre, tim, row0, x.cbase + (j * kFBox + 16 * g16) / 8, v0, v1, pol_last);
      }
    }
    if (pend) {
      ++pend_n;
    } else {
      pend = &p;
      pend_slot = x.slot;
      pend_c = x.c;
      pend_sb = sb;
      pend_n = 1;
    }
    if (*abort_flag) {
      drain_tma(bar, phase, tma_pending, wc.timeout_ns);
      return;
    }
  }
  if (pend) publish_unit(*pend, pend_slot, lane, pend_n);
}

// --------------------------------------------------------------- epilogue

// Store one 32-column piece: values v_re[j], v_im[j] of V(a, b0 + j).
template <bool IS_INT>
__device__ __forceinline__ void store_piece(const uint32_t (&re)[32], const uint32_t (&im)[32],
                                            const Params& p, int f, int a, int b0, bool add) {
  using T = typename std::conditional<IS_INT, int, float>::type;
  const Geometry& g = p.g;
  T* out = static_cast<T*>(p.out);
  auto val = [&](uint32_t u) -> T {
    if constexpr (IS_INT) {
      return __float2int_rn(__uint_as_float(u));
    } else {
      return __uint_as_float(u);
    }
  };
  // Two polarisations, overwrite, 32-byte aligned output: the lanes of a
  // station's two rows (a, a ^ 1; both valid or both not, n being even)
  // exchange halves so that each writes whole 32-byte baseline records.
  const bool pairs = g.P == 2 && !add && (reinterpret_cast<uintptr_t>(out) & 31) == 0;
  const bool valid = a < p.n;
  if (!valid && !pairs) return;
  // Real channel, row station and first column station (packed channels:
  // columns of another channel of the pack fall outside 0 <= s2 <= s1).
  int fr = f, s1 = a / g.P, s2_0 = b0 / g.P;
  if (p.pack > 1) {
    const int j = s1 / p.Nr;
    s1 -= j * p.Nr;
    s2_0 -= j * p.Nr;
    fr = f * p.pack + j;
  }
  const int64_t krow = static_cast<int64_t>(fr) * p.NBr + static_cast<int64_t>(s1) * (s1 + 1) / 2;
  if (pairs) {
    const int p1 = a & 1;
    uint32_t* o8 = reinterpret_cast<uint32_t*>(out + krow * 8);  // record of s2 at o8 + 8 s2
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      // This lane's products for column stations 2m (A) and 2m + 1 (B) of the piece.
      uint32_t A[4], B[4], rec[8];
      auto bits = [&](uint32_t u) -> uint32_t {  // the stored word: int32 value or fp32 bits
        if constexpr (IS_INT) {
          return static_cast<uint32_t>(val(u));
        } else {
          return u;
        }
      };
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        A[2 * q] = bits(re[4 * m + q]);
        A[2 * q + 1] = bits(im[4 * m + q]);
        B[2 * q] = bits(re[4 * m + 2 + q]);
        B[2 * q + 1] = bits(im[4 * m + 2 + q]);
      }
      // Row p1 = 0 writes baseline 2m, row p1 = 1 baseline 2m + 1; each sends
      // the partner the half it needs.
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t got = __shfl_xor_sync(0xffffffffu, p1 ? A[k] : B[k], 1);
        rec[k] = p1 ? got : A[k];
        rec[4 + k] = p1 ? B[k] : got;
      }
      const int s2 = s2_0 + 2 * m + p1;
      if (valid && s2 >= 0 && s2 <= s1)
        ptx::st_global_v8_hint(o8 + 8 * static_cast<int64_t>(s2), rec, ptx::l2_policy_evict_first());
    }
  } else if (g.P == 2) {
    const int p1 = a & 1;
    using V4 = typename std::conditional<IS_INT, int4, float4>::type;
    V4* o4 = reinterpret_cast<V4*>(out + (krow * 4 + p1 * 2) * 2);  // (p1,0),(p1,1) of s2 at o4[2 s2]
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      V4 old[8];
      if (add) {
        // Loads of a half first: independent of the stores that follow.
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int s2 = s2_0 + 8 * h + j;
          if (s2 >= 0 && s2 <= s1) old[j] = o4[2 * s2];
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int jj = 8 * h + j;
        const int s2 = s2_0 + jj;
        if (s2 >= 0 && s2 <= s1) {
          V4 v;
          v.x = val(re[2 * jj]);
          v.y = val(im[2 * jj]);
          v.z = val(re[2 * jj + 1]);
          v.w = val(im[2 * jj + 1]);
          if (add) {
            v.x += old[j].x;
            v.y += old[j].y;
            v.z += old[j].z;
            v.w += old[j].w;
          }
          o4[2 * s2] = v;
        }
      }
    }
  } else {
    using V2 = typename std::conditional<IS_INT, int2, float2>::type;
    V2* o2 = reinterpret_cast<V2*>(out + krow * 2);  // baseline s2 at o2[s2]
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      V2 old[8];
      if (add) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int s2 = s2_0 + 8 * h + j;
          if (s2 >= 0 && s2 <= s1) old[j] = o2[s2];
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int jj = 8 * h + j;
        const int s2 = s2_0 + jj;
        if (s2 >= 0 && s2 <= s1) {
          V2 v;
          v.x = val(re[jj]);
          v.y = val(im[jj]);
          if (add) {
            v.x += old[j].x;
            v.y += old[j].y;
          }
          o2[s2] = v;
        }
      }
    }
  }
}

// Undo the operand scales of float input: V(a, b0 + j) *= 2^(e_a + e_b).
template <int FMT>
__device__ __forceinline__ void scale_piece(uint32_t (&re)[32], uint32_t (&im)[32], const Params& p,
                                            int f, int a, int b0) {
  const unsigned* am = p.in_amax + static_cast<int64_t>(f) * p.n;
  const int ea = a < p.n ? scale_exp<FMT>(am[a]) : 0;
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const int b = b0 + j;
    const float sc = exp2i(ea + (b < p.n ? scale_exp<FMT>(am[b]) : 0));
    re[j] = __float_as_uint(__uint_as_float(re[j]) * sc);
    im[j] = __float_as_uint(__uint_as_float(im[j]) * sc);
  }
}

// FP64 block sums: acc64 = (first chunk and not accumulating ? 0 : acc64) +
// piece; the last chunk of the integration also stores its fp32 rounding.
__device__ __forceinline__ void store_piece_f64(const uint32_t (&re)[32], const uint32_t (&im)[32],
                                                const Params& p, int f, int a, int b0, bool first,
                                                bool last) {
  const int P = p.g.P;
  // Every lane of the warp joins the pairs path's exchanges; rows past n
  // (the ragged last block) only skip their memory accesses.
  const bool valid = a < p.n;
  if (!valid && !(P == 2 && p.pack == 1)) return;
  int s1 = a / P, joff = 0, fr = f;
  const int p1 = a - s1 * P;
  if (p.pack > 1) {  // packed channels: real channel and stations
    const int j = s1 / p.Nr;
    joff = j * p.Nr;
    s1 -= joff;
    fr = f * p.pack + j;
  }
  const int64_t krow = static_cast<int64_t>(fr) * p.NBr + static_cast<int64_t>(s1) * (s1 + 1) / 2;
  const bool load_old = !first || p.accumulate;
  // The running sum outlives this drain unless it is the integration's last
  // one and calls do not accumulate.
  const bool keep = !last || p.accumulate;
  double2* ws = reinterpret_cast<double2*>(p.acc64);
  float2* out = static_cast<float2*>(p.out);
  if (P == 2 && p.pack == 1) {
    // As the int32 store's pairs path: the lanes of a station's two
    // polarisation rows (a, a ^ 1) exchange halves so that each holds one
    // whole baseline record {(0,0), (0,1), (1,0), (1,1)}: the p1 = 0 lane the
    // record of column station 2m, the p1 = 1 lane that of 2m + 1.  A lane
    // then moves 64 contiguous bytes of running sums (and 32 of output), and
    // a lane pair 128 contiguous bytes of one baseline row.
    const int s2_0 = b0 / 2;
    // Groups of MG records: the running sums of a group are loaded before
    // any of its stores (the compiler cannot move a load above a store to
    // the same buffer), so their memory latencies overlap.
    constexpr int MG = 2;
#pragma unroll
    for (int h = 0; h < 8 / MG; ++h) {
      double2 old[MG][4];
      if (load_old) {
#pragma unroll
        for (int mm = 0; mm < MG; ++mm) {
          const int s2 = s2_0 + 2 * (MG * h + mm) + p1;
          const bool ok = valid && s2 <= s1;
#pragma unroll
          for (int k = 0; k < 4; ++k)
            old[mm][k] = ok ? ws[(krow + s2) * 4 + k] : make_double2(0.0, 0.0);
        }
      }
#pragma unroll
      for (int mm = 0; mm < MG; ++mm) {
        const int m = MG * h + mm;
        float own[4], got[4];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const float r0 = __uint_as_float(re[4 * m + q]), i0 = __uint_as_float(im[4 * m + q]);
          const float r1 = __uint_as_float(re[4 * m + 2 + q]), i1 = __uint_as_float(im[4 * m + 2 + q]);
          own[2 * q] = p1 ? r1 : r0;
          own[2 * q + 1] = p1 ? i1 : i0;
          got[2 * q] = __shfl_xor_sync(0xffffffffu, p1 ? r0 : r1, 1);
          got[2 * q + 1] = __shfl_xor_sync(0xffffffffu, p1 ? i0 : i1, 1);
        }
        // Products (p1', p2) of the record: row p1' = 0 from the p1 = 0 lane.
        double2 v[4];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const float* r0 = p1 ? got : own;  // row 0 of the record
          const float* r1 = p1 ? own : got;  // row 1
          v[q] = make_double2(r0[2 * q], r0[2 * q + 1]);
          v[2 + q] = make_double2(r1[2 * q], r1[2 * q + 1]);
        }
        const int s2 = s2_0 + 2 * m + p1;
        if (!valid || s2 > s1) continue;
        double2* w4 = ws + (krow + s2) * 4;
        if (load_old) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            v[k].x += old[mm][k].x;
            v[k].y += old[mm][k].y;
          }
        }
        if (keep) {
#pragma unroll
          for (int k = 0; k < 4; ++k) w4[k] = v[k];
        }
        if (last) {
          uint32_t rec[8];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            rec[2 * k] = __float_as_uint(static_cast<float>(v[k].x));
            rec[2 * k + 1] = __float_as_uint(static_cast<float>(v[k].y));
          }
          ptx::st_global_v8_hint(out + (krow + s2) * 4, rec, ptx::l2_policy_evict_first());
        }
      }
    }
    return;
  }
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const int b = b0 + j;
    const int s2v = b / P, p2 = b - s2v * P, s2 = s2v - joff;
    if (s2 < 0 || s2 > s1) continue;
    const int64_t idx = (krow + s2) * P * P + p1 * P + p2;
    double2 v = make_double2(static_cast<double>(__uint_as_float(re[j])),
                             static_cast<double>(__uint_as_float(im[j])));
    if (load_old) {
      const double2 o = ws[idx];
      v.x += o.x;
      v.y += o.y;
    }
    if (!last || p.accumulate) ws[idx] = v;
    if (last) out[idx] = make_float2(static_cast<float>(v.x), static_cast<float>(v.y));
  }
}

// Transposed blocks (CTA pairs): this thread's row a lies in a row block
// above the piece's columns b0 .. b0 + 31 (every b > a), so the stored lower
// entries are the mirror ones, V[b][a] = conj(V[a][b]): baseline
// (s1, s2) = (s_b, s_a), polarisation product p_b * P + p_a.  Packed
// channels never occur here (they have one block row).
template <bool IS_INT>
__device__ __forceinline__ void store_piece_tr(const uint32_t (&re)[32], const uint32_t (&im)[32],
                                               const Params& p, int f, int a, int b0, bool add) {
  using T = typename std::conditional<IS_INT, int, float>::type;
  const Geometry& g = p.g;
  T* out = static_cast<T*>(p.out);
  const int P = g.P;
  const int sa = a / P, pa = a - sa * P;
  // The stored word of the conjugate: int32 value or fp32 bits.
  auto re_bits = [](uint32_t u) -> uint32_t {
    if constexpr (IS_INT) {
      return static_cast<uint32_t>(__float2int_rn(__uint_as_float(u)));
    } else {
      return u;
    }
  };
  auto im_bits = [](uint32_t u) -> uint32_t {  // of -im
    if constexpr (IS_INT) {
      return static_cast<uint32_t>(-__float2int_rn(__uint_as_float(u)));
    } else {
      return u ^ 0x80000000u;
    }
  };
  const bool pairs = P == 2 && !add && (reinterpret_cast<uintptr_t>(out) & 31) == 0;
  if (pairs) {
    // Lanes (2i, 2i + 1) hold pols 0 and 1 of station s_a.  For column
    // stations s_b0 + 2k (written by the pa = 0 lane) and s_b0 + 2k + 1 (by
    // the pa = 1 lane) each lane needs its partner's two products of that
    // column station: one exchange of 4 words per k gives both lanes whole
    // 32-byte records, {(0,0), (0,1), (1,0), (1,1)} x {re, im}.
    const bool row_ok = a < p.n;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      uint32_t own[4], got[4];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        // Columns 4k + q (station 2k) and 4k + 2 + q (station 2k + 1): the
        // pa = 0 lane keeps the first and sends the second, pa = 1 the reverse.
        const uint32_t r0 = re_bits(re[4 * k + q]), i0 = im_bits(im[4 * k + q]);
        const uint32_t r1 = re_bits(re[4 * k + 2 + q]), i1 = im_bits(im[4 * k + 2 + q]);
        own[2 * q] = pa ? r1 : r0;
        own[2 * q + 1] = pa ? i1 : i0;
        got[2 * q] = __shfl_xor_sync(0xffffffffu, pa ? r0 : r1, 1);
        got[2 * q + 1] = __shfl_xor_sync(0xffffffffu, pa ? i0 : i1, 1);
      }
      uint32_t rec[8];
#pragma unroll
      for (int q = 0; q < 2; ++q) {  // products (p_b = q, p_a = 0) and (q, 1)
        rec[4 * q + 0] = pa ? got[2 * q] : own[2 * q];
        rec[4 * q + 1] = pa ? got[2 * q + 1] : own[2 * q + 1];
        rec[4 * q + 2] = pa ? own[2 * q] : got[2 * q];
        rec[4 * q + 3] = pa ? own[2 * q + 1] : got[2 * q + 1];
      }
      const int sb = b0 / 2 + 2 * k + pa;
      if (row_ok && sb < g.N) {
        const int64_t rec_idx =
            static_cast<int64_t>(f) * p.NBr + static_cast<int64_t>(sb) * (sb + 1) / 2 + sa;
        ptx::st_global_v8_hint(reinterpret_cast<uint32_t*>(out) + rec_idx * 8, rec,
                               ptx::l2_policy_evict_first());
      }
    }
    return;
  }
  if (a >= p.n) return;
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const int b = b0 + j;
    if (b >= p.n) continue;
    const int sb = b / P, pb = b - sb * P;
    const int64_t idx =
        ((static_cast<int64_t>(f) * p.NBr + static_cast<int64_t>(sb) * (sb + 1) / 2 + sa) * P + pb) * P + pa;
    uint32_t w[2] = {re_bits(re[j]), im_bits(im[j])};
    T* o = out + idx * 2;
    if (add) {
      o[0] += *reinterpret_cast<const T*>(&w[0]);
      o[1] += *reinterpret_cast<const T*>(&w[1]);
    } else if constexpr (IS_INT) {
      *reinterpret_cast<int2*>(o) = make_int2(static_cast<int>(w[0]), static_cast<int>(w[1]));
    } else {
      *reinterpret_cast<float2*>(o) = make_float2(__uint_as_float(w[0]), __uint_as_float(w[1]));
    }
  }
}

// FP64 block sums of a transposed block (see store_piece_f64, store_piece_tr).
__device__ __forceinline__ void store_piece_f64_tr(const uint32_t (&re)[32], const uint32_t (&im)[32],
                                                   const Params& p, int f, int a, int b0, bool first,
                                                   bool last) {
  if (a >= p.n) return;
  const int P = p.g.P;
  const int sa = a / P, pa = a - sa * P;
  const bool load_old = !first || p.accumulate;
  double2* ws = reinterpret_cast<double2*>(p.acc64);
  float2* out = static_cast<float2*>(p.out);
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const int b = b0 + j;
    if (b >= p.n) continue;
    const int sb = b / P, pb = b - sb * P;
    const int64_t idx =
        ((static_cast<int64_t>(f) * p.NBr + static_cast<int64_t>(sb) * (sb + 1) / 2 + sa) * P + pb) * P + pa;
    double2 v = make_double2(static_cast<double>(__uint_as_float(re[j])),
                             -static_cast<double>(__uint_as_float(im[j])));
    if (load_old) {
      const double2 o = ws[idx];
      v.x += o.x;
      v.y += o.y;
    }
    if (!last || p.accumulate) ws[idx] = v;
    if (last) out[idx] = make_float2(static_cast<float>(v.x), static_cast<float>(v.y));
  }
}

// ------------------------------------------------------------------ kernel

// Per-launch constants of the item loop: CTA pairs walk the items by
// cluster, single CTAs by block.
template <int SHAPE>
__device__ __forceinline__ long long item_first() {
  return SHAPE == kShapePair ? static_cast<long long>(blockIdx.x >> 1) : static_cast<long long>(blockIdx.x);
}
template <int SHAPE>
__device__ __forceinline__ long long item_stride() {
  return SHAPE == kShapePair ? static_cast<long long>(gridDim.x >> 1) : static_cast<long long>(gridDim.x);
}

template <bool IS_INT, int DT, int FMT, bool MULTI, int SHAPE>
__device__ __forceinline__ void planar_body(const Batch& bt) {
  constexpr bool PAIR = SHAPE == kShapePair;
  constexpr bool WIDE = SHAPE == kShapeWide;
  using C = Cfg<SHAPE, FMT, DT>;
  constexpr int kStages = C::kStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  const uint32_t sbase = ptx::smem_u32(smem);
  const uint32_t bar0 = sbase + C::kBarOff;
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (kStages + s); };
  auto pfull_bar = [&](int s) { return bar0 + 8u * (2 * kStages + s); };  // PAIR only
  constexpr int kB = (PAIR ? 3 : 2) * kStages;
  auto accf_bar = [&](int b) { return bar0 + 8u * (kB + b); };
  auto acce_bar = [&](int b) { return bar0 + 8u * (kB + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (kB + 4);
  auto conv_bar = [&](int w) { return bar0 + 8u * (kB + 5 + w); };
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(smem + C::kBarOff + C::kNumBars * 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  // K-blocks per exact accumulation chunk of the item whose first step stage s
  // holds: the producer (which has waited for the channel) writes it before the
  // stage's arrive, so the MMA thread reads it after its wait with no global
  // round trip of its own.
  volatile int* item_chunk = reinterpret_cast<volatile int*>(tmem_holder + 2);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = PAIR ? ptx::cluster_ctarank() : 0u;
  const bool leader = rank == 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(full_bar(s), 1);
      ptx::mbar_init(empty_bar(s), 1);
      if (PAIR) ptx::mbar_init(pfull_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(accf_bar(b), 1);
      ptx::mbar_init(acce_bar(b), (PAIR ? 2 : 1) * kNumEpiWarps);
    }
    ptx::mbar_init(drain_bar, 1);
    for (int w = 0; w < conv_warps<FMT, DT>(); ++w) ptx::mbar_init(conv_bar(w), 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
    ptx::fence_proxy_async_smem();
  }
  if (warp == 1) {
    if constexpr (PAIR) {
      ptx::tmem_alloc_pair(ptx::smem_u32(tmem_holder), kTmemCols);
      ptx::tmem_relinquish_pair();
    } else {
      ptx::tmem_alloc(ptx::smem_u32(tmem_holder), kTmemCols);
      ptx::tmem_relinquish();
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if constexpr (PAIR) ptx::cluster_sync();  // both CTAs' barriers exist before any remote arrive
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  // Hi/lo operands: 22-bit products lose accuracy in a long fp32 TMEM
  // accumulation, so the MMA restarts its accumulator (buffer 0) every
  // 64-sample K-block and the epilogue adds each block into a round-to-nearest
  // fp32 running sum held in TMEM columns 256..511 (not with 128 x 256 items,
  // whose accumulators fill the 512 columns).
  constexpr bool kTmemSum = FMT == kFmtHiLo;
  static_assert(!(kTmemSum && WIDE), "hi/lo operands need TMEM columns 256..511 for their sums");
  // One accumulator set in TMEM (no double buffer) for 128 x 256 items:
  // D_re in columns 0..255, D_im in 256..511.  Other shapes alternate two
  // sets {D_re, D_im} of 128 + 128 columns.
  constexpr bool kOneSet = kTmemSum || WIDE;
  constexpr int TB = FmtT<FMT>::kTile;
  const ptx::WaitCtl wc{bt.sub[0].timeout_ns, bt.sub[0].status, abort_flag};
  const long long nitems = table_end<MULTI>(bt.item_base, bt.nsub);
  const long long it0 = item_first<SHAPE>(), istep = item_stride<SHAPE>();

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int issued_phase[kStages];
      for (int s = 0; s < kStages; ++s) issued_phase[s] = -1;
      bool ok = true;
      int sb = 0, ready_chan = -1, ready_sb = -1, chan_chunk = 1;
      const uint64_t pol_last = ptx::l2_policy_evict_last();  // tiles are shared by the channel's blocks
      for (long long it = it0; ok && it < nitems; it += istep) {
        sb = advance_sub<MULTI>(bt.item_base, bt.nsub, it, sb);
        const Params& p = bt.sub[sb];
        const Blk k = item_block<SHAPE>(p, it - bt.item_base[sb], rank);
        const int slot = k.f % p.ring_slots;
        if (k.f != ready_chan || sb != ready_sb) {
          const unsigned gen = static_cast<unsigned>(k.f / p.ring_slots);
          if (!wait_counter(p.ready + slot, (gen + 1) * static_cast<unsigned>(p.units_per_chan), p,
                            abort_flag)) {
            ok = false;
            break;
          }
          ready_chan = k.f;
          ready_sb = sb;
          chan_chunk = chunk_kblocks(p, k.f);  // the channel is converted: its max |x| is final
        }
        const bool diag = SHAPE == kShape128 && k.a == k.b;
        for (int st = 0; ok && st < p.nkb * FmtT<FMT>::kSteps; ++st) {
          // Step st: K-block kb; HI/LO steps j = 0, 1, 2 take (H, H), (L, H), (H, L).
          const int kb = st / FmtT<FMT>::kSteps, j = st - kb * FmtT<FMT>::kSteps;
          const int kta = kb + (j == 1 ? p.nkb : 0);
          const int ktb = kb + (j == 2 ? p.nkb : 0);
          if (!ptx::wait_bounded(empty_bar(stage), phase ^ 1u, wc)) {
            ok = false;
            break;
          }
          const uint32_t dst = sbase + stage * C::kStageBytes;
          const uint32_t fb = full_bar(stage);
          if (st == 0) item_chunk[stage] = chan_chunk;  // published by the arrive below
          if constexpr (PAIR) {
            // A: this CTA's row block (not needed by an idle CTA); B: this
            // CTA's half of the column block (always: the leader's MMA reads it).
            constexpr int HB = TB / 2;
            ptx::mbar_arrive_expect_tx(fb, k.idle ? 2 * HB : 2 * TB + 2 * HB);
            if (!k.idle) {
              ptx::bulk_load_hint(dst, ring_tile<FMT>(p, slot, 0, kta, k.a), TB, fb, pol_last);
              ptx::bulk_load_hint(dst + TB, ring_tile<FMT>(p, slot, 1, kta, k.a), TB, fb, pol_last);
            }
            ptx::bulk_load_hint(dst + 2 * TB, ring_tile<FMT>(p, slot, 0, ktb, k.b) + rank * HB, HB, fb,
                                pol_last);
            ptx::bulk_load_hint(dst + 2 * TB + HB, ring_tile<FMT>(p, slot, 1, ktb, k.b) + rank * HB, HB,
                                fb, pol_last);
          } else if constexpr (WIDE) {
            // Ar, Ai; then Br of both column blocks back to back (one 256-row
            // operand: the second tile starts 16 groups on), and Bi likewise.
            const bool two = k.b2 >= 0;
            ptx::mbar_arrive_expect_tx(fb, two ? 6 * TB : 4 * TB);
            ptx::bulk_load_hint(dst, ring_tile<FMT>(p, slot, 0, kta, k.a), TB, fb, pol_last);
            ptx::bulk_load_hint(dst + TB, ring_tile<FMT>(p, slot, 1, kta, k.a), TB, fb, pol_last);
            ptx::bulk_load_hint(dst + 2 * TB, ring_tile<FMT>(p, slot, 0, ktb, k.b), TB, fb, pol_last);
            ptx::bulk_load_hint(dst + 4 * TB, ring_tile<FMT>(p, slot, 1, ktb, k.b), TB, fb, pol_last);
            if (two) {
              ptx::bulk_load_hint(dst + 3 * TB, ring_tile<FMT>(p, slot, 0, ktb, k.b2), TB, fb, pol_last);
              ptx::bulk_load_hint(dst + 5 * TB, ring_tile<FMT>(p, slot, 1, ktb, k.b2), TB, fb, pol_last);
            }
          } else {
            const bool same = diag && kta == ktb;
            ptx::mbar_arrive_expect_tx(fb, same ? 2 * TB : 4 * TB);
            ptx::bulk_load_hint(dst, ring_tile<FMT>(p, slot, 0, kta, k.a), TB, fb, pol_last);
            ptx::bulk_load_hint(dst + TB, ring_tile<FMT>(p, slot, 1, kta, k.a), TB, fb, pol_last);
            if (!same) {
              ptx::bulk_load_hint(dst + 2 * TB, ring_tile<FMT>(p, slot, 0, ktb, k.b), TB, fb, pol_last);
              ptx::bulk_load_hint(dst + 3 * TB, ring_tile<FMT>(p, slot, 1, ktb, k.b), TB, fb, pol_last);
            }
          }
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
                 ptx::globaltimer() - t0 < wc.timeout_ns) {
          }
        }
      }
    }
  } else if (warp == 1 && PAIR && !leader) {
    // ------------------------------------------------ peer relay (pairs)
    // Forwards each completed stage of this CTA to the leader's pfull.
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int sb = 0;
      for (long long it = it0; ok && it < nitems; it += istep) {
        sb = advance_sub<MULTI>(bt.item_base, bt.nsub, it, sb);
        const Params& p = bt.sub[sb];
        for (int st = 0; st < p.nkb * FmtT<FMT>::kSteps; ++st) {
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
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t u = 0;
      bool ok = true;
      bool issued_any = false;
      int sb = 0;
      for (long long it = it0; ok && it < nitems; it += istep) {
        sb = advance_sub<MULTI>(bt.item_base, bt.nsub, it, sb);
        const Params& p = bt.sub[sb];
        const Blk k = item_block<SHAPE>(p, it - bt.item_base[sb], rank);
        const bool diag = SHAPE == kShape128 && k.a == k.b;
        // MMA shape.  128 x 128: M = 128 rows, N trimmed to the block's valid
        // columns (rounded up to 16), so ragged edge blocks skip the zero
        // columns.  Pairs: M = 256 (both row blocks), N = 128, 64 per CTA.
        // 128 x 256: N = 128 + the second block's valid columns.
        uint32_t idesc;
        if constexpr (PAIR) {
          idesc = ptx::idesc_f16_f32(2 * kBlk, kBlk);
        } else {
          // (The second column block of a 128 x 256 item sits right after the
          // first in shared memory, whatever their block indices.)
          const bool two = WIDE && k.b2 >= 0;
          const int last_b = two ? k.b2 : k.b;
          const int ncols = (two ? kBlk : 0) + min(kBlk, p.n - last_b * kBlk);
          idesc = ptx::idesc_f16_f32(kBlk, (ncols + 15) & ~15);
        }
        const uint32_t idesc_negb = idesc | (1u << 14);
        // The item's first stage (its data and its chunk length).  Waiting for
        // it again in the step loop returns at once: the stage cannot complete
        // another phase before these MMAs release it.
        if (!ptx::wait_bounded(full_bar(stage), phase, wc) ||
            (PAIR && !ptx::wait_bounded(pfull_bar(stage), phase, wc))) {
          ok = false;
          break;
        }
        const int chunk_kb = item_chunk[stage];
        const int nchunks = (p.nkb + chunk_kb - 1) / chunk_kb;
        // The item's first step needs no second wait.
        bool waited = true;
        for (int ch = 0; ok && ch < nchunks; ++ch) {
          const int kb0 = ch * chunk_kb;
          const int kb1 = min(p.nkb, kb0 + chunk_kb);
          // Accumulation groups: the whole chunk, or one K-block per group when
          // the epilogue sums 64-sample fp32 blocks in TMEM (buffer 0 only).
          const int gstep = kTmemSum ? 1 : (kb1 - kb0);
          for (int g0 = kb0; ok && g0 < kb1; g0 += gstep) {
          const int g1 = min(kb1, g0 + gstep);
          const uint32_t ab = kOneSet ? 0u : (u & 1u);
          const uint32_t ap = kOneSet ? (u & 1u) : ((u >> 1) & 1u);
          if (!ptx::wait_bounded(acce_bar(ab), ap ^ 1u, wc)) {
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t d_re = tmem + ab * 256;
          const uint32_t d_im = d_re + (WIDE ? 256 : 128);
          for (int st = g0 * FmtT<FMT>::kSteps; st < g1 * FmtT<FMT>::kSteps; ++st) {
            if (!waited && (!ptx::wait_bounded(full_bar(stage), phase, wc) ||
                            (PAIR && !ptx::wait_bounded(pfull_bar(stage), phase, wc)))) {
              ok = false;
              break;
            }
            waited = false;
            const int nstage = stage + 1 == kStages ? 0 : stage + 1;
            const uint32_t nphase = stage + 1 == kStages ? phase ^ 1u : phase;
            ptx::tc_fence_after();
            const uint32_t ar = sbase + stage * C::kStageBytes;
            const uint32_t ai = ar + TB;
            uint32_t br, bi;
            if constexpr (PAIR) {
              br = ar + 2 * TB;
              bi = br + TB / 2;
            } else if constexpr (WIDE) {
              br = ar + 2 * TB;
              bi = ar + 4 * TB;
            } else {
              const bool same = diag && (FMT != kFmtHiLo || st % 3 == 0);
              br = same ? ar : ar + 2 * TB;
              bi = same ? ai : ar + 3 * TB;
            }
            // Descriptors of the stage's four operands; K-step kk adds its byte
            // offset (16-byte units) to the address field, which cannot carry:
            // every shared-memory address is below 256 KiB.
            constexpr uint32_t SBO = FmtT<FMT>::kSbo;
            const uint64_t dar0 = ptx::interleave_kmajor_desc(ar, kCoreBytes, SBO);
            const uint64_t dai0 = ptx::interleave_kmajor_desc(ai, kCoreBytes, SBO);
            const uint64_t dbr0 = ptx::interleave_kmajor_desc(br, kCoreBytes, SBO);
            const uint64_t dbi0 = ptx::interleave_kmajor_desc(bi, kCoreBytes, SBO);
#pragma unroll
            for (int kk = 0; kk < FmtT<FMT>::kChunks / 2; ++kk) {
              const uint32_t acc = (st > g0 * FmtT<FMT>::kSteps || kk > 0) ? 1u : 0u;
              // K-step kk covers 16-byte chunks 2kk and 2kk + 1 (16 fp16 or 32 e4m3 samples).
              const uint64_t kd = static_cast<uint64_t>(kk * 2 * kCoreBytes) >> 4;
              const uint64_t dar = dar0 + kd, dai = dai0 + kd, dbr = dbr0 + kd, dbi = dbi0 + kd;

              if constexpr (PAIR && FMT == kFmtF8) {
                ptx::mma_f8_ss_pair(d_re, dar, dbr, idesc, acc);       // Re += Ar Br^T
                ptx::mma_f8_ss_pair(d_re, dai, dbi, idesc, 1u);        // Re += Ai Bi^T
                ptx::mma_f8_ss_pair(d_im, dai, dbr, idesc, acc);       // Im += Ai Br^T
                ptx::mma_f8_ss_pair(d_im, dar, dbi, idesc_negb, 1u);   // Im -= Ar Bi^T
              } else if constexpr (PAIR) {
                ptx::mma_f16_ss_pair(d_re, dar, dbr, idesc, acc);
                ptx::mma_f16_ss_pair(d_re, dai, dbi, idesc, 1u);
                ptx::mma_f16_ss_pair(d_im, dai, dbr, idesc, acc);
                ptx::mma_f16_ss_pair(d_im, dar, dbi, idesc_negb, 1u);
              } else if constexpr (FMT == kFmtF8) {
                ptx::mma_f8_ss(d_re, dar, dbr, idesc, acc);
                ptx::mma_f8_ss(d_re, dai, dbi, idesc, 1u);
                ptx::mma_f8_ss(d_im, dai, dbr, idesc, acc);
                ptx::mma_f8_ss(d_im, dar, dbi, idesc_negb, 1u);
              } else {
                ptx::mma_f16_ss(d_re, dar, dbr, idesc, acc);
                ptx::mma_f16_ss(d_re, dai, dbi, idesc, 1u);
                ptx::mma_f16_ss(d_im, dai, dbr, idesc, acc);
                ptx::mma_f16_ss(d_im, dar, dbi, idesc_negb, 1u);
              }
            }
            issued_any = true;
            if constexpr (PAIR) {
              ptx::mma_commit_pair_mc(empty_bar(stage), 0x3);
            } else {
              ptx::mma_commit(empty_bar(stage));
            }
            stage = nstage;
            phase = nphase;

          }
          if (!ok) break;
          if constexpr (PAIR) {
            ptx::mma_commit_pair_mc(accf_bar(ab), 0x3);
          } else {
            ptx::mma_commit(accf_bar(ab));
          }
          ++u;
          }
        }
      }
      if (!ok && issued_any) {
        if constexpr (PAIR) {
          ptx::mma_commit_pair_mc(drain_bar, 0x1);
        } else {
          ptx::mma_commit(drain_bar);
        }
        const uint64_t t0 = ptx::globaltimer();
        while (!ptx::mbar_try_wait(drain_bar, 0) && ptx::globaltimer() - t0 < wc.timeout_ns) {
        }
      }
    }
  } else if (warp < 2 + kNumEpiWarps) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;
    const uint32_t t_lanes = tmem + (static_cast<uint32_t>(q * 32) << 16);
    uint32_t u = 0;
    bool ok = true;
    int sb = 0;
    // Accumulator b has been read: local arrive, or remote on the leader's barrier.
    auto release_acc = [&](uint32_t ab) {
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (!PAIR || leader)
          ptx::mbar_arrive(acce_bar(ab));
        else
          ptx::mbar_arrive_remote(ptx::mapa_shared(acce_bar(ab), 0));
      }
    };
    for (long long it = it0; ok && it < nitems; it += istep) {
      sb = advance_sub<MULTI>(bt.item_base, bt.nsub, it, sb);
      const Params& p = bt.sub[sb];
      const int P = p.g.P;
      const Blk k = item_block<SHAPE>(p, it - bt.item_base[sb], rank);
      const int f = k.f;
      const int a = k.a * kBlk + q * 32 + lane;  // this thread's row input
      // The item's column blocks and, per block, the pieces piece0..last this
      // warp stores: for a block on or below the diagonal those that can reach
      // the lower station triangle (packed channels: only from the first
      // column of the lowest row's real channel on); for a mirrored block
      // every piece with a valid column.
      const int nblk = (WIDE && k.b2 >= 0) ? 2 : 1;
      int cb[2] = {k.b, k.b2}, first_p[2] = {0, 0}, last_p[2] = {-1, -1};
      for (int j = 0; j < nblk; ++j) {
        const int b = cb[j];
        if (k.idle) continue;
        if (b > k.a) {
          for (int piece = 0; piece < kBlk / 32; ++piece)
            if (b * kBlk + piece * 32 < p.n) last_p[j] = piece;
        } else {
          const int s1_hi = min(p.g.N - 1, (k.a * kBlk + q * 32 + 31) / P);
          for (int piece = 0; piece < kBlk / 32; ++piece)
            if ((b * kBlk + piece * 32) / P <= s1_hi) last_p[j] = piece;
          if (p.pack > 1) {
            const int col0 = (k.a * kBlk + q * 32) / P / p.Nr * p.Nr * P;  // first column of that channel
            first_p[j] = max(0, (col0 - b * kBlk) / 32);
            if (first_p[j] > last_p[j]) last_p[j] = -1;  // no row of this warp is valid
          }
        }
      }
      // The last block with pieces to read releases the accumulator after them.
      const int jlast = (nblk == 2 && last_p[1] >= 0) ? 1 : (last_p[0] >= 0 ? 0 : -1);
      const bool rdy = channel_ready(p, f, abort_flag);
      if (!__all_sync(0xffffffffu, rdy)) {
        ok = false;
        break;
      }
      const int chunk_kb = chunk_kblocks(p, f);
      const int nchunks = (p.nkb + chunk_kb - 1) / chunk_kb;
      for (int ch = 0; ok && ch < nchunks; ++ch) {
        const int kb0 = ch * chunk_kb;
        const int kb1 = min(p.nkb, kb0 + chunk_kb);
        const int gstep = kTmemSum ? 1 : (kb1 - kb0);
        const bool add = p.accumulate || ch > 0;
        const bool last_chunk = ch == nchunks - 1;
        // FP64 block sums: chunks pair off, (0, 1), (2, 3), ...  The first
        // chunk of a pair stays in its TMEM accumulator (`hold`); the second's
        // drain adds it in fp32 (a correctly rounded sum of the two partials,
        // what an fp64 add rounded back would give) and updates the float64
        // running sum once per pair: half the passes over it, none at all for
        // an integration of two chunks.  Needs the two accumulator sets.
        const bool f64pair = !IS_INT && !kOneSet && p.acc64 != nullptr;
        const bool hold = f64pair && (ch % 2 == 0) && ch + 1 < nchunks;
        const bool paired = f64pair && (ch % 2 == 1);
        const bool first = f64pair ? ch < 2 : ch == 0;
        for (int g0 = kb0; g0 < kb1; g0 += gstep) {
          // TMEM running sum: the first group of a chunk starts it, the last
          // one is stored; groups in between only add into it.
          const bool gfirst = g0 == kb0, glast = g0 + gstep >= kb1;
          const uint32_t ab = kOneSet ? 0u : (u & 1u);
          const uint32_t ap = kOneSet ? (u & 1u) : ((u >> 1) & 1u);
          if constexpr (!IS_INT) {
            // FP64 block sums: while the MMAs run, bring into L2 the running
            // sums this drain will read: each lane of a row's pair prefetches
            // half of the row's records in the block (one bulk request).
            if (p.acc64 && !hold && (!first || p.accumulate) && glast && P == 2 && p.pack == 1 && a < p.n) {
              const int s1 = a / 2;
              const int64_t krow = static_cast<int64_t>(f) * p.NBr + static_cast<int64_t>(s1) * (s1 + 1) / 2;
              for (int j = 0; j < nblk; ++j) {
                const int b = cb[j];
                if (b > k.a) continue;  // mirrored blocks write other rows
                const int lo = b * (kBlk / 2), hi = min(b * (kBlk / 2) + kBlk / 2 - 1, s1);
                const int half = (hi - lo + 2) / 2;
                const int from = lo + (a & 1) * half, cnt = min(half, hi - from + 1);
                if (cnt > 0)
                  ptx::bulk_prefetch_l2(reinterpret_cast<const double2*>(p.acc64) + (krow + from) * 4,
                                        static_cast<uint32_t>(cnt) * 64u);
              }
            }
          }
          const bool got = ptx::wait_bounded(accf_bar(ab), ap, wc);
          if (!__all_sync(0xffffffffu, got)) {
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          // The item's last group is complete, so every MMA of the item (in
          // both CTAs of a pair) has read its operands: the item is done with
          // its ring slot.  (Released here, off the MMA thread's path.)
          if (last_chunk && glast && q == 0 && lane == 0 && leader)
            red_release_add(p.done + (f % p.ring_slots), 1u);
          if (hold) {  // drained with the next chunk
            ++u;
            continue;
          }
          if (paired) {
            // Add the held chunk into this one inside TMEM and free it at
            // once, so the next item's MMAs need not wait for the stores.
            for (int j = 0; j < nblk; ++j) {
              const uint32_t c_re = ab * 256, c_im = ab * 256 + 128;
              const uint32_t h_re = (ab ^ 1u) * 256, h_im = (ab ^ 1u) * 256 + 128;
#pragma unroll 1
              for (int piece = first_p[j]; piece <= last_p[j]; ++piece) {
                uint32_t vr[32], vi[32], sr[32], si[32];
                ptx::tmem_ld_32x32b_x32(t_lanes + c_re + piece * 32, vr);
                ptx::tmem_ld_32x32b_x32(t_lanes + c_im + piece * 32, vi);
                ptx::tmem_ld_32x32b_x32(t_lanes + h_re + piece * 32, sr);
                ptx::tmem_ld_32x32b_x32(t_lanes + h_im + piece * 32, si);
                ptx::tmem_wait_ld();
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                  vr[jj] = __float_as_uint(__uint_as_float(vr[jj]) + __uint_as_float(sr[jj]));
                  vi[jj] = __float_as_uint(__uint_as_float(vi[jj]) + __uint_as_float(si[jj]));
                }
                ptx::tmem_st_32x32b_x32(t_lanes + c_re + piece * 32, vr);
                ptx::tmem_st_32x32b_x32(t_lanes + c_im + piece * 32, vi);
              }
            }
            ptx::tmem_wait_st();
            release_acc(ab ^ 1u);
          }
          if (jlast < 0) release_acc(ab);
          for (int j = 0; j < nblk; ++j) {
            const int b = cb[j];
            // TMEM columns of block j: D_re and D_im of its 128 columns.
            const uint32_t c_re = WIDE ? j * kBlk : ab * 256;
            const uint32_t c_im = WIDE ? 256 + j * kBlk : ab * 256 + 128;
#pragma unroll 1
            for (int piece = first_p[j]; piece <= last_p[j]; ++piece) {
              uint32_t vr[32], vi[32];
              ptx::tmem_ld_32x32b_x32(t_lanes + c_re + piece * 32, vr);
              ptx::tmem_ld_32x32b_x32(t_lanes + c_im + piece * 32, vi);
              if constexpr (kTmemSum) {
               if (!gfirst) {
                uint32_t sr[32], si[32];
                ptx::tmem_ld_32x32b_x32(t_lanes + 256 + piece * 32, sr);
                ptx::tmem_ld_32x32b_x32(t_lanes + 384 + piece * 32, si);
                ptx::tmem_wait_ld();
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                  vr[jj] = __float_as_uint(__uint_as_float(vr[jj]) + __uint_as_float(sr[jj]));
                  vi[jj] = __float_as_uint(__uint_as_float(vi[jj]) + __uint_as_float(si[jj]));
                }
               }
              }
              ptx::tmem_wait_ld();
              if (j == jlast && piece == last_p[j]) release_acc(ab);
              if (kTmemSum && !glast) {
                ptx::tmem_st_32x32b_x32(t_lanes + 256 + piece * 32, vr);
                ptx::tmem_st_32x32b_x32(t_lanes + 384 + piece * 32, vi);
                continue;
              }
              const int b0 = b * kBlk + piece * 32;
              const bool tr = b > k.a;  // a mirrored block
              if constexpr (IS_INT) {
                if (tr)
                  store_piece_tr<true>(vr, vi, p, f, a, b0, add);
                else
                  store_piece<true>(vr, vi, p, f, a, b0, add);
              } else {
                if (p.in_amax) scale_piece<FMT>(vr, vi, p, f, a, b0);
                // A drain that is both the first and the last of the running
                // sum (one chunk, or one chunk pair, without accumulation
                // across calls) only rounds to fp32: the plain store.
                if (p.acc64 && !(first && last_chunk && !p.accumulate)) {
                  if (tr)
                    store_piece_f64_tr(vr, vi, p, f, a, b0, first, last_chunk);
                  else
                    store_piece_f64(vr, vi, p, f, a, b0, first, last_chunk);
                } else {
                  // With block sums on, this drain holds the whole
                  // integration: it overwrites `out` (a paired chunk's
                  // ch > 0 must not make it add).
                  const bool add_out = add && !p.acc64;
                  if (tr)
                    store_piece_tr<false>(vr, vi, p, f, a, b0, add_out);
                  else
                    store_piece<false>(vr, vi, p, f, a, b0, add_out);
                }
              }
            }
          }
          if (kTmemSum && !glast) ptx::tmem_wait_st();
          ++u;
        }
      }
    }
  } else {
    // ---------------------------------------------------------- converters
    const int cw = warp - (2 + kNumEpiWarps);
    const uint32_t cbuf = sbase + C::kConvOff + cw * kConvBufBytes;
    if constexpr (DT == 0) {
      if (bt.sub[0].tma_in) {  // set for every subarray or for none
        converter_tma<FMT, MULTI>(bt, cbuf, conv_bar(cw), cw, lane, abort_flag);
      } else {
        converter_direct<DT, FMT, MULTI>(bt, cw, lane, abort_flag);
      }
    } else {
      if (bt.sub[0].tma_in) {
        converter_tma_float<DT, FMT, MULTI>(bt, cbuf, conv_bar(cw), cw, lane, abort_flag);
      } else {
        converter_direct<DT, FMT, MULTI>(bt, cw, lane, abort_flag);
      }
    }
  }

  // ------------------------------------------------------------- teardown
  ptx::tc_fence_before();
  __syncthreads();
  if constexpr (PAIR) ptx::cluster_sync();  // no SM still reads the other's shared memory or TMEM
  if (warp == 1) {
    ptx::tc_fence_after();
    if constexpr (PAIR) {
      ptx::tmem_dealloc_pair(tmem, kTmemCols);
    } else {
      ptx::tmem_dealloc(tmem, kTmemCols);
    }
  }
}

template <bool IS_INT, int DT, int FMT, bool MULTI>
__global__ void __launch_bounds__(threads_of<FMT, DT>(), 1) planar_kernel(const __grid_constant__ Batch bt) {
  planar_body<IS_INT, DT, FMT, MULTI, kShape128>(bt);
}

// 128 x 256 items: one CTA, N = 256 MMAs.
template <bool IS_INT, int DT, int FMT, bool MULTI>
__global__ void __launch_bounds__(threads_of<FMT, DT>(), 1) planar_wide_kernel(const __grid_constant__ Batch bt) {
  if constexpr (FMT != kFmtHiLo) planar_body<IS_INT, DT, FMT, MULTI, kShapeWide>(bt);
}

// CTA pairs: the cluster shape is part of the kernel, so no launch can run it
// without its peer.
template <bool IS_INT, int DT, int FMT, bool MULTI>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(threads_of<FMT, DT>(), 1)
    planar_pair_kernel(const __grid_constant__ Batch bt) {
  planar_body<IS_INT, DT, FMT, MULTI, kShapePair>(bt);
}

}  // namespace
}  // namespace xc
