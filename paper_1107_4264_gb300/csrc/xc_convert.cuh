// xc_convert.cuh -- device code shared by the fused X-engine kernels: the
// kernel parameters, global release/acquire counters and the converter
// warps that form fp16 K-major operands in the L2-resident ring.
//
// Converter: each input element of a channel is widened/rounded to fp16 and
// transposed once (register transpose: a lane loads 4 rows x 16 samples as
// 32-bit/64-bit/128-bit words and byte-permutes them into per-row runs of 8
// samples), written into the channel's ring slot and published through
// ready[slot]; a slot is reused only when done[slot] shows every block of
// its previous channel has read it.
#pragma once

#include <cuda_fp16.h>

#include "xc_launch.h"
#include "xc_ptx.cuh"

namespace xc {
namespace conv {

constexpr int kUnitRows = 128;  // converter unit: 128 rows x 64 samples
constexpr int kUnitT = 64;
constexpr int kNumConvWarps = 4;
constexpr int kConvBarrier = 1;  // named barrier of the converter warps

struct XeParams {
  Geometry g;
  const void* in;
  int in_dtype;
  void* out;
  int accumulate;
  int ntiles;          // lower blocks per channel
  long long nitems;    // ntiles * F
  int nkb;             // Tp / 64
  int chunk_kb;        // K-blocks per accumulation unit
  __half* ring;        // [ring_slots][R][Tp]
  int ring_slots;
  unsigned* ready;     // [ring_slots]
  unsigned* done;      // [ring_slots]
  int row_units;       // ceil(R / 128)
  int units_per_chan;  // row_units * Tp / 64
  int vec4;            // R % 4 == 0: 4-row vector loads
  unsigned long long timeout_ns;
  int* status;
};

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

// Bounded wait until *p >= target.  Gives up if the CTA is aborting, another
// CTA has recorded a failure, or timeout_ns passes.
static __device__ __noinline__ bool wait_counter(const unsigned* p, unsigned target, const XeParams& prm,
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

// -------------------------------------------------------------- converter

// Four consecutive input components (rows r .. r+3) of sample t, channel f.
template <int DT>
struct Quad;
template <>
struct Quad<0> {
  uint32_t w;
};
template <>
struct Quad<1> {
  uint2 w;
};
template <>
struct Quad<2> {
  float4 w;
};

template <int DT>
__device__ __forceinline__ void load_quad(const void* in, int64_t idx, Quad<DT>& q) {
  if constexpr (DT == 0) {
    q.w = __ldg(reinterpret_cast<const uint32_t*>(static_cast<const int8_t*>(in) + idx));
  } else if constexpr (DT == 1) {
    q.w = __ldg(reinterpret_cast<const uint2*>(static_cast<const __half*>(in) + idx));
  } else {
    q.w = __ldg(reinterpret_cast<const float4*>(static_cast<const float*>(in) + idx));
  }
}

template <int DT>
__device__ __forceinline__ void zero_quad(Quad<DT>& q) {
  if constexpr (DT == 0) {
    q.w = 0u;
  } else if constexpr (DT == 1) {
    q.w = make_uint2(0u, 0u);
  } else {
    q.w = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// fp16x2 of (component j of sample a, component j of sample b).
template <int DT>
__device__ __forceinline__ uint32_t pair_half2(const Quad<DT>& a, const Quad<DT>& b, int j) {
  if constexpr (DT == 0) {
    // Bytes j of both words into the low bytes of the two halves, then
    // 0x6400 | (x ^ 0x80) is the fp16 value 1152 + x; subtract 1152 exactly.
    // Selector nibble 0 = j (byte j of a), nibble 2 = j + 4 (byte j of b):
    // d = [a_j, a_0, b_j, a_0]; the mask keeps bytes 0 and 2.
    uint32_t d = __byte_perm(a.w, b.w, static_cast<uint32_t>(j) | (static_cast<uint32_t>(j + 4) << 8));
    d = (d & 0x00FF00FFu) ^ 0x64806480u;
    __half2 h = *reinterpret_cast<__half2*>(&d);
    h = __hsub2(h, __half2(__float2half_rn(1152.f), __float2half_rn(1152.f)));
    return *reinterpret_cast<uint32_t*>(&h);
  } else if constexpr (DT == 1) {
    const uint32_t wa = (j < 2) ? a.w.x : a.w.y;
    const uint32_t wb = (j < 2) ? b.w.x : b.w.y;
    const uint32_t sel = (j & 1) ? 0x7632u : 0x5410u;  // high or low halves of both
    return __byte_perm(wa, wb, sel);
  } else {
    const float fa = (j == 0) ? a.w.x : (j == 1) ? a.w.y : (j == 2) ? a.w.z : a.w.w;
    const float fb = (j == 0) ? b.w.x : (j == 1) ? b.w.y : (j == 2) ? b.w.z : b.w.w;
    __half2 h = __floats2half2_rn(fa, fb);
    return *reinterpret_cast<uint32_t*>(&h);
  }
}

template <int DT>
__device__ __forceinline__ __half scalar_half(const void* in, int64_t idx) {
  if constexpr (DT == 0) {
    return __int2half_rn(static_cast<int>(static_cast<const int8_t*>(in)[idx]));
  } else if constexpr (DT == 1) {
    return static_cast<const __half*>(in)[idx];
  } else {
    return __float2half_rn(static_cast<const float*>(in)[idx]);
  }
}

// Converter work.  A unit is 128 rows x 64 samples of one channel; a batch
// is up to kNumConvWarps consecutive units of the same channel and row block
// (consecutive 64-sample blocks), one unit per converter warp.  Batches are
// taken in channel order, b = blockIdx.x + k * gridDim.x, and published with
// one proxy fence and one release per batch.
struct Batch {
  int c;      // channel
  int slot;   // ring slot of the channel
  int rb;     // row block
  int tb0;    // first 64-sample block of the batch
  int n;      // units in the batch
};

__device__ __forceinline__ Batch batch_of(const XeParams& p, long long b) {
  const int tblocks = p.g.Tp / kUnitT;
  const int bpr = (tblocks + kNumConvWarps - 1) / kNumConvWarps;  // batches per row block
  const int bpc = bpr * p.row_units;                              // batches per channel
  Batch x;
  x.c = static_cast<int>(b / bpc);
  const int j = static_cast<int>(b % bpc);
  x.slot = x.c % p.ring_slots;
  x.rb = j / bpr;
  x.tb0 = (j % bpr) * kNumConvWarps;
  x.n = min(kNumConvWarps, tblocks - x.tb0);
  return x;
}

// Issue the 16 loads of this lane's 4 rows (r .. r+3) x 16 samples (tb ..):
// zeros past T or R.
template <int DT>
__device__ __forceinline__ void load_group(const XeParams& p, int c, int r, int tb,
                                           Quad<DT> (&q)[16]) {
  const Geometry& g = p.g;
  const bool row_ok = r < g.R;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int t = tb + i;
    if (row_ok && t < g.T)
      load_quad<DT>(p.in, (static_cast<int64_t>(t) * g.F + c) * g.R + r, q[i]);
    else
      zero_quad<DT>(q[i]);
  }
}

// Widen/round, transpose in registers and write 4 rows x 16 samples (two
// 16-byte runs per row) into the ring slot.
template <int DT>
__device__ __forceinline__ void store_group(const XeParams& p, int slot, int r, int tb,
                                            const Quad<DT> (&q)[16]) {
  const Geometry& g = p.g;
  if (r >= g.R) return;
  __half* dst_base = p.ring + (static_cast<int64_t>(slot) * g.R + r) * g.Tp + tb;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    uint32_t h[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) h[i] = pair_half2<DT>(q[2 * i], q[2 * i + 1], j);
    uint4* dst = reinterpret_cast<uint4*>(dst_base + static_cast<int64_t>(j) * g.Tp);
    dst[0] = make_uint4(h[0], h[1], h[2], h[3]);
    dst[1] = make_uint4(h[4], h[5], h[6], h[7]);
  }
}

// Any row count: one component at a time (rows that are not a multiple of 4).
template <int DT>
__device__ __forceinline__ void convert_group_scalar(const XeParams& p, int c, int slot, int r,
                                                     int tb) {
  const Geometry& g = p.g;
  for (int j = 0; j < 4; ++j) {
    const int rr = r + j;
    if (rr >= g.R) break;
    __half* dst = p.ring + (static_cast<int64_t>(slot) * g.R + rr) * g.Tp + tb;
    for (int i = 0; i < 16; ++i) {
      const int t = tb + i;
      dst[i] = (t < g.T) ? scalar_half<DT>(p.in, (static_cast<int64_t>(t) * g.F + c) * g.R + rr)
                         : __float2half_rn(0.f);
    }
  }
}

__device__ __forceinline__ void conv_sync() {
  asm volatile("bar.sync %0, %1;" ::"r"(kConvBarrier), "r"(32 * kNumConvWarps));
}

// Before the first write of channel c into its slot: the slot's previous
// channel (c - ring_slots) must have been read by all of its blocks.
__device__ __forceinline__ bool claim_slot(const XeParams& p, int c, int cw, int lane,
                                           volatile int* abort_flag) {
  const unsigned gen = static_cast<unsigned>(c / p.ring_slots);
  if (gen > 0) {
    if (cw == 0 && lane == 0)
      wait_counter(p.done + (c % p.ring_slots), gen * static_cast<unsigned>(p.ntiles), p, abort_flag);
    conv_sync();
    if (*abort_flag) return false;
  }
  // No proxy fence here: every TMA read of the slot's previous channel has
  // completed (its data sat in shared memory before the MMA thread released
  // done[slot]), so the generic writes that follow cannot reach it.
  return true;
}

template <int DT>
__device__ __forceinline__ void converter_loop(const XeParams& p, int cw, int lane, volatile int* abort_flag) {
  const int tblocks = p.g.Tp / kUnitT;
  const int bpr = (tblocks + kNumConvWarps - 1) / kNumConvWarps;
  const long long total = static_cast<long long>(p.g.F) * bpr * p.row_units;
  int claimed = -1;
  Quad<DT> qa[16], qb[16];
  long long b = blockIdx.x;
  // Prefetch the first group of this warp's unit in the first batch.
  Batch x = batch_of(p, b < total ? b : 0);
  if (p.vec4 && b < total && cw < x.n)
    load_group<DT>(p, x.c, x.rb * kUnitRows + 4 * lane, (x.tb0 + cw) * kUnitT, qa);
  for (; b < total; b += gridDim.x) {
    x = batch_of(p, b);
    const long long bn = b + gridDim.x;
    const Batch xn = batch_of(p, bn < total ? bn : b);
    if (x.c != claimed) {
      if (!claim_slot(p, x.c, cw, lane, abort_flag)) return;
      claimed = x.c;
    }
    const int r = x.rb * kUnitRows + 4 * lane;
    if (cw < x.n) {
      const int t0 = (x.tb0 + cw) * kUnitT;
      if (p.vec4) {
        // Four 16-sample groups; the loads of the next group (or of the next
        // batch's first group) are in flight while one is converted.
        load_group<DT>(p, x.c, r, t0 + 16, qb);
        store_group<DT>(p, x.slot, r, t0, qa);
        load_group<DT>(p, x.c, r, t0 + 32, qa);
        store_group<DT>(p, x.slot, r, t0 + 16, qb);
        load_group<DT>(p, x.c, r, t0 + 48, qb);
        store_group<DT>(p, x.slot, r, t0 + 32, qa);
        if (bn < total && cw < xn.n)
          load_group<DT>(p, xn.c, xn.rb * kUnitRows + 4 * lane, (xn.tb0 + cw) * kUnitT, qa);
        store_group<DT>(p, x.slot, r, t0 + 48, qb);
      } else {
        for (int gq = 0; gq < 4; ++gq) convert_group_scalar<DT>(p, x.c, x.slot, r, t0 + 16 * gq);
      }
    } else if (p.vec4 && bn < total && cw < xn.n) {
      load_group<DT>(p, xn.c, xn.rb * kUnitRows + 4 * lane, (xn.tb0 + cw) * kUnitT, qa);
    }
    fence_proxy_async_global();
    conv_sync();
    if (cw == 0 && lane == 0) red_release_add(p.ready + x.slot, static_cast<unsigned>(x.n));
    if (*abort_flag) return;
  }
}

}  // namespace conv
}  // namespace xc
