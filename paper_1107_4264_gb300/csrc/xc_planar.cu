// xc_planar.cu -- host side of the planar tensor-core X-engine (the kernel
// template is xc_planar_kernel.cuh): the single-CTA instantiations, the
// float scale pre-pass, the kernel parameter block, the ring geometry and
// the launch (single CTAs, or CTA pairs from xc_planar_pair.cu).
#include "xc_planar_kernel.cuh"

namespace xc {

// The CTA-pair and 128 x 256 instantiations live in xc_planar_pair.cu and
// xc_planar_wide.cu (compiled in parallel with this file).
const void* planar_pair_select(int in_dtype, int fmt, bool multi);
const void* planar_wide_select(int in_dtype, int fmt, bool multi);

static_assert(kShape128 == kPlanar128 && kShapePair == kPlanarPair && kShapeWide == kPlanarWide,
              "tile shape codes");

namespace {

template <bool IS_INT, int DT, int FMT, bool MULTI = false>
const void* kernel_of() {
  return reinterpret_cast<const void*>(planar_kernel<IS_INT, DT, FMT, MULTI>);
}

// Batches of several subarrays take 8-bit input.
const void* select_kernel(int in_dtype, int fmt, bool multi) {
  if (in_dtype == 0) {
    if (fmt == kFmtF8) return multi ? nullptr : kernel_of<true, 0, kFmtF8>();
    return multi ? kernel_of<true, 0, kFmtF16, true>() : kernel_of<true, 0, kFmtF16>();
  }
  if (multi) return nullptr;
  if (in_dtype != 1 && in_dtype != 2) return nullptr;
  const bool h = in_dtype == 1;
  switch (fmt) {
    case kFmtF16: return h ? kernel_of<false, 1, kFmtF16>() : kernel_of<false, 2, kFmtF16>();
    case kFmtHiLo: return h ? kernel_of<false, 1, kFmtHiLo>() : kernel_of<false, 2, kFmtHiLo>();
    case kFmtF8: return h ? kernel_of<false, 1, kFmtF8>() : kernel_of<false, 2, kFmtF8>();
    default: return nullptr;
  }
}

// Scale pre-pass for float input: amax[f][a] = max over t of the largest
// component of g_a x_a(t) (fp32 bits; non-negative floats order as
// unsigned integers).  A thread per (input, channel, 128-sample range);
// a warp reads 32 consecutive inputs of one sample row.
template <int DT>
__global__ void __launch_bounds__(128) input_amax_kernel(const void* __restrict__ in,
                                                         const float2* __restrict__ gains,
                                                         unsigned* __restrict__ amax, Geometry g,
                                                         int n, int gain_n) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const int f = blockIdx.y;
  if (a >= n) return;
  const int t0 = blockIdx.z * 128;
  const int t1 = min(g.T, t0 + 128);
  const float2 ga = gains ? gains[a % gain_n] : make_float2(1.f, 0.f);
  float m = 0.f;
#pragma unroll 8
  for (int t = t0; t < t1; ++t) {
    const int64_t idx = (static_cast<int64_t>(t) * g.F + f) * n + a;
    float2 v;
    if constexpr (DT == 1) {
      v = __half22float2(static_cast<const __half2*>(in)[idx]);
    } else {
      v = static_cast<const float2*>(in)[idx];
    }
    if (gains) v = make_float2(ga.x * v.x - ga.y * v.y, ga.x * v.y + ga.y * v.x);
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  atomicMax(amax + static_cast<int64_t>(f) * n + a, __float_as_uint(m));
}

int fmt_kt(int fmt) { return fmt == kFmtHiLo ? 2 : 1; }
int fmt_tile_bytes(int fmt) { return fmt == kFmtF8 ? (1 << 13) : (1 << 14); }

// Kernel parameters of one subarray.
Params sub_params(const XeLaunch& L, int shape) {
  Params p;
  p.g = L.g;
  p.n = L.g.N * L.g.P;
  p.in = L.in;
  p.out = L.out;
  p.accumulate = L.accumulate;
  p.nib = (p.n + kBlk - 1) / kBlk;
  p.ntiles = p.nib * (p.nib + 1) / 2;
  p.ipc = shape != kShape128 ? pair_items(p.nib) : p.ntiles;
  p.nitems = static_cast<long long>(p.ipc) * L.g.F;
  p.nkb = L.g.Tp / kBK;
  p.is_int = L.in_dtype == 0 ? 1 : 0;
  const int fmt = p.is_int ? (L.fmt == kFmtF8 ? kFmtF8 : kFmtF16) : L.fmt;
  p.nkt = fmt_kt(fmt) * p.nkb;
  p.amax = L.amax;
  p.gains = static_cast<const float2*>(L.gains);
  p.in_amax = p.is_int ? nullptr : L.in_amax;
  p.acc64 = p.is_int ? nullptr : L.acc64;
  p.f_chunk_kb = p.nkb;
  if (p.acc64 && L.f64_block > 0) p.f_chunk_kb = std::max(1, std::min(p.nkb, L.f64_block / kBK));
  p.ring = static_cast<uint8_t*>(L.ring);
  p.ring_slots = L.ring_slots;
  p.ready = L.counters;
  p.done = L.counters + L.ring_slots;
  p.row_units = 2 * p.nib;
  p.units_per_chan = p.row_units * p.nkb * (kBK / kUnitT);
  p.tma_in = 0;
  p.timeout_ns = L.timeout_ns;
  p.status = L.status;
  p.test_no_publish = L.test_no_publish;
  p.pack = std::max(1, L.pack);
  p.Nr = L.g.N / p.pack;
  p.NBr = static_cast<int64_t>(p.Nr) * (p.Nr + 1) / 2;
  p.gain_n = p.Nr * L.g.P;
  return p;
}

}  // namespace

int64_t planar_slot_bytes(const Geometry& g, int fmt) {
  const int64_t nib = (static_cast<int64_t>(g.N) * g.P + kBlk - 1) / kBlk;
  return 2 * fmt_kt(fmt) * (g.Tp / kBK) * nib * fmt_tile_bytes(fmt);
}

Geometry planar_geometry(const Geometry& g, int* pack) {
  int k = 1;
  const int64_t n = static_cast<int64_t>(g.N) * g.P;
  if (n <= kBlk / 2) {
    for (int c = static_cast<int>(kBlk / n); c >= 2; --c) {
      if (g.F % c == 0) {
        k = c;
        break;
      }
    }
  }
  Geometry v = g;
  v.N = g.N * k;
  v.F = g.F / k;
  v.R = g.R * k;
  v.NB = static_cast<int64_t>(v.N) * (v.N + 1) / 2;
  if (pack) *pack = k;
  return v;
}

int planar_ring_slots(const Geometry& g, int grid, int fmt) {
  // The persistent CTAs keep about grid / blocks_per_channel channels in
  // flight; the converters need room ahead of them.
  const int64_t nib = (static_cast<int64_t>(g.N) * g.P + kBlk - 1) / kBlk;
  const int64_t blocks = std::max<int64_t>(1, nib * (nib + 1) / 2);
  const int64_t inflight = (grid + blocks - 1) / blocks;
  int64_t n = (inflight * 8 + 4) / 5 + 4;
  const int64_t cap =
      std::max<int64_t>(2, (256ll << 20) / std::max<int64_t>(planar_slot_bytes(g, fmt), 1));
  n = std::max<int64_t>(4, std::min<int64_t>(std::min<int64_t>(kMaxRingSlots, cap), n));
  return static_cast<int>(std::min<int64_t>(n, g.F));
}

int planar_default_shape(const Geometry& g, int fmt) {
  // 128 x 128 measured fastest for the Large-N geometry (the larger shapes
  // move fewer operand bytes per MAC but put more channels in flight than
  // the L2-resident ring can run ahead of); the batch tuner tries all three.
  (void)g;
  (void)fmt;
  return kShape128;
}

cudaError_t planar_prepare(const XeLaunch* subs, const CUtensorMap* const* maps, int nsub,
                           PlanarKernel* k, int shape) {
  if (nsub < 1 || nsub > kMaxSub || !subs || !k) return cudaErrorInvalidValue;
  const int dt = subs[0].in_dtype;
  // 8-bit input: fp16 operands, or e4m3 when asked for (exact for |x| <= 16).
  auto fmt_of = [](const XeLaunch& L) {
    return L.in_dtype == 0 ? (L.fmt == kFmtF8 ? kFmtF8 : kFmtF16) : L.fmt;
  };
  const int fmt = fmt_of(subs[0]);
  Batch* b = reinterpret_cast<Batch*>(k->args);
  memset(b, 0, sizeof(Batch));
  b->nsub = nsub;
  bool all_tma = true;
  for (int i = 0; i < nsub; ++i) {
    if (subs[i].in_dtype != dt || fmt_of(subs[i]) != fmt) return cudaErrorInvalidValue;
    if (subs[i].ring_slots < 1 || subs[i].ring_slots > kMaxRingSlots) return cudaErrorInvalidValue;
    b->sub[i] = sub_params(subs[i], shape);
    if (maps && maps[i]) {
      b->maps[i] = *maps[i];
    } else {
      all_tma = false;
    }
    b->item_base[i + 1] = b->item_base[i] + (b->sub[i].nkb > 0 ? b->sub[i].nitems : 0);
    b->unit_base[i + 1] = b->unit_base[i] +
                          (b->sub[i].nkb > 0 ? static_cast<long long>(subs[i].g.F) * b->sub[i].units_per_chan : 0);
  }
  for (int i = 0; i < nsub; ++i) b->sub[i].tma_in = all_tma ? 1 : 0;
  const bool pair = shape == kShapePair;
  switch (shape) {
    case kShape128: k->func = select_kernel(dt, fmt, nsub > 1); break;
    case kShapePair: k->func = planar_pair_select(dt, fmt, nsub > 1); break;
    case kShapeWide: k->func = planar_wide_select(dt, fmt, nsub > 1); break;
    default: k->func = nullptr;
  }
  if (!k->func) return cudaErrorInvalidValue;
  const bool f8 = fmt == kFmtF8 && dt == 0;  // the e4m3 plan of 8-bit input
  k->block = f8 ? threads_of<kFmtF8, 0>() : threads_of<kFmtF16, 0>();
  k->smem = shape == kShapePair
                ? (f8 ? Cfg<kShapePair, kFmtF8, 0>::kSmemBytes : Cfg<kShapePair, kFmtF16, 0>::kSmemBytes)
                : (shape == kShapeWide
                       ? (f8 ? Cfg<kShapeWide, kFmtF8, 0>::kSmemBytes : Cfg<kShapeWide, kFmtF16, 0>::kSmemBytes)
                       : (f8 ? Cfg<kShape128, kFmtF8, 0>::kSmemBytes : Cfg<kShape128, kFmtF16, 0>::kSmemBytes));
  k->shape = shape;
  cudaError_t e = cudaFuncSetAttribute(k->func, cudaFuncAttributeMaxDynamicSharedMemorySize, k->smem);
  if (e != cudaSuccess) return e;
  // Every CTA must be resident at once: the operand ring couples them.
  const long long items = b->item_base[nsub];
  if (pair) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(std::max(2, subs[0].grid & ~1)));
    cfg.blockDim = dim3(static_cast<unsigned>(k->block));
    cfg.dynamicSmemBytes = static_cast<size_t>(k->smem);
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, k->func, &cfg);
    if (e != cudaSuccess) return e;
    if (clusters < 1) return cudaErrorInvalidConfiguration;
    const long long ncl = std::min<long long>({static_cast<long long>(clusters), subs[0].grid / 2, items});
    k->grid = static_cast<int>(2 * ncl);
  } else {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k->func, k->block, static_cast<size_t>(k->smem));
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long resident = static_cast<long long>(per_sm) * subs[0].grid;
    k->grid = static_cast<int>(std::min<long long>({items, static_cast<long long>(subs[0].grid), resident}));
  }
  return cudaSuccess;
}

cudaError_t planar_setup(const XeLaunch* subs, int nsub, cudaStream_t s) {
  for (int i = 0; i < nsub; ++i) {
    const XeLaunch& L = subs[i];
    const int n = L.g.N * L.g.P;
    cudaError_t e = cudaMemsetAsync(L.counters, 0, 2 * sizeof(unsigned) * L.ring_slots, s);
    if (e == cudaSuccess && L.in_dtype == 0)
      e = cudaMemsetAsync(L.amax, 0, sizeof(unsigned) * L.g.F, s);
    if (e != cudaSuccess) return e;
    if (L.in_dtype != 0 && L.in_amax) {
      e = cudaMemsetAsync(L.in_amax, 0, sizeof(unsigned) * L.g.F * static_cast<size_t>(n), s);
      if (e != cudaSuccess) return e;
      const dim3 ag((n + 127) / 128, L.g.F, (L.g.T + 127) / 128);
      if (ag.z > 65535u) return cudaErrorInvalidConfiguration;
      const float2* gains = static_cast<const float2*>(L.gains);
      const int gain_n = n / std::max(1, L.pack);
      if (L.in_dtype == 1)
        input_amax_kernel<1><<<ag, 128, 0, s>>>(L.in, gains, L.in_amax, L.g, n, gain_n);
      else
        input_amax_kernel<2><<<ag, 128, 0, s>>>(L.in, gains, L.in_amax, L.g, n, gain_n);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t planar_launch(PlanarKernel& k, cudaStream_t s) {
  if (k.grid <= 0) return cudaSuccess;
  void* args[1] = {k.args};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(k.grid));
  cfg.blockDim = dim3(static_cast<unsigned>(k.block));
  cfg.dynamicSmemBytes = static_cast<size_t>(k.smem);
  cfg.stream = s;
  // The persistent CTAs wait on each other through the operand ring, so all
  // of them must be resident at once.  A cooperative launch guarantees that
  // or fails up front (cudaErrorCooperativeLaunchTooLarge, e.g. when part of
  // the GPU's SMs are held by another context), instead of a kernel whose
  // waits run out.  CTA-pair kernels rely on the cluster occupancy query of
  // planar_prepare instead.
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = k.shape == kShapePair ? 0 : 1;
  return cudaLaunchKernelExC(&cfg, k.func, args);
}

cudaError_t launch_planar(const CUtensorMap* in_map, const XeLaunch& L, int shape, cudaStream_t s) {
  static thread_local PlanarKernel k;
  const CUtensorMap* maps[1] = {in_map};
  cudaError_t e = planar_prepare(&L, maps, 1, &k, shape);
  if (e == cudaSuccess && k.grid > 0) e = planar_setup(&L, 1, s);
  if (e == cudaSuccess) e = planar_launch(k, s);
  return e;
}

}  // namespace xc
