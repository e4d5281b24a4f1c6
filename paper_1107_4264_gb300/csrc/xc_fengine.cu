// F-engine of the FX correlator (Sec. 2): each station's signal is Fourier
// transformed in blocks of F consecutive complex samples,
//     X_t(f) = scale * sum_{m<F} x(t F + m) exp(-2 pi i f m / F),
// optionally after a polyphase front end (taps h[p][m] over ntaps
// consecutive blocks: x(t F + m) becomes sum_p h[p][m] x((t + p) F + m)),
// and the result is written in the X-engine's input order [T][F][N][P]
// (station fastest, then channel, then block: the corner turn of Sec. 2,
// in the ordering of Sec. 4.1).  Input is station-major [N][P][T F]: the
// F-engine is independent per station, the X-engine per channel.
//
// One CTA transforms G = 8192 / F (or 16384 / F) blocks (G consecutive inputs
// a = s P + p of one block index t) in shared memory and writes them
// corner-turned, so each output channel f receives G consecutive inputs in one
// contiguous run.
//
// Each transform is a Stockham radix-16 FFT (a radix-2/4/8 first pass when
// log2 F is not a multiple of 4, so that only radix-16 passes carry
// twiddles): a team of F / 16 threads, each holding 16 points in registers
// per pass.  Pass p combines 16 sub-transforms of length
// L into one of length 16 L:
//     A'[i][q L + k] = sum_r W_16^{q r} (W_{16 L}^{k r} A[i + (F / 16 L) r][k]),
// read at flat index j + r F / 16 and written at (j - k) 16 + k + q L, where
// j = i L + k.  The 16-point DFTs run in registers as 4 x 4 (Cooley-Tukey)
// with constant twiddles; the pass twiddles W_{16 L}^{k r} come from one
// sincospif per butterfly and a product tree of its powers.  Shared-memory
// rows are padded (one float2 per 16, and a row stride chosen per F) so that
// the strided pass writes and the corner-turn reads avoid bank conflicts.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "xc_launch.h"

namespace xc {
namespace {

constexpr int kPts = 16;  // points per thread per pass
// A CTA holds 2^LOGP points (G = 2^LOGP / F transforms, 2^LOGP / 16 threads):
// 2^13 with two CTAs per SM, or 2^14 with one, whose longer corner-turn runs
// (G consecutive inputs per channel) fill whole 32-byte sectors for 8-bit output.

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }  // -i a

// W_16^e = exp(-2 pi i e / 16); e is a compile-time constant after unrolling.
__device__ __forceinline__ float2 w16(int e) {
  // cos(r pi / 8) for r = 0..4
  const float c0 = 1.f, c1 = 0.92387953251128674f, c2 = 0.70710678118654752f,
              c3 = 0.38268343236508977f, c4 = 0.f;
  const int q = (e & 15) >> 2, r = e & 3;
  const float cr = r == 0 ? c0 : r == 1 ? c1 : r == 2 ? c2 : c3;  // cos(r pi/8)
  const float sr = r == 0 ? c4 : r == 1 ? c3 : r == 2 ? c2 : c1;  // sin(r pi/8)
  // rotate (cr, sr) by q quarter turns: cos and sin of (4 q + r) pi / 8
  const float co = q == 0 ? cr : q == 1 ? -sr : q == 2 ? -cr : sr;
  const float si = q == 0 ? sr : q == 1 ? cr : q == 2 ? -sr : -cr;
  return make_float2(co, -si);
}

// X[q] = sum_r x[r] W_R^{q r}, natural order in and out.
template <int R>
__device__ __forceinline__ void dft(const float2* x, float2* X);

template <>
__device__ __forceinline__ void dft<2>(const float2* x, float2* X) {
  X[0] = cadd(x[0], x[1]);
  X[1] = csub(x[0], x[1]);
}

template <>
__device__ __forceinline__ void dft<4>(const float2* x, float2* X) {
  const float2 t0 = cadd(x[0], x[2]), t1 = csub(x[0], x[2]);
  const float2 t2 = cadd(x[1], x[3]), t3 = mul_mi(csub(x[1], x[3]));
  X[0] = cadd(t0, t2);
  X[2] = csub(t0, t2);
  X[1] = cadd(t1, t3);
  X[3] = csub(t1, t3);
}

// 8 = 4 (inner, over n1 of x[2 n1 + n2]) x 2 (outer, over n2).
template <>
__device__ __forceinline__ void dft<8>(const float2* x, float2* X) {
  float2 a[4], b[4], A[4], B[4];
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
    a[n1] = x[2 * n1];
    b[n1] = x[2 * n1 + 1];
  }
  dft<4>(a, A);
  dft<4>(b, B);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    const float2 bt = cmul(B[k1], w16(2 * k1));  // W_8^{k1}
    X[k1] = cadd(A[k1], bt);
    X[k1 + 4] = csub(A[k1], bt);
  }
}

// 16 = 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2.
template <>
__device__ __forceinline__ void dft<16>(const float2* x, float2* X) {
  float2 Y[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    float2 a[4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) a[n1] = x[4 * n1 + n2];
    dft<4>(a, Y[n2]);
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1)
      if (n2 * k1 == 4) {
        Y[n2][k1] = mul_mi(Y[n2][k1]);  // W_16^4 = -i
      } else if (n2 > 0) {
        Y[n2][k1] = cmul(Y[n2][k1], w16(n2 * k1));
      }
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 c[4], C[4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) c[n2] = Y[n2][k1];
    dft<4>(c, C);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) X[k1 + 4 * k2] = C[k2];
  }
}

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

// float2 elements between the padded rows of consecutive transforms: at least
// F + F / 16, congruent mod 16 to 16 / min(G, 16), so that a warp's
// corner-turn reads (G rows, 32 / G bins each) spread over all banks.
__host__ __device__ __forceinline__ int row_stride(int F, int G) {
  const int target = 16 / (G < 16 ? G : 16);
  const int base = F + F / 16;
  return base + (((target - base) % 16) + 16) % 16;
}

template <int DT>
__device__ __forceinline__ float2 load_sample(const void* in, int64_t i) {
  if constexpr (DT == 0) {
    const char2 c = static_cast<const char2*>(in)[i];
    return make_float2(static_cast<float>(c.x), static_cast<float>(c.y));
  } else if constexpr (DT == 1) {
    return __half22float2(static_cast<const __half2*>(in)[i]);
  } else {
    return static_cast<const float2*>(in)[i];
  }
}

// Second half of a Stockham pass of radix R combining sub-transforms of
// length L into R L, for a transform of length F held in buf (padded): this
// thread's butterflies j, j + F/16, ... (C = 16 / R of them) have their
// inputs in v; twiddle (L > 1), DFT, store.
template <int R, int F, int L>
__device__ __forceinline__ void pass_body(float2 (&v)[kPts], float2* buf, int j) {
  constexpr int tpf = F / kPts, C = kPts / R, Lp = L * R;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int jj = j + c * tpf;
    const int k = jj & (L - 1);
    if constexpr (L > 1) {
      float s, co;
      sincospif(static_cast<float>(k) * (2.f / static_cast<float>(Lp)), &s, &co);
      float2 pw[R];  // pw[r] = W_{R L}^{k r}, as a product tree (depth log2 R)
      pw[1] = make_float2(co, -s);
#pragma unroll
      for (int r = 2; r < R; ++r) pw[r] = cmul(pw[r >> 1], pw[r - (r >> 1)]);
#pragma unroll
      for (int r = 1; r < R; ++r) v[c * R + r] = cmul(v[c * R + r], pw[r]);
    }
    float2 X[R];
    dft<R>(v + c * R, X);
    const int o = (jj - k) * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if constexpr (L % 16 == 0) {
        buf[pad16(o) + q * (L + L / 16)] = X[q];  // q L is a multiple of 16
      } else {
        buf[pad16(o + q * L)] = X[q];
      }
    }
  }
  __syncthreads();
}

// A pass after the first: inputs from shared memory.
template <int R, int F, int L>
__device__ __forceinline__ void pass_smem(float2 (&v)[kPts], float2* buf, int j) {
  constexpr int tpf = F / kPts, C = kPts / R, S = F / R;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int jj = j + c * tpf;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if constexpr (S % 16 == 0) {
        v[c * R + r] = buf[pad16(jj) + r * (S + S / 16)];  // r S is a multiple of 16
      } else {
        v[c * R + r] = buf[pad16(jj + r * S)];
      }
    }
  }
  __syncthreads();  // every thread has read its inputs before any output overwrites them
  pass_body<R, F, L>(v, buf, j);
}

// Radix-16 passes from sub-transform length L up to F.
template <int F, int L>
__device__ __forceinline__ void later_passes(float2 (&v)[kPts], float2* buf, int j) {
  if constexpr (L < F) {
    pass_smem<16, F, L>(v, buf, j);
    later_passes<F, L * 16>(v, buf, j);
  }
}

// in [n][T F] complex (in_dt: 0 int8, 1 fp16, 2 fp32), out [T][F][n] complex
// (out_dt: 0 int8 requantised, 1 fp16, 2 fp32), F = 2^LOGF; T input blocks.
// taps (NULL: none) is [ntaps][F] real: output block t transforms
// sum_p taps[p][m] x((t + p) F + m).  grid = (T - ntaps + 1, ceil(n / G)),
// block = 2^LOGP / 16 threads, dynamic shared memory G row_stride(F, G) float2.
template <int LOGF, int LOGP>
__global__ void __launch_bounds__((1 << LOGP) / kPts, (1 << 14) >> LOGP)
    fengine_kernel(const void* __restrict__ in, void* __restrict__ out, int n, int T, float scale,
                   int in_dt, int out_dt, const float* __restrict__ taps, int ntaps) {
  constexpr int F = 1 << LOGF;
  constexpr int G = (1 << LOGP) / F, LOGG = LOGP - LOGF;
  constexpr int kFThreads = (1 << LOGP) / kPts;
  constexpr int tpf = F / kPts;
  extern __shared__ float2 fsm[];
  const int stride = row_stride(F, G);
  const int g = threadIdx.x >> (LOGF - 4);  // transform of this thread within the CTA
  const int j = threadIdx.x & (tpf - 1);
  const int t = blockIdx.x;
  const int a0 = blockIdx.y * G;
  const int a = a0 + g;
  float2* buf = fsm + g * stride;

  // First pass (L = 1, no twiddles) takes the remainder radix R0 = F / 16^k,
  // so that every twiddled pass is radix 16; inputs straight from global:
  // butterfly jj = j + c F/16 reads x[jj + r F / R0].
  constexpr int R0 = (LOGF % 4 == 0) ? 16 : (1 << (LOGF % 4));
  float2 v[kPts];
  {
    const int64_t base = (static_cast<int64_t>(a) * T + t) * F + j;
    auto at = [](int e) { return (e / R0) * tpf + (e % R0) * (F / R0); };  // e = c R0 + r
    if (a >= n) {
#pragma unroll
      for (int e = 0; e < kPts; ++e) v[e] = make_float2(0.f, 0.f);
    } else if (taps) {
      // Polyphase front end: tap-weighted sum of ntaps consecutive blocks;
      // per tap, eight taps and eight samples are loaded before they are used.
#pragma unroll
      for (int e = 0; e < kPts; ++e) v[e] = make_float2(0.f, 0.f);
      auto accumulate = [&](auto dt) {
        constexpr int DT = decltype(dt)::value;
#pragma unroll 1
        for (int p = 0; p < ntaps; ++p) {
          const float* hp = taps + static_cast<int64_t>(p) * F + j;
          const int64_t bp = base + static_cast<int64_t>(p) * F;
#pragma unroll
          for (int e0 = 0; e0 < kPts; e0 += 8) {
            float h[8];
            float2 xs[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              h[e] = __ldg(hp + at(e0 + e));
              xs[e] = load_sample<DT>(in, bp + at(e0 + e));
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              v[e0 + e].x = fmaf(h[e], xs[e].x, v[e0 + e].x);
              v[e0 + e].y = fmaf(h[e], xs[e].y, v[e0 + e].y);
            }
          }
        }
      };
      if (in_dt == 0) {
        accumulate(std::integral_constant<int, 0>());
      } else if (in_dt == 1) {
        accumulate(std::integral_constant<int, 1>());
      } else {
        accumulate(std::integral_constant<int, 2>());
      }
    } else if (in_dt == 0) {
#pragma unroll
      for (int e = 0; e < kPts; ++e) v[e] = load_sample<0>(in, base + at(e));
    } else if (in_dt == 1) {
#pragma unroll
      for (int e = 0; e < kPts; ++e) v[e] = load_sample<1>(in, base + at(e));
    } else {
#pragma unroll
      for (int e = 0; e < kPts; ++e) v[e] = load_sample<2>(in, base + at(e));
    }
    pass_body<R0, F, 1>(v, buf, j);
  }
  later_passes<F, R0>(v, buf, j);

  // Corner turn: out[t][f][a0 .. a0 + G) from the G transforms' bins f.
  // Thread (gg, f0) writes bins f0 + i F/16, i < 16.
  const int gg = threadIdx.x & (G - 1);
  if (a0 + gg >= n) return;
  constexpr int step = kFThreads >> LOGG;  // = F / 16
  const int f0 = threadIdx.x >> LOGG;
  const float2* src = fsm + gg * stride;
  const int64_t o0 = static_cast<int64_t>(t) * F * n + static_cast<int64_t>(f0) * n + a0 + gg;
  const int64_t ostep = static_cast<int64_t>(step) * n;
#pragma unroll
  for (int i = 0; i < kPts; ++i) {
    float2 X;
    if constexpr (step % 16 == 0) {
      X = src[pad16(f0) + i * (step + step / 16)];
    } else {
      X = src[pad16(f0 + i * step)];
    }
    const int64_t o = o0 + i * ostep;
    if (out_dt == 1) {
      static_cast<__half2*>(out)[o] = __floats2half2_rn(X.x * scale, X.y * scale);
    } else if (out_dt == 0) {
      // Requantised to 8 bits: nearest integer (ties to even), saturated at +-127.
      const int qr = max(-127, min(127, __float2int_rn(X.x * scale)));
      const int qi = max(-127, min(127, __float2int_rn(X.y * scale)));
      static_cast<char2*>(out)[o] = make_char2(static_cast<signed char>(qr), static_cast<signed char>(qi));
    } else {
      static_cast<float2*>(out)[o] = make_float2(X.x * scale, X.y * scale);
    }
  }
}

template <int LOGF, int LOGP>
cudaError_t launch_fp(const void* in, int in_dt, void* out, int out_dt, int n, int T, float scale,
                      const float* taps, int ntaps, cudaStream_t s) {
  constexpr int F = 1 << LOGF, G = (1 << LOGP) / F;
  const size_t smem = static_cast<size_t>(G) * row_stride(F, G) * sizeof(float2);
  if ((n + G - 1) / G > 65535) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(fengine_kernel<LOGF, LOGP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const dim3 grid(static_cast<unsigned>(T - ntaps + 1), static_cast<unsigned>((n + G - 1) / G));
  fengine_kernel<LOGF, LOGP><<<grid, (1 << LOGP) / kPts, smem, s>>>(in, out, n, T, scale, in_dt,
                                                                    out_dt, taps, ntaps);
  return cudaGetLastError();
}

// CTA size by output type: 8-bit codes (2 bytes per complex value) take the
// larger CTA, whose corner-turn runs cover whole 32-byte sectors.
template <int LOGF>
cudaError_t launch_f(const void* in, int in_dt, void* out, int out_dt, int n, int T, float scale,
                     const float* taps, int ntaps, cudaStream_t s) {
  if (out_dt == 0) return launch_fp<LOGF, 14>(in, in_dt, out, out_dt, n, T, scale, taps, ntaps, s);
  return launch_fp<LOGF, 13>(in, in_dt, out, out_dt, n, T, scale, taps, ntaps, s);
}

}  // namespace

cudaError_t launch_fengine(const void* in, int in_dtype, void* out, int out_dtype, int n, int F,
                           int T, float scale, const float* taps, int ntaps, cudaStream_t s) {
  if (n <= 0 || T <= 0 || in_dtype < 0 || in_dtype > 2 || out_dtype < 0 || out_dtype > 2 ||
      ntaps < 1 || ntaps > T || (!taps && ntaps != 1))
    return cudaErrorInvalidValue;
  switch (F) {
    case 16: return launch_f<4>(in, in_dtype, out, out_dtype, n, T, scale, taps, ntaps, s);
    case 32: return launch_f<5>(in, in_dtype, out, out_dtype, n, T, scale, taps, ntaps, s);
    case 64: return launch_f<6>(in, in_dtype, out, out_dtype, n, T, scale, taps, ntaps, s);
    case 128: return launch_f<7>(in, in_dtype, out, out_dtype, n, T, scale, taps, ntaps, s);
    case 256: return launch_f<8>(in, in_dtype, out, out_dtype, n, T, scale, taps, ntaps, s);
    case 512: return launch_f<9>(in, in_dtype, out, out_dtype, n, T, scale, taps, ntaps, s);
    case 1024: return launch_f<10>(in, in_dtype, out, out_dtype, n, T, scale, taps, ntaps, s);
    case 2048: return launch_f<11>(in, in_dtype, out, out_dtype, n, T, scale, taps, ntaps, s);
    case 4096: return launch_f<12>(in, in_dtype, out, out_dtype, n, T, scale, taps, ntaps, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace xc
