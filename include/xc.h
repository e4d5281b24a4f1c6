/*
 * xc.h -- C ABI of the GB300 (sm_103a) X-engine.
 *
 * The X-engine is the cross-multiply stage of an FX correlator (Clark,
 * La Plante & Greenhill, Sec. 2.1): for every frequency channel f it
 * accumulates, over an integration of T samples, the self outer products of
 * the station signal vector (Eq. outer),
 *
 *     V_f[a][b] = sum_{t<T} x_f(t)[a] * conj(x_f(t)[b]),
 *
 * where a = s*P + p runs over N stations times P polarisations (dual
 * polarisation, Sec. 2.1).  V_f is Hermitian, so only the lower triangle of
 * station pairs is produced: N(N+1)/2 baselines (autocorrelations included),
 * each with all P*P polarisation products.
 *
 * LAYOUTS (all arrays dense, row-major, no padding)
 *   input   in [T][F][N][P][2]  -- corner-turned order of Sec. 4.1: station
 *           fastest, then channel, then time; {re, im} interleaved.
 *           Element type from xc_dtype: int8 (XC_CI8, Sec. 5 8-bit input),
 *           IEEE fp16 (XC_CF16) or fp32 (XC_CF32).
 *   output  out[F][N(N+1)/2][P*P][2] -- baseline k(s1,s2) = s1(s1+1)/2 + s2
 *           for 0 <= s2 <= s1 < N (the lower-triangle block order of
 *           Sec. 4.2), polarisation product index p1*P + p2, {re, im}:
 *             out[f][k(s1,s2)][p1*P+p2] = sum_t x[t][f][s1][p1] * conj(x[t][f][s2][p2]).
 *           Element type: int32 for XC_CI8 input (exact integer sums),
 *           fp32 for float input.  Diagonal baselines hold all P*P products
 *           (the yx product is the conjugate of xy).
 *
 * MEMORY AND OWNERSHIP
 *   Every data pointer passed to a call is owned by the caller.  Device
 *   pointers must be device memory of the handle's device, 16-byte aligned.
 *   The handle owns its workspace (allocated at xc_create), its streams and
 *   events, and its device status word.
 *
 * STREAMS
 *   `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Calls are stream-ordered and asynchronous: they return once
 *   the work is queued.  A handle may be used by one host thread at a time,
 *   and one call's work must finish before another call on the same handle
 *   starts on a different stream (the workspace is shared).
 *
 * ERRORS
 *   Calls return an xc_status; nothing aborts the process.  The status of
 *   the last call on this thread is kept in xc_last_error(), with a message
 *   in xc_last_error_message().  Kernel-side failures (a bounded wait that
 *   ran out) are recorded in the handle's device status word and reported
 *   by xc_synchronize() as XC_ERR_TIMEOUT.
 */
#ifndef XC_H
#define XC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xc_handle xc_handle; /* opaque, owned by the library */

/* Input sample type; samples are complex, {re, im} interleaved. */
typedef enum {
  XC_CI8 = 0,  /* two's-complement 8-bit integers (Sec. 5) */
  XC_CF16 = 1, /* IEEE half */
  XC_CF32 = 2  /* IEEE single */
} xc_dtype;

typedef enum {
  XC_OK = 0,
  XC_ERR_INVALID_ARG = 1,   /* NULL pointer, a size <= 0, npol not 1 or 2, bad option */
  XC_ERR_UNSUPPORTED = 2,   /* valid request this build does not implement */
  XC_ERR_OVERFLOW_RISK = 3, /* XC_CI8: ntime > XC_CI8_MAX_NTIME, or |x| > 16 on XC_PREC_FP8 */
  XC_ERR_ALIGNMENT = 4,     /* a device pointer not 16-byte aligned */
  XC_ERR_CUDA = 5,          /* a CUDA runtime/driver call failed */
  XC_ERR_TIMEOUT = 6,       /* a kernel's bounded wait ran out */
  XC_ERR_OOM = 7,           /* device or pinned allocation failed */
  XC_ERR_NO_DEVICE = 8      /* no CUDA device, or not an sm_103 device */
} xc_status;

/*
 * Largest ntime accepted for XC_CI8: every visibility component is a sum of
 * 2T products of magnitude <= 128*128, and must fit int32
 * (T * 2 * 127^2 < 2^31 for the symmetric range used by the paper's 8-bit
 * samples).  Longer integrations are split by the caller into several calls
 * (see XC_OPT_ACCUMULATE), with int32 range their responsibility.
 */
#define XC_CI8_MAX_NTIME 66572

/*
 * Create an engine for fixed sizes on the current CUDA device.
 *   nstation N >= 1, npol P in {1, 2}, nfreq F >= 1 (at most 65535),
 *   ntime T >= 1.
 * Allocates the workspace: a ring of tensor-core operand tiles for the
 * channels in flight (about 1.6 x 152 / (blocks per channel) + 4 channel
 * slots, at most 256 MiB; 60 MiB for N=256 x 2 pols, T=1000, sized to stay
 * in L2), plus counters and a status word.  Small arrays (N*P <= 64) have k
 * consecutive channels correlated together in one tensor-core block (k the
 * largest divisor of F with k*N*P <= 128); this is internal and changes
 * neither layouts nor results.  Returns NULL on error; the reason is in
 * xc_last_error().
 */
xc_handle* xc_create(int nstation, int npol, int nfreq, int ntime, xc_dtype in_dtype);

/*
 * One integration (Eq. outer over T samples for all F channels).
 *   in  : device, layout and type above, T*F*N*P*2 elements.
 *   out : device, F*N(N+1)/2*P*P*2 elements of int32 (XC_CI8) or fp32.
 *         Overwritten, or added to when XC_OPT_ACCUMULATE is 1 (the
 *         chunked integration of Sec. 5, Algorithm 1).
 * Stream-ordered on `stream`.
 */
xc_status xc_correlate(xc_handle* h, const void* in, void* out, void* stream);

/*
 * Adjoint of xc_correlate for float input (the paper has no adjoint; this is
 * the differentiable form of the engine).  With G the dense P*N x P*N matrix
 * holding grad_out on the stored (lower-triangle) entries and zero elsewhere,
 * H = G + G^H and y = g*x (gains, unit unless set):
 *     grad_in[t][f] = conj(g) * (H_f y_f(t)).
 *   grad_out: device fp32, layout of `out`; in: the forward's input
 *   (re-read, nothing of the forward is stored); grad_in: device fp32,
 *   layout of `in`.  The gain gradient is kept for xc_get_grad_gains.
 *   Arithmetic: with the default XC_ENGINE_TENSOR, a tcgen05 complex GEMM on
 *   split hi/lo fp16 operands (per-channel power-of-two scales, three MMAs
 *   per step: about 22 significant bits) with fp32 accumulation; with
 *   XC_ENGINE_FP32, FP32 on the CUDA cores.  Allocates an F*n*n complex
 *   workspace (and, on the tensor cores, the hi/lo operand tiles) on first
 *   use.  Needs XC_CF32 input (XC_ERR_UNSUPPORTED otherwise).
 */
xc_status xc_correlate_backward(xc_handle* h, const void* grad_out, const void* in, void* grad_in,
                                void* stream);

/*
 * Complex gains (not in the paper; the calibration term of the
 * differentiable form): one gain per (station, polarisation), applied to the
 * voltages before correlation, y = g x, so that V_ab = g_a conj(g_b) V_ab
 * of the ungained input.  Float input only (XC_CI8 handles return
 * XC_ERR_UNSUPPORTED); used by the planar tensor-core and the FP32 engines.
 *   gains: device cf32 [N][P] {re, im}, copied into the handle (synchronous);
 *          NULL clears them (unit gains).
 */
xc_status xc_set_gains(xc_handle* h, const void* gains);

/*
 * Gradient of the loss with respect to the gains from the last
 * xc_correlate_backward on `stream`: grad_g_a = sum_{f,t} conj(x_a) (H_f y)_a.
 *   grad_gains: device cf32 [N][P] (written, stream-ordered).
 */
xc_status xc_get_grad_gains(xc_handle* h, void* grad_gains, void* stream);

/* Free a handle (NULL-safe).  Synchronises the handle's own streams first. */
void xc_destroy(xc_handle* h);

/* ------------------------------------------------------------- extensions */

/* Status of the last call made on this host thread. */
xc_status xc_last_error(void);
/* Human-readable message of the last error on this host thread. */
const char* xc_last_error_message(void);
/* Static name of a status code. */
const char* xc_status_string(xc_status s);

/* Option keys for xc_set_option. */
enum {
  XC_OPT_ENGINE = 1,     /* XC_ENGINE_* below (default XC_ENGINE_TENSOR) */
  XC_OPT_ACCUMULATE = 2, /* 0: out = V (default); 1: out += V */
  XC_OPT_TIMEOUT_MS = 3, /* bound on any in-kernel wait, milliseconds (default 2000) */
  XC_OPT_PROFILE = 4,    /* 1: time every kernel with CUDA events (see xc_kernel_times) */
  XC_OPT_PRECISION = 5,  /* XC_ENGINE_TENSOR: XC_PREC_* (default FP16; 8-bit input: FP16 or FP8) */
  XC_OPT_FP64_BLOCK = 6, /* float input, XC_ENGINE_TENSOR: T_blk > 0 enables FP64 block sums */
  XC_OPT_TILE = 7,       /* XC_ENGINE_TENSOR tile shape: XC_TILE_* below (default XC_TILE_AUTO) */
  /* Test hook for the failure-detection path (XC_ENGINE_TENSOR): 1 makes the
   * operand converters skip publishing converted units, so every wait of the
   * kernel's consumers runs out after XC_OPT_TIMEOUT_MS; the kernel then
   * finishes its in-flight copies and MMAs, frees its tensor memory and
   * returns, and xc_synchronize reports XC_ERR_TIMEOUT.  Never set it outside
   * tests: the output is not computed. */
  XC_OPT_TEST_NO_PUBLISH = 100
};
/* 8-bit input takes XC_PREC_FP16 (default, exact for all int8) or
 * XC_PREC_FP8: e4m3 operands at twice the tensor rate and half the operand
 * bytes, exact when every |x| <= 16 (4-bit to 5-bit digitiser data); a
 * larger value makes xc_synchronize report XC_ERR_OVERFLOW_RISK.
 * Operand precision of float input on XC_ENGINE_TENSOR (Sec. 5 leaves the
 * precision of float voltages open).  Every
 * form scales each (channel, input) by a power of two 2^-e chosen from a
 * pre-pass over the integration (largest component of g x), so any finite
 * fp32 input is in range, and undoes it exactly in the epilogue; all forms
 * accumulate in fp32.
 *   XC_PREC_FP16: fp16 operands (11-bit significand).
 *   XC_PREC_HILO: y 2^-e = h + l with h, l fp16; V from h h^H + l h^H + h l^H
 *     (the l l^H term is dropped): about 22 significant bits, 3x the MMAs.
 *   XC_PREC_FP8 : e4m3 operands (4-bit significand), tcgen05 kind::f8f6f4.
 * FP64 block sums (XC_OPT_FP64_BLOCK = T_blk, a multiple of 64, 0 = off):
 * the fp32 accumulator of each T_blk-sample block is added into a float64
 * running sum that the handle owns (allocated on first use, 16 bytes per
 * visibility); `out` receives its fp32 rounding after every call.  With
 * XC_OPT_ACCUMULATE = 1 the running sum continues across calls (the caller's
 * `out` is not read); with 0 it restarts every call.  Setting the option to a
 * positive value zeroes the running sum (after waiting for the device). */
enum { XC_PREC_FP16 = 0, XC_PREC_HILO = 1, XC_PREC_FP8 = 2 };
/* Tile shapes of XC_ENGINE_TENSOR (results are identical; only speed differs):
 *   XC_TILE_128 : 128 x 128 complex blocks of V, one per CTA (tcgen05
 *     cta_group::1, two TMEM accumulator sets).
 *   XC_TILE_PAIR: two 128 x 128 blocks sharing a column block per pair of
 *     CTAs on two SMs, one 256 x 128 MMA per step (tcgen05 cta_group::2);
 *     each SM stages its 128 rows and half of the 128 columns.
 *   XC_TILE_WIDE: two 128 x 128 blocks sharing a row block per CTA, one
 *     128 x 256 MMA per step (N = 256; one TMEM accumulator set): a quarter
 *     fewer shared-memory and L2 operand bytes per MAC than XC_TILE_128.  Not
 *     with XC_PREC_HILO (XC_ERR_UNSUPPORTED at the call).
 *   XC_TILE_SMALL: the small-array engine (8-bit input, fp16 operands or,
 *     with XC_PREC_FP8, e4m3 operands for |x| <= 16 with the same range
 *     report; W = 2 * nstation * npol in {16, 32, 64, 128, 256}).  Each input is two
 *     real rows (re, im) of 128-row tiles; a tile holds 128 / W channels
 *     (W <= 128) or a channel spans two tiles (W = 256).  Per 16-sample step
 *     128 x 128 MMAs form the real Gram matrix of the tile rows (one MMA, or
 *     three for the lower tile blocks at W = 256), whose 2 x 2 sub-blocks
 *     give V (Sec. 4.4's diagonal blocks at twice the planar density).
 *     Operands are converted straight into shared memory: no operand ring,
 *     one read of the input.  When the channel groups
 *     (ceil(nfreq * W / 128)) are fewer than twice the SM count, T is split
 *     across CTAs and partial sums are added with integer atomics into the
 *     output, which the call zeroes first unless XC_OPT_ACCUMULATE is set.
 *     XC_ERR_UNSUPPORTED at the call for other sizes, input types or
 *     operand forms, and for batch handles.
 *   XC_TILE_AUTO: XC_TILE_SMALL where it applies (see
 *     xc_small_engine_channels; an input pointer that is not 16-byte aligned
 *     keeps the planar engine), else
 *     XC_TILE_128, the fastest planar shape measured on the Large-N
 *     workload.  A batch handle takes the shape xc_batch_tune chose
 *     (XC_TILE_AUTO restores the default). */
enum { XC_TILE_AUTO = 0, XC_TILE_128 = 1, XC_TILE_PAIR = 2, XC_TILE_WIDE = 3, XC_TILE_SMALL = 4 };
/* Engines:
 *   XC_ENGINE_TENSOR (default): one fused persistent tcgen05 kernel in
 *     planar complex form (real and imaginary fp16 operand planes, four MMAs
 *     per 16-sample step into separate real and imaginary accumulators,
 *     128 x 128 complex blocks); operands are formed once per channel into a
 *     small ring that stays in L2.
 *   XC_ENGINE_TENSOR_1CTA: fused kernel in interleaved real form
 *     (G = Y Y^T over 128 x 128 real blocks, 2x2 combine in the epilogue).
 *   XC_ENGINE_TENSOR_PAIR: the interleaved form on CTA pairs
 *     (tcgen05 cta_group::2, 256 x 256 real blocks over two SMs).
 *   XC_ENGINE_FP32: the plain FP32 CUDA-core form of the same X-engine
 *     (register tile over a shared-memory double buffer, after the paper's
 *     kernel 11, Sec. 4.4), kept as the same-GPU comparator.
 *   XC_ENGINE_TENSOR_2PASS: the same tensor-core arithmetic with operand
 *     formation as a separate pass through a full fp16 copy of the
 *     integration in device memory (allocated when this engine is selected). */
enum {
  XC_ENGINE_TENSOR = 0,
  XC_ENGINE_FP32 = 1,
  XC_ENGINE_TENSOR_2PASS = 2,
  XC_ENGINE_TENSOR_1CTA = 3,
  XC_ENGINE_TENSOR_PAIR = 4
};

xc_status xc_set_option(xc_handle* h, int key, long long value);

/*
 * Wait for `stream`, then read and clear the handle's device status word.
 * Returns XC_ERR_TIMEOUT if a kernel gave up on a bounded wait since the
 * last check, XC_ERR_CUDA on a CUDA error, else XC_OK.
 */
xc_status xc_synchronize(xc_handle* h, void* stream);

/*
 * Integrated pipeline (Sec. 5, Algorithm 1): n_integrations consecutive
 * integrations stored back to back in pinned host memory are copied to the
 * device through two staging buffers on a side copy stream, each copy
 * overlapping the correlation of the previous integration on `stream`.
 *   host_in : pinned host memory, n_integrations * (T*F*N*P*2) samples.
 *   out     : device.  With XC_OPT_ACCUMULATE = 0 it holds n_integrations
 *             outputs back to back (one per integration); with 1, a single
 *             output that all integrations are added into (Algorithm 1).
 *   host_out: optional pinned host memory of the same size as `out`; when
 *             not NULL each integration's output is also copied back on a
 *             second side stream once computed.
 * Returns once all work is queued.  The correlations and the copies out are
 * ordered after work queued earlier on `stream`, and later work on `stream`
 * after this call's copies out.  The copies in wait only for their staging
 * buffer (so they overlap an earlier call's last copies out): `host_in` must
 * already hold its data when the call is made.
 */
xc_status xc_correlate_stream(xc_handle* h, const void* host_in, int n_integrations, void* out,
                              void* host_out, void* stream);

/*
 * Kernel timing, for profiling runs (XC_OPT_PROFILE = 1).  While enabled,
 * every launch is bracketed by CUDA events recorded on the launching stream.
 * This call waits for those events and returns, per kernel class, the summed
 * device time in milliseconds and the number of launches since the last
 * reset:  index 0 = operand formation, 1 = X-engine kernel (tensor-core or
 * FP32).  ms and launches each point to 2 elements (either may be NULL).
 */
xc_status xc_kernel_times(xc_handle* h, double* ms, long long* launches, int reset);

/* Sizes (bytes) of one integration's input and output. */
size_t xc_input_bytes(const xc_handle* h);
size_t xc_output_bytes(const xc_handle* h);

/*
 * Lower-triangle block map of Sec. 4.2: block (bx, by), 0 <= bx <= by, has
 * linear index g = by(by+1)/2 + bx.  xc_tri_coords inverts it with the
 * paper's b_y = floor(-1/2 + sqrt(1/4 + 2g)), corrected to exact integers.
 * Host-side helpers (no device work), exposed for tests and schedulers.
 */
int64_t xc_tri_index(int64_t bx, int64_t by);
void xc_tri_coords(int64_t g, int64_t* bx, int64_t* by);

/*
 * Channels the tensor-core engine correlates together in one 128-input block
 * for these sizes (see xc_create): k, the largest divisor of nfreq with
 * k * nstation * npol <= 128, when nstation * npol <= 64; else 1.  Host-side,
 * no device work; returns 0 for sizes xc_create rejects (a size <= 0, npol
 * not 1 or 2, more than 2^30 rows).
 */
int xc_channels_packed(int nstation, int npol, int nfreq);

/*
 * Channels per channel group of the small-array engine (XC_TILE_SMALL) for
 * these sizes: 128 / (2 * nstation * npol) when that product is 16, 32, 64
 * or 128, 1 when it is 256 (a channel spans two 128-row tiles), else 0 (the
 * planar engine serves the sizes).  Host-side, no device
 * work.  With XC_TILE_AUTO an 8-bit, fp16-operand handle of such sizes runs
 * on the small-array engine, and xc_channels_packed does not apply to it.
 */
int xc_small_engine_channels(int nstation, int npol);

/*
 * No-allocation X-engine (the paper has no counterpart; this is a service
 * for callers of this library).
 *
 * Some callers cannot call cudaMalloc: a real-time correlator loop that
 * reserved all of its memory at start-up and may not allocate afterwards
 * (an allocation can stall the device and break a budget sized in advance),
 * an application whose device memory is entirely held by another allocator,
 * or a plug-in whose host forbids allocation inside its processing callback.
 * xc_create allocates the operand workspace, so those callers use this call
 * instead: it runs the same tensor-core kernel as xc_correlate with default
 * options (the small-array engine for 8-bit input of the sizes
 * xc_small_engine_channels accepts, else the planar engine's default tile
 * shape, FP16 operands with the same per-input power-of-two scaling for float
 * input and the same exact chunks for 8-bit input), so its visibilities are
 * identical to xc_correlate's, and it allocates nothing, neither device nor
 * host memory.
 *
 * Its scratch is a static device array of XC_NOALLOC_SCRATCH_BYTES that
 * every GPU loading the library holds until the process exits.  The planar
 * engine keeps in it the kernel's counters, the scale pre-pass maxima
 * (nfreq*npol*nstation words for float input) and as many operand-ring
 * channel slots as fit; one slot is 2*P*N rows (rounded up to 128) x ntime
 * (rounded up to 64) x 2 bytes.  A size where not even one slot fits is
 * rejected with XC_ERR_UNSUPPORTED (message in xc_last_error_message()).
 * The small-array engine uses only the status word.
 *
 *   sizes, in_dtype, in, out: as for xc_create / xc_correlate.
 *   status: optional caller-owned device int; a kernel whose bounded wait
 *           gives up ORs 1 into it (the caller zeroes it).  NULL: not reported.
 *   stream: cudaStream_t as void*; the call is stream-ordered and returns
 *           once the work is queued.
 * The first call on each device does a one-time set-up with that device
 * current: it looks up the device address of the static scratch, and with
 * CUDA's lazy module loading (the default) that also loads the library's
 * device code and creates its 64 MiB array.  Make that first call at
 * start-up, before any stream capture and outside any section that must not
 * allocate (or set CUDA_MODULE_LOADING=EAGER so the load happens when the
 * context is created).  A failed set-up is retried by the next call.  Every
 * call on a device shares the one scratch array, so calls whose work overlaps
 * on the GPU (different streams, or different host threads, without ordering
 * between them) race and corrupt each other's results: order them.
 */
#define XC_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
xc_status xc_correlate_noalloc(int nstation, int npol, int nfreq, int ntime, xc_dtype in_dtype,
                               const void* in, void* out, int* status, void* stream);

/*
 * F-engine (Sec. 2, the FX correlator): channelises each station's signal by
 * Fourier transforming blocks of nchan consecutive complex samples, and
 * writes the result corner-turned, in exactly the input layout xc_correlate
 * takes (station fastest, then channel, then block; Sec. 4.1), so the two
 * calls chain on one stream with no reordering in between:
 *
 *   out[t][f][s][p] = scale * sum_{m < nchan} in[s][p][t nchan + m] exp(-2 pi i f m / nchan)
 *
 *   in:  device, [nstation][npol][nblock * nchan] complex samples ({re, im}
 *        interleaved) of in_dtype (XC_CI8, XC_CF16 or XC_CF32): each station
 *        and polarisation's sample stream, contiguous in time.
 *   out: device, [nblock][nchan][nstation][npol] complex of out_dtype; it is
 *        xc_correlate's input for nfreq = nchan, ntime = nblock.
 *        XC_CF16 / XC_CF32: the value above, rounded to the type.
 *        XC_CI8: requantised to 8 bits, each component rounded to the nearest
 *        integer (ties to even) and saturated at +-127, the form the 8-bit
 *        X-engine correlates exactly (Sec. 5: 8-bit X-engine input).  The
 *        rounding decision is taken on the fp32 value, so a component within
 *        about 1e-6 relative of a half-integer may round the other way than
 *        in exact arithmetic.
 *   nchan: a power of two from 16 to 4096 (else XC_ERR_UNSUPPORTED); channel
 *        f is DFT bin f (DC first, not re-centred).
 *   scale: real factor on every output.  The paper leaves the normalisation
 *        open; 1/sqrt(nchan) keeps the transform unitary, and with fp16
 *        output it keeps 8-bit input in range (|out| <= 128 sqrt(2 nchan)).
 *   stream: cudaStream_t as void*; stream-ordered, returns once queued.
 * Buffers are caller-owned and 16-byte aligned (XC_ERR_ALIGNMENT); NULL or
 * sizes <= 0 give XC_ERR_INVALID_ARG; more than 65535 * 8192 / nchan
 * station-polarisations (65535 * 16384 / nchan for XC_CI8 output) give
 * XC_ERR_UNSUPPORTED.  Arithmetic is fp32 throughout (radix-16 FFT), about
 * 1e-6 relative before the output rounding.
 */
xc_status xc_channelize(const void* in, xc_dtype in_dtype, int nstation, int npol, int nchan,
                        int nblock, float scale, void* out, xc_dtype out_dtype, void* stream);

/*
 * Polyphase F-engine (not in the paper; the usual F-engine filter in front
 * of the DFT): as xc_channelize, but each output block is the DFT of ntaps
 * consecutive input blocks weighted by real taps,
 *
 *   out[t][f][s][p] = scale * sum_m exp(-2 pi i f m / nchan)
 *                             * sum_{q < ntaps} taps[q][m] in[s][p][(t + q) nchan + m]
 *
 * for the nblock - ntaps + 1 output blocks (out holds that many).
 *   taps: device, [ntaps][nchan] float32, 16-byte aligned (e.g. a windowed
 *         sinc prototype of ntaps * nchan coefficients); NULL is
 *         XC_ERR_INVALID_ARG.  ntaps from 1 to min(64, nblock).
 * Everything else as xc_channelize; one unit tap gives xc_channelize.
 */
xc_status xc_channelize_pfb(const void* in, xc_dtype in_dtype, int nstation, int npol, int nchan,
                            int nblock, const float* taps, int ntaps, float scale, void* out,
                            xc_dtype out_dtype, void* stream);

/*
 * Batched form: many subarrays of uneven size correlated by ONE persistent
 * tensor-core launch (Sec. 4.2's channel-major block raster continued from
 * one subarray to the next), replayed from a CUDA graph captured on first
 * use.  For an array split into independent subarrays, or many small arrays
 * sharing one GPU (the small-N regime Sec. 6 discusses: small subarrays alone
 * leave most SMs idle, together they fill the GPU).
 *
 * xc_batch_create: nsub in [1, XC_BATCH_MAX_SUB]; nstation / nfreq / ntime:
 *   host arrays of nsub sizes (each as for xc_create); one npol and one input
 *   type for all (XC_CI8 only: bit-exact int32 visibilities).  Returns NULL
 *   on error (xc_last_error()).  The handle owns every subarray's operand
 *   ring and counters; free it with xc_destroy.  xc_correlate on a batch
 *   handle returns XC_ERR_UNSUPPORTED; xc_set_option accepts ACCUMULATE,
 *   TIMEOUT_MS and PROFILE.
 * xc_batch_correlate: in[i] / out[i] are device pointers (16-byte aligned)
 *   in the layouts of xc_correlate for subarray i; arrays of nsub pointers
 *   in host memory, read during the call.  Stream-ordered; one graph launch
 *   per call.  Calls on one handle must be ordered with each other (they
 *   share the rings and counters).
 * xc_batch_tune: times each candidate schedule on the given buffers with
 *   `reps` timed launches each (after one warm-up), keeps the fastest for
 *   later calls, and writes the mean milliseconds of every candidate to
 *   ms[XC_BATCH_CANDIDATES] (-1 for candidates not timed) and the winner to
 *   *best (either may be NULL).  Candidate c (the tile shapes of XC_OPT_TILE
 *   and the launch's schedule; every candidate computes the same result):
 *     c % 3        work-list order: as given, largest subarray first,
 *                  smallest first;
 *     (c / 3) % 2  operand-ring depth: 1x, 2x;
 *     (c / 6) % 2  channel packing of subarrays with nstation*npol <= 64
 *                  (see xc_create): on, off (only tried when some subarray
 *                  packs);
 *     c / 12       tile shape: 128 x 128, CTA pair, 128 x 256.
 *   With a tuning file set (xc_batch_set_cache) that holds this batch's
 *   choice, the choice is applied without timing (ms[c] gets its recorded
 *   time); otherwise the winner is appended to the file.  Synchronises
 *   `stream`.
 * xc_batch_set_cache: names a tuning file (NULL or "" for none) for this
 *   handle's xc_batch_tune; lines are "<key>\t<candidate>\t<ms>", the last
 *   line of a key counts, and the file is meant for one GPU model.
 * xc_batch_cache_key: the key of a batch (the library version, npol, input
 *   type and every subarray's nstation:nfreq:ntime in order) into buf;
 *   returns its length, or -1 if it does not fit or an argument is bad.
 * xc_batch_cache_lookup: the candidate a tuning file records for a key, or
 *   -1 (no file, no such line).  Host-side helpers, no device work.
 */
#define XC_BATCH_MAX_SUB 8
#define XC_BATCH_CANDIDATES 36
xc_handle* xc_batch_create(int nsub, const int* nstation, const int* nfreq, const int* ntime,
                           int npol, xc_dtype in_dtype);
xc_status xc_batch_correlate(xc_handle* h, const void* const* in, void* const* out, void* stream);
xc_status xc_batch_tune(xc_handle* h, const void* const* in, void* const* out, void* stream,
                        int reps, double* ms, int* best);
xc_status xc_batch_set_cache(xc_handle* h, const char* path);
int xc_batch_cache_key(int nsub, const int* nstation, const int* nfreq, const int* ntime, int npol,
                       xc_dtype in_dtype, char* buf, size_t len);
int xc_batch_cache_lookup(const char* path, const char* key);

/* Library version string. */
const char* xc_version(void);

/*
 * Diagnostics (not in the paper): the FP32 CUDA-core peak that the plain
 * FP32 X-engine's fraction of peak is quoted against, measured rather than
 * computed from a nominal clock.  Launches, on `stream`, 4 CTAs of 512
 * threads per SM of the current device, each thread running 8 independent
 * fused multiply-add chains for 16 * iterations rounds; *flops receives the
 * floating-point operations launched (2 per FFMA).  The caller times the
 * launch (CUDA events on `stream`).  sink: device float[4 * SM count],
 * written only in a case that cannot occur (it keeps the chains live).
 */
xc_status xc_fp32_peak_probe(long long iterations, void* sink, void* stream, long long* flops);

#ifdef __cplusplus
}
#endif

#endif /* XC_H */
