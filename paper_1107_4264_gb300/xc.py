"""Python binding of the C ABI in ``include/xc.h`` (ctypes; marshalling only).

The functions carry the C names (``xc_create``, ``xc_correlate``, ...) and
take raw pointers; :class:`Correlator` adds torch-tensor conveniences
(allocation of outputs, the current CUDA stream) on top.  Every step of the
X-engine runs in the library's CUDA kernels: there is no Python or CPU
fallback, and a missing library raises immediately.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libxc.so")

XC_CI8, XC_CF16, XC_CF32 = 0, 1, 2
XC_OK = 0
XC_ERR_INVALID_ARG = 1
XC_ERR_UNSUPPORTED = 2
XC_ERR_OVERFLOW_RISK = 3
XC_ERR_ALIGNMENT = 4
XC_ERR_CUDA = 5
XC_ERR_TIMEOUT = 6
XC_ERR_OOM = 7
XC_ERR_NO_DEVICE = 8
XC_OPT_ENGINE, XC_OPT_ACCUMULATE, XC_OPT_TIMEOUT_MS, XC_OPT_PROFILE = 1, 2, 3, 4
XC_OPT_PRECISION, XC_OPT_FP64_BLOCK, XC_OPT_TILE = 5, 6, 7
XC_TILE_AUTO, XC_TILE_128, XC_TILE_PAIR, XC_TILE_WIDE, XC_TILE_SMALL = 0, 1, 2, 3, 4
XC_OPT_TEST_NO_PUBLISH = 100
XC_PREC_FP16, XC_PREC_HILO, XC_PREC_FP8 = 0, 1, 2
(XC_ENGINE_TENSOR, XC_ENGINE_FP32, XC_ENGINE_TENSOR_2PASS, XC_ENGINE_TENSOR_1CTA,
 XC_ENGINE_TENSOR_PAIR) = 0, 1, 2, 3, 4
XC_CI8_MAX_NTIME = 66572
XC_BATCH_MAX_SUB = 8
XC_BATCH_CANDIDATES = 36

# Symbols declared in include/xc.h (checked by the tests against the header).
EXPORTS = [
    "xc_create", "xc_correlate", "xc_correlate_backward", "xc_destroy", "xc_last_error",
    "xc_last_error_message", "xc_status_string", "xc_set_option", "xc_synchronize",
    "xc_correlate_stream", "xc_input_bytes", "xc_output_bytes", "xc_tri_index", "xc_tri_coords",
    "xc_version", "xc_kernel_times", "xc_correlate_noalloc", "xc_set_gains", "xc_get_grad_gains",
    "xc_batch_create", "xc_batch_correlate", "xc_batch_tune", "xc_channelize",
    "xc_channelize_pfb", "xc_channels_packed", "xc_small_engine_channels", "xc_fp32_peak_probe", "xc_batch_set_cache",
    "xc_batch_cache_key", "xc_batch_cache_lookup",
]

_lib: Optional[ctypes.CDLL] = None


class XcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (status_string(status) if _lib else status, message))
        self.status = status


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    sig = {
        "xc_create": ([i32, i32, i32, i32, i32], vp),
        "xc_correlate": ([vp, vp, vp, vp], i32),
        "xc_correlate_backward": ([vp, vp, vp, vp, vp], i32),
        "xc_destroy": ([vp], None),
        "xc_last_error": ([], i32),
        "xc_last_error_message": ([], ctypes.c_char_p),
        "xc_status_string": ([i32], ctypes.c_char_p),
        "xc_set_option": ([vp, i32, ctypes.c_longlong], i32),
        "xc_synchronize": ([vp, vp], i32),
        "xc_correlate_stream": ([vp, vp, i32, vp, vp, vp], i32),
        "xc_input_bytes": ([vp], sz),
        "xc_output_bytes": ([vp], sz),
        "xc_tri_index": ([i64, i64], i64),
        "xc_tri_coords": ([i64, ctypes.POINTER(i64), ctypes.POINTER(i64)], None),
        "xc_version": ([], ctypes.c_char_p),
        "xc_kernel_times": ([vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                             i32], i32),
        "xc_correlate_noalloc": ([i32, i32, i32, i32, i32, vp, vp, vp, vp], i32),
        "xc_set_gains": ([vp, vp], i32),
        "xc_get_grad_gains": ([vp, vp, vp], i32),
        "xc_batch_create": ([i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                             i32, i32], vp),
        "xc_batch_correlate": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp], i32),
        "xc_batch_tune": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, i32,
                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)], i32),
        "xc_channelize": ([vp, i32, i32, i32, i32, i32, ctypes.c_float, vp, i32, vp], i32),
        "xc_channelize_pfb": ([vp, i32, i32, i32, i32, i32, vp, i32, ctypes.c_float, vp, i32, vp], i32),
        "xc_channels_packed": ([i32, i32, i32], i32),
        "xc_small_engine_channels": ([i32, i32], i32),
        "xc_fp32_peak_probe": ([ctypes.c_longlong, vp, vp, ctypes.POINTER(ctypes.c_longlong)], i32),
        "xc_batch_set_cache": ([vp, ctypes.c_char_p], i32),
        "xc_batch_cache_key": ([i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32), i32, i32,
                                ctypes.c_char_p, sz], i32),
        "xc_batch_cache_lookup": ([ctypes.c_char_p, ctypes.c_char_p], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libxc.so (built by ``__graft_entry__.build()``).  Raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libxc.so is not built (%s); run __graft_entry__.build()" % path)
        _lib = _bind(ctypes.CDLL(path))
    return _lib


def _check(status: int) -> int:
    if status != XC_OK:
        raise XcError(status, xc_last_error_message())
    return status


# ------------------------------------------------------------ C-named calls

def xc_create(nstation: int, npol: int, nfreq: int, ntime: int, in_dtype: int) -> int:
    h = load().xc_create(nstation, npol, nfreq, ntime, in_dtype)
    if not h:
        raise XcError(xc_last_error(), xc_last_error_message())
    return h


def xc_correlate(h: int, in_ptr: int, out_ptr: int, stream: int = 0) -> int:
    return load().xc_correlate(h, in_ptr, out_ptr, stream)


def xc_correlate_backward(h: int, grad_out_ptr: int, in_ptr: int, grad_in_ptr: int,
                          stream: int = 0) -> int:
    return load().xc_correlate_backward(h, grad_out_ptr, in_ptr, grad_in_ptr, stream)


def xc_destroy(h: int) -> None:
    load().xc_destroy(h)


def xc_last_error() -> int:
    return load().xc_last_error()


def xc_last_error_message() -> str:
    return load().xc_last_error_message().decode()


def status_string(s: int) -> str:
    return load().xc_status_string(s).decode()


xc_status_string = status_string


def xc_set_option(h: int, key: int, value: int) -> int:
    return load().xc_set_option(h, key, value)


def xc_synchronize(h: int, stream: int = 0) -> int:
    return load().xc_synchronize(h, stream)


def xc_correlate_stream(h: int, host_in_ptr: int, n_integrations: int, out_ptr: int,
                        host_out_ptr: int = 0, stream: int = 0) -> int:
    return load().xc_correlate_stream(h, host_in_ptr, n_integrations, out_ptr, host_out_ptr,
                                      stream)


def xc_input_bytes(h: int) -> int:
    return load().xc_input_bytes(h)


def xc_output_bytes(h: int) -> int:
    return load().xc_output_bytes(h)


def xc_tri_index(bx: int, by: int) -> int:
    return load().xc_tri_index(bx, by)


def xc_tri_coords(g: int):
    bx, by = ctypes.c_int64(), ctypes.c_int64()
    load().xc_tri_coords(g, ctypes.byref(bx), ctypes.byref(by))
    return bx.value, by.value


def xc_kernel_times(h: int, reset: bool = True):
    """((formation_ms, main_ms), (formation_launches, main_launches))."""
    ms = (ctypes.c_double * 2)()
    n = (ctypes.c_longlong * 2)()
    _check(load().xc_kernel_times(h, ms, n, int(reset)))
    return (ms[0], ms[1]), (n[0], n[1])


def xc_set_gains(h: int, gains_ptr: int) -> int:
    return load().xc_set_gains(h, gains_ptr or None)


def xc_get_grad_gains(h: int, grad_ptr: int, stream: int = 0) -> int:
    return load().xc_get_grad_gains(h, grad_ptr, stream)


XC_NOALLOC_SCRATCH_BYTES = 64 * 1024 * 1024


def xc_correlate_noalloc(nstation: int, npol: int, nfreq: int, ntime: int, in_dtype: int,
                         in_ptr: int, out_ptr: int, status_ptr: int = 0, stream: int = 0) -> int:
    """The X-engine without any allocation, for callers that may not allocate
    device memory (they cannot create a handle, which allocates a workspace):
    scratch is the library's static device array of XC_NOALLOC_SCRATCH_BYTES.
    Same result as xc_correlate; calls that overlap on the GPU race."""
    return load().xc_correlate_noalloc(nstation, npol, nfreq, ntime, in_dtype, in_ptr, out_ptr,
                                       status_ptr or None, stream)


def xc_channelize(in_ptr: int, in_dtype: int, nstation: int, npol: int, nchan: int, nblock: int,
                  scale: float, out_ptr: int, out_dtype: int, stream: int = 0) -> int:
    return load().xc_channelize(in_ptr, in_dtype, nstation, npol, nchan, nblock, scale, out_ptr,
                                out_dtype, stream)


def xc_channelize_pfb(in_ptr: int, in_dtype: int, nstation: int, npol: int, nchan: int,
                      nblock: int, taps_ptr: int, ntaps: int, scale: float, out_ptr: int,
                      out_dtype: int, stream: int = 0) -> int:
    return load().xc_channelize_pfb(in_ptr, in_dtype, nstation, npol, nchan, nblock, taps_ptr,
                                    ntaps, scale, out_ptr, out_dtype, stream)


def xc_version() -> str:
    return load().xc_version().decode()


def xc_fp32_peak_probe(iterations: int, sink_ptr: int, stream: int = 0) -> int:
    """Launch the FP32 FFMA peak probe; returns the flops launched (time it with
    CUDA events on `stream`)."""
    flops = ctypes.c_longlong(0)
    _check(load().xc_fp32_peak_probe(iterations, sink_ptr, stream, ctypes.byref(flops)))
    return flops.value


# ------------------------------------------------------ torch convenience

_DTYPES = {"int8": XC_CI8, "float16": XC_CF16, "float32": XC_CF32}


class Correlator:
    """One engine for fixed (nstation, npol, nfreq, ntime, dtype).

    Tensors: input ``[T][F][N][P][2]`` (int8 / float16 / float32) on the
    handle's CUDA device; output ``[F][N(N+1)/2][P*P][2]`` int32 (int8 input)
    or float32.
    """

    def __init__(self, nstation: int, npol: int, nfreq: int, ntime: int, dtype: str = "int8",
                 engine: int = XC_ENGINE_TENSOR, accumulate: bool = False,
                 timeout_ms: Optional[int] = None, precision: int = XC_PREC_FP16,
                 fp64_block: int = 0, tile: int = XC_TILE_AUTO):
        import torch
        self._torch = torch
        self.nstation, self.npol, self.nfreq, self.ntime = nstation, npol, nfreq, ntime
        self.dtype = dtype
        self.h = xc_create(nstation, npol, nfreq, ntime, _DTYPES[dtype])
        self.set_option(XC_OPT_ENGINE, engine)
        self.set_option(XC_OPT_ACCUMULATE, int(accumulate))
        if timeout_ms is not None:
            self.set_option(XC_OPT_TIMEOUT_MS, timeout_ms)
        if precision != XC_PREC_FP16:
            self.set_option(XC_OPT_PRECISION, precision)
        if fp64_block:
            self.set_option(XC_OPT_FP64_BLOCK, fp64_block)
        if tile != XC_TILE_AUTO:
            self.set_option(XC_OPT_TILE, tile)

    @property
    def in_shape(self):
        return (self.ntime, self.nfreq, self.nstation, self.npol, 2)

    @property
    def out_shape(self):
        nb = self.nstation * (self.nstation + 1) // 2
        return (self.nfreq, nb, self.npol * self.npol, 2)

    @property
    def out_dtype(self):
        return self._torch.int32 if self.dtype == "int8" else self._torch.float32

    def set_option(self, key: int, value: int) -> None:
        _check(xc_set_option(self.h, key, int(value)))

    def new_output(self, n: int = 1, device=None):
        shape = self.out_shape if n == 1 else (n,) + self.out_shape
        return self._torch.zeros(shape, dtype=self.out_dtype,
                                 device=device or self._torch.device("cuda"))

    def _stream(self, stream) -> int:
        s = stream if stream is not None else self._torch.cuda.current_stream()
        return s.cuda_stream

    def correlate(self, x, out=None, stream=None, sync: bool = False):
        assert x.is_cuda and x.is_contiguous() and tuple(x.shape) == self.in_shape, x.shape
        if out is None:
            out = self.new_output(device=x.device)
        assert out.is_cuda and out.is_contiguous() and out.dtype == self.out_dtype
        _check(xc_correlate(self.h, x.data_ptr(), out.data_ptr(), self._stream(stream)))
        if sync:
            self.synchronize(stream)
        return out

    def correlate_stream(self, host_in, n_integrations: int, out, host_out=None, stream=None):
        assert host_in.is_contiguous() and not host_in.is_cuda
        _check(xc_correlate_stream(self.h, host_in.data_ptr(), n_integrations, out.data_ptr(),
                                   0 if host_out is None else host_out.data_ptr(),
                                   self._stream(stream)))
        return out

    def set_gains(self, gains) -> None:
        """Complex gains [N][P][2] float32 on the device (None clears them)."""
        if gains is None:
            _check(xc_set_gains(self.h, 0))
            return
        g = gains.detach().to(self._torch.float32).contiguous()
        assert g.is_cuda and tuple(g.shape) == (self.nstation, self.npol, 2), g.shape
        _check(xc_set_gains(self.h, g.data_ptr()))

    def correlate_backward(self, grad_out, x, grad_in=None, stream=None):
        """grad_in = conj(g) (G + G^H)(g x) for float32 input; returns grad_in."""
        assert grad_out.is_cuda and grad_out.is_contiguous() and grad_out.dtype == self._torch.float32
        assert x.is_cuda and x.is_contiguous() and x.dtype == self._torch.float32
        if grad_in is None:
            grad_in = self._torch.empty_like(x)
        _check(xc_correlate_backward(self.h, grad_out.data_ptr(), x.data_ptr(), grad_in.data_ptr(),
                                     self._stream(stream)))
        return grad_in

    def grad_gains(self, stream=None):
        """Gain gradient [N][P][2] from the last correlate_backward."""
        out = self._torch.empty((self.nstation, self.npol, 2), dtype=self._torch.float32,
                                device=self._torch.device("cuda"))
        _check(xc_get_grad_gains(self.h, out.data_ptr(), self._stream(stream)))
        return out

    def kernel_times(self, reset: bool = True):
        return xc_kernel_times(self.h, reset)

    def synchronize(self, stream=None) -> None:
        _check(xc_synchronize(self.h, self._stream(stream)))

    def close(self) -> None:
        if getattr(self, "h", None):
            xc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ F-engine


def channelize(x, nchan: int, scale: float = 1.0, out_dtype: str = "float16", out=None,
               stream=None, taps=None):
    """F-engine: ``x[N][P][T*nchan][2]`` (int8, float16 or float32 on the GPU,
    each station's complex stream) -> ``[T][nchan][N][P][2]`` of ``out_dtype``,
    the DFT of every block of nchan samples times ``scale``, already in
    :class:`Correlator`'s input layout; ``out_dtype="int8"`` requantises each
    component to the nearest integer, saturated at +-127.  With ``taps``
    (float32 ``[ntaps][nchan]`` on the GPU) a polyphase front end weights
    ntaps consecutive blocks before each DFT and T - ntaps + 1 blocks come
    out.  Stream-ordered (current stream by default); raises XcError on a bad
    argument."""
    import torch
    assert x.is_cuda and x.is_contiguous() and x.dim() == 4 and x.shape[-1] == 2
    N, P, L, _ = x.shape
    if L % nchan:
        raise ValueError("samples per stream (%d) not a multiple of nchan (%d)" % (L, nchan))
    T = L // nchan
    ntaps = 1 if taps is None else taps.shape[0]
    if taps is not None:
        assert taps.is_cuda and taps.is_contiguous() and taps.dtype == torch.float32
        assert tuple(taps.shape) == (ntaps, nchan)
    Tout = T - ntaps + 1
    odt = {"int8": torch.int8, "float16": torch.float16, "float32": torch.float32}[out_dtype]
    if out is None:
        out = torch.empty((max(Tout, 0), nchan, N, P, 2), dtype=odt, device=x.device)
    assert out.is_contiguous() and out.dtype == odt and tuple(out.shape) == (Tout, nchan, N, P, 2)
    s = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
    idt = _DTYPES[str(x.dtype).replace("torch.", "")]
    if taps is None:
        _check(xc_channelize(x.data_ptr(), idt, N, P, nchan, T, float(scale), out.data_ptr(),
                             _DTYPES[out_dtype], s))
    else:
        _check(xc_channelize_pfb(x.data_ptr(), idt, N, P, nchan, T, taps.data_ptr(), ntaps,
                                 float(scale), out.data_ptr(), _DTYPES[out_dtype], s))
    return out


# ------------------------------------------------------------ autograd


def correlate_autograd(engine: "Correlator", x, gains):
    """Visibilities of float32 voltages ``x[T][F][N][P][2]`` with complex gains
    ``gains[N][P][2]`` applied first, differentiable in both (backward through
    the library's adjoint kernel; the forward's input is re-read, nothing
    else is stored)."""
    import torch

    class _Correlate(torch.autograd.Function):
        @staticmethod
        def forward(ctx, xx, gg):
            engine.set_gains(gg)
            out = engine.correlate(xx.detach().contiguous())
            ctx.save_for_backward(xx, gg)
            return out

        @staticmethod
        def backward(ctx, grad_out):
            xx, gg = ctx.saved_tensors
            engine.set_gains(gg)
            grad_x = engine.correlate_backward(grad_out.contiguous(), xx.detach().contiguous())
            grad_g = engine.grad_gains()
            return grad_x, grad_g

    return _Correlate.apply(x, gains)


# ------------------------------------------------------------ batched form


def xc_batch_create(nstation, nfreq, ntime, npol: int, in_dtype: int) -> int:
    n = len(nstation)
    arr = ctypes.c_int * n
    h = load().xc_batch_create(n, arr(*nstation), arr(*nfreq), arr(*ntime), npol, in_dtype)
    if not h:
        raise XcError(xc_last_error(), xc_last_error_message())
    return h


def _ptr_array(ptrs):
    return (ctypes.c_void_p * len(ptrs))(*ptrs)


def xc_batch_correlate(h: int, in_ptrs, out_ptrs, stream: int = 0) -> int:
    return load().xc_batch_correlate(h, _ptr_array(in_ptrs), _ptr_array(out_ptrs), stream)


def xc_batch_tune(h: int, in_ptrs, out_ptrs, stream: int = 0, reps: int = 3):
    ms = (ctypes.c_double * XC_BATCH_CANDIDATES)()
    best = ctypes.c_int(-1)
    _check(load().xc_batch_tune(h, _ptr_array(in_ptrs), _ptr_array(out_ptrs), stream, reps, ms,
                                ctypes.byref(best)))
    return list(ms), best.value


def xc_batch_set_cache(h: int, path: Optional[str]) -> int:
    return load().xc_batch_set_cache(h, path.encode() if path else None)


def xc_batch_cache_key(nstation, nfreq, ntime, npol: int, in_dtype: int) -> str:
    n = len(nstation)
    arr = ctypes.c_int * n
    buf = ctypes.create_string_buffer(512)
    k = load().xc_batch_cache_key(n, arr(*nstation), arr(*nfreq), arr(*ntime), npol, in_dtype, buf, 512)
    if k < 0:
        raise ValueError("bad batch key arguments")
    return buf.value.decode()


def xc_batch_cache_lookup(path: str, key: str) -> int:
    return load().xc_batch_cache_lookup(path.encode(), key.encode())


class BatchCorrelator:
    """Subarrays ``[(nstation, nfreq, ntime), ...]`` (8-bit input, one npol)
    correlated by one persistent launch replayed from a CUDA graph."""

    def __init__(self, subs, npol: int = 2, timeout_ms: Optional[int] = None):
        import torch
        self._torch = torch
        self.subs = [tuple(int(v) for v in s) for s in subs]
        self.npol = npol
        self.h = xc_batch_create([s[0] for s in self.subs], [s[1] for s in self.subs],
                                 [s[2] for s in self.subs], npol, XC_CI8)
        if timeout_ms is not None:
            _check(xc_set_option(self.h, XC_OPT_TIMEOUT_MS, timeout_ms))

    def in_shape(self, i: int):
        N, F, T = self.subs[i]
        return (T, F, N, self.npol, 2)

    def out_shape(self, i: int):
        N, F, _ = self.subs[i]
        return (F, N * (N + 1) // 2, self.npol * self.npol, 2)

    def new_outputs(self, device=None):
        dev = device or self._torch.device("cuda")
        return [self._torch.zeros(self.out_shape(i), dtype=self._torch.int32, device=dev)
                for i in range(len(self.subs))]

    def _check_bufs(self, xs, outs):
        assert len(xs) == len(self.subs) and len(outs) == len(self.subs)
        for i, (x, o) in enumerate(zip(xs, outs)):
            assert x.is_cuda and x.is_contiguous() and x.dtype == self._torch.int8
            assert tuple(x.shape) == self.in_shape(i), (i, x.shape)
            assert o.is_cuda and o.is_contiguous() and o.dtype == self._torch.int32
            assert tuple(o.shape) == self.out_shape(i), (i, o.shape)

    def set_option(self, key: int, value: int) -> None:
        _check(xc_set_option(self.h, key, int(value)))

    def correlate(self, xs, outs=None, stream=None, sync: bool = False):
        if outs is None:
            outs = self.new_outputs(xs[0].device)
        self._check_bufs(xs, outs)
        s = (stream or self._torch.cuda.current_stream()).cuda_stream
        _check(xc_batch_correlate(self.h, [x.data_ptr() for x in xs], [o.data_ptr() for o in outs], s))
        if sync:
            _check(xc_synchronize(self.h, s))
        return outs

    def set_cache(self, path: Optional[str]) -> None:
        """Tuning file for tune(): a recorded choice is applied without timing."""
        _check(xc_batch_set_cache(self.h, path))

    def tune(self, xs, outs, reps: int = 3, stream=None):
        self._check_bufs(xs, outs)
        s = (stream or self._torch.cuda.current_stream()).cuda_stream
        return xc_batch_tune(self.h, [x.data_ptr() for x in xs], [o.data_ptr() for o in outs], s, reps)

    def synchronize(self, stream=None) -> None:
        s = (stream or self._torch.cuda.current_stream()).cuda_stream
        _check(xc_synchronize(self.h, s))

    def kernel_times(self, reset: bool = True):
        return xc_kernel_times(self.h, reset)

    def close(self) -> None:
        if getattr(self, "h", None):
            xc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
