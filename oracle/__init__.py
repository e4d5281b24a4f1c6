"""CPU oracle for the X-engine -- test infrastructure, not the product.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` import this package.  It wraps ``xc_oracle.c`` (plain C loops,
int64 / FP64 accumulation) through ctypes.  The C source states which passage
of Clark, La Plante & Greenhill each function follows:

* ``correlate_i8`` / ``correlate_f64`` -- Sec. 2.1 Eq. (outer) with the dual
  polarisation, lower-triangle packing of Sec. 2.1 / Sec. 4.2 and the input
  ordering of Sec. 4.1;
* ``backward_f64`` -- the adjoint of the float form (not in the paper);
* ``channelize_f64`` -- the F-engine of Sec. 2 (blockwise DFT of each
  station's signal) with the corner turn into the X-engine's input order;
  ``requantise_i8`` -- its 8-bit requantisation (nearest integer, ties to
  even, saturated at +-127), the 8-bit X-engine input of Sec. 5;
  ``channelize_pfb_f64`` -- the same with a polyphase front end (taps
  h[p][m] over ntaps consecutive blocks; not in the paper).

Arrays use the engine's layouts: input ``[T][F][N][P][2]``, output
``[F][N(N+1)/2][P*P][2]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libxc_oracle.so")
_lib: Optional[ctypes.CDLL] = None


def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile the oracle with gcc (-O2, OpenMP).  Returns the library path."""
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    i64, i32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
    lib.xco_baseline_index.argtypes = [i64, i64]
    lib.xco_baseline_index.restype = i64
    lib.xco_num_baselines.argtypes = [i64]
    lib.xco_num_baselines.restype = i64
    lib.xco_num_threads.argtypes = []
    lib.xco_num_threads.restype = i32
    lib.xco_set_num_threads.argtypes = [i32]
    lib.xco_set_num_threads.restype = None
    lib.xco_correlate_i8.argtypes = [vp, i32, i32, i32, i32, vp, i32, vp]
    lib.xco_correlate_i8.restype = i32
    lib.xco_correlate_f64.argtypes = [vp, vp, i32, i32, i32, i32, vp, i32, vp]
    lib.xco_correlate_f64.restype = i32
    lib.xco_backward_f64.argtypes = [vp, vp, vp, i32, i32, i32, i32, vp, vp]
    lib.xco_backward_f64.restype = i32
    lib.xco_channelize_f64.argtypes = [vp, i32, i32, i32, i32, ctypes.c_double, vp, i32, vp]
    lib.xco_channelize_f64.restype = i32
    lib.xco_channelize_pfb_f64.argtypes = [vp, i32, i32, i32, i32, vp, i32, ctypes.c_double, vp]
    lib.xco_channelize_pfb_f64.restype = i32
    return lib


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Load (building first if needed) the oracle library."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def num_baselines(nstation: int) -> int:
    return nstation * (nstation + 1) // 2


def num_threads(lib: Optional[ctypes.CDLL] = None) -> int:
    return int((lib or load()).xco_num_threads())


def set_num_threads(n: int, lib: Optional[ctypes.CDLL] = None) -> None:
    (lib or load()).xco_set_num_threads(int(n))


def correlate_i8(x: np.ndarray, chans: Optional[Sequence[int]] = None,
                 lib: Optional[ctypes.CDLL] = None) -> np.ndarray:
    """Integer visibilities (int64) of int8 input ``x[T][F][N][P][2]``.

    Returns ``[len(chans) or F][N(N+1)/2][P*P][2]`` int64.
    """
    lib = lib or load()
    x = np.ascontiguousarray(x, dtype=np.int8)
    T, F, N, P, two = x.shape
    assert two == 2
    ch = None if chans is None else np.ascontiguousarray(np.asarray(chans, dtype=np.int32))
    nch = F if ch is None else len(ch)
    out = np.zeros((nch, num_baselines(N), P * P, 2), dtype=np.int64)
    rc = lib.xco_correlate_i8(_ptr(x), N, P, F, T, None if ch is None else _ptr(ch), nch, _ptr(out))
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    return out


def correlate_f64(x: np.ndarray, gains: Optional[np.ndarray] = None,
                  chans: Optional[Sequence[int]] = None,
                  lib: Optional[ctypes.CDLL] = None) -> np.ndarray:
    """FP64 visibilities of float input ``x[T][F][N][P][2]`` with optional
    complex gains ``gains[N][P][2]`` applied to the voltages first."""
    lib = lib or load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    T, F, N, P, two = x.shape
    assert two == 2
    g = None if gains is None else np.ascontiguousarray(gains, dtype=np.float64).reshape(N, P, 2)
    ch = None if chans is None else np.ascontiguousarray(np.asarray(chans, dtype=np.int32))
    nch = F if ch is None else len(ch)
    out = np.zeros((nch, num_baselines(N), P * P, 2), dtype=np.float64)
    rc = lib.xco_correlate_f64(_ptr(x), None if g is None else _ptr(g), N, P, F, T,
                               None if ch is None else _ptr(ch), nch, _ptr(out))
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    return out


def backward_f64(x: np.ndarray, grad_out: np.ndarray, gains: Optional[np.ndarray] = None,
                 lib: Optional[ctypes.CDLL] = None):
    """FP64 adjoint: returns ``(grad_x[T][F][N][P][2], grad_g[N][P][2])``."""
    lib = lib or load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    T, F, N, P, _ = x.shape
    go = np.ascontiguousarray(grad_out, dtype=np.float64)
    assert go.shape == (F, num_baselines(N), P * P, 2)
    g = None if gains is None else np.ascontiguousarray(gains, dtype=np.float64).reshape(N, P, 2)
    gx = np.zeros_like(x)
    gg = np.zeros((N, P, 2), dtype=np.float64)
    rc = lib.xco_backward_f64(_ptr(x), None if g is None else _ptr(g), _ptr(go), N, P, F, T,
                              _ptr(gx), _ptr(gg))
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    return gx, gg


def channelize_f64(x: np.ndarray, nchan: int, scale: float = 1.0,
                   sel: Optional[Sequence[Sequence[int]]] = None,
                   lib: Optional[ctypes.CDLL] = None) -> np.ndarray:
    """F-engine: ``x[N][P][T*nchan][2]`` (each station's complex stream) ->
    ``X[T][nchan][N][P][2]`` with ``X[t][f] = scale * sum_m x[t*nchan + m]
    exp(-2 pi i f m / nchan)``; with ``sel`` (a list of (t, f) pairs) only
    those outputs, as ``[len(sel)][N][P][2]``."""
    lib = lib or load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    N, P, L, two = x.shape
    assert two == 2 and L % nchan == 0
    T = L // nchan
    s = None if sel is None else np.ascontiguousarray(np.asarray(sel, dtype=np.int32).reshape(-1, 2))
    nout = T * nchan if s is None else len(s)
    out = np.zeros((nout, N, P, 2), dtype=np.float64)
    rc = lib.xco_channelize_f64(_ptr(x), N, P, nchan, T, float(scale),
                                None if s is None else _ptr(s), 0 if s is None else len(s), _ptr(out))
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    return out if s is not None else out.reshape(T, nchan, N, P, 2)


def requantise_i8(X: np.ndarray) -> np.ndarray:
    """8-bit requantisation of F-engine output: each component rounded to the
    nearest integer (ties to even) and saturated at +-127, as int8."""
    return np.clip(np.rint(np.asarray(X, dtype=np.float64)), -127, 127).astype(np.int8)


def channelize_pfb_f64(x: np.ndarray, taps: np.ndarray, scale: float = 1.0,
                       lib: Optional[ctypes.CDLL] = None) -> np.ndarray:
    """Polyphase F-engine: ``taps[ntaps][nchan]`` real, ``x[N][P][T*nchan][2]``
    -> ``X[T-ntaps+1][nchan][N][P][2]`` with ``X[t][f] = scale * sum_m
    exp(-2 pi i f m / nchan) sum_p taps[p][m] x[(t+p)*nchan + m]``."""
    lib = lib or load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    h = np.ascontiguousarray(taps, dtype=np.float64)
    N, P, L, two = x.shape
    ntaps, F = h.shape
    assert two == 2 and L % F == 0
    T = L // F
    out = np.zeros((T - ntaps + 1, F, N, P, 2), dtype=np.float64)
    rc = lib.xco_channelize_pfb_f64(_ptr(x), N, P, F, T, _ptr(h), ntaps, float(scale), _ptr(out))
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    return out
