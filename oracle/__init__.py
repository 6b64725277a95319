"""FP64 CPU oracle for one t-FDP iteration (arXiv 2303.03964).

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()``, and the CPU-baseline
leg and the reference arm of ``bench.py`` may import this package (``build()`` compiles
it). The GPU library shares no code with it.

This module only marshals numpy arrays into the C oracle (``tfdp_oracle.c``); every
step of the arithmetic is there, each function citing the section or equation of the
paper it follows. See the header of ``tfdp_oracle.c`` for the sign convention and the
readings taken where the paper is silent.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None

GRID_PAPER = 0
GRID_SNAP_H = 1

_d = ctypes.c_double
_i64 = ctypes.c_int64
_i32 = ctypes.c_int
_p = ctypes.c_void_p


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        sigs = {
            "or_num_threads": ([], _i32),
            "or_tforce": ([_d, _d], _d),
            "or_rep_exact": ([_i64, _p, _p, _d, _i64, _i64, _p], None),
            "or_rep_exact_rows": ([_i64, _p, _p, _d, _i64, _p, _p], None),
            "or_att": ([_i64, _i64, _p, _p, _p, _d, _d, _p], None),
            "or_energy": ([_i64, _p, _i64, _p, _p, _p, _d, _d, _d], _d),
            "or_grid_policy": ([_i64, _p, _i32, _i32, _i32, _i32, _p], None),
            "or_box_f32": ([ctypes.c_float, ctypes.c_float, ctypes.c_float, _i32], _i32),
            "or_lagrange": ([_i32, _d, _p], None),
            "or_fft": ([_i64, _p, _p, _i32], None),
            "or_fft2": ([_i64, _p, _p, _i32], None),
            "or_conv_grid_fft": ([_i64, _i64, _d, _d, _i32, _p, _p], _i32),
            "or_conv_grid_direct": ([_i64, _d, _d, _i32, _p, _p], None),
            "or_rep_fft": ([_i64, _p, _p, _p, _d, _i32, _d, _d, _i32, _i64, _p], _i32),
            "or_step_size": ([_i64, _i64, _d, _d], _d),
            "or_k_of_iter": ([_i32, _i64, _i64], _i32),
            "or_update": ([_i64, _p, _p, _d], None),
            "or_iterate": ([_i64, _i64, _p, _p, _p, _p, _d, _d, _d, _i32, _i32, _i32, _i32, _i32,
                            _i64, _d, _d, _i64, _i64, _i64], _i32),
        }
        for name, (args, res) in sigs.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _LIB = lib
    return _LIB


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(_p)


def num_threads() -> int:
    return int(_lib().or_num_threads())


def tforce(d: float, phi: float) -> float:
    """t-force f(d) = d / (1 + d^2)^phi, Sec. 3.2 Eq. (forcefunction)."""
    return float(_lib().or_tforce(float(d), float(phi)))


def _weights(w, n):
    """Per-node local-refinement weights as a contiguous FP64 array (None: all 1)."""
    if w is None:
        return None
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(-1))
    if w.shape[0] != n:
        raise ValueError("one weight per node")
    return w


def _wptr(w):
    return _ptr(w) if w is not None else None


def rep_exact(xy, gamma: float, rows=None, w=None):
    """Exact repulsion of Eq. (repfK), FP64. ``rows`` selects target rows (all by default);
    ``w`` are per-node repulsion weights r_i (pair force scaled by r_i r_j)."""
    xy = _f64(xy).reshape(-1, 2)
    n = xy.shape[0]
    w = _weights(w, n)
    if rows is None:
        out = np.zeros((n, 2))
        _lib().or_rep_exact(n, _ptr(xy), _wptr(w), gamma, 0, n, _ptr(out))
        return out
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    out = np.zeros((rows.shape[0], 2))
    _lib().or_rep_exact_rows(n, _ptr(xy), _wptr(w), gamma, rows.shape[0], _ptr(rows), _ptr(out))
    return out


def attraction(edges, xy, alpha: float, beta: float, w=None):
    """alpha-weighted attraction of Eq. (newforce) over undirected ``edges`` (m x 2);
    ``w`` are per-node attraction weights a_i (edge force scaled by a_i a_j)."""
    xy = _f64(xy).reshape(-1, 2)
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    w = _weights(w, xy.shape[0])
    out = np.zeros_like(xy)
    _lib().or_att(xy.shape[0], e.shape[0], _ptr(e), _ptr(xy), _wptr(w), alpha, beta, _ptr(out))
    return out


def energy(xy, edges, alpha: float, beta: float, gamma: float, wr=None, wa=None) -> float:
    xy = _f64(xy).reshape(-1, 2)
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    wr, wa = _weights(wr, xy.shape[0]), _weights(wa, xy.shape[0])
    return float(_lib().or_energy(xy.shape[0], _ptr(xy), e.shape[0], _ptr(e), _wptr(wr), _wptr(wa),
                                  alpha, beta, gamma))


def grid_policy(xy_f32, k: int, n_int_min: int = 50, grid_max: int = 1 << 30,
                policy: int = GRID_SNAP_H):
    """Grid descriptor (lo, h, n_int, G, L) of Sec. 3.4 from FP32 positions."""
    xyf = np.ascontiguousarray(np.asarray(xy_f32, dtype=np.float32).reshape(-1, 2))
    out = np.zeros(5)
    _lib().or_grid_policy(xyf.shape[0], _ptr(xyf), k, n_int_min, grid_max, policy, _ptr(out))
    return {"lo": out[0], "h": out[1], "n_int": int(out[2]), "G": int(out[3]), "L": out[4]}


def box_f32(x: float, lo: float, h: float, n_int: int) -> int:
    return int(_lib().or_box_f32(float(np.float32(x)), float(np.float32(lo)),
                                 float(np.float32(h)), n_int))


def lagrange(k: int, u: float):
    w = np.zeros(k)
    _lib().or_lagrange(k, float(u), _ptr(w))
    return w


def fft(z, inverse: bool = False):
    """Own radix-2 FFT (1D for 1D input, 2D square for 2D input); inverse has no 1/N."""
    z = np.asarray(z, dtype=np.complex128)
    re = np.ascontiguousarray(z.real.copy())
    im = np.ascontiguousarray(z.imag.copy())
    sign = 1 if inverse else -1
    if z.ndim == 1:
        _lib().or_fft(z.shape[0], _ptr(re), _ptr(im), sign)
    else:
        assert z.shape[0] == z.shape[1]
        _lib().or_fft2(z.shape[0], _ptr(re), _ptr(im), sign)
    return re + 1j * im


def conv_grid(channels, spacing: float, gamma: float, P=None, direct: bool = False):
    """Grid interaction of Sec. 3.4 for (nch, G, G) channels with node spacing ``spacing``."""
    c = _f64(channels)
    if c.ndim == 2:
        c = c[None]
    nch, G, _ = c.shape
    out = np.zeros_like(c)
    if direct:
        _lib().or_conv_grid_direct(G, spacing, gamma, nch, _ptr(c), _ptr(out))
    else:
        if P is None:
            P = 1
            while P < 2 * G - 1:
                P *= 2
        rc = _lib().or_conv_grid_fft(G, P, spacing, gamma, nch, _ptr(c), _ptr(out))
        if rc != 0:
            raise RuntimeError("or_conv_grid_fft failed: %d" % rc)
    return out


def rep_fft(xy, gamma: float, k: int, grid=None, P=None, xy_f32=None, n_int_min: int = 50,
            grid_max: int = 1 << 30, policy: int = GRID_SNAP_H, w=None):
    """ibFFT repulsion of Sec. 3.4 (paper's three-sum form), FP64.

    ``grid`` is a dict (lo, h, n_int); when omitted it comes from ``grid_policy`` on the
    FP32 positions. ``xy_f32`` are the FP32 positions used for the box decision
    (default: ``xy`` rounded to FP32).
    """
    xy = _f64(xy).reshape(-1, 2)
    xyf = (np.ascontiguousarray(np.asarray(xy_f32, dtype=np.float32).reshape(-1, 2))
           if xy_f32 is not None else xy.astype(np.float32))
    if grid is None:
        grid = grid_policy(xyf, k, n_int_min, grid_max, policy)
    n_int = int(grid["n_int"])
    G = n_int * k
    if P is None:
        P = 1
        while P < 2 * G - 1:
            P *= 2
    w = _weights(w, xy.shape[0])
    out = np.zeros_like(xy)
    rc = _lib().or_rep_fft(xy.shape[0], _ptr(xy), _ptr(xyf), _wptr(w), gamma, k, float(grid["lo"]),
                           float(grid["h"]), n_int, int(P), _ptr(out))
    if rc != 0:
        raise RuntimeError("or_rep_fft failed: %d" % rc)
    return out


def step_size(t: int, T: int, s0: float, smin: float) -> float:
    return float(_lib().or_step_size(t, T, s0, smin))


def k_of_iter(k: int, t: int, T: int) -> int:
    """k of iteration t of a T-iteration run; k = 0 is the dynamic strategy of Sec. 3.4
    "Choices of k" (1 for the first 90 % of the iterations, 2 for the next 5 %, then 3)."""
    return int(_lib().or_k_of_iter(k, t, T))


def update(xy, D, s: float):
    xy = _f64(xy).reshape(-1, 2).copy()
    D = _f64(D).reshape(-1, 2)
    _lib().or_update(xy.shape[0], _ptr(xy), _ptr(D), s)
    return xy


def iterate(xy, edges, iters: int, alpha=0.1, beta=8.0, gamma=2.0, mode="exact", k=3,
            n_int_min=50, grid_max=1 << 30, policy=GRID_SNAP_H, P=0, s0=1.0, smin=0.01,
            T=300, t0=0, wrep=None, watt=None):
    """Run ``iters`` synchronous t-FDP iterations from iteration index ``t0``; k = 0 takes
    k per iteration from the dynamic strategy (``k_of_iter``); ``wrep`` / ``watt`` are the
    per-node local-refinement weights (None: all 1)."""
    xy = _f64(xy).reshape(-1, 2).copy()
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    wr, wa = _weights(wrep, xy.shape[0]), _weights(watt, xy.shape[0])
    m = {"exact": 0, "fft": 1}[mode]
    rc = _lib().or_iterate(xy.shape[0], e.shape[0], _ptr(e), _ptr(xy), _wptr(wr), _wptr(wa), alpha,
                           beta, gamma, m, k, n_int_min, grid_max, policy, P, s0, smin, T, t0, iters)
    if rc != 0:
        raise RuntimeError("or_iterate failed: %d" % rc)
    return xy
