"""Python binding of the t-FDP C ABI (include/tfdp.h): argument marshalling only.

Every step of an iteration runs in the CUDA library libtfdp.so; this module converts
numpy arrays / torch tensors to pointers and status codes to exceptions. Importing it
raises if the library has not been built (``__graft_entry__.build()`` or
``python paper_2303_03964_gb300/build.py``): there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtfdp.so")

REP_EXACT, REP_FFT, REP_AUTO = 0, 1, 2  # REP_AUTO: resolved by n at creation / set_params
PREC_FP32, PREC_BF16X3 = 0, 1
GRID_PAPER, GRID_SNAP_H = 0, 1
K_DYNAMIC = 0  # k_interp: the dynamic k schedule (1, then 2, then 3)
WEIGHT_MAX = 64.0  # largest local-refinement weight
DEBUG_GRID_CHARGES, DEBUG_GRID_OUTPUT, DEBUG_SORT_PERM, DEBUG_CELL_START = 1, 2, 3, 4
INJECT_FFT_ALLOC, INJECT_SCAN_STALL = 1, 2  # failure-detection test hooks (tfdp_debug_inject)
FLAG_NONFINITE, FLAG_BOX_RANGE, FLAG_SORT_RANGE, FLAG_WAIT_TIMEOUT = 1, 2, 4, 8  # device_flags bits
STAGES = ["sort", "spread", "spectrum", "rows_fwd", "cols", "rows_inv", "gather_update",
          "exact", "edge_update", "attract"]

STATUS = {0: "TFDP_OK", 1: "TFDP_ERR_INVALID_ARG", 2: "TFDP_ERR_BAD_GRAPH",
          3: "TFDP_ERR_PARAM_RANGE", 4: "TFDP_ERR_OUT_OF_MEMORY", 5: "TFDP_ERR_CUDA",
          6: "TFDP_ERR_TIMEOUT", 7: "TFDP_ERR_BUSY", 8: "TFDP_ERR_DEVICE_CHECK"}


class TfdpError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        self.name = STATUS.get(status, "TFDP_ERR_%d" % status)
        super().__init__("%s failed: %s%s" % (where, self.name, (" (" + detail + ")") if detail else ""))


class Params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("gamma", ctypes.c_double),
                ("k_interp", ctypes.c_int32), ("n_int_min", ctypes.c_int32),
                ("grid_max", ctypes.c_int32), ("grid_policy", ctypes.c_int32),
                ("rep_mode", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("step0", ctypes.c_double), ("step_min", ctypes.c_double),
                ("total_iters", ctypes.c_int32), ("reserved", ctypes.c_int32 * 7)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class Stats(ctypes.Structure):
    _fields_ = [("iteration", ctypes.c_int64), ("net_frep", ctypes.c_double * 2),
                ("grid_lo", ctypes.c_double), ("grid_h", ctypes.c_double),
                ("grid_n_int", ctypes.c_int32), ("grid_G", ctypes.c_int32),
                ("fft_P", ctypes.c_int32), ("spectrum_builds", ctypes.c_int32),
                ("device_flags", ctypes.c_int32), ("kernels_per_iteration", ctypes.c_int32),
                ("grid_k", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}
        d["net_frep"] = (self.net_frep[0], self.net_frep[1])
        return d


_p = ctypes.c_void_p
_SIGS = {
    "tfdp_status_str": ([ctypes.c_int], ctypes.c_char_p),
    "tfdp_last_cuda_error": ([], ctypes.c_char_p),
    "tfdp_params_default": ([ctypes.POINTER(Params)], ctypes.c_int),
    "tfdp_params_check": ([ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "tfdp_create_graph": ([ctypes.c_int64, ctypes.c_int64, _p, _p, ctypes.c_uint64,
                           ctypes.POINTER(Params), _p, ctypes.POINTER(_p)], ctypes.c_int),
    "tfdp_set_params": ([_p, ctypes.POINTER(Params)], ctypes.c_int),
    "tfdp_get_params": ([_p, ctypes.POINTER(Params)], ctypes.c_int),
    "tfdp_set_positions": ([_p, _p, ctypes.c_int], ctypes.c_int),
    "tfdp_set_node_weights": ([_p, _p, _p, ctypes.c_int], ctypes.c_int),
    "tfdp_run": ([_p, _p, ctypes.c_int32, _p], ctypes.c_int),
    "tfdp_get_positions": ([_p, _p, ctypes.c_int], ctypes.c_int),
    "tfdp_iterate": ([_p, ctypes.c_int32], ctypes.c_int),
    "tfdp_set_iteration": ([_p, ctypes.c_int64], ctypes.c_int),
    "tfdp_eval_forces": ([_p, _p, _p, ctypes.c_int], ctypes.c_int),
    "tfdp_get_stats": ([_p, ctypes.POINTER(Stats)], ctypes.c_int),
    "tfdp_synchronize": ([_p], ctypes.c_int),
    "tfdp_set_stage_timing": ([_p, ctypes.c_int], ctypes.c_int),
    "tfdp_set_stage_timing_mask": ([_p, ctypes.c_uint32], ctypes.c_int),
    "tfdp_get_stage_times": ([_p, ctypes.POINTER(ctypes.c_float), ctypes.c_int], ctypes.c_int),
    "tfdp_destroy_graph": ([_p], ctypes.c_int),
    "tfdp_debug_fetch": ([_p, ctypes.c_int, _p, ctypes.c_size_t], ctypes.c_int),
    "tfdp_debug_inject": ([_p, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "tfdp_exact_repulsion_noalloc": ([_p, ctypes.c_int64, ctypes.c_double, _p, _p], ctypes.c_int),
    "tfdp_batch_create": ([ctypes.c_int32, _p, _p, _p, _p, _p, _p, ctypes.POINTER(_p)], ctypes.c_int),
    "tfdp_batch_iterate": ([_p, ctypes.c_int32], ctypes.c_int),
    "tfdp_batch_eval_forces": ([_p, ctypes.c_int32, _p, _p, ctypes.c_int], ctypes.c_int),
    "tfdp_batch_get_positions": ([_p, ctypes.c_int32, _p, ctypes.c_int], ctypes.c_int),
    "tfdp_batch_get_stats": ([_p, ctypes.c_int32, ctypes.POINTER(Stats)], ctypes.c_int),
    "tfdp_batch_synchronize": ([_p], ctypes.c_int),
    "tfdp_batch_destroy": ([_p], ctypes.c_int),
    "tfdp_batch_grid_blocks": ([_p], ctypes.c_int32),
    "tfdp_batch_autotune": ([_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "tfdp_batch_phase_parts": ([_p], ctypes.c_int32),
    "tfdp_batch_set_phase_launches": ([_p, ctypes.c_int32], ctypes.c_int),
    "tfdp_batch_num_parts": ([_p], ctypes.c_int32),
    "tfdp_batch_plan": ([ctypes.c_int32, _p, _p, _p, _p, _p, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                         _p, _p], ctypes.c_int),
    "tfdp_graph_set_stream": ([_p, _p], ctypes.c_int),
    "tfdp_graph_footprint": ([ctypes.c_int64, ctypes.c_int64, _p, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "tfdp_server_create": ([ctypes.c_size_t, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_p)], ctypes.c_int),
    "tfdp_server_submit": ([_p, ctypes.c_int64, ctypes.c_int64, _p, _p, _p, ctypes.c_int32,
                            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "tfdp_server_update": ([_p, ctypes.c_int64, _p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "tfdp_server_poll": ([_p, _p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32], ctypes.c_int),
    "tfdp_server_get_positions": ([_p, ctypes.c_int64, _p], ctypes.c_int),
    "tfdp_server_release": ([_p, ctypes.c_int64], ctypes.c_int),
    "tfdp_server_get_stats": ([_p, _p], ctypes.c_int),
    "tfdp_server_destroy": ([_p], ctypes.c_int),
}

NOALLOC_MAX_N = 16384


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libtfdp.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


lib = _load()


def _check(status, where):
    if status != 0:
        detail = lib.tfdp_last_cuda_error().decode() if status in (4, 5) else ""
        raise TfdpError(status, where, detail)


def params_default(**overrides) -> Params:
    p = Params()
    _check(lib.tfdp_params_default(ctypes.byref(p)), "tfdp_params_default")
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def params_check(p: Params):
    ok = ctypes.c_int(0)
    _check(lib.tfdp_params_check(ctypes.byref(p), ctypes.byref(ok)), "tfdp_params_check")
    return bool(ok.value)


def _is_torch_cuda(x):
    return hasattr(x, "is_cuda") and hasattr(x, "data_ptr") and x.is_cuda


def _check_device_f32(t, numel, what):
    """A CUDA tensor passed as a device pointer: contiguous float32 with `numel` values."""
    import torch

    if t.dtype != torch.float32:
        raise TypeError("%s must be float32" % what)
    if not t.is_contiguous() or t.numel() != numel:
        raise ValueError("%s must be contiguous with %d values" % (what, numel))


def _host_f32(x, n):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32).reshape(n, 2))
    return a


class Graph:
    """One graph on the current CUDA device (wraps a tfdp_graph handle)."""

    def __init__(self, n, edges, xy0=None, params=None, seed=0, stream=0):
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
        self.n = int(n)
        self.m = int(e.shape[0])
        self._edges = e
        xp = None
        if xy0 is not None:
            xp = _host_f32(xy0, self.n)
        self._params = params if params is not None else params_default()
        h = _p()
        st = lib.tfdp_create_graph(self.n, self.m, e.ctypes.data_as(_p) if self.m else None,
                                   xp.ctypes.data_as(_p) if xp is not None else None,
                                   ctypes.c_uint64(seed), ctypes.byref(self._params),
                                   _p(stream or 0), ctypes.byref(h))
        _check(st, "tfdp_create_graph")
        self._h = h

    # ------------------------------------------------------------ lifecycle
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib.tfdp_destroy_graph(self._h)
            self._h = _p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------ parameters
    def set_params(self, params: Params = None, **overrides):
        p = Params()
        ctypes.memmove(ctypes.byref(p), ctypes.byref(params or self._params), ctypes.sizeof(Params))
        for k, v in overrides.items():
            setattr(p, k, v)
        _check(lib.tfdp_set_params(self._h, ctypes.byref(p)), "tfdp_set_params")
        self._params = p

    def get_params(self) -> Params:
        p = Params()
        _check(lib.tfdp_get_params(self._h, ctypes.byref(p)), "tfdp_get_params")
        return p

    # ------------------------------------------------------------ positions
    def set_positions(self, xy):
        if _is_torch_cuda(xy):
            _check_device_f32(xy, 2 * self.n, "xy")
            _check(lib.tfdp_set_positions(self._h, _p(xy.data_ptr()), 1), "tfdp_set_positions")
        else:
            a = _host_f32(xy, self.n)
            _check(lib.tfdp_set_positions(self._h, a.ctypes.data_as(_p), 0), "tfdp_set_positions")

    def set_node_weights(self, w_rep=None, w_att=None):
        """Local-refinement weights (n each; None: all 1): repulsion between i and j scaled by
        w_rep[i] w_rep[j], attraction along edge (i, j) by w_att[i] w_att[j]. Both numpy
        (host) or both CUDA tensors (device)."""
        dev = _is_torch_cuda(w_rep) or _is_torch_cuda(w_att)
        keep, ptrs = [], []
        for w in (w_rep, w_att):
            if w is None:
                ptrs.append(None)
            elif dev:
                if not _is_torch_cuda(w):
                    raise TypeError("weights must both be CUDA tensors or both host arrays")
                _check_device_f32(w, self.n, "weight")
                ptrs.append(_p(w.data_ptr()))
            else:
                a = np.ascontiguousarray(np.asarray(w, dtype=np.float32).reshape(-1))
                if a.shape[0] != self.n:
                    raise ValueError("one weight per node")
                keep.append(a)
                ptrs.append(a.ctypes.data_as(_p))
        _check(lib.tfdp_set_node_weights(self._h, ptrs[0], ptrs[1], 1 if dev else 0), "tfdp_set_node_weights")

    def get_positions(self, out=None):
        """Positions as an (n, 2) float32 numpy array, or into `out` (numpy or CUDA tensor)."""
        if out is not None and _is_torch_cuda(out):
            _check_device_f32(out, 2 * self.n, "out")
            _check(lib.tfdp_get_positions(self._h, _p(out.data_ptr()), 1), "tfdp_get_positions")
            return out
        a = out if out is not None else np.empty((self.n, 2), dtype=np.float32)
        if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags.c_contiguous
                and a.size == 2 * self.n):
            raise ValueError("out must be a contiguous float32 numpy array of n x 2 values")
        _check(lib.tfdp_get_positions(self._h, a.ctypes.data_as(_p), 0), "tfdp_get_positions")
        return a

    # ------------------------------------------------------------ compute
    def run(self, xy_in, iters, xy_out):
        """Upload `xy_in` (host, (n, 2) float32; None keeps the positions), run `iters`
        iterations and download into `xy_out` (host, (n, 2) float32) in one call."""
        src = None if xy_in is None else _host_f32(xy_in, self.n)  # kept alive across the call
        pin = None if src is None else src.ctypes.data_as(_p)
        if not (isinstance(xy_out, np.ndarray) and xy_out.dtype == np.float32 and xy_out.flags.c_contiguous
                and xy_out.size == 2 * self.n):
            raise ValueError("xy_out must be a contiguous float32 numpy array of n x 2 values")
        _check(lib.tfdp_run(self._h, pin, int(iters), xy_out.ctypes.data_as(_p)), "tfdp_run")
        return xy_out

    def iterate(self, iters=1):
        _check(lib.tfdp_iterate(self._h, int(iters)), "tfdp_iterate")

    def set_iteration(self, t):
        _check(lib.tfdp_set_iteration(self._h, int(t)), "tfdp_set_iteration")

    def eval_forces(self):
        """(frep, fatt) at the current positions, each (n, 2) float32."""
        fr = np.empty((self.n, 2), dtype=np.float32)
        fa = np.empty((self.n, 2), dtype=np.float32)
        _check(lib.tfdp_eval_forces(self._h, fr.ctypes.data_as(_p), fa.ctypes.data_as(_p), 0),
               "tfdp_eval_forces")
        return fr, fa

    def stats(self) -> dict:
        s = Stats()
        _check(lib.tfdp_get_stats(self._h, ctypes.byref(s)), "tfdp_get_stats")
        return s.as_dict()

    def set_stage_timing(self, enable=True):
        _check(lib.tfdp_set_stage_timing(self._h, 1 if enable else 0), "tfdp_set_stage_timing")

    def set_stage_timing_mask(self, stages):
        """Time only the named stages (an iterable of STAGES names); empty turns it off."""
        mask = 0
        for name in stages:
            mask |= 1 << STAGES.index(name)
        _check(lib.tfdp_set_stage_timing_mask(self._h, mask), "tfdp_set_stage_timing_mask")

    def stage_times(self) -> dict:
        ms = (ctypes.c_float * len(STAGES))()
        _check(lib.tfdp_get_stage_times(self._h, ms, len(STAGES)), "tfdp_get_stage_times")
        return {name: float(ms[i]) for i, name in enumerate(STAGES)}

    def synchronize(self):
        _check(lib.tfdp_synchronize(self._h), "tfdp_synchronize")

    def debug_inject(self, what, value):
        """Failure-detection test hook (INJECT_FFT_ALLOC / INJECT_SCAN_STALL, see tfdp.h)."""
        _check(lib.tfdp_debug_inject(self._h, int(what), int(value)), "tfdp_debug_inject")

    def debug_fetch(self, what):
        s = self.stats()
        G, n_int = s["grid_G"], s["grid_n_int"]
        if what == DEBUG_GRID_CHARGES:
            a = np.empty((3, G, G), dtype=np.float32)
        elif what == DEBUG_GRID_OUTPUT:
            a = np.empty((G, G, 4), dtype=np.float32)
        elif what == DEBUG_SORT_PERM:
            a = np.empty(self.n, dtype=np.int32)
        elif what == DEBUG_CELL_START:
            a = np.empty(n_int * n_int + 1, dtype=np.int32)
        else:
            raise ValueError(what)
        _check(lib.tfdp_debug_fetch(self._h, int(what), a.ctypes.data_as(_p), a.nbytes),
               "tfdp_debug_fetch")
        return a


def exact_repulsion_noalloc(xy, frep, gamma=2.0, stream=0):
    """Exact repulsion into a caller-owned CUDA tensor without any device allocation.

    For callers that cannot allocate device memory (a framework's caching allocator
    owns the pool, or a latency-critical loop must not risk cudaMalloc / cudaFree
    synchronising the device). ``xy`` and ``frep`` are contiguous float32 CUDA tensors
    of shape (n, 2), n <= NOALLOC_MAX_N. Asynchronous on ``stream``. All calls share one
    fixed scratch array in the library: calls that may overlap on the GPU race.
    """
    import torch

    if not (_is_torch_cuda(xy) and _is_torch_cuda(frep)):
        raise TypeError("xy and frep must be CUDA tensors")
    if xy.dtype != torch.float32 or frep.dtype != torch.float32:
        raise TypeError("xy and frep must be float32")
    if xy.dim() != 2 or xy.shape[1] != 2 or tuple(frep.shape) != tuple(xy.shape):
        raise ValueError("xy and frep must both have shape (n, 2)")
    if not (xy.is_contiguous() and frep.is_contiguous()):
        raise ValueError("xy and frep must be contiguous")
    cur = torch.cuda.current_device()
    if xy.device.index != cur or frep.device.index != cur:
        raise ValueError("xy and frep must be on the current CUDA device (%d)" % cur)
    n = xy.shape[0]
    _check(lib.tfdp_exact_repulsion_noalloc(_p(xy.data_ptr()), n, float(gamma),
                                            _p(frep.data_ptr()), _p(stream or 0)),
           "tfdp_exact_repulsion_noalloc")
    return frep


def _graph_arrays(graphs):
    """Per-graph host arrays and pointer tables of a list of (n, edges, xy0)."""
    B = len(graphs)
    n = np.array([int(g[0]) for g in graphs], dtype=np.int64)
    edges = [np.ascontiguousarray(np.asarray(g[1], dtype=np.int32).reshape(-1, 2)) for g in graphs]
    xy = [_host_f32(g[2], int(g[0])) for g in graphs]
    m = np.array([e.shape[0] for e in edges], dtype=np.int64)
    eptr = (_p * B)(*[e.ctypes.data if e.shape[0] else None for e in edges])
    xptr = (_p * B)(*[x.ctypes.data for x in xy])
    return n, m, edges, xy, eptr, xptr


def batch_plan(graphs, base=None, max_error_ratio=1.5, min_error_bound=0.0, probes=2):
    """Grid autotuner (tfdp_batch_plan): per graph, the k_interp and grid cap with the
    cheapest FFT whose measured repulsion error is within max(max_error_ratio x the error
    of ``base`` (None: defaults), min_error_bound). Returns (list of Params, numpy array
    of errors)."""
    B = len(graphs)
    n, m, edges, xy, eptr, xptr = _graph_arrays(graphs)
    out = (Params * B)()
    err = np.zeros(B, dtype=np.float64)
    _check(lib.tfdp_batch_plan(B, n.ctypes.data_as(_p), m.ctypes.data_as(_p), ctypes.cast(eptr, _p),
                               ctypes.cast(xptr, _p), ctypes.byref(base) if base is not None else None,
                               float(max_error_ratio), float(min_error_bound), int(probes), ctypes.cast(out, _p),
                               err.ctypes.data_as(_p)),
           "tfdp_batch_plan")
    params = []
    for i in range(B):
        p = Params()
        ctypes.memmove(ctypes.byref(p), ctypes.byref(out[i]), ctypes.sizeof(Params))
        params.append(p)
    return params, err


class Batch:
    """Many graphs advanced together (wraps tfdp_batch).

    ``graphs`` is a list of (n, edges (m x 2 int32), xy0 (n x 2 float32)); ``params`` is
    None (defaults) or one Params per graph; graphs with the same (k_interp, FFT size)
    form a part, whose iterations run as one launch per phase (default) or as one
    cooperative persistent launch (``set_phase_launches``, ``autotune``).
    """

    def __init__(self, graphs, params=None, stream=0):
        B = len(graphs)
        self.B = B
        self._n, m, self._edges, self._xy, eptr, xptr = _graph_arrays(graphs)
        prm = None
        if params is not None:
            prm = (Params * B)()
            for i, p in enumerate(params):
                ctypes.memmove(ctypes.byref(prm[i]), ctypes.byref(p), ctypes.sizeof(Params))
        h = _p()
        _check(lib.tfdp_batch_create(B, self._n.ctypes.data_as(_p), m.ctypes.data_as(_p),
                                     ctypes.cast(eptr, _p), ctypes.cast(xptr, _p),
                                     ctypes.cast(prm, _p) if prm is not None else None,
                                     _p(stream or 0), ctypes.byref(h)), "tfdp_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib.tfdp_batch_destroy(self._h)
            self._h = _p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def iterate(self, iters=1):
        _check(lib.tfdp_batch_iterate(self._h, int(iters)), "tfdp_batch_iterate")

    def synchronize(self):
        _check(lib.tfdp_batch_synchronize(self._h), "tfdp_batch_synchronize")

    def eval_forces(self, g):
        n = int(self._n[g])
        fr = np.empty((n, 2), dtype=np.float32)
        fa = np.empty((n, 2), dtype=np.float32)
        _check(lib.tfdp_batch_eval_forces(self._h, int(g), fr.ctypes.data_as(_p), fa.ctypes.data_as(_p), 0),
               "tfdp_batch_eval_forces")
        return fr, fa

    def get_positions(self, g):
        a = np.empty((int(self._n[g]), 2), dtype=np.float32)
        _check(lib.tfdp_batch_get_positions(self._h, int(g), a.ctypes.data_as(_p), 0), "tfdp_batch_get_positions")
        return a

    def stats(self, g):
        s = Stats()
        _check(lib.tfdp_batch_get_stats(self._h, int(g), ctypes.byref(s)), "tfdp_batch_get_stats")
        return s.as_dict()

    def grid_blocks(self):
        return int(lib.tfdp_batch_grid_blocks(self._h))

    def phase_parts(self):
        """Parts that run one launch per phase (the rest: one cooperative launch)."""
        return int(lib.tfdp_batch_phase_parts(self._h))

    def set_phase_launches(self, on=True):
        """One launch per phase (True) or the cooperative persistent launch (False)."""
        _check(lib.tfdp_batch_set_phase_launches(self._h, 1 if on else 0), "tfdp_batch_set_phase_launches")

    def num_parts(self):
        return int(lib.tfdp_batch_num_parts(self._h))

    def autotune(self, trials=3):
        c = ctypes.c_int32(0)
        _check(lib.tfdp_batch_autotune(self._h, int(trials), ctypes.byref(c)), "tfdp_batch_autotune")
        return int(c.value)


def graph_footprint(n, m, params=None):
    """Device bytes a graph of n nodes and m edges would take."""
    out = ctypes.c_size_t(0)
    _check(lib.tfdp_graph_footprint(int(n), int(m), ctypes.byref(params) if params is not None else None,
                                    ctypes.byref(out)), "tfdp_graph_footprint")
    return int(out.value)


class Done(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_int64), ("job_id", ctypes.c_int64), ("kind", ctypes.c_int32),
                ("iters", ctypes.c_int32), ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("active", ctypes.c_int32), ("peak_active", ctypes.c_int32), ("waiting", ctypes.c_int32),
                ("jobs", ctypes.c_int32), ("used_bytes", ctypes.c_size_t), ("budget_bytes", ctypes.c_size_t),
                ("node_iterations", ctypes.c_int64), ("reserved", ctypes.c_int32 * 8)]


class Server:
    """Interactive layout serving with continuous batching (wraps tfdp_server)."""

    def __init__(self, budget_bytes, max_active=8, chunk_iters=10):
        h = _p()
        _check(lib.tfdp_server_create(int(budget_bytes), int(max_active), int(chunk_iters), ctypes.byref(h)),
               "tfdp_server_create")
        self._h = h
        self._n = {}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib.tfdp_server_destroy(self._h)
            self._h = _p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, n, edges, xy0, params=None, iters=300):
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
        x = _host_f32(xy0, n)
        job, req = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(lib.tfdp_server_submit(self._h, int(n), e.shape[0], e.ctypes.data_as(_p) if e.shape[0] else None,
                                      x.ctypes.data_as(_p), ctypes.byref(params) if params is not None else None,
                                      int(iters), ctypes.byref(job), ctypes.byref(req)), "tfdp_server_submit")
        self._n[job.value] = int(n)
        return job.value, req.value

    def update(self, job, params, iters=50):
        req = ctypes.c_int64(0)
        _check(lib.tfdp_server_update(self._h, int(job), ctypes.byref(params), int(iters), ctypes.byref(req)),
               "tfdp_server_update")
        return req.value

    def poll(self, max_items=256, wait_ms=0):
        buf = (Done * max_items)()
        c = ctypes.c_int32(0)
        _check(lib.tfdp_server_poll(self._h, buf, int(max_items), ctypes.byref(c), int(wait_ms)), "tfdp_server_poll")
        return [{f: getattr(buf[i], f) for f, _ in Done._fields_ if f != "reserved"} for i in range(c.value)]

    def positions(self, job):
        a = np.empty((self._n[job], 2), dtype=np.float32)
        _check(lib.tfdp_server_get_positions(self._h, int(job), a.ctypes.data_as(_p)), "tfdp_server_get_positions")
        return a

    def release(self, job):
        _check(lib.tfdp_server_release(self._h, int(job)), "tfdp_server_release")

    def stats(self):
        s = ServerStats()
        _check(lib.tfdp_server_get_stats(self._h, ctypes.byref(s)), "tfdp_server_get_stats")
        return {f: getattr(s, f) for f, _ in ServerStats._fields_ if f != "reserved"}
