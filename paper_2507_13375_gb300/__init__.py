"""GB300-native layer assignment (GAP-LA, arxiv 2507.13375): Python binding.

This module only marshals arguments to the C ABI of include/gapla.h
(libgapla.so, built in-tree for sm_103a); every step of the round runs in the
library's CUDA kernels.  PyTorch provides device memory and streams.  There is
no CPU path: without the built library every call raises.

Functions with the C names (``la_create``, ``la_load_grid``, ``la_load_nets``,
``la_assign_round``, ``la_elmore``, ``la_elmore_backward``, ...) take the
context handle first; ``LayerAssigner`` wraps them, and ``ElmoreFn`` exposes
the Elmore delay and its hand-written adjoint as a ``torch.autograd.Function``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgapla.so")

LA_OK, LA_ERR_INVALID, LA_ERR_CUDA, LA_ERR_OOM, LA_ERR_STATE, LA_ERR_TIMEOUT, LA_ERR_DEVICE_CHECK = range(7)
LA_MODE_PLAIN, LA_MODE_BATCHED = 0, 1
LA_WEIGHTS_EQ4, LA_WEIGHTS_ADJOINT = 0, 1
LA_MAX_LAYERS = 16
_STATUS = {0: "LA_OK", 1: "LA_ERR_INVALID", 2: "LA_ERR_CUDA", 3: "LA_ERR_OOM", 4: "LA_ERR_STATE",
           5: "LA_ERR_TIMEOUT", 6: "LA_ERR_DEVICE_CHECK"}
# Default round weights (the paper prints none; Fig. 10 sweeps them).
DEFAULT_WEIGHTS = dict(w_cong=1.0, w_via=1.0, w_cap=0.1, w_d=1e-3, hist_w=1.0)

# Every symbol include/gapla.h declares.
EXPORTS = ("la_create", "la_destroy", "la_last_error", "la_set_stream", "la_device_bytes", "la_check",
           "la_launch_count",
           "la_load_grid", "la_load_nets", "la_assign_round", "la_get_assignment", "la_set_assignment",
           "la_get_net_cost", "la_get_state", "la_set_state", "la_rc_from_assignment", "la_elmore",
           "la_elmore_backward", "la_elmore_assignment", "la_reweight_adjoint", "la_get_weights",
           "la_inject_fault", "la_probe_fp64", "la_commit_demand", "la_logistic_pin_weight",
           "la_partition_batches", "la_elmore_static")
LA_STATIC_MAX_NODES = 1 << 21


class LaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class GridDesc(ctypes.Structure):
    _fields_ = [("X", ctypes.c_int32), ("Y", ctypes.c_int32), ("L", ctypes.c_int32),
                ("dir", ctypes.c_void_p), ("cap", ctypes.c_void_p), ("unit_r", ctypes.c_void_p),
                ("unit_c", ctypes.c_void_p), ("via_r", ctypes.c_void_p), ("via_c", ctypes.c_double),
                ("ofw", ctypes.c_void_p)]


class NetDesc(ctypes.Structure):
    _fields_ = [("num_nets", ctypes.c_int64), ("num_nodes", ctypes.c_int64), ("net_ptr", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("parent", ctypes.c_void_p),
                ("pin_layer", ctypes.c_void_p), ("sink_cap", ctypes.c_void_p), ("kappa", ctypes.c_void_p),
                ("r_drv", ctypes.c_void_p), ("batch", ctypes.c_void_p)]


class RoundParams(ctypes.Structure):
    _fields_ = [("w_cong", ctypes.c_double), ("w_via", ctypes.c_double), ("w_cap", ctypes.c_double),
                ("w_d", ctypes.c_double), ("hist_w", ctypes.c_double), ("mode", ctypes.c_int32),
                ("weights", ctypes.c_int32), ("reset", ctypes.c_int32), ("no_look_ahead", ctypes.c_int32),
                ("tail_threshold", ctypes.c_int32), ("force_split", ctypes.c_int32),
                ("local_demand", ctypes.c_int32), ("reweight_adjoint", ctypes.c_int32)]


class RoundStats(ctypes.Structure):
    _fields_ = [("total_cost", ctypes.c_double), ("tof", ctypes.c_double), ("relu_overflow", ctypes.c_int64),
                ("vias", ctypes.c_int64), ("wl", ctypes.c_int64),
                ("wl_per_layer", ctypes.c_int64 * LA_MAX_LAYERS), ("ms", ctypes.c_double),
                ("ms_dp", ctypes.c_double), ("ms_backtrack", ctypes.c_double), ("ms_demand", ctypes.c_double),
                ("launches", ctypes.c_int64), ("batch_split", ctypes.c_int32), ("batch_block", ctypes.c_int32),
                ("batch_big_nets", ctypes.c_int64), ("batch_cached", ctypes.c_int32), ("batch_trials", ctypes.c_int32),
                ("batch_tune_ms", ctypes.c_double), ("batch_levels", ctypes.c_int32),
                ("batch_tail_level", ctypes.c_int32), ("batch_graph_captured", ctypes.c_int32)]


_lib = None


def library() -> ctypes.CDLL:
    """The loaded libgapla.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, P = ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER
    sig = {
        "la_create": [P(vp), ctypes.c_int, vp], "la_destroy": [vp], "la_set_stream": [vp, vp],
        "la_device_bytes": [vp, P(ctypes.c_size_t)], "la_check": [vp], "la_launch_count": [vp, P(ctypes.c_int64)],
        "la_load_grid": [vp, P(GridDesc)], "la_load_nets": [vp, P(NetDesc)],
        "la_assign_round": [vp, P(RoundParams), P(RoundStats)],
        "la_get_assignment": [vp, vp, vp, vp], "la_set_assignment": [vp, vp, vp, vp],
        "la_get_net_cost": [vp, vp], "la_get_state": [vp, vp, vp], "la_set_state": [vp, vp, vp],
        "la_rc_from_assignment": [vp, vp, vp], "la_elmore": [vp, vp, vp, vp],
        "la_elmore_backward": [vp, vp, vp, vp, vp, vp], "la_elmore_assignment": [vp, vp],
        "la_reweight_adjoint": [vp],
        "la_get_weights": [vp, i32, vp, vp], "la_inject_fault": [vp, ctypes.c_int],
        "la_probe_fp64": [ctypes.c_int, vp, P(ctypes.c_double)],
        "la_commit_demand": [vp, vp, P(RoundStats)],
        "la_logistic_pin_weight": [vp, vp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double, vp,
                                   vp],
        "la_partition_batches": [vp, vp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, vp,
                                 P(ctypes.c_int32), vp],
        "la_elmore_static": [P(NetDesc), vp, vp, vp, i32, vp, ctypes.c_double, vp, vp, vp, vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.la_last_error.argtypes = [vp]
    lib.la_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check(ctx, status):
    if status != LA_OK:
        msg = library().la_last_error(ctx)
        raise LaError(status, msg.decode() if msg else "")


def _dev(x, dtype, device):
    """A contiguous CUDA tensor of `dtype` (copied from numpy/torch if needed)."""
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x))
    return x.to(device=device, dtype=dtype).contiguous()


# ----------------------------- C-named calls -----------------------------
def la_create(device: int = 0, stream=None):
    lib = library()
    h = ctypes.c_void_p()
    if stream is None:
        stream = torch.cuda.current_stream(device).cuda_stream
    st = lib.la_create(ctypes.byref(h), int(device), ctypes.c_void_p(stream))
    if st != LA_OK:
        raise LaError(st, lib.la_last_error(None).decode())
    return h


def la_destroy(ctx):
    library().la_destroy(ctx)


def la_set_stream(ctx, stream):
    _check(ctx, library().la_set_stream(ctx, ctypes.c_void_p(stream)))


def la_check(ctx):
    _check(ctx, library().la_check(ctx))


def la_launch_count(ctx) -> int:
    n = ctypes.c_int64()
    _check(ctx, library().la_launch_count(ctx, ctypes.byref(n)))
    return int(n.value)


def la_device_bytes(ctx) -> int:
    n = ctypes.c_size_t()
    _check(ctx, library().la_device_bytes(ctx, ctypes.byref(n)))
    return int(n.value)


def la_load_grid(ctx, grid: dict, device: int = 0):
    """grid: X, Y, L, dir, cap (public edge layout), unit_r, unit_c, via_r, via_c, ofw."""
    keep = [np.ascontiguousarray(grid["dir"], np.int8), np.ascontiguousarray(grid["unit_r"], np.float64),
            np.ascontiguousarray(grid["unit_c"], np.float64), np.ascontiguousarray(grid["via_r"], np.float64),
            np.ascontiguousarray(grid["ofw"], np.float64)]
    cap = _dev(grid["cap"], torch.int32, device)
    d = GridDesc(int(grid["X"]), int(grid["Y"]), int(grid["L"]), keep[0].ctypes.data, cap.data_ptr(),
                 keep[1].ctypes.data, keep[2].ctypes.data, keep[3].ctypes.data, float(grid["via_c"]),
                 keep[4].ctypes.data)
    _check(ctx, library().la_load_grid(ctx, ctypes.byref(d)))
    torch.cuda.current_stream(device).synchronize()


def la_load_nets(ctx, forest: dict, device: int = 0):
    """forest: net_ptr, x, y, parent, pin_layer, sink_cap, kappa, r_drv (numpy or torch); an optional
    "batch" (int32 per net) splits a round into sequential batches."""
    t = dict(net_ptr=_dev(forest["net_ptr"], torch.int64, device), x=_dev(forest["x"], torch.int32, device),
             y=_dev(forest["y"], torch.int32, device), parent=_dev(forest["parent"], torch.int32, device),
             pin_layer=_dev(forest["pin_layer"], torch.int8, device),
             sink_cap=_dev(forest["sink_cap"], torch.float64, device),
             kappa=_dev(forest["kappa"], torch.float64, device), r_drv=_dev(forest["r_drv"], torch.float64, device))
    batch = forest.get("batch")
    if batch is not None:
        t["batch"] = _dev(batch, torch.int32, device)
    d = NetDesc(int(t["r_drv"].numel()), int(t["x"].numel()), *(t[k].data_ptr() for k in
                ("net_ptr", "x", "y", "parent", "pin_layer", "sink_cap", "kappa", "r_drv")),
                t["batch"].data_ptr() if batch is not None else None)
    _check(ctx, library().la_load_nets(ctx, ctypes.byref(d)))


def la_assign_round(ctx, mode: int = LA_MODE_PLAIN, weights: int = LA_WEIGHTS_EQ4, reset: bool = False,
                    stats: bool = True, look_ahead: bool = True, tail_threshold: int = 0, force_split: int = 0,
                    local_demand: bool = False, reweight_adjoint: bool = False, **w):
    ww = dict(DEFAULT_WEIGHTS)
    ww.update(w)
    p = RoundParams(ww["w_cong"], ww["w_via"], ww["w_cap"], ww["w_d"], ww["hist_w"], int(mode), int(weights),
                    1 if reset else 0, 0 if look_ahead else 1, int(tail_threshold), int(force_split),
                    1 if local_demand else 0, int(reweight_adjoint))
    if not stats:
        _check(ctx, library().la_assign_round(ctx, ctypes.byref(p), None))
        return None
    s = RoundStats()
    _check(ctx, library().la_assign_round(ctx, ctypes.byref(p), ctypes.byref(s)))
    return dict(total_cost=s.total_cost, tof=s.tof, relu_overflow=s.relu_overflow, vias=s.vias, wl=s.wl,
                wl_per_layer=list(s.wl_per_layer), ms=s.ms, ms_dp=s.ms_dp, ms_backtrack=s.ms_backtrack,
                ms_demand=s.ms_demand, launches=s.launches, batch_split=s.batch_split, batch_block=s.batch_block,
                batch_big_nets=s.batch_big_nets, batch_cached=s.batch_cached, batch_trials=s.batch_trials,
                batch_tune_ms=s.batch_tune_ms, batch_levels=s.batch_levels, batch_tail_level=s.batch_tail_level,
                batch_graph_captured=s.batch_graph_captured)


def la_commit_demand(ctx, demand, stats: bool = True):
    """End a local-demand round with the demand summed over every shard."""
    if not stats:
        _check(ctx, library().la_commit_demand(ctx, _ptr(demand), None))
        return None
    s = RoundStats()
    _check(ctx, library().la_commit_demand(ctx, _ptr(demand), ctypes.byref(s)))
    return dict(tof=s.tof, relu_overflow=s.relu_overflow)


def la_get_assignment(ctx, layer, b, t):
    _check(ctx, library().la_get_assignment(ctx, _ptr(layer), _ptr(b), _ptr(t)))


def la_set_assignment(ctx, layer, b, t):
    _check(ctx, library().la_set_assignment(ctx, _ptr(layer), _ptr(b), _ptr(t)))


def la_get_net_cost(ctx, J):
    _check(ctx, library().la_get_net_cost(ctx, _ptr(J)))


def la_get_state(ctx, demand, history):
    _check(ctx, library().la_get_state(ctx, _ptr(demand), _ptr(history)))


def la_set_state(ctx, demand, history):
    _check(ctx, library().la_set_state(ctx, _ptr(demand), _ptr(history)))


def la_rc_from_assignment(ctx, R, C):
    _check(ctx, library().la_rc_from_assignment(ctx, _ptr(R), _ptr(C)))


def la_elmore(ctx, R, C, delay):
    _check(ctx, library().la_elmore(ctx, _ptr(R), _ptr(C), _ptr(delay)))


def la_elmore_assignment(ctx, delay):
    _check(ctx, library().la_elmore_assignment(ctx, _ptr(delay)))


def la_elmore_backward(ctx, R, C, grad, dR, dC):
    _check(ctx, library().la_elmore_backward(ctx, _ptr(R), _ptr(C), _ptr(grad), _ptr(dR), _ptr(dC)))


def la_reweight_adjoint(ctx):
    _check(ctx, library().la_reweight_adjoint(ctx))


def la_get_weights(ctx, source, W, rho):
    _check(ctx, library().la_get_weights(ctx, int(source), _ptr(W), _ptr(rho)))


def la_inject_fault(ctx, code: int):
    """The next step of the context that can fail in this way reports `code`
    from the host side (a test hook: nothing faults on the device)."""
    _check(ctx, library().la_inject_fault(ctx, int(code)))


def la_logistic_pin_weight(pin_layer, slack, wns: float, k: float = 10.0, b: float = 0.3, stream=None):
    """Sec. III-C pin weights (CUDA tensors in, a new float64 tensor out): the
    logistic of slack / WNS at pins, 0 elsewhere (see include/gapla.h)."""
    lib = library()
    pin_layer, slack = pin_layer.contiguous(), slack.contiguous()
    if pin_layer.dtype != torch.int8 or slack.dtype != torch.float64 or pin_layer.numel() != slack.numel():
        raise LaError(LA_ERR_INVALID, "la_logistic_pin_weight: int8 pin_layer and float64 slack of one length")
    w = torch.empty_like(slack)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    st = lib.la_logistic_pin_weight(_ptr(pin_layer), _ptr(slack), int(slack.numel()), float(wns), float(k), float(b),
                                    _ptr(w), ctypes.c_void_p(stream))
    if st != LA_OK:
        raise LaError(st, lib.la_last_error(None).decode())
    return w


def la_partition_batches(crit, slack=None, critical_frac: float = 0.5, slack_ratio: float = 0.7, stream=None):
    """Alg. 1's partition of the nets into batches on the GPU (see
    include/gapla.h): per-net criticality and optional slack (CUDA float64
    tensors) -> (int32 batch ids, number of batches)."""
    lib = library()
    crit = crit.contiguous()
    if crit.dtype != torch.float64 or (slack is not None and (slack.dtype != torch.float64
                                                              or slack.numel() != crit.numel())):
        raise LaError(LA_ERR_INVALID, "la_partition_batches: float64 crit and slack of one length")
    slack = None if slack is None else slack.contiguous()
    out = torch.empty(crit.numel(), dtype=torch.int32, device=crit.device)
    nb = ctypes.c_int32()
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    st = lib.la_partition_batches(_ptr(crit), _ptr(slack), int(crit.numel()), float(critical_frac),
                                  float(slack_ratio), _ptr(out), ctypes.byref(nb), ctypes.c_void_p(stream))
    if st != LA_OK:
        raise LaError(st, lib.la_last_error(None).decode())
    return out, int(nb.value)


def la_probe_fp64(device: int = 0, stream=None) -> float:
    """FP64 fused multiply-adds per second that this GPU sustains (measured)."""
    lib = library()
    if stream is None:
        stream = torch.cuda.current_stream(device).cuda_stream
    r = ctypes.c_double()
    st = lib.la_probe_fp64(int(device), ctypes.c_void_p(stream), ctypes.byref(r))
    if st != LA_OK:
        raise LaError(st, lib.la_last_error(None).decode())
    return float(r.value)


def la_elmore_static(nets: dict, layer, b, t, L: int, via_r, via_c: float, R, C, delay, stream=None,
                     num_nodes: int | None = None):
    """The allocation-free Elmore forward pass (see include/gapla.h).

    nets: CUDA tensors net_ptr (int64), parent (int32), pin_layer (int8),
    sink_cap and r_drv (float64); layer, b, t (int8), R, C, delay (float64):
    CUDA tensors in input order, all on the current CUDA device.  The library
    allocates nothing on the device for this call.  The types, device and
    sizes are checked here before the C call (the C side sees bare pointers);
    `num_nodes` overrides the node count passed to C (only to exercise the
    library's own size refusal: the arrays are not read then)."""
    lib = library()
    L = int(L)
    keep = np.ascontiguousarray(via_r, np.float64).ravel()
    if keep.size < L - 1:
        raise LaError(LA_ERR_INVALID, f"la_elmore_static: via_r has {keep.size} entries, needs L - 1 = {L - 1}")
    dev = torch.device("cuda", torch.cuda.current_device())
    V = int(nets["parent"].numel())
    N = int(nets["r_drv"].numel())
    want = dict(net_ptr=(torch.int64, N + 1), parent=(torch.int32, V), pin_layer=(torch.int8, V),
                sink_cap=(torch.float64, V), r_drv=(torch.float64, N))
    arrays = [(k, nets[k]) + want[k] for k in want]
    arrays += [(k, x, dt, V) for k, x, dt in (("layer", layer, torch.int8), ("b", b, torch.int8),
                                              ("t", t, torch.int8), ("R", R, torch.float64),
                                              ("C", C, torch.float64), ("delay", delay, torch.float64))]
    for k, x, dt, n in arrays:
        if not isinstance(x, torch.Tensor) or x.device != dev or x.dtype != dt or not x.is_contiguous():
            raise LaError(LA_ERR_INVALID, f"la_elmore_static: {k} must be a contiguous {dt} tensor on {dev}")
        if num_nodes is None and x.numel() != n:
            raise LaError(LA_ERR_INVALID, f"la_elmore_static: {k} has {x.numel()} entries, needs {n}")
    z = lambda k: nets[k].data_ptr() if k in nets and nets[k] is not None else None
    d = NetDesc(N, int(num_nodes if num_nodes is not None else V),
                z("net_ptr"), z("x"), z("y"), z("parent"), z("pin_layer"), z("sink_cap"), z("kappa"), z("r_drv"))
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    st = lib.la_elmore_static(ctypes.byref(d), _ptr(layer), _ptr(b), _ptr(t), L, keep.ctypes.data,
                              float(via_c), _ptr(R), _ptr(C), _ptr(delay), ctypes.c_void_p(stream))
    if st != LA_OK:
        raise LaError(st, lib.la_last_error(None).decode())


# ------------------------------ convenience ------------------------------
class LayerAssigner:
    """Owns one library context on one CUDA device; arrays are torch CUDA tensors."""

    def __init__(self, device: int = 0):
        self.device = int(device)
        self.dev = torch.device("cuda", self.device)
        self.ctx = la_create(self.device)
        self.V = self.N = self.E = 0

    def _sync_stream(self):
        la_set_stream(self.ctx, torch.cuda.current_stream(self.device).cuda_stream)

    def close(self):
        if self.ctx is not None:
            la_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_grid(self, grid: dict):
        self._sync_stream()
        la_load_grid(self.ctx, grid, self.device)
        L, X, Y = int(grid["L"]), int(grid["X"]), int(grid["Y"])
        self.E = sum(Y * (X - 1) if int(grid["dir"][l]) == 0 else X * (Y - 1) for l in range(L))

    def load_nets(self, forest: dict):
        self._sync_stream()
        la_load_nets(self.ctx, forest, self.device)
        self.N = int(len(forest["r_drv"]))
        self.V = int(len(forest["x"]))

    def assign_round(self, mode=LA_MODE_PLAIN, weights=LA_WEIGHTS_EQ4, reset=False, stats=True, look_ahead=True,
                     tail_threshold=0, force_split=0, local_demand=False, reweight_adjoint=False, **w):
        self._sync_stream()
        return la_assign_round(self.ctx, mode, weights, reset, stats, look_ahead, tail_threshold, force_split,
                               local_demand, reweight_adjoint, **w)

    def commit_demand(self, D, stats=True):
        """D: the demand summed over every shard (public layout, int32, this device)."""
        self._sync_stream()
        return la_commit_demand(self.ctx, _dev(D, torch.int32, self.dev), stats)

    def get_assignment(self):
        self._sync_stream()
        out = [torch.empty(self.V, dtype=torch.int8, device=self.dev) for _ in range(3)]
        la_get_assignment(self.ctx, *out)
        return tuple(out)

    def set_assignment(self, layer, b, t):
        self._sync_stream()
        la_set_assignment(self.ctx, *(_dev(x, torch.int8, self.dev) for x in (layer, b, t)))

    def get_net_cost(self):
        self._sync_stream()
        J = torch.empty(self.N, dtype=torch.float64, device=self.dev)
        la_get_net_cost(self.ctx, J)
        return J

    def get_state(self):
        self._sync_stream()
        D = torch.empty(self.E, dtype=torch.int32, device=self.dev)
        H = torch.empty(self.E, dtype=torch.int32, device=self.dev)
        la_get_state(self.ctx, D, H)
        return D, H

    def set_state(self, D=None, H=None):
        self._sync_stream()
        la_set_state(self.ctx, None if D is None else _dev(D, torch.int32, self.dev),
                     None if H is None else _dev(H, torch.int32, self.dev))

    def rc_from_assignment(self):
        self._sync_stream()
        R = torch.empty(self.V, dtype=torch.float64, device=self.dev)
        C = torch.empty_like(R)
        la_rc_from_assignment(self.ctx, R, C)
        return R, C

    def elmore(self, R, C):
        self._sync_stream()
        R, C = R.contiguous(), C.contiguous()
        d = torch.empty_like(R)
        la_elmore(self.ctx, R, C, d)
        return d

    def elmore_assignment(self):
        """Elmore delays (input order) of the current assignment, R and C taken
        from its layers inside the level passes."""
        self._sync_stream()
        d = torch.empty(self.V, dtype=torch.float64, device=self.dev)
        la_elmore_assignment(self.ctx, d)
        return d

    def elmore_backward(self, R, C, grad):
        self._sync_stream()
        dR, dC = torch.empty_like(R), torch.empty_like(C)
        la_elmore_backward(self.ctx, R.contiguous(), C.contiguous(), grad.contiguous(), dR, dC)
        return dR, dC

    def reweight_adjoint(self):
        self._sync_stream()
        la_reweight_adjoint(self.ctx)

    def get_weights(self, source=LA_WEIGHTS_EQ4):
        self._sync_stream()
        W = torch.empty(self.V, dtype=torch.float64, device=self.dev)
        rho = torch.empty_like(W)
        la_get_weights(self.ctx, source, W, rho)
        return W, rho

    def device_bytes(self) -> int:
        return la_device_bytes(self.ctx)

    def launch_count(self) -> int:
        return la_launch_count(self.ctx)


class ElmoreFn(torch.autograd.Function):
    """delay = Elmore(R_seg, C_seg) on the assigner's current assignment; the
    backward pass is the library's adjoint kernel (dL/dR_seg, dL/dC_seg)."""

    @staticmethod
    def forward(ctx, assigner: LayerAssigner, R, C):
        ctx.assigner = assigner
        ctx.save_for_backward(R, C)
        return assigner.elmore(R.detach(), C.detach())

    @staticmethod
    def backward(ctx, grad):
        R, C = ctx.saved_tensors
        dR, dC = ctx.assigner.elmore_backward(R.detach(), C.detach(), grad.contiguous())
        return None, dR, dC
