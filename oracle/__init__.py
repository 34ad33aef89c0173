"""Plain FP64 CPU oracle of the GAP-LA layer-assignment round (arxiv 2507.13375).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg (``bench.py`` cpu_baseline / ``--impl reference``)
may import this package.  The CUDA library (``paper_2507_13375_gb300``) never
imports it, and the two share no code: the only thing both consume is the
seeded input of ``forestgen``.

Contents
  la_oracle.c  the DP of Alg. 3 (every via stack enumerated per parent layer),
               the root selection and backtrack of Alg. 4, the demand / via /
               history update, the Eq. 4 weights and the look-ahead r_est of
               Sec. III-D, the Elmore delay (Sec. II-C, III-D) and its adjoint.
  brute.py     independent pure-Python pins: the cost J of an assignment
               evaluated straight from the RC model, brute-force enumeration
               of all layer vectors of tiny nets, and the textbook O(n^2)
               Elmore path sum.

Parity status of each function (what pins it, see tests/test_oracle_pins.py):
  dp           pinned: = brute force exactly when w_d = 0 (separable) and when
               all unit R are equal with zero via R (the look-ahead is then the
               exact upstream resistance), and on single-segment nets for any
               parameters; J = cost of the returned assignment evaluated from
               the RC model.  In general only J(brute) <= J(dp) holds: the
               look-ahead DP is a heuristic (Sec. III-D).
  penalty      pinned to the closed form exp() values of Eq. 3 and the
               saturation bounds.
  demand       pinned by invariants (per-GCell layer sums = 2D demand,
               total = wirelength, vias = stack heights, H update).
  elmore       pinned to the textbook path sum, the distributed-wire closed
               form, and the d_34 = R_34 (C4+C5+C6+C7) example of Sec. III-D.
  elmore_backward  pinned to the closed forms dT/dR = Wsum Cdown and
               dT/dC = sum of R Wsum above, and to central differences.
  logistic_pin_weight  pinned to the logistic's fixed points: 1/2 at
               slack / WNS = b, about 1 at the worst slack, symmetry
               w(b + d) + w(b - d) = 1, monotone in the slack ratio.
  partition_batches  pinned by hand-built nets on every interval edge of
               Alg. 1 (criticality halvings, slack edges 1 - j^2/100) and by
               the interval rule checked net by net in exact arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_LIBDIR, "liboracle.so")
_lib = None

# Default weights of the round (the paper prints none; Fig. 10 sweeps them).
DEFAULT_WEIGHTS = dict(w_cong=1.0, w_via=1.0, w_cap=0.1, w_d=1e-3, hist_w=1.0)


def build(force: bool = False) -> str:
    """Compile la_oracle.c into oracle/_lib/liboracle.so (gcc, -ffp-contract=off)."""
    src = os.path.join(_HERE, "la_oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                           "-ffp-contract=off", "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


class _Grid(ctypes.Structure):
    _fields_ = [("X", ctypes.c_int32), ("Y", ctypes.c_int32), ("L", ctypes.c_int32),
                ("dir", ctypes.c_void_p), ("cap", ctypes.c_void_p), ("unit_r", ctypes.c_void_p),
                ("unit_c", ctypes.c_void_p), ("via_r", ctypes.c_void_p), ("via_c", ctypes.c_double),
                ("ofw", ctypes.c_void_p)]


class _Forest(ctypes.Structure):
    _fields_ = [("num_nets", ctypes.c_int64), ("num_nodes", ctypes.c_int64),
                ("net_ptr", ctypes.c_void_p), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("parent", ctypes.c_void_p), ("pin_layer", ctypes.c_void_p),
                ("sink_cap", ctypes.c_void_p), ("kappa", ctypes.c_void_p), ("r_drv", ctypes.c_void_p)]


class _Weights(ctypes.Structure):
    _fields_ = [("w_cong", ctypes.c_double), ("w_via", ctypes.c_double), ("w_cap", ctypes.c_double),
                ("w_d", ctypes.c_double), ("hist_w", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [("vias", ctypes.c_int64), ("wl", ctypes.c_int64), ("relu_overflow", ctypes.c_int64),
                ("tof", ctypes.c_double), ("wl_per_layer", ctypes.c_int64 * 16)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, P = ctypes.c_void_p, ctypes.POINTER
        lib.or_num_edges.restype = ctypes.c_int64
        lib.or_num_edges.argtypes = [P(_Grid)]
        lib.or_penalty_table.argtypes = [P(_Grid), vp]
        lib.or_penalty.argtypes = [P(_Grid), vp, vp, ctypes.c_double, vp]
        lib.or_weights_eq4.argtypes = [P(_Grid), P(_Forest), vp, vp]
        lib.or_dp.restype = ctypes.c_int
        lib.or_dp.argtypes = [P(_Grid), P(_Forest), P(_Weights), vp, vp, vp, ctypes.c_int64,
                              ctypes.c_int64, ctypes.c_int] + [vp] * 6
        lib.or_demand.argtypes = [P(_Grid), P(_Forest), vp, vp, vp, vp, vp, vp, P(_Stats)]
        lib.or_rc_from_assignment.argtypes = [P(_Grid), P(_Forest), vp, vp, vp]
        lib.or_elmore.argtypes = [P(_Grid), P(_Forest)] + [vp] * 8
        lib.or_elmore_backward.argtypes = [P(_Grid), P(_Forest)] + [vp] * 11
        lib.or_logistic_pin_weight.argtypes = [ctypes.c_int64, vp, vp, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, vp]
        lib.or_partition_batches.restype = ctypes.c_int32
        lib.or_partition_batches.argtypes = [ctypes.c_int64, vp, vp, ctypes.c_double, ctypes.c_double, vp]
        for fn in ("or_penalty_table", "or_penalty", "or_weights_eq4", "or_demand",
                   "or_rc_from_assignment", "or_elmore", "or_elmore_backward", "or_logistic_pin_weight"):
            getattr(lib, fn).restype = None
        _lib = lib
    return _lib


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


class _Keep:
    """Holds converted arrays alive while the C structs point at them."""

    def __init__(self):
        self.refs = []

    def ptr(self, a, dtype):
        a = _c(a, dtype)
        self.refs.append(a)
        return a.ctypes.data


def _grid(grid, keep):
    g = _Grid()
    g.X, g.Y, g.L = int(grid["X"]), int(grid["Y"]), int(grid["L"])
    g.dir = keep.ptr(grid["dir"], np.int8)
    g.cap = keep.ptr(grid["cap"], np.int32)
    g.unit_r = keep.ptr(grid["unit_r"], np.float64)
    g.unit_c = keep.ptr(grid["unit_c"], np.float64)
    g.via_r = keep.ptr(grid["via_r"], np.float64)
    g.via_c = float(grid["via_c"])
    g.ofw = keep.ptr(grid["ofw"], np.float64)
    return g


def _forest(forest, keep):
    f = _Forest()
    f.num_nets, f.num_nodes = int(forest["num_nets"]), int(forest["num_nodes"])
    f.net_ptr = keep.ptr(forest["net_ptr"], np.int64)
    f.x = keep.ptr(forest["x"], np.int32)
    f.y = keep.ptr(forest["y"], np.int32)
    f.parent = keep.ptr(forest["parent"], np.int32)
    f.pin_layer = keep.ptr(forest["pin_layer"], np.int8)
    f.sink_cap = keep.ptr(forest["sink_cap"], np.float64)
    f.kappa = keep.ptr(forest["kappa"], np.float64)
    f.r_drv = keep.ptr(forest["r_drv"], np.float64)
    return f


def _weights(w):
    ww = dict(DEFAULT_WEIGHTS)
    ww.update(w or {})
    x = _Weights()
    for k in ("w_cong", "w_via", "w_cap", "w_d", "hist_w"):
        setattr(x, k, float(ww[k]))
    return x


def num_edges(grid) -> int:
    keep = _Keep()
    return int(_load().or_num_edges(ctypes.byref(_grid(grid, keep))))


def penalty_table(grid) -> np.ndarray:
    """T[l, s, k+64]: llround(min(ofw_l e^{s k} 2^24, 2^48)), s index 0 -> 0.5, 1 -> 1.5."""
    keep = _Keep()
    T = np.empty((int(grid["L"]), 2, 129), np.int64)
    _load().or_penalty_table(ctypes.byref(_grid(grid, keep)), T.ctypes.data)
    return T


def penalty(grid, D, H, hist_w: float) -> np.ndarray:
    """Per-edge congestion penalty (int64, 2^-24 units) of snapshot (D, H)."""
    keep = _Keep()
    pen = np.empty(num_edges(grid), np.int64)
    _load().or_penalty(ctypes.byref(_grid(grid, keep)), keep.ptr(D, np.int32), keep.ptr(H, np.int32),
                       float(hist_w), pen.ctypes.data)
    return pen


def weights_eq4(grid, forest):
    """(W, r_est) of the plain mode: Eq. 4 max criticality and distance-based r_est."""
    keep = _Keep()
    V = int(forest["num_nodes"])
    W, rho = np.empty(V), np.empty(V)
    _load().or_weights_eq4(ctypes.byref(_grid(grid, keep)), ctypes.byref(_forest(forest, keep)),
                           W.ctypes.data, rho.ctypes.data)
    return W, rho


def dp(grid, forest, weights, pen, W, rho, nets=None, threads: int = 0, tables: bool = False) -> dict:
    """Alg. 3 + Alg. 4 on the nets in range `nets` = (lo, hi) (default: all).

    Returns layer, b, t (int8, V; only the range's nodes are written), J (f64, N;
    only the range), threads used, and with tables=True the per-(node, layer)
    A and Cc tables (NaN where the layer is not a candidate)."""
    keep = _Keep()
    V, N, L = int(forest["num_nodes"]), int(forest["num_nets"]), int(grid["L"])
    lo, hi = (0, N) if nets is None else nets
    out = dict(layer=np.full(V, -1, np.int8), b=np.full(V, -1, np.int8), t=np.full(V, -1, np.int8),
               J=np.full(N, np.nan))
    A = Cc = None
    if tables:
        A = np.full((V, L), np.nan)
        Cc = np.full((V, L), np.nan)
    w = _weights(weights)
    used = _load().or_dp(ctypes.byref(_grid(grid, keep)), ctypes.byref(_forest(forest, keep)),
                         ctypes.byref(w), keep.ptr(pen, np.int64), keep.ptr(W, np.float64),
                         keep.ptr(rho, np.float64), int(lo), int(hi), int(threads),
                         out["layer"].ctypes.data, out["b"].ctypes.data, out["t"].ctypes.data,
                         out["J"].ctypes.data, A.ctypes.data if tables else None,
                         Cc.ctypes.data if tables else None)
    if used < 0:
        raise RuntimeError("oracle DP found a node without a valid via stack")
    out["threads"] = used
    if tables:
        out["A"], out["Cc"] = A, Cc
    return out


def demand(grid, forest, layer, b, t, H_in):
    """Demand D of an assignment, H_out = H_in + max(0, D - C), and statistics."""
    keep = _Keep()
    E = num_edges(grid)
    D, H = np.empty(E, np.int32), np.empty(E, np.int32)
    st = _Stats()
    _load().or_demand(ctypes.byref(_grid(grid, keep)), ctypes.byref(_forest(forest, keep)),
                      keep.ptr(layer, np.int8), keep.ptr(b, np.int8), keep.ptr(t, np.int8),
                      keep.ptr(H_in, np.int32), D.ctypes.data, H.ctypes.data, ctypes.byref(st))
    stats = dict(vias=st.vias, wl=st.wl, relu_overflow=st.relu_overflow, tof=st.tof,
                 wl_per_layer=np.array(st.wl_per_layer[: int(grid["L"])], np.int64))
    return D, H, stats


def assign_round(grid, forest, weights=None, D=None, H=None, W=None, rho=None, threads: int = 0,
                 tables: bool = False) -> dict:
    """One full round from snapshot (D, H) (zeros if None): penalty, DP, backtrack,
    then the new demand and history.  W/rho default to the Eq. 4 weights."""
    ww = dict(DEFAULT_WEIGHTS)
    ww.update(weights or {})
    E = num_edges(grid)
    D = np.zeros(E, np.int32) if D is None else D
    H = np.zeros(E, np.int32) if H is None else H
    if W is None or rho is None:
        W, rho = weights_eq4(grid, forest)
    pen = penalty(grid, D, H, ww["hist_w"])
    out = dp(grid, forest, ww, pen, W, rho, threads=threads, tables=tables)
    Dn, Hn, st = demand(grid, forest, out["layer"], out["b"], out["t"], H)
    st["total_cost"] = float(np.sum(out["J"]))
    out.update(D=Dn, H=Hn, stats=st, pen=pen, W=W, rho=rho)
    return out


def _net_subset(forest, nets):
    """The sub-forest of the nets in `nets` (ascending), with the node ids of
    the original forest that it keeps."""
    ptr = forest["net_ptr"]
    sizes = (ptr[1:] - ptr[:-1])[nets]
    nodes = np.concatenate([np.arange(ptr[n], ptr[n + 1]) for n in nets]) if len(nets) else np.zeros(0, np.int64)
    sub = {k: forest[k][nodes] for k in ("x", "y", "parent", "pin_layer", "sink_cap", "kappa")}
    sub["r_drv"] = forest["r_drv"][nets]
    sub["net_ptr"] = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    sub["num_nets"], sub["num_nodes"] = len(nets), int(len(nodes))
    return sub, nodes


def assign_round_batches(grid, forest, batch, weights=None, D=None, H=None, W=None, rho=None, layer_prev=None,
                         threads: int = 0) -> dict:
    """A round in sequential batches (Sec. III-A; Alg. 2 over the batches BS):
    the batches go in increasing batch id.  Batch k is assigned against the
    demand in which the nets of batches < k carry their new assignment of this
    round and every other net its previous one (`layer_prev`; none in a round
    that starts from D = 0).  H is the round's start history throughout; after
    the last batch the new demand and history follow as in a single round."""
    ww = dict(DEFAULT_WEIGHTS)
    ww.update(weights or {})
    E = num_edges(grid)
    N, V = int(forest["num_nets"]), int(forest["num_nodes"])
    D_cur = (np.zeros(E, np.int64) if D is None else D.astype(np.int64)).copy()
    H = np.zeros(E, np.int32) if H is None else H
    if W is None or rho is None:
        W, rho = weights_eq4(grid, forest)
    layer, b, t = np.full(V, -1, np.int8), np.full(V, -1, np.int8), np.full(V, -1, np.int8)
    J = np.full(N, np.nan)
    zeros = np.zeros(E, np.int32)
    net_of = np.repeat(np.arange(N), np.diff(forest["net_ptr"]))
    for k in np.unique(batch):
        nets = np.nonzero(batch == k)[0]
        pen = penalty(grid, np.minimum(D_cur, np.iinfo(np.int32).max).astype(np.int32), H, ww["hist_w"])
        out = dp(grid, forest, ww, pen, W, rho, threads=threads)
        sel = batch[net_of] == k
        layer[sel], b[sel], t[sel] = out["layer"][sel], out["b"][sel], out["t"][sel]
        J[nets] = out["J"][nets]
        sub, nodes = _net_subset(forest, nets)
        Dn, _, _ = demand(grid, sub, layer[nodes], b[nodes], t[nodes], zeros)
        D_cur += Dn
        if layer_prev is not None:
            Do, _, _ = demand(grid, sub, layer_prev[nodes], b[nodes], t[nodes], zeros)
            D_cur -= Do
    Dn, Hn, st = demand(grid, forest, layer, b, t, H)
    st["total_cost"] = float(np.sum(J))
    return dict(layer=layer, b=b, t=t, J=J, D=Dn, H=Hn, stats=st, W=W, rho=rho)


def rc_from_assignment(grid, forest, layer):
    keep = _Keep()
    V = int(forest["num_nodes"])
    R, C = np.empty(V), np.empty(V)
    _load().or_rc_from_assignment(ctypes.byref(_grid(grid, keep)), ctypes.byref(_forest(forest, keep)),
                                  keep.ptr(layer, np.int8), R.ctypes.data, C.ctypes.data)
    return R, C


def elmore(grid, forest, layer, b, t, R_seg, C_seg) -> np.ndarray:
    """Elmore delay at every node's pin point (pin nodes) or junction (others)."""
    keep = _Keep()
    V = int(forest["num_nodes"])
    delay, s1, s2 = np.empty(V), np.empty(V), np.empty(V)
    _load().or_elmore(ctypes.byref(_grid(grid, keep)), ctypes.byref(_forest(forest, keep)),
                      keep.ptr(layer, np.int8), keep.ptr(b, np.int8), keep.ptr(t, np.int8),
                      keep.ptr(R_seg, np.float64), keep.ptr(C_seg, np.float64), delay.ctypes.data,
                      s1.ctypes.data, s2.ctypes.data)
    return delay


def elmore_backward(grid, forest, layer, b, t, R_seg, C_seg, grad_delay):
    """(dR_seg, dC_seg, Wsum, U_J) of L = sum grad_delay * delay."""
    keep = _Keep()
    V = int(forest["num_nodes"])
    dR, dC, Ws, UJ, s1 = (np.empty(V) for _ in range(5))
    _load().or_elmore_backward(ctypes.byref(_grid(grid, keep)), ctypes.byref(_forest(forest, keep)),
                               keep.ptr(layer, np.int8), keep.ptr(b, np.int8), keep.ptr(t, np.int8),
                               keep.ptr(R_seg, np.float64), keep.ptr(C_seg, np.float64),
                               keep.ptr(grad_delay, np.float64), dR.ctypes.data, dC.ctypes.data,
                               Ws.ctypes.data, UJ.ctypes.data, s1.ctypes.data)
    return dR, dC, Ws, UJ


def adjoint_weights(grid, forest, layer, b, t):
    """(W, r_est) of the adjoint mode: Wsum and U_J with g = kappa on the
    assignment's own RC tree (R = len r, C = len c)."""
    R, C = rc_from_assignment(grid, forest, layer)
    g = np.where(np.asarray(forest["pin_layer"]) >= 0, forest["kappa"], 0.0)
    _, _, Ws, UJ = elmore_backward(grid, forest, layer, b, t, R, C, g)
    return Ws, UJ


def logistic_pin_weight(pin_layer, slack, wns: float, k: float = 10.0, b: float = 0.3):
    """Sec. III-C pin weights: 1 / (1 + e^{-k (slack / WNS - b)}) at pins, 0 elsewhere."""
    keep = _Keep()
    V = len(pin_layer)
    w = np.empty(V)
    _load().or_logistic_pin_weight(V, keep.ptr(pin_layer, np.int8), keep.ptr(slack, np.float64), float(wns),
                                   float(k), float(b), w.ctypes.data)
    return w


def partition_batches(crit, slack=None, critical_frac: float = 0.5, slack_ratio: float = 0.7):
    """Alg. 1's partition of the nets into batches: (batch ids, number of batches)."""
    keep = _Keep()
    N = len(crit)
    out = np.empty(N, np.int32)
    nb = _load().or_partition_batches(N, keep.ptr(crit, np.float64),
                                      None if slack is None else keep.ptr(slack, np.float64),
                                      float(critical_frac), float(slack_ratio), out.ctypes.data)
    return out, int(nb)
