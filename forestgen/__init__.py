"""Seeded synthetic inputs for layer assignment (shared by the CUDA path's tests,
the benchmark and the CPU oracle).

This package generates data only: GCell grids with per-layer edge capacities,
per-layer unit R/C stacks, and net forests of straight-segment 2D routing trees.
It contains none of the layer-assignment arithmetic.

The five workloads follow the shapes of the paper's benchmarks (Table II:
10 routing layers, 0.1-12 M nets, grids of 386^2 to 3719^2 GCells); the designs
themselves are not available, so these seeded generators stand in for them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_LIBDIR, "libforestgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile forestgen.c into forestgen/_lib/libforestgen.so (gcc, no -march)."""
    src = os.path.join(_HERE, "forestgen.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                           "-ffp-contract=off", "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [("X", ctypes.c_int32), ("Y", ctypes.c_int32), ("L", ctypes.c_int32),
                ("cap_lo", ctypes.c_int32), ("cap_hi", ctypes.c_int32),
                ("block_frac", ctypes.c_double), ("num_nets", ctypes.c_int64),
                ("pin_dist", ctypes.c_int32), ("pin_a", ctypes.c_int32), ("pin_b", ctypes.c_int32),
                ("pin_p", ctypes.c_double), ("clustered", ctypes.c_int32),
                ("n_centres", ctypes.c_int32), ("sigma", ctypes.c_double),
                ("rdrv_lo", ctypes.c_double), ("rdrv_hi", ctypes.c_double),
                ("csink_lo", ctypes.c_double), ("csink_hi", ctypes.c_double),
                ("kappa_lo", ctypes.c_double), ("kappa_hi", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("threads", ctypes.c_int32)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        lib.fg_grid_edges.restype = ctypes.c_int64
        lib.fg_grid_edges.argtypes = [ctypes.c_int32] * 3
        lib.fg_grid_cap.restype = None
        lib.fg_grid_cap.argtypes = [P(_Params), ctypes.c_void_p]
        lib.fg_generate.restype = ctypes.c_void_p
        lib.fg_generate.argtypes = [P(_Params)]
        lib.fg_num_nodes.restype = ctypes.c_int64
        lib.fg_num_nodes.argtypes = [ctypes.c_void_p]
        lib.fg_export.restype = None
        lib.fg_export.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 8
        lib.fg_free.restype = None
        lib.fg_free.argtypes = [ctypes.c_void_p]
        _lib = lib
    return _lib


@dataclass
class Workload:
    """One synthetic layer-assignment workload: grid, layer stack and net forest."""
    name: str
    X: int
    Y: int
    L: int
    cap: tuple            # (lo, hi) uniform integer capacity per (layer, edge)
    block_frac: float     # fraction of (layer, edge) capacities halved
    num_nets: int
    pin_dist: int         # 0 uniform [a,b]; 1: 2+Geometric(p) capped at b; 2: Zipf(p) on [a,b]
    pin_a: int
    pin_b: int
    pin_p: float
    clustered: bool
    unit_r: tuple         # ohm per GCell edge, per layer
    unit_c: tuple         # fF per GCell edge, per layer
    rounds: int
    via_r: object = 2.0   # ohm per via between adjacent layers (one value, or L-1 values)
    via_c: float = 0.05   # fF per via
    n_centres: int = 64
    sigma: float = 20.0
    rdrv: tuple = (50.0, 500.0)
    csink: tuple = (1.0, 5.0)
    kappa: tuple = (0.0, 1.0)
    note: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def dirs(self):
        """Alternating preferred directions, layer 0 horizontal (0 = H, 1 = V)."""
        return tuple(l % 2 for l in range(self.L))

    def scaled(self, num_nets: int) -> "Workload":
        """Same grid and distributions with a different net count."""
        import dataclasses
        return dataclasses.replace(self, num_nets=num_nets, name=f"{self.name}[{num_nets} nets]")


def _pairs(v):
    return tuple(x for x in v for _ in range(2))


_R5 = tuple(8.0 * 10.0 ** (-l / 11.0) for l in range(12))
_C5 = tuple(0.20 - 0.05 * l / 11.0 for l in range(12))

WORKLOADS = {
    1: Workload("plain-64x64x6-2k", 64, 64, 6, (6, 12), 0.0, 2000, 0, 2, 8, 0.0, False,
                (8, 8, 4, 4, 1, 1), (0.20, 0.20, 0.18, 0.18, 0.15, 0.15), rounds=1,
                note="2k nets, uniform pins U{2..8}, 1 round"),
    2: Workload("plain-512x512x10-500k", 512, 512, 10, (8, 16), 0.05, 500_000, 1, 2, 64, 0.4, True,
                _pairs((8.0, 4.0, 2.0, 1.0, 0.5)), _pairs((0.20, 0.19, 0.18, 0.16, 0.15)), rounds=3,
                note="500k nets, 2+Geom(0.4)<=64 clustered pins, 3 negotiation rounds"),
    4: Workload("zipf-1024x1024x10-2M", 1024, 1024, 10, (8, 16), 0.05, 2_000_000, 2, 2, 4096, 1.6, True,
                _pairs((8.0, 4.0, 2.0, 1.0, 0.5)), _pairs((0.20, 0.19, 0.18, 0.16, 0.15)), rounds=5,
                note="2M nets, Zipf(1.6) pins on [2,4096], 5 rounds"),
    5: Workload("full-2048x2048x12-12M", 2048, 2048, 12, (8, 20), 0.10, 12_000_000, 1, 2, 256, 0.35, True,
                _R5, _C5, rounds=5,
                note="12M nets, 2+Geom(0.35)<=256 clustered pins, 5 rounds"),
}
# Config 3 is config 2's forest with a fixed assignment (Elmore + adjoint).
WORKLOADS[3] = WORKLOADS[2]

# The modified NanGate 45 nm stack of the paper's Table I (10 metal layers: R in
# kOhm/um, C in fF/um, the via resistance up to the next layer in kOhm), read
# with a GCell edge of 1 um: R per GCell = 1000 R Ohm, C per GCell = C fF, via
# R = 1000 Rvia Ohm.
NANGATE45_R_KOHM_UM = (5.4286e-3, 3.5714e-3, 3.5714e-3, 1.5e-3, 1.5e-3, 1.5e-3, 1.875e-4, 1.875e-4, 3.75e-5, 3.75e-5)
NANGATE45_C_FF_UM = (7.41819e-2, 6.74606e-2, 8.88758e-2, 1.07121e-1, 1.08964e-1, 1.02044e-1, 1.10436e-1,
                     9.69714e-2, 3.6864e-2, 2.8042e-2)
NANGATE45_VIA_KOHM = (5e-3, 5e-3, 5e-3, 3e-3, 3e-3, 3e-3, 1e-3, 1e-3, 0.5e-3)
WORKLOADS[6] = Workload("nangate45-1024x1024x10-2M", 1024, 1024, 10, (8, 16), 0.05, 2_000_000, 1, 2, 64, 0.4, True,
                        tuple(1000.0 * r for r in NANGATE45_R_KOHM_UM), NANGATE45_C_FF_UM, rounds=3,
                        via_r=tuple(1000.0 * r for r in NANGATE45_VIA_KOHM),
                        note="Table I stack, 2M nets, 2+Geom(0.4)<=64 clustered pins, 3 rounds")


def _params(w: Workload, seed: int, threads: int = 0) -> _Params:
    p = _Params()
    p.X, p.Y, p.L = w.X, w.Y, w.L
    p.cap_lo, p.cap_hi = w.cap
    p.block_frac = w.block_frac
    p.num_nets = w.num_nets
    p.pin_dist, p.pin_a, p.pin_b, p.pin_p = w.pin_dist, w.pin_a, w.pin_b, w.pin_p
    p.clustered = 1 if w.clustered else 0
    p.n_centres, p.sigma = w.n_centres, w.sigma
    p.rdrv_lo, p.rdrv_hi = w.rdrv
    p.csink_lo, p.csink_hi = w.csink
    p.kappa_lo, p.kappa_hi = w.kappa
    p.seed = seed & 0xFFFFFFFFFFFFFFFF
    p.threads = threads
    return p


def grid_edges(X: int, Y: int, L: int) -> int:
    """Number of GCell edges over all layers (H layer: Y*(X-1), V layer: X*(Y-1))."""
    return int(_load().fg_grid_edges(X, Y, L))


def make_grid(w: Workload, seed: int = 0, threads: int = 0) -> dict:
    """Grid of workload `w`: capacities (int32, public edge layout) and the layer stack."""
    lib = _load()
    p = _params(w, seed, threads)
    E = grid_edges(w.X, w.Y, w.L)
    cap = np.empty(E, dtype=np.int32)
    lib.fg_grid_cap(ctypes.byref(p), cap.ctypes.data)
    return dict(X=w.X, Y=w.Y, L=w.L, dir=np.array(w.dirs, dtype=np.int8), cap=cap,
                unit_r=np.array(w.unit_r, dtype=np.float64), unit_c=np.array(w.unit_c, dtype=np.float64),
                via_r=(np.array(w.via_r, dtype=np.float64) if isinstance(w.via_r, (tuple, list))
                       else np.full(w.L - 1, w.via_r, dtype=np.float64)), via_c=float(w.via_c),
                ofw=np.ones(w.L, dtype=np.float64))


def make_forest(w: Workload, seed: int = 0, threads: int = 0) -> dict:
    """Net forest of workload `w` as CSR numpy arrays (see forestgen.c)."""
    lib = _load()
    p = _params(w, seed, threads)
    h = lib.fg_generate(ctypes.byref(p))
    try:
        V = int(lib.fg_num_nodes(h))
        N = w.num_nets
        out = dict(net_ptr=np.empty(N + 1, np.int64), x=np.empty(V, np.int32), y=np.empty(V, np.int32),
                   parent=np.empty(V, np.int32), pin_layer=np.empty(V, np.int8),
                   sink_cap=np.empty(V, np.float64), kappa=np.empty(V, np.float64),
                   r_drv=np.empty(N, np.float64))
        lib.fg_export(h, *(out[k].ctypes.data for k in
                           ("net_ptr", "x", "y", "parent", "pin_layer", "sink_cap", "kappa", "r_drv")))
    finally:
        lib.fg_free(h)
    out["num_nets"] = N
    out["num_nodes"] = V
    return out


def subset_forest(forest: dict, nets) -> dict:
    """The nets with the given indices, renumbered as a forest of their own."""
    nets = np.asarray(nets, dtype=np.int64)
    ptr = forest["net_ptr"]
    lens = ptr[nets + 1] - ptr[nets]
    idx = np.concatenate([np.arange(ptr[n], ptr[n + 1]) for n in nets]) if len(nets) else np.zeros(0, np.int64)
    out = {k: forest[k][idx] for k in ("x", "y", "parent", "pin_layer", "sink_cap", "kappa")}
    out["net_ptr"] = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    out["r_drv"] = forest["r_drv"][nets].copy()
    out["num_nets"] = len(nets)
    out["num_nodes"] = int(out["net_ptr"][-1])
    return out
