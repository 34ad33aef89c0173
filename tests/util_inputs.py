"""Seeded input builders for the tests (data only: no layer-assignment arithmetic)."""
from __future__ import annotations

import dataclasses
import os

import numpy as np

import forestgen as fg

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# Tiny nets for brute force: 12x12 grid, 4 layers, 2-4 pins (<= 6 segments).
TINY = fg.Workload("tiny-12x12x4", 12, 12, 4, (0, 6), 0.2, 200, 0, 2, 4, 0.0, False,
                   (8.0, 6.0, 2.0, 1.0), (0.20, 0.19, 0.17, 0.15), rounds=1)


def tiny(**kw) -> fg.Workload:
    return dataclasses.replace(TINY, **kw)


def random_snapshot(E: int, seed: int, dmax: int = 9, hmax: int = 3):
    """A demand/history snapshot (D, H) with congestion on many edges."""
    rng = np.random.default_rng(seed)
    return (rng.integers(0, dmax, E).astype(np.int32), rng.integers(0, hmax, E).astype(np.int32))


def forest_from_rows(rows, r_drv: float) -> dict:
    """One-net forest from (parent_local, x, y, pin_layer, sink_cap, kappa) rows."""
    par, x, y, pin, cs, kap = zip(*rows)
    V = len(rows)
    return dict(num_nets=1, num_nodes=V, net_ptr=np.array([0, V], np.int64),
                x=np.array(x, np.int32), y=np.array(y, np.int32), parent=np.array(par, np.int32),
                pin_layer=np.array(pin, np.int8), sink_cap=np.array(cs, np.float64),
                kappa=np.array(kap, np.float64), r_drv=np.array([r_drv], np.float64))


def read_fig6():
    """The Fig. 6 tree: list of (node id, parent id or None, x, y, pin, cap, kappa)."""
    rows = []
    with open(os.path.join(GOLDEN, "fig6_rc_tree.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            n, p, x, y, pin, cap, kap = line.split()
            rows.append((int(n), None if p == "-" else int(p), int(x), int(y), int(pin), float(cap), float(kap)))
    return rows


def read_table1():
    """Table I rows: (name, R kOhm/um, C fF/um, upper-via R kOhm or None)."""
    rows = []
    with open(os.path.join(GOLDEN, "table1_nangate45.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, r, c, v = line.split()
            rows.append((name, float(r), float(c), None if v == "-" else float(v)))
    return rows


def simple_grid(X, Y, L, unit_r, unit_c, via_r, via_c, cap=8):
    E = fg.grid_edges(X, Y, L)
    return dict(X=X, Y=Y, L=L, dir=np.array([l % 2 for l in range(L)], np.int8),
                cap=np.full(E, cap, np.int32), unit_r=np.array(unit_r, np.float64),
                unit_c=np.array(unit_c, np.float64), via_r=np.array(via_r, np.float64),
                via_c=float(via_c), ofw=np.ones(L, np.float64))
