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


def merge_forests(parts) -> dict:
    """Concatenate one-or-more-net forests into one forest."""
    out = {k: np.concatenate([p[k] for p in parts]) for k in
           ("x", "y", "parent", "pin_layer", "sink_cap", "kappa", "r_drv")}
    sizes = np.concatenate([np.diff(p["net_ptr"]) for p in parts])
    out["net_ptr"] = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    out["num_nets"] = len(sizes)
    out["num_nodes"] = int(out["net_ptr"][-1])
    return out


def edge_case_forest(X: int, Y: int, L: int, seed: int = 0) -> dict:
    """Hand-made nets covering the degenerate shapes: a single-node net, a
    2-pin straight net, a long zig-zag chain (deep tree), a star with four
    sons, a Steiner node with three sons, pins on upper layers, a sink merged
    into the driver's GCell, and a branch that ends without a pin."""
    rng = np.random.default_rng(seed)
    nets = []
    u = lambda: float(rng.uniform(0.1, 1.0))
    # single node (all pins in the driver's GCell)
    nets.append(forest_from_rows([(-1, 3, 3, 0, 2.0, 0.7)], r_drv=200.0))
    # 2-pin straight
    nets.append(forest_from_rows([(-1, 1, 1, 0, 0.0, 0.0), (0, 9, 1, 0, 3.0, u())], r_drv=120.0))
    # zig-zag chain: H, V, H, V, ... with a pin every fourth node
    rows = [(-1, 0, 0, 0, 0.0, 0.0)]
    x, y = 0, 0
    depth = min(X, Y) - 2
    for i in range(1, depth):
        if i % 2:
            x += 1
        else:
            y += 1
        pin = int(rng.integers(0, L)) if i % 4 == 0 else -1
        rows.append((i - 1, x, y, pin, 1.5 if pin >= 0 else 0.0, u() if pin >= 0 else 0.0))
    rows[-1] = rows[-1][:3] + (0, 2.5, u())
    nets.append(forest_from_rows(rows, r_drv=300.0))
    # star: driver in the middle, four straight sons
    cx, cy = X // 2, Y // 2
    nets.append(forest_from_rows([(-1, cx, cy, 0, 0.0, 0.0), (0, cx + 5, cy, 0, 1.0, u()),
                                  (0, cx - 4, cy, 1, 2.0, u()), (0, cx, cy + 3, 0, 1.5, u()),
                                  (0, cx, cy - 6, 2 % L, 2.5, u())], r_drv=90.0))
    # Steiner node (no pin) with three sons, one of them carrying a further son
    nets.append(forest_from_rows([(-1, 2, 2, 0, 0.0, 0.0), (0, 2, 8, -1, 0.0, 0.0), (1, 7, 8, 0, 1.0, u()),
                                  (1, 2, 12 % Y, 0, 2.0, u()), (1, 0, 8, L - 1, 1.0, u()),
                                  (4, 0, 10, 0, 3.0, u())], r_drv=60.0))
    # sink merged into the driver node, and a son
    nets.append(forest_from_rows([(-1, 5, 5, 0, 4.0, 0.9), (0, 5, 1, 0, 1.0, 0.2)], r_drv=400.0))
    # a dangling branch: a leaf without a pin, and a bend without a pin below it
    nets.append(forest_from_rows([(-1, 4, 4, 0, 0.0, 0.0), (0, 9, 4, 0, 1.5, u()), (0, 4, 7, -1, 0.0, 0.0),
                                  (2, 1, 7, -1, 0.0, 0.0)], r_drv=150.0))
    return merge_forests(nets)


# Exact-tie cases for the tie rules (w_d = 0, no via cost, zero snapshot): on
# a 4-layer stack (0 H, 1 V, 2 H, 3 V) with equal unit R and C, two layers of
# one direction whose overflow weights are equal give exactly equal keys.
TIE_WEIGHTS = dict(w_cong=1.0, w_via=0.0, w_cap=0.0, w_d=0.0, hist_w=1.0)


def tie_grid(ofw):
    grid = simple_grid(12, 12, 4, (1.0, 1.0, 1.0, 1.0), (0.2, 0.2, 0.2, 0.2), (1.0, 1.0, 1.0), 0.0, cap=8)
    grid["ofw"] = np.array(ofw, np.float64)
    return grid


def son_tie_case():
    """A root (driver pin on layer 0) with an H leaf and a V leaf, both with a
    pin on layer 0; layer 3 (V) is cheaper (overflow weight 1/2), so the root's
    stack reaches layer 3 and holds both H layers 0 and 2, whose keys for the
    H leaf are equal.  Returns (grid, forest, the documented layers and
    stacks): the son takes the lowest of its tied layers."""
    forest = forest_from_rows([(-1, 2, 2, 0, 0.0, 0.0), (0, 6, 2, 0, 1.0, 0.5), (0, 2, 7, 0, 1.0, 0.5)], r_drv=100.0)
    return tie_grid((1.0, 1.0, 1.0, 0.5)), forest, [0, 0, 3], [(0, 3), (0, 0), (0, 3)]


def stack_tie_case():
    """A root (driver pin on layer 0), an H bend v without a pin, and a V leaf
    c below it with a pin on layer 0; layer 0 is dearer for wires (overflow
    weight 3), so v goes on layer 2, and c's layers 1 and 3 have equal keys.
    At v the stacks [1, 2] and [2, 3] tie on cost and on via count, and wider
    ones tie on cost.  Returns (grid, forest, the documented layers and
    stacks): fewest vias, then the lowest b."""
    forest = forest_from_rows([(-1, 2, 2, 0, 0.0, 0.0), (0, 8, 2, -1, 0.0, 0.0), (1, 8, 7, 0, 1.0, 0.5)],
                              r_drv=100.0)
    return tie_grid((3.0, 1.0, 1.0, 1.0)), forest, [0, 2, 1], [(0, 2), (1, 2), (0, 1)]
