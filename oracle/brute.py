"""Independent pure-Python pins for the oracle (TEST INFRASTRUCTURE ONLY).

Nothing here calls la_oracle.c; everything is written again from the model:

* ``net_cost``: the cost J of one net under a given assignment, evaluated
  directly on the RC tree (Sec. II-C Elmore delay with the pi-model of
  Sec. III-B) in exact rational arithmetic:
      J = sum over segments v of  w_cong 2^-24 K_v + w_cap C_v
                                + w_d W_v R_v (C_v/2 + Cd(v))
                                + w_d W_v Rvia(l_p, l_v) (C_v + Cd(v))
        + sum over nodes of (w_via + w_cap vc) (t - b)
        + sum over pin nodes of w_d kappa_v Rvia(l_v, p_v) Cs_v
        + w_d W_root R_drv Cd(root)
  where Cd(v) is the capacitance hanging below v's junction (vias at v, its
  pin, and every son's segment and subtree).  This is the weighted Elmore sum
  sum_x W(x) R_x Cdown(x) over the resistors x of the tree, plus the
  congestion, via and capacitance terms.
* ``brute_force``: min of ``net_cost`` over every layer vector (each segment on
  a layer of its direction), with minimal via stacks (the hull of the
  junction layer, the pin and the sons' layers).
* ``elmore_path_sum``: the textbook Elmore delay, delay(s) = sum over caps k of
  R_common(s, k) C_k, on an explicitly built RC tree, O(n^2).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass
from fractions import Fraction as Fr

import numpy as np


@dataclass
class Net:
    x: list
    y: list
    parent: list       # local, -1 at 0
    pin_layer: list
    sink_cap: list
    kappa: list
    r_drv: float

    @property
    def m(self):
        return len(self.x)

    def sons(self, v):
        return [c for c in range(self.m) if self.parent[c] == v]

    def segment(self, v):
        """(dir, line, lo, hi) of the segment from v to its parent."""
        p = self.parent[v]
        if self.y[v] == self.y[p]:
            return 0, self.y[v], min(self.x[v], self.x[p]), max(self.x[v], self.x[p])
        assert self.x[v] == self.x[p]
        return 1, self.x[v], min(self.y[v], self.y[p]), max(self.y[v], self.y[p])


def nets_of(forest, max_nets=None):
    """Split a forestgen forest into Net objects."""
    out = []
    ptr = forest["net_ptr"]
    N = int(forest["num_nets"]) if max_nets is None else min(max_nets, int(forest["num_nets"]))
    for n in range(N):
        a, b = int(ptr[n]), int(ptr[n + 1])
        out.append(Net([int(v) for v in forest["x"][a:b]], [int(v) for v in forest["y"][a:b]],
                       [int(v) for v in forest["parent"][a:b]], [int(v) for v in forest["pin_layer"][a:b]],
                       [float(v) for v in forest["sink_cap"][a:b]], [float(v) for v in forest["kappa"][a:b]],
                       float(forest["r_drv"][n])))
    return out


def _rvia(via_r, a, b):
    lo, hi = min(a, b), max(a, b)
    return sum((Fr(via_r[k]) for k in range(lo, hi)), Fr(0))


def edge_id(grid, l, line, e):
    X, Y, dirs = int(grid["X"]), int(grid["Y"]), list(grid["dir"])
    off = 0
    for k in range(l):
        off += Y * (X - 1) if dirs[k] == 0 else X * (Y - 1)
    per = X - 1 if dirs[l] == 0 else Y - 1
    return off + line * per + e


def eq4_weights(net):
    """W_v = max sink criticality in the subtree of v (Eq. 4, downstream)."""
    W = [Fr(net.kappa[v]) if net.pin_layer[v] >= 0 else Fr(0) for v in range(net.m)]
    for v in reversed(range(1, net.m)):
        p = net.parent[v]
        W[p] = max(W[p], W[v])
    return W


def hull_stacks(net, lay):
    """Minimal via stack at each node: hull of junction layer, pin and sons' layers."""
    bt = []
    for v in range(net.m):
        s = {lay[v]} | {lay[c] for c in net.sons(v)}
        if net.pin_layer[v] >= 0:
            s.add(net.pin_layer[v])
        bt.append((min(s), max(s)))
    return bt


def net_cost(grid, net, lay, bt, pen, W, w) -> Fr:
    """Exact cost J of one net under assignment `lay` (junction layers) and
    via stacks `bt`, straight from the RC model (see module docstring)."""
    r = [Fr(v) for v in grid["unit_r"]]
    c = [Fr(v) for v in grid["unit_c"]]
    via_r = [float(v) for v in grid["via_r"]]
    vc = Fr(float(grid["via_c"]))
    w_cong, w_via, w_cap, w_d = (Fr(float(w[k])) for k in ("w_cong", "w_via", "w_cap", "w_d"))
    m = net.m
    seg = [None] + [net.segment(v) for v in range(1, m)]
    Cseg = [Fr(0)] + [(seg[v][3] - seg[v][2]) * c[lay[v]] for v in range(1, m)]
    Rseg = [Fr(0)] + [(seg[v][3] - seg[v][2]) * r[lay[v]] for v in range(1, m)]
    Cd = [Fr(0)] * m
    for v in reversed(range(m)):
        s = vc * (bt[v][1] - bt[v][0]) + Fr(net.sink_cap[v])
        for s_ in net.sons(v):
            s += Cseg[s_] + Cd[s_]
        Cd[v] = s
    J = Fr(0)
    for v in range(1, m):
        d, line, lo, hi = seg[v]
        K = sum(int(pen[edge_id(grid, lay[v], line, e)]) for e in range(lo, hi))
        J += w_cong * Fr(K, 1 << 24) + w_cap * Cseg[v]
        J += w_d * W[v] * Rseg[v] * (Cseg[v] / 2 + Cd[v])
        J += w_d * W[v] * _rvia(via_r, lay[net.parent[v]], lay[v]) * (Cseg[v] + Cd[v])
    for v in range(m):
        J += (w_via + w_cap * vc) * (bt[v][1] - bt[v][0])
        if net.pin_layer[v] >= 0:
            J += w_d * Fr(net.kappa[v]) * _rvia(via_r, lay[v], net.pin_layer[v]) * Fr(net.sink_cap[v])
    J += w_d * W[0] * Fr(net.r_drv) * Cd[0]
    return J


def brute_force(grid, net, pen, w, W=None):
    """(min J, list of minimising layer vectors) over all direction-legal layer
    vectors, stacks = hulls.  W defaults to the Eq. 4 weights."""
    W = eq4_weights(net) if W is None else [Fr(float(x)) for x in W]
    dirs = list(grid["dir"])
    L = int(grid["L"])
    choices = [[net.pin_layer[0]]]
    for v in range(1, net.m):
        d = net.segment(v)[0]
        choices.append([l for l in range(L) if dirs[l] == d])
    best, arg = None, []
    for lay in itertools.product(*choices):
        J = net_cost(grid, net, list(lay), hull_stacks(net, list(lay)), pen, W, w)
        if best is None or J < best:
            best, arg = J, [list(lay)]
        elif J == best:
            arg.append(list(lay))
    return best, arg


# ---------------------------------------------------------------------------
# Textbook Elmore delay on an explicit RC tree
# ---------------------------------------------------------------------------
def rc_tree(grid, net, lay, bt, R_seg, C_seg):
    """Explicit RC tree: list of (parent index, resistance, capacitance) with the
    source as index -1.  Returns (nodes, out_index per net node)."""
    via_r = [float(v) for v in grid["via_r"]]
    vc = float(grid["via_c"])
    nodes = []   # (parent, R, C)
    J = [None] * net.m
    out = [None] * net.m

    def add(par, R, C):
        nodes.append([par, R, C])
        return len(nodes) - 1

    J[0] = add(-1, net.r_drv, vc * (bt[0][1] - bt[0][0]))
    for v in range(1, net.m):
        p = net.parent[v]
        X = add(J[p], float(_rvia(via_r, lay[p], lay[v])), 0.5 * C_seg[v])
        J[v] = add(X, R_seg[v], 0.5 * C_seg[v] + vc * (bt[v][1] - bt[v][0]))
    for v in range(net.m):
        if net.pin_layer[v] >= 0:
            out[v] = add(J[v], float(_rvia(via_r, lay[v], net.pin_layer[v])), net.sink_cap[v])
        else:
            out[v] = J[v]
    return nodes, out


def elmore_path_sum(nodes, target):
    """delay(target) = sum over every cap k of R_common(target, k) * C_k."""
    def path(i):
        s = set()
        while i != -1:
            s.add(i)
            i = nodes[i][0]
        return s
    pt = path(target)
    total = 0.0
    for k in range(len(nodes)):
        common = pt & path(k)
        total += sum(nodes[i][1] for i in common) * nodes[k][2]
    return total
