"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks an oracle function against something other than itself:
brute-force enumeration (exact rational arithmetic), the textbook Elmore path
sum, closed forms, the worked example of Sec. III-D, Table I values, and
invariants.  None of these tests touches the GPU.
"""
from __future__ import annotations

import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import forestgen as fg
import oracle
import oracle.brute as br
from util_inputs import (forest_from_rows, random_snapshot, read_fig6, read_table1, simple_grid, tiny)

W_ALL = dict(oracle.DEFAULT_WEIGHTS)


def _round_on(grid, forest, weights, seed):
    E = oracle.num_edges(grid)
    D, H = random_snapshot(E, seed)
    return oracle.assign_round(grid, forest, weights, D=D, H=H)


def _net_assignment(forest, out, n):
    a, b = int(forest["net_ptr"][n]), int(forest["net_ptr"][n + 1])
    lay = [int(v) for v in out["layer"][a:b]]
    bt = list(zip([int(v) for v in out["b"][a:b]], [int(v) for v in out["t"][a:b]]))
    W = [Fr(float(x)) for x in out["W"][a:b]]
    return lay, bt, W


def _random_pin_layers(forest, L, seed):
    """The forest with every pin moved to a random layer (the generator puts
    them on layer 0)."""
    pin = forest["pin_layer"].copy()
    on = pin >= 0
    pin[on] = np.random.default_rng(seed).integers(0, L, int(on.sum())).astype(pin.dtype)
    return dict(forest, pin_layer=pin)


def _check_against_brute(wl, weights, seed, zero_via=False, max_seg=6, expect_exact=True, pins_random=False):
    grid = fg.make_grid(wl, seed)
    forest = fg.make_forest(wl, seed)
    if pins_random:
        forest = _random_pin_layers(forest, wl.L, seed)
    if zero_via:
        grid["via_r"] = np.zeros_like(grid["via_r"])
    ww = dict(W_ALL, **weights)
    out = _round_on(grid, forest, ww, seed)
    checked = gaps = 0
    for n, net in enumerate(br.nets_of(forest)):
        if net.m - 1 > max_seg:
            continue
        lay, bt, W = _net_assignment(forest, out, n)
        Jdp = out["J"][n]
        # bookkeeping: the DP's J equals the cost of its own assignment
        Jev = br.net_cost(grid, net, lay, bt, out["pen"], W, ww)
        assert abs(float(Jev) - Jdp) <= 1e-12 * abs(Jdp), (n, float(Jev), Jdp)
        assert bt == br.hull_stacks(net, lay), n
        Jb, _ = br.brute_force(grid, net, out["pen"], ww, W)
        assert float(Jb) <= Jdp * (1 + 1e-12), (n, float(Jb), Jdp)
        if expect_exact:
            assert Jdp <= float(Jb) * (1 + 1e-12), (n, float(Jb), Jdp)
        elif Jdp > float(Jb) * (1 + 1e-12):
            gaps += 1
        checked += 1
    assert checked >= 100
    return gaps


# ---------------------------------------------------------------------------
# The DP of Alg. 3 / Alg. 4 against brute force
# ---------------------------------------------------------------------------
def test_dp_equals_brute_force_when_cost_is_separable():
    """w_d = 0: congestion + via + capacitance only; the tree DP is exact."""
    _check_against_brute(tiny(), dict(w_d=0.0), seed=11)


def test_dp_equals_brute_force_when_lookahead_is_exact():
    """All unit R equal and zero via R: the distance-based r_est is the exact
    weighted upstream resistance, so f' orders candidates exactly (Sec. III-D)."""
    _check_against_brute(tiny(unit_r=(3.0, 3.0, 3.0, 3.0)), dict(w_d=5e-3), seed=12, zero_via=True)


def test_dp_equals_brute_force_with_pins_on_upper_layers():
    """Every pin on a random layer: a node with a pin above layer 0 has several
    stack bottoms, and the root's junction sits above layer 0.  Exact cases:
    w_d = 0 (separable) and the exact look-ahead."""
    wl = tiny()
    forest = _random_pin_layers(fg.make_forest(wl, 14), wl.L, 14)
    # the shapes are there among the small nets: several-son nodes and roots
    # with a pin above layer 0
    nets = [n for n in br.nets_of(forest) if n.m - 1 <= 6]
    multi = sum(1 for n in nets for v in range(n.m)
                if n.pin_layer[v] > 0 and sum(1 for u in range(n.m) if n.parent[u] == v) >= 2)
    assert multi >= 20
    _check_against_brute(wl, dict(w_d=0.0), seed=14, pins_random=True)
    _check_against_brute(tiny(unit_r=(3.0, 3.0, 3.0, 3.0)), dict(w_d=5e-3), seed=15, zero_via=True,
                         pins_random=True)
    # and with via R and a strong delay weight (the pin's via delay term is
    # live): J(brute) <= J(DP), and the DP's J is the cost of its own assignment
    _check_against_brute(tiny(pin_a=3, pin_b=5, num_nets=250, unit_r=(40.0, 30.0, 2.0, 1.0)),
                         dict(w_d=0.05, w_cong=1e-3), seed=16, max_seg=7, expect_exact=False, pins_random=True)


def test_dp_equals_brute_force_on_single_segment_nets():
    """2-pin nets with one straight segment: the only choice is its layer."""
    wl = tiny(pin_a=2, pin_b=2, num_nets=400)
    grid, forest = fg.make_grid(wl, 13), fg.make_forest(wl, 13)
    ww = dict(W_ALL, w_d=0.05)
    out = _round_on(grid, forest, ww, 13)
    n_single = 0
    for n, net in enumerate(br.nets_of(forest)):
        if net.m != 2:
            continue
        lay, bt, W = _net_assignment(forest, out, n)
        Jb, _ = br.brute_force(grid, net, out["pen"], ww, W)
        assert abs(out["J"][n] - float(Jb)) <= 1e-12 * float(Jb)
        n_single += 1
    assert n_single >= 50


def test_dp_is_a_heuristic_in_general_but_keeps_its_books():
    """Strong delay weight, unequal unit R, via R: J(brute) <= J(DP) and the DP's
    J is the cost of its own assignment.  The look-ahead is a heuristic, so
    some nets are above the optimum."""
    wl = tiny(pin_a=3, pin_b=5, num_nets=250, unit_r=(40.0, 30.0, 2.0, 1.0))
    gaps = _check_against_brute(wl, dict(w_d=0.05, w_cong=1e-3), seed=7, max_seg=7, expect_exact=False)
    assert gaps > 0


def test_assignment_invariants():
    """Every segment on a layer of its direction, stacks = hulls, root on its pin."""
    wl = fg.WORKLOADS[1].scaled(300)
    grid, forest = fg.make_grid(wl, 3), fg.make_forest(wl, 3)
    out = _round_on(grid, forest, W_ALL, 3)
    dirs = grid["dir"]
    for n, net in enumerate(br.nets_of(forest)):
        lay, bt, _ = _net_assignment(forest, out, n)
        assert lay[0] == net.pin_layer[0]
        for v in range(1, net.m):
            assert dirs[lay[v]] == net.segment(v)[0]
        assert bt == br.hull_stacks(net, lay)


# ---------------------------------------------------------------------------
# Congestion penalty (reading of Eq. 3)
# ---------------------------------------------------------------------------
E_CONST = 2.718281828459045  # Euler's number


def test_penalty_table_closed_form():
    grid = simple_grid(4, 4, 2, (1, 1), (1, 1), (1,), 0.0)
    grid["ofw"] = np.array([1.0, 2.0])
    T = oracle.penalty_table(grid)
    s24 = 1 << 24
    assert T[0, 0, 64] == s24 and T[0, 1, 64] == s24           # e^0 = 1
    assert T[1, 0, 64] == 2 * s24                               # ofw = 2
    assert T[0, 0, 64 + 2] == round(E_CONST * s24)              # s = 0.5, k = 2 -> e
    assert T[0, 0, 64 - 2] == round(s24 / E_CONST)              # k = -2 -> 1/e
    assert abs(T[0, 1, 64 + 2] - E_CONST ** 3 * s24) <= 2       # s = 1.5, k = 2 -> e^3
    assert T[0, 0, 128] == 1 << 48 and T[0, 1, 128] == 1 << 48  # saturated
    assert (np.diff(T, axis=2) >= 0).all()                      # non-decreasing in k
    assert T[0, 0, 0] == 0                                      # e^-32 2^24 rounds to 0


def test_penalty_clamps_the_overflow_at_minus_64():
    """The reading clamps k = D + 1 - C to [-64, 64]: with a large overflow
    weight the entries near the low end are non-zero, ofw e^{k/2} 2^24 rounded
    (1e8 e^-32 2^24 = 21.25, 1e8 e^-31.5 2^24 = 35.03), and every k below
    -64 takes the k = -64 value."""
    grid = simple_grid(4, 4, 2, (1, 1), (1, 1), (1,), 0.0)
    grid["ofw"] = np.array([1e8, 1.0])
    E = oracle.num_edges(grid)
    cap = np.full(E, 200, np.int32)
    D = np.zeros(E, np.int32)
    D[1] = 136   # k = -63
    D[2] = 135   # k = -64
    grid["cap"] = cap
    pen = oracle.penalty(grid, D, np.zeros(E, np.int32), hist_w=1.0)
    assert pen[0] == 21 and pen[2] == 21 and pen[1] == 35   # k = -199 clamps to -64


def test_penalty_values_and_saturation():
    grid = simple_grid(3, 3, 2, (1, 1), (1, 1), (1,), 0.0)
    E = oracle.num_edges(grid)
    cap = np.array([4, 0, 5, 2, 7, 1, 0, 3, 9, 6, 2, 8][:E], np.int32)
    grid["cap"] = cap
    D = np.arange(E, dtype=np.int32) % 5
    H = np.zeros(E, np.int32)
    H[3] = 2
    H[5] = 2_000_000_000
    pen = oracle.penalty(grid, D, H, hist_w=1.0)
    T = oracle.penalty_table(grid)
    for e in range(E):
        l = 0 if e < 6 else 1
        k = int(np.clip(D[e] + 1 - cap[e], -64, 64))
        base = int(T[l, 0 if cap[e] > 0 else 1, k + 64])
        want = min(base + (1 << 24) * int(H[e]), 1 << 48)
        assert pen[e] == want, e
    assert pen[5] == 1 << 48


# ---------------------------------------------------------------------------
# Weights (Eq. 4) and r_est on the Fig. 6 tree, by hand
# ---------------------------------------------------------------------------
def _fig6_forest():
    rows = read_fig6()
    ids = [r[0] for r in rows]
    loc = {n: i for i, n in enumerate(ids)}
    return forest_from_rows([(-1 if p is None else loc[p], x, y, pin, cap, kap)
                             for (_, p, x, y, pin, cap, kap) in rows], r_drv=120.0), loc


def test_eq4_weights_and_rest_by_hand():
    forest, loc = _fig6_forest()
    grid = simple_grid(8, 8, 4, (4.0, 3.0, 2.0, 1.0), (0.2, 0.2, 0.2, 0.2), (1.0, 1.0, 1.0), 0.0)
    W, rho = oracle.weights_eq4(grid, forest)
    k5, k7 = 0.3, 0.8
    # downstream max criticality (Eq. 4): edge 3->4 sees sinks 5 and 7, etc.
    want_W = {3: k7, 4: k7, 5: k5, 6: k7, 7: k7}
    for n, wv in want_W.items():
        assert W[loc[n]] == wv
    rH, rV = (4.0 + 2.0) / 2, (3.0 + 1.0) / 2
    r3 = k7 * 120.0
    r4 = r3 + k7 * 3 * rH        # 3 -> 4: horizontal, 3 edges
    r5 = r4 + k5 * 4 * rV        # 4 -> 5: vertical, 4 edges
    r6 = r4 + k7 * 3 * rH        # 4 -> 6: horizontal, 3 edges
    r7 = r6 + k7 * 2 * rV        # 6 -> 7: vertical, 2 edges
    for n, want in {3: r3, 4: r4, 5: r5, 6: r6, 7: r7}.items():
        assert rho[loc[n]] == pytest.approx(want, rel=1e-15)
    # only sinks carry a criticality: a large kappa on a node without a pin
    # changes neither W nor r_est
    nopin = forest["pin_layer"] < 0
    assert nopin.any()
    f2 = dict(forest, kappa=np.where(nopin, 5.0, forest["kappa"]))
    W2, rho2 = oracle.weights_eq4(grid, f2)
    assert np.array_equal(W2, W) and np.array_equal(rho2, rho)


# ---------------------------------------------------------------------------
# Demand, vias and history
# ---------------------------------------------------------------------------
def test_demand_invariants():
    wl = fg.WORKLOADS[1]
    grid, forest = fg.make_grid(wl, 5), fg.make_forest(wl, 5)
    E = oracle.num_edges(grid)
    D0, H0 = random_snapshot(E, 5)
    out = oracle.assign_round(grid, forest, W_ALL, D=D0, H=H0)
    D, H, st = out["D"], out["H"], out["stats"]
    X, Y, L = wl.X, wl.Y, wl.L
    # 2D demand from the segments alone (no layers)
    d2h = np.zeros((Y, X - 1), np.int64)
    d2v = np.zeros((X, Y - 1), np.int64)
    ptr = forest["net_ptr"]
    net_of = np.repeat(np.arange(forest["num_nets"]), np.diff(ptr))
    wl_total = 0
    for v in np.nonzero(forest["parent"] >= 0)[0]:
        p = ptr[net_of[v]] + forest["parent"][v]
        if forest["y"][v] == forest["y"][p]:
            a, b = sorted((forest["x"][v], forest["x"][p]))
            d2h[forest["y"][v], a:b] += 1
        else:
            a, b = sorted((forest["y"][v], forest["y"][p]))
            d2v[forest["x"][v], a:b] += 1
        wl_total += b - a
    sumH = np.zeros_like(d2h)
    sumV = np.zeros_like(d2v)
    off = 0
    for l in range(L):
        n_e = Y * (X - 1) if l % 2 == 0 else X * (Y - 1)
        blk = D[off:off + n_e]
        if l % 2 == 0:
            sumH += blk.reshape(Y, X - 1)
        else:
            sumV += blk.reshape(X, Y - 1)
        off += n_e
    assert (sumH == d2h).all() and (sumV == d2v).all()
    assert D.sum() == wl_total == st["wl"] == st["wl_per_layer"].sum()
    assert st["vias"] == int(np.sum(out["t"].astype(np.int64) - out["b"]))
    over = D.astype(np.int64) - grid["cap"]
    assert (H == H0 + np.maximum(over, 0)).all()
    assert st["relu_overflow"] == np.maximum(over, 0).sum()
    s = np.where(grid["cap"] > 0, 0.5, 1.5)
    assert st["tof"] == pytest.approx(np.sum(np.exp(s * over)), rel=1e-12)
    # Eq. 3 is linear in the per-layer overflow weights: the totals with one
    # layer weighted at a time, scaled and summed, give the total of any weights
    w = np.linspace(0.5, 3.0, L)
    tof_w = oracle.demand(grid | dict(ofw=w), forest, out["layer"], out["b"], out["t"], H0)[2]["tof"]
    parts = [oracle.demand(grid | dict(ofw=np.eye(L)[l]), forest, out["layer"], out["b"], out["t"], H0)[2]["tof"]
             for l in range(L)]
    assert tof_w == pytest.approx(float(np.dot(w, parts)), rel=1e-12)
    assert max(parts) < st["tof"]


# ---------------------------------------------------------------------------
# Elmore delay (Sec. II-C, III-D) and its adjoint
# ---------------------------------------------------------------------------
def test_elmore_equals_textbook_path_sum():
    wl = fg.WORKLOADS[1].scaled(120)
    grid, forest = fg.make_grid(wl, 9), fg.make_forest(wl, 9)
    out = _round_on(grid, forest, W_ALL, 9)
    R, C = oracle.rc_from_assignment(grid, forest, out["layer"])
    delay = oracle.elmore(grid, forest, out["layer"], out["b"], out["t"], R, C)
    for n, net in enumerate(br.nets_of(forest)):
        a = int(forest["net_ptr"][n])
        lay, bt, _ = _net_assignment(forest, out, n)
        nodes, outi = br.rc_tree(grid, net, lay, bt, R[a:a + net.m], C[a:a + net.m])
        for v in range(net.m):
            assert delay[a + v] == pytest.approx(br.elmore_path_sum(nodes, outi[v]), rel=1e-12)


@pytest.mark.parametrize("pieces", [1, 2, 3, 5, 8, 13])
def test_elmore_distributed_wire_closed_form(pieces):
    """Driver R_d, a wire R, C cut into n equal pi pieces, load C_L:
    delay = R_d (C + C_L) + R C / 2 + R C_L for every n."""
    Rd, Rw, Cw, CL = 350.0, 80.0, 12.0, 4.5
    rows = [(-1, 0, 0, 0, 0.0, 0.0)] + [(i - 1, i, 0, -1, 0.0, 0.0) for i in range(1, pieces)]
    rows.append((pieces - 1, pieces, 0, 0, CL, 1.0))
    forest = forest_from_rows(rows, r_drv=Rd)
    grid = simple_grid(pieces + 2, 4, 2, (1, 1), (1, 1), (0.0,), 0.0)
    V = pieces + 1
    lay = np.zeros(V, np.int8)
    R = np.full(V, Rw / pieces); C = np.full(V, Cw / pieces)
    R[0] = C[0] = 0.0
    delay = oracle.elmore(grid, forest, lay, lay, lay, R, C)
    want = Rd * (Cw + CL) + Rw * Cw / 2 + Rw * CL
    assert delay[-1] == pytest.approx(want, rel=1e-14)


def test_elmore_worked_example_d34():
    """d_34 = R_34 (C4 + C5 + C6 + C7) (Sec. III-D) with pi-lumped node caps."""
    forest, loc = _fig6_forest()
    grid = simple_grid(8, 8, 4, (4.0, 3.0, 2.0, 1.0), (0.2, 0.25, 0.3, 0.35), (0.0, 0.0, 0.0), 0.07)
    V = 5
    lay = np.array([0, 2, 1, 0, 3], np.int8)   # nodes 3,4,5,6,7 (H, H, V, H, V)
    b = np.array([0, 0, 0, 0, 0], np.int8)
    t = np.array([2, 2, 1, 3, 3], np.int8)     # hulls of junction, pin and sons
    R, C = oracle.rc_from_assignment(grid, forest, lay)
    d = oracle.elmore(grid, forest, lay, b, t, R, C)
    vc = 0.07
    seg = {4: loc[4], 5: loc[5], 6: loc[6], 7: loc[7]}
    # pi-model node caps: half of each incident segment + vias + pin
    Cn = {
        4: C[seg[4]] / 2 + C[seg[5]] / 2 + C[seg[6]] / 2 + vc * 2,
        5: C[seg[5]] / 2 + vc * 1 + 2.0,
        6: C[seg[6]] / 2 + C[seg[7]] / 2 + vc * 3,
        7: C[seg[7]] / 2 + vc * 3 + 3.5,
    }
    d34 = d[loc[4]] - d[loc[3]]
    assert d34 == pytest.approx(R[seg[4]] * (Cn[4] + Cn[5] + Cn[6] + Cn[7]), rel=1e-13)


def test_elmore_on_table1_layers():
    """One straight segment on each metal layer of Table I (per-um values, 1 um
    GCells): delay = (R_d + Rv)(C + C_L) + R (C/2 + C_L) + Rv C_L, Rv = the
    via path from metal1 (pins) to the layer."""
    rows = read_table1()
    L = len(rows)
    unit_r = [r for (_, r, _, _) in rows]
    unit_c = [c for (_, _, c, _) in rows]
    via_r = [v for (_, _, _, v) in rows[:-1]]
    grid = simple_grid(40, 40, L, unit_r, unit_c, via_r, 0.0)
    Rd, CL, length = 1.2, 1.7, 30
    for l in range(L):
        horiz = l % 2 == 0
        rows_f = [(-1, 0, 0, 0, 0.0, 0.0), (0, length if horiz else 0, 0 if horiz else length, 0, CL, 1.0)]
        forest = forest_from_rows(rows_f, r_drv=Rd)
        lay = np.array([0, l], np.int8)
        b = np.array([0, 0], np.int8)
        t = np.array([l, l], np.int8)
        R, C = oracle.rc_from_assignment(grid, forest, lay)
        d = oracle.elmore(grid, forest, lay, b, t, R, C)
        Rv = math.fsum(via_r[:l])
        Rw, Cw = length * unit_r[l], length * unit_c[l]
        want = (Rd + Rv) * (Cw + CL) + Rw * (Cw / 2 + CL) + Rv * CL
        assert d[1] == pytest.approx(want, rel=1e-13), rows[l][0]


def _adjoint_case(seed, nets=60):
    wl = fg.WORKLOADS[1].scaled(nets)
    grid, forest = fg.make_grid(wl, seed), fg.make_forest(wl, seed)
    out = _round_on(grid, forest, W_ALL, seed)
    R, C = oracle.rc_from_assignment(grid, forest, out["layer"])
    g = np.where(forest["pin_layer"] >= 0, forest["kappa"], 0.0)
    return grid, forest, out, R, C, g


def test_adjoint_equals_central_differences():
    """T = sum kappa delay is affine in each single R or C, so central
    differences are exact up to rounding."""
    grid, forest, out, R, C, g = _adjoint_case(21)
    lay, b, t = out["layer"], out["b"], out["t"]
    dR, dC, _, _ = oracle.elmore_backward(grid, forest, lay, b, t, R, C, g)

    def T(Rx, Cx):
        return float(np.dot(g, oracle.elmore(grid, forest, lay, b, t, Rx, Cx)))

    rng = np.random.default_rng(0)
    for v in rng.choice(np.nonzero(forest["parent"] >= 0)[0], 40, replace=False):
        h = 1e-3 * R[v]
        Rp, Rm = R.copy(), R.copy()
        Rp[v] += h; Rm[v] -= h
        assert dR[v] == pytest.approx((T(Rp, C) - T(Rm, C)) / (2 * h), rel=1e-6)
        h = 1e-3 * C[v]
        Cp, Cm = C.copy(), C.copy()
        Cp[v] += h; Cm[v] -= h
        assert dC[v] == pytest.approx((T(R, Cp) - T(R, Cm)) / (2 * h), rel=1e-6)


def test_adjoint_cap_gradient_equals_common_path_sum():
    """dT/dcap(y) = sum_s kappa_s R_common(s, y) on the explicit RC tree; the
    segment cap is split half/half between its two ends (pi-model)."""
    grid, forest, out, R, C, g = _adjoint_case(22, nets=40)
    lay_all, b_all, t_all = out["layer"], out["b"], out["t"]
    dR, dC, Ws, _ = oracle.elmore_backward(grid, forest, lay_all, b_all, t_all, R, C, g)
    for n, net in enumerate(br.nets_of(forest)):
        a = int(forest["net_ptr"][n])
        lay, bt, _ = _net_assignment(forest, out, n)
        nodes, outi = br.rc_tree(grid, net, lay, bt, R[a:a + net.m], C[a:a + net.m])

        def path(i):
            s = set()
            while i != -1:
                s.add(i)
                i = nodes[i][0]
            return s

        sinks = [(outi[v], g[a + v]) for v in range(net.m) if g[a + v] != 0.0]
        for v in range(1, net.m):
            # node indices of X_v and J_v in rc_tree's construction order
            Xi = 2 * v - 1
            Ji = 2 * v
            gX = sum(k * sum(nodes[i][1] for i in path(s) & path(Xi)) for s, k in sinks)
            gJ = sum(k * sum(nodes[i][1] for i in path(s) & path(Ji)) for s, k in sinks)
            assert dC[a + v] == pytest.approx(0.5 * (gX + gJ), rel=1e-12, abs=1e-300)
            # dT/dR_v = Cdown(J_v) * (criticality below v)
            below = [s for s, k in sinks if Ji in path(s)]
            cd = sum(nodes[k][2] for k in range(len(nodes)) if Ji in path(k))
            kap = sum(k for s, k in sinks if s in below)
            assert dR[a + v] == pytest.approx(cd * kap, rel=1e-12, abs=1e-300)


def test_sequential_batches_oracle():
    """Sequential batches (Sec. III-A): one batch is the snapshot round; with
    several, batch k's choice is the DP against the demand its predecessors
    left, and the final demand is the demand of the final assignment."""
    import forestgen as fg

    wl = fg.WORKLOADS[2].scaled(3000)
    grid, forest = fg.make_grid(wl, 5), fg.make_forest(wl, 5)
    N = int(forest["num_nets"])
    one = oracle.assign_round_batches(grid, forest, np.zeros(N, np.int32))
    ref = oracle.assign_round(grid, forest)
    for k in ("layer", "b", "t", "D", "H"):
        assert np.array_equal(one[k], ref[k])
    assert np.array_equal(one["J"], ref["J"])
    rng = np.random.default_rng(1)
    batch = rng.integers(0, 3, N).astype(np.int32)
    r1 = oracle.assign_round_batches(grid, forest, batch)
    Dchk, _, _ = oracle.demand(grid, forest, r1["layer"], r1["b"], r1["t"], np.zeros_like(r1["D"]))
    assert np.array_equal(Dchk, r1["D"])
    # batch 0 sees an empty map, so its nets match the snapshot round from zero
    net_of = np.repeat(np.arange(N), np.diff(forest["net_ptr"]))
    sel0 = batch[net_of] == 0
    assert np.array_equal(r1["layer"][sel0], ref["layer"][sel0])
    # the last batch sees batches 0 and 1 committed: its nets match a DP on that map
    sub, nodes = oracle._net_subset(forest, np.nonzero(batch < 2)[0])
    D01, _, _ = oracle.demand(grid, sub, r1["layer"][nodes], r1["b"][nodes], r1["t"][nodes], np.zeros_like(r1["D"]))
    pen = oracle.penalty(grid, D01, np.zeros_like(D01), oracle.DEFAULT_WEIGHTS["hist_w"])
    W, rho = oracle.weights_eq4(grid, forest)
    out = oracle.dp(grid, forest, oracle.DEFAULT_WEIGHTS, pen, W, rho)
    sel2 = batch[net_of] == 2
    assert np.array_equal(out["layer"][sel2], r1["layer"][sel2])
    assert not np.array_equal(r1["layer"], ref["layer"])  # the order changes the outcome


def test_sequential_batches_from_a_previous_assignment():
    """A round after a previous one, in sequential batches (Sec. III-A): batch
    k sees the nets of batches < k on their new layers and every other net on
    its previous layer, against the round's start history.  The map the last
    batch sees is rebuilt here from that composite assignment by the demand
    count alone."""
    import forestgen as fg

    wl = fg.WORKLOADS[2].scaled(3000)
    grid, forest = fg.make_grid(wl, 6), fg.make_forest(wl, 6)
    N = int(forest["num_nets"])
    prev = oracle.assign_round(grid, forest)
    # one batch from the previous state is the snapshot round
    one = oracle.assign_round_batches(grid, forest, np.zeros(N, np.int32), D=prev["D"], H=prev["H"],
                                      layer_prev=prev["layer"])
    snap = oracle.assign_round(grid, forest, D=prev["D"], H=prev["H"])
    for k in ("layer", "b", "t", "D", "H"):
        assert np.array_equal(one[k], snap[k])
    batch = np.random.default_rng(2).integers(0, 3, N).astype(np.int32)
    r = oracle.assign_round_batches(grid, forest, batch, D=prev["D"], H=prev["H"], layer_prev=prev["layer"])
    net_of = np.repeat(np.arange(N), np.diff(forest["net_ptr"]))
    last = batch[net_of] == 2
    seen = np.where(last, prev["layer"], r["layer"]).astype(np.int8)
    D_seen, _, _ = oracle.demand(grid, forest, seen, r["b"], r["t"], np.zeros_like(prev["D"]))
    pen = oracle.penalty(grid, D_seen, prev["H"], oracle.DEFAULT_WEIGHTS["hist_w"])
    W, rho = oracle.weights_eq4(grid, forest)
    out = oracle.dp(grid, forest, oracle.DEFAULT_WEIGHTS, pen, W, rho)
    assert np.array_equal(out["layer"][last], r["layer"][last])
    assert not np.array_equal(r["layer"], snap["layer"])  # the batches change the outcome


def test_history_raises_the_penalty_of_a_round():
    """Negotiation (Sec. I, Eq. 3's penalty with the history term): a 2-pin
    straight net on an empty map takes the lowest horizontal layer (no vias);
    with history on that layer's edges of the route it moves to the other
    horizontal layer, and history elsewhere changes nothing."""
    grid = simple_grid(12, 6, 4, (1.0, 1.0, 1.0, 1.0), (0.2, 0.2, 0.2, 0.2), (1.0, 1.0, 1.0), 0.05)
    forest = forest_from_rows([(-1, 2, 3, 0, 0.0, 0.0), (0, 8, 3, 0, 1.0, 0.5)], r_drv=100.0)
    E = oracle.num_edges(grid)
    zero = np.zeros(E, np.int32)
    base = oracle.assign_round(grid, forest, D=zero, H=zero)
    assert int(base["layer"][1]) == 0
    # layer 0 (H) is the first block of the public layout: row y = 3, edges x = 2 .. 7
    per_row = grid["X"] - 1
    H = zero.copy()
    H[3 * per_row + 2: 3 * per_row + 8] = 50
    moved = oracle.assign_round(grid, forest, D=zero, H=H)
    assert int(moved["layer"][1]) == 2
    H_off = zero.copy()
    H_off[1 * per_row + 2: 1 * per_row + 8] = 50  # another row
    same = oracle.assign_round(grid, forest, D=zero, H=H_off)
    assert int(same["layer"][1]) == 0 and same["J"][0] == base["J"][0]


def test_adjoint_weights_come_from_sinks_only():
    """The adjoint weights (g = kappa at the sinks): W(v) = the sum of the
    sinks' kappa below v, whatever kappa a node without a pin carries."""
    forest, loc = _fig6_forest()
    grid = simple_grid(8, 8, 4, (4.0, 3.0, 2.0, 1.0), (0.2, 0.2, 0.2, 0.2), (1.0, 1.0, 1.0), 0.05)
    nopin = forest["pin_layer"] < 0
    assert nopin.any()
    f2 = dict(forest, kappa=np.where(nopin, 5.0, forest["kappa"]))
    out = oracle.assign_round(grid, f2)
    Ws, _ = oracle.adjoint_weights(grid, f2, out["layer"], out["b"], out["t"])
    par = f2["parent"]
    for v in range(len(par)):
        want, stack = 0.0, [v]
        while stack:  # the subtree of v, by its parent links
            u = stack.pop()
            if f2["pin_layer"][u] >= 0:
                want += float(f2["kappa"][u])
            stack += [c for c in range(len(par)) if par[c] == u]
        assert Ws[v] == pytest.approx(want, rel=1e-15), v


# ---------------------------------------------------------------------------
# Tie rules (reading of Alg. 3, Kernel 1 and Kernel 2): exact ties resolved as
# documented, checked against the full set of brute-force minimisers
# ---------------------------------------------------------------------------
def _tie_check(case):
    from util_inputs import TIE_WEIGHTS

    grid, forest, want_layers, want_stacks = case
    out = oracle.assign_round(grid, forest, TIE_WEIGHTS)
    net = br.nets_of(forest)[0]
    lay, bt, W = _net_assignment(forest, out, 0)
    Jb, arg = br.brute_force(grid, net, out["pen"], TIE_WEIGHTS, W)
    # w_d = 0: the DP is exact; the case has several minimisers
    assert out["J"][0] == float(Jb)
    assert len(arg) >= 2 and lay in arg
    assert lay == want_layers
    assert bt == want_stacks
    return arg


def test_son_takes_its_lowest_tied_layer():
    """Kernel 1: inside a stack, a son whose keys tie on two layers takes the
    lower one (here the H leaf on layer 0, not 2)."""
    from util_inputs import son_tie_case

    arg = _tie_check(son_tie_case())
    assert [0, 2, 3] in arg  # the other minimiser, which the rule excludes


def test_stack_tie_fewest_vias_then_lowest_bottom():
    """Kernel 2: stacks of equal f' are ordered by via count, then by their
    bottom layer (here [1, 2] over [2, 3] at the bend, so the leaf goes on
    layer 1, not 3; and not the wider [0, 2] a lowest-bottom-first order
    would take)."""
    from util_inputs import stack_tie_case

    arg = _tie_check(stack_tie_case())
    assert [0, 2, 3] in arg


# ---------------------------------------------------------------------------
# Pin weights (Sec. III-C) and Alg. 1's partition (Sec. III-A)
# ---------------------------------------------------------------------------
def test_logistic_pin_weight_fixed_points():
    """The logistic of the slack ratio x = slack / WNS: exactly 1/2 at x = b,
    close to 1 at the worst slack (x = 1: the paper's "nearly 1"), small for
    positive slack, symmetric about b, increasing in x, 0 off the pins."""
    k, b = 10.0, 0.3
    x = np.array([0.3, 1.0, -0.5, 0.0, 0.3 + 0.125, 0.3 - 0.125, 0.3 + 0.25, 0.3 - 0.25, 0.15, 0.8, 0.99])
    pin = np.zeros(len(x) + 1, np.int8)
    pin[-1] = -1
    slack = np.append(x, 5.0)          # WNS = -1: the slack ratio is -slack
    w = oracle.logistic_pin_weight(pin, -slack, -1.0, k, b)
    assert w[0] == 0.5
    assert 0.999 < w[1] < 1.0
    assert w[2] < 1e-3 and w[3] < 0.05
    for i in (4, 6):
        assert abs(w[i] + w[i + 1] - 1.0) <= 2.0 ** -52
    xs, first = np.unique(x, return_index=True)
    assert np.all(np.diff(w[first]) > 0)
    assert w[-1] == 0.0


def test_partition_on_interval_edges():
    """Nets placed on every interval edge of Alg. 1: criticality C = 8 with
    critical_frac 1/4 gives [8, 8], [4, 8), [2, 4); slack with WNS = -100 and
    slack_ratio 0.7 gives slack = WNS, (WNS, 0.99 WNS], (0.99 WNS, 0.96 WNS],
    ..., (0.75 WNS, 0.64 WNS]; the rest last; ids without gaps."""
    crit = np.array([8, 4, 6, 2, 3.9999, 0.5, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0])
    slack = np.array([-1, -1, -1, -1, -1, -100, -99, -99.5, -98.9, -96, -71, -69, 0.0, -100.0])
    got, nb = oracle.partition_batches(crit, slack, critical_frac=0.25, slack_ratio=0.7)
    # net by net: critical interval k, semi-critical interval j, or the rest
    keys = [("c", 0), ("c", 1), ("c", 1), ("c", 2), ("c", 2),  # 8, 4, 6, 2, 3.9999
            ("s", 0), ("s", 1), ("s", 1), ("s", 2), ("s", 2),  # -100, -99, -99.5, -98.9, -96
            ("s", 6), ("r", 0), ("r", 0), ("s", 0)]             # -71, -69 (> 0.7 WNS), 0, -100
    rank = {"c": 0, "s": 1, "r": 2}
    order = sorted(set(keys), key=lambda t: (rank[t[0]], t[1]))
    want = [order.index(t) for t in keys]
    assert list(got) == want and nb == len(order) == 8
    # without slack: critical nets, then one batch
    got2, nb2 = oracle.partition_batches(crit, None, critical_frac=0.25)
    assert list(got2) == [0, 1, 1, 2, 2, 3, 3, 3, 3, 3, 3, 3, 3, 3] and nb2 == 4


def test_partition_matches_exact_intervals():
    """Random criticalities and slacks: each net's batch follows from its
    interval computed in exact rational arithmetic, and the batch ids are
    those intervals in Alg. 1's order."""
    rng = np.random.default_rng(4)
    N = 3000
    crit = rng.uniform(0, 10, N) ** 2
    slack = rng.uniform(-50, 20, N)
    got, nb = oracle.partition_batches(crit, slack, critical_frac=0.1, slack_ratio=0.7)
    C, W = Fr(float(crit.max())), Fr(float(slack.min()))
    keys = []
    for c, s in zip(crit, slack):
        c, s = Fr(float(c)), Fr(float(s))
        if c >= Fr(1, 10) * C:
            k = 0 if c == C else next(k for k in range(1, 200) if c >= C / 2 ** k)
            keys.append((0, k))
        elif s <= Fr(7, 10) * W:
            j = 0 if s == W else next(j for j in range(1, 200) if s <= W * (1 - Fr(j * j, 100)))
            keys.append((1, j))
        else:
            keys.append((2, 0))
    order = sorted(set(keys))
    assert nb == len(order)
    assert list(got) == [order.index(t) for t in keys]
