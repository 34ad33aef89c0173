"""The seeded input generator: determinism and the directed-tree structure."""
import numpy as np

import forestgen as fg
from util_inputs import tiny


def test_deterministic_and_thread_independent():
    wl = fg.WORKLOADS[2].scaled(5000)
    a = fg.make_forest(wl, seed=4, threads=1)
    b = fg.make_forest(wl, seed=4, threads=7)
    for k in ("net_ptr", "x", "y", "parent", "pin_layer", "sink_cap", "kappa", "r_drv"):
        assert np.array_equal(a[k], b[k]), k
    ga, gb = fg.make_grid(wl, 4, threads=1), fg.make_grid(wl, 4, threads=5)
    assert np.array_equal(ga["cap"], gb["cap"])
    c = fg.make_forest(wl, seed=5)
    assert not np.array_equal(a["x"], c["x"])


def test_directed_tree_has_straight_segments_and_parents_first():
    """Every tree edge is a straight H/V run (Sec. III-B: nodes are added at
    bends); parent < child inside a net; the root carries the driver pin."""
    wl = fg.WORKLOADS[1]
    f = fg.make_forest(wl, 0)
    ptr, par = f["net_ptr"], f["parent"]
    net_of = np.repeat(np.arange(f["num_nets"]), np.diff(ptr))
    local = np.arange(f["num_nodes"]) - ptr[net_of]
    assert (par[local == 0] == -1).all() and (par[local > 0] >= 0).all()
    assert (par[local > 0] < local[local > 0]).all()
    assert (f["pin_layer"][local == 0] == 0).all()
    v = np.nonzero(local > 0)[0]
    p = ptr[net_of[v]] + par[v]
    dx, dy = f["x"][v] - f["x"][p], f["y"][v] - f["y"][p]
    assert (((dx == 0) ^ (dy == 0))).all()
    # bend nodes (no pin) have exactly one son and turn the corner
    bend = v[f["pin_layer"][v] < 0]
    nsons = np.bincount(ptr[net_of[v]] + par[v], minlength=f["num_nodes"])
    assert (nsons[bend] == 1).all()


def test_l_shaped_edge_becomes_two_segments_and_a_bend_node():
    """Fig. 5: net 2 has 4 nodes in 2D and 5 in the directed tree, the extra one
    at the bend.  A 2-pin net whose pins differ in x and y gives 3 nodes."""
    wl = tiny(pin_a=2, pin_b=2, num_nets=300)
    f = fg.make_forest(wl, 1)
    sizes = np.diff(f["net_ptr"])
    for n in range(300):
        a = f["net_ptr"][n]
        if sizes[n] == 3:
            assert f["pin_layer"][a + 1] == -1 and f["parent"][a + 2] == 1
            assert f["x"][a + 1] == f["x"][a + 2] and f["y"][a + 1] == f["y"][a]
    assert set(np.unique(sizes)) <= {1, 2, 3} and (sizes == 3).sum() > 100


def test_nangate45_workload_is_table1():
    """The NanGate45 workload's stack is the paper's Table I read with a 1 um
    GCell edge (R per GCell in Ohm = 1000 x kOhm/um; via R in Ohm)."""
    from util_inputs import read_table1

    rows = read_table1()
    g = fg.make_grid(fg.WORKLOADS[6].scaled(50), 0)
    assert g["L"] == len(rows) == 10
    assert np.allclose(g["unit_r"], [1000.0 * r for _, r, _, _ in rows], rtol=1e-12)
    assert np.allclose(g["unit_c"], [c for _, _, c, _ in rows], rtol=1e-12)
    assert np.allclose(g["via_r"], [1000.0 * v for _, _, _, v in rows[:-1]], rtol=1e-12)
