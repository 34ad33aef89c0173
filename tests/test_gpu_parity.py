"""GPU (CUDA, sm_103a) vs the FP64 CPU oracle, element by element.

Layers, via stacks, demand, history and vias must match bit for bit; the
per-net costs J (FP64, same expression trees on both sides) are compared
exactly too, and the total cost within 1e-9 relative."""
import numpy as np
import pytest

import forestgen as fg
import oracle
from util_inputs import edge_case_forest, merge_forests, random_snapshot, simple_grid

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def la():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2507_13375_gb300 as la

    la.library()
    return la


def gpu_round(a, weights, reset=False, weights_src=0):
    st = a.assign_round(reset=reset, weights=weights_src, **weights)
    layer, b, t = (x.cpu().numpy() for x in a.get_assignment())
    D, H = (x.cpu().numpy() for x in a.get_state())
    J = a.get_net_cost().cpu().numpy()
    return dict(layer=layer, b=b, t=t, D=D, H=H, J=J, stats=st)


def assert_same_round(got, ref, label=""):
    assert np.array_equal(got["layer"], ref["layer"]), f"{label}: layers differ at " \
        f"{np.nonzero(got['layer'] != ref['layer'])[0][:10]}"
    assert np.array_equal(got["b"], ref["b"]) and np.array_equal(got["t"], ref["t"]), f"{label}: via stacks"
    assert np.array_equal(got["J"], ref["J"]), f"{label}: max |dJ|/J = " \
        f"{np.max(np.abs(got['J'] - ref['J']) / np.maximum(np.abs(ref['J']), 1e-300))}"
    assert np.array_equal(got["D"], ref["D"]), f"{label}: demand"
    assert np.array_equal(got["H"], ref["H"]), f"{label}: history"
    s, r = got["stats"], ref["stats"]
    assert s["vias"] == r["vias"] and s["wl"] == r["wl"] and s["relu_overflow"] == r["relu_overflow"]
    assert list(s["wl_per_layer"][: len(r["wl_per_layer"])]) == list(r["wl_per_layer"])
    # Eq. 3 total overflow sums one term per GCell edge; summed sequentially
    # (oracle) or by blocks (GPU), n non-negative terms agree to n * 2^-53
    n_edges = len(got["D"])
    assert s["tof"] == pytest.approx(r["tof"], rel=max(1e-12, 2.0 * n_edges * 2.0 ** -53))
    assert s["total_cost"] == pytest.approx(r["total_cost"], rel=1e-9)


def ref_round(grid, forest, weights, D=None, H=None, W=None, rho=None):
    """The oracle's round; its stats carry total_cost = sum of J."""
    return oracle.assign_round(grid, forest, weights, D=D, H=H, W=W, rho=rho)


def _assigner(la, grid, forest):
    a = la.LayerAssigner(0)
    a.load_grid(grid)
    a.load_nets(forest)
    return a


def test_round_config1(la):
    wl = fg.WORKLOADS[1]
    grid, forest = fg.make_grid(wl, 0), fg.make_forest(wl, 0)
    a = _assigner(la, grid, forest)
    got = gpu_round(a, la.DEFAULT_WEIGHTS, reset=True)
    ref = ref_round(grid, forest, la.DEFAULT_WEIGHTS)
    assert_same_round(got, ref)


@pytest.mark.parametrize("weights", [dict(w_d=0.0), dict(w_d=5e-2, w_cong=1e-2), dict(w_via=0.0, w_cap=0.0),
                                     dict(hist_w=3.0, w_d=2e-3)])
def test_round_random_snapshot(la, weights):
    """Congested random snapshot (D, H) and several weight mixes, 3 rounds,
    each round's oracle fed the GPU's previous (D, H)."""
    wl = fg.WORKLOADS[2].scaled(20000)
    grid, forest = fg.make_grid(wl, 3), fg.make_forest(wl, 3)
    ww = dict(la.DEFAULT_WEIGHTS, **weights)
    a = _assigner(la, grid, forest)
    D, H = random_snapshot(len(grid["cap"]), 3, dmax=18, hmax=4)
    a.set_state(D, H)
    for r in range(3):
        got = gpu_round(a, ww)
        ref = ref_round(grid, forest, ww, D=D, H=H)
        assert_same_round(got, ref, f"round {r}")
        D, H = got["D"], got["H"]


def test_multi_round_config2_full(la):
    """500k nets, 3 negotiation rounds; round r's oracle starts from the GPU's
    round r-1 snapshot."""
    wl = fg.WORKLOADS[2]
    grid, forest = fg.make_grid(wl, 0), fg.make_forest(wl, 0)
    a = _assigner(la, grid, forest)
    D = H = None
    for r in range(wl.rounds):
        got = gpu_round(a, la.DEFAULT_WEIGHTS, reset=(r == 0))
        ref = ref_round(grid, forest, la.DEFAULT_WEIGHTS, D=D, H=H)
        assert_same_round(got, ref, f"round {r}")
        D, H = got["D"], got["H"]


@pytest.mark.parametrize("L", [2, 4, 6, 12, 16])
def test_edge_cases_and_layer_counts(la, L):
    X, Y = 24, 20
    rng = np.random.default_rng(L)
    unit_r = list(np.round(rng.uniform(0.5, 9.0, L), 3))
    unit_c = list(np.round(rng.uniform(0.1, 0.3, L), 3))
    grid = simple_grid(X, Y, L, unit_r, unit_c, list(rng.uniform(0.5, 4.0, L - 1)), 0.04)
    grid["cap"] = rng.integers(0, 5, len(grid["cap"])).astype(np.int32)
    forest = merge_forests([edge_case_forest(X, Y, L, seed=L),
                            fg.make_forest(fg.Workload("e", X, Y, L, (1, 4), 0.0, 300, 0, 2, 9, 0.0, False,
                                                       tuple(unit_r), tuple(unit_c), 1), seed=L)])
    a = _assigner(la, grid, forest)
    for r in range(2):
        D, H = (None, None) if r == 0 else (got["D"], got["H"])
        got = gpu_round(a, dict(la.DEFAULT_WEIGHTS, w_d=2e-2), reset=(r == 0))
        ref = ref_round(grid, forest, dict(la.DEFAULT_WEIGHTS, w_d=2e-2), D=D, H=H)
        assert_same_round(got, ref, f"L={L} r={r}")


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_long_lines_take_the_global_demand_path(la, mode):
    """Lines too long for the shared-memory difference array (13000 positions x
    2 layers) take the global-atomics demand pass and the separate scan; the
    result is the oracle's either way."""
    X, Y, L = 13000, 6, 4
    grid = simple_grid(X, Y, L, [6.0, 5.0, 2.0, 1.5], [0.2, 0.19, 0.17, 0.15], [2.0, 2.0, 2.0], 0.05, cap=2)
    wl = fg.Workload("long", X, Y, L, (1, 3), 0.0, 400, 0, 2, 12, 0.0, False, (6.0, 5.0, 2.0, 1.5),
                     (0.2, 0.19, 0.17, 0.15), 1)
    forest = fg.make_forest(wl, seed=2)
    a = _assigner(la, grid, forest)
    m = la.LA_MODE_PLAIN if mode == "plain" else la.LA_MODE_BATCHED
    D = H = None
    for r in range(2):
        st = a.assign_round(mode=m, reset=(r == 0), **la.DEFAULT_WEIGHTS)
        got = dict(zip(("layer", "b", "t"), (x.cpu().numpy() for x in a.get_assignment())))
        got["D"], got["H"] = (x.cpu().numpy() for x in a.get_state())
        got["J"] = a.get_net_cost().cpu().numpy()
        got["stats"] = st
        ref = ref_round(grid, forest, la.DEFAULT_WEIGHTS, D=D, H=H)
        assert_same_round(got, ref, f"{mode} r={r}")
        D, H = got["D"], got["H"]


def test_non_alternating_directions(la):
    X, Y, L = 16, 16, 6
    dirs = np.array([0, 0, 1, 1, 0, 1], np.int8)
    E = sum(Y * (X - 1) if d == 0 else X * (Y - 1) for d in dirs)
    rng = np.random.default_rng(5)
    grid = dict(X=X, Y=Y, L=L, dir=dirs, cap=rng.integers(0, 6, E).astype(np.int32),
                unit_r=np.array([6.0, 5.0, 4.0, 3.0, 1.0, 0.7]), unit_c=np.array([0.2, 0.21, 0.18, 0.17, 0.15, 0.16]),
                via_r=np.array([1.0, 2.0, 1.5, 3.0, 0.5]), via_c=0.03, ofw=np.array([1.0, 2.0, 1.0, 0.5, 1.0, 1.5]))
    wl = fg.Workload("nd", X, Y, L, (1, 4), 0.0, 400, 0, 2, 7, 0.0, False, tuple(grid["unit_r"]),
                     tuple(grid["unit_c"]), 1)
    forest = fg.make_forest(wl, 9)
    a = _assigner(la, grid, forest)
    got = gpu_round(a, dict(la.DEFAULT_WEIGHTS, w_d=1e-2), reset=True)
    ref = ref_round(grid, forest, dict(la.DEFAULT_WEIGHTS, w_d=1e-2))
    assert_same_round(got, ref)


def test_elmore_and_adjoint_config3(la):
    """Config 3: the 500k-net forest of config 2 with a fixed assignment;
    FP64 delays and d(sum kappa delay)/d(R, C) against the oracle, and central
    differences through the GPU path on 1000 sampled nets."""
    wl = fg.WORKLOADS[3]
    grid, forest = fg.make_grid(wl, 0), fg.make_forest(wl, 0)
    a = _assigner(la, grid, forest)
    a.assign_round(reset=True, **la.DEFAULT_WEIGHTS)
    layer, b, t = (x.cpu().numpy() for x in a.get_assignment())
    R, C = a.rc_from_assignment()
    Rr, Cr = oracle.rc_from_assignment(grid, forest, layer)
    assert np.array_equal(R.cpu().numpy(), Rr) and np.array_equal(C.cpu().numpy(), Cr)
    g = np.where(forest["pin_layer"] >= 0, forest["kappa"], 0.0)
    gt = torch.from_numpy(g).cuda()
    Rg, Cg = R.clone().requires_grad_(True), C.clone().requires_grad_(True)
    delay = la.ElmoreFn.apply(a, Rg, Cg)
    (delay * gt).sum().backward()
    d_ref = oracle.elmore(grid, forest, layer, b, t, Rr, Cr)
    dR_ref, dC_ref, _, _ = oracle.elmore_backward(grid, forest, layer, b, t, Rr, Cr, g)
    np.testing.assert_allclose(delay.detach().cpu().numpy(), d_ref, rtol=1e-10, atol=0)
    np.testing.assert_allclose(Rg.grad.cpu().numpy(), dR_ref, rtol=1e-10, atol=0)
    np.testing.assert_allclose(Cg.grad.cpu().numpy(), dC_ref, rtol=1e-10, atol=0)
    # central differences on 1000 sampled nets (T is affine in each R and C)
    rng = np.random.default_rng(0)
    ptr = forest["net_ptr"]
    nets = rng.choice(forest["num_nets"], 1000, replace=False)
    cand = np.array([ptr[n] + 1 + rng.integers(0, ptr[n + 1] - ptr[n] - 1) for n in nets if ptr[n + 1] - ptr[n] > 1])
    R0, C0 = R.clone(), C.clone()

    def dT(Rp, Cp, Rm, Cm):
        # delays differ only inside the perturbed net: subtract first, then sum
        return float(torch.dot(a.elmore(Rp, Cp) - a.elmore(Rm, Cm), gt))

    dRg, dCg = Rg.grad.cpu().numpy(), Cg.grad.cpu().numpy()
    checked = 0
    for v in cand[:1000]:
        for which, arr, grad in ((0, R0, dRg), (1, C0, dCg)):
            h = 1e-3 * float(arr[v])
            if h == 0.0:
                continue
            p, m = arr.clone(), arr.clone()
            p[v] += h
            m[v] -= h
            fd = (dT(p, C0, m, C0) if which == 0 else dT(R0, p, R0, m)) / (2 * h)
            assert grad[v] == pytest.approx(fd, rel=1e-6, abs=1e-300), (which, int(v))
            checked += 1
    assert checked >= 1500


def test_adjoint_reweighted_round(la):
    """Rounds reweighted by the adjoint sensitivities (W = sum of kappa below,
    r_est = weighted upstream R of the previous assignment)."""
    wl = fg.WORKLOADS[2].scaled(30000)
    grid, forest = fg.make_grid(wl, 4), fg.make_forest(wl, 4)
    a = _assigner(la, grid, forest)
    got = gpu_round(a, la.DEFAULT_WEIGHTS, reset=True)
    for r in range(2):
        a.reweight_adjoint()
        W, rho = (x.cpu().numpy() for x in a.get_weights(la.LA_WEIGHTS_ADJOINT))
        Wr, rhor = oracle.adjoint_weights(grid, forest, got["layer"], got["b"], got["t"])
        assert np.array_equal(W, Wr) and np.array_equal(rho, rhor)
        D, H = got["D"], got["H"]
        got = gpu_round(a, la.DEFAULT_WEIGHTS, weights_src=la.LA_WEIGHTS_ADJOINT)
        ref = ref_round(grid, forest, la.DEFAULT_WEIGHTS, D=D, H=H, W=Wr, rho=rhor)
        assert_same_round(got, ref, f"adjoint {r}")


def test_eq4_weights_match_oracle(la):
    wl = fg.WORKLOADS[2].scaled(20000)
    grid, forest = fg.make_grid(wl, 8), fg.make_forest(wl, 8)
    a = _assigner(la, grid, forest)
    W, rho = (x.cpu().numpy() for x in a.get_weights(la.LA_WEIGHTS_EQ4))
    Wr, rhor = oracle.weights_eq4(grid, forest)
    assert np.array_equal(W, Wr) and np.array_equal(rho, rhor)


@pytest.mark.parametrize("case", ["bent_segment", "parent_order", "outside", "root_without_pin", "negative_cap",
                                  "cap_without_pin", "net_ptr"])
def test_malformed_forest_is_rejected(la, case):
    wl = fg.WORKLOADS[1].scaled(50)
    grid, forest = fg.make_grid(wl, 1), fg.make_forest(wl, 1)
    bad = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in forest.items()}
    v = int(bad["net_ptr"][3]) + 1
    if case == "bent_segment":
        bad["x"][v] += 1
        bad["y"][v] += 1
    elif case == "parent_order":
        bad["parent"][v] = v - int(bad["net_ptr"][3]) + 1
    elif case == "outside":
        bad["x"][v] = wl.X + 3
    elif case == "root_without_pin":
        bad["pin_layer"][int(bad["net_ptr"][5])] = -1
    elif case == "negative_cap":
        bad["sink_cap"][v] = -1.0
    elif case == "cap_without_pin":
        bad["sink_cap"][int(np.flatnonzero(bad["pin_layer"] < 0)[0])] = 1.0
    elif case == "net_ptr":
        bad["net_ptr"][4] = bad["net_ptr"][6]
    a = la.LayerAssigner(0)
    a.load_grid(grid)
    with pytest.raises(la.LaError) as e:
        a.load_nets(bad)
    assert e.value.status == la.LA_ERR_INVALID
    # the context is still usable
    a.load_nets(forest)
    a.assign_round(reset=True)


# ---------------------------------------------------------------------------
# Batched form (size buckets, persistent block-per-net kernels, autotuner,
# CUDA graph): bit-identical to the plain form and to the oracle.
# ---------------------------------------------------------------------------
def _rounds(a, la, mode, n, weights=None, adjoint=False, tail_threshold=0):
    out = []
    for r in range(n):
        src = la.LA_WEIGHTS_ADJOINT if (adjoint and r > 0) else la.LA_WEIGHTS_EQ4
        st = a.assign_round(mode=mode, reset=(r == 0), weights=src, tail_threshold=tail_threshold,
                            **(weights or la.DEFAULT_WEIGHTS))
        got = dict(zip(("layer", "b", "t"), (x.cpu().numpy() for x in a.get_assignment())))
        got["D"], got["H"] = (x.cpu().numpy() for x in a.get_state())
        got["J"] = a.get_net_cost().cpu().numpy()
        got["stats"] = st
        out.append(got)
        if adjoint:
            a.reweight_adjoint()
    return out


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_pins_on_upper_layers(la, mode):
    """Every pin on a random layer (the generator puts them on layer 0): a
    several-son node with a pin above layer 0 and a root whose driver pin is
    there enumerate several stack bottoms (the scan over b repeats for every
    son, without the per-top record), with its first sons staged in shared
    memory; two rounds against the oracle, the second from the GPU's
    snapshot."""
    wl = fg.WORKLOADS[2].scaled(30000)
    grid, forest = fg.make_grid(wl, 11), fg.make_forest(wl, 11)
    rng = np.random.default_rng(11)
    pin = forest["pin_layer"].copy()
    on = pin >= 0
    pin[on] = rng.integers(0, wl.L, int(on.sum())).astype(pin.dtype)
    forest = dict(forest, pin_layer=pin)
    # the case is there: several-son nodes with a pin above layer 0
    par, ptr = forest["parent"], forest["net_ptr"]
    net_of = np.repeat(np.arange(len(ptr) - 1), np.diff(ptr))
    gp = np.where(par >= 0, ptr[net_of] + par, -1)
    sons = np.bincount(gp[gp >= 0], minlength=len(par))
    assert int(((sons >= 2) & (pin > 0) & (par >= 0)).sum()) > 100
    assert int(((sons >= 2) & (pin > 0) & (par < 0)).sum()) > 100
    m = la.LA_MODE_PLAIN if mode == "plain" else la.LA_MODE_BATCHED
    a = _assigner(la, grid, forest)
    D = H = None
    for r in range(2):
        st = a.assign_round(mode=m, reset=(r == 0), **la.DEFAULT_WEIGHTS)
        layer, b, t = (x.cpu().numpy() for x in a.get_assignment())
        Dg, Hg = (x.cpu().numpy() for x in a.get_state())
        got = dict(layer=layer, b=b, t=t, D=Dg, H=Hg, J=a.get_net_cost().cpu().numpy(), stats=st)
        ref = ref_round(grid, forest, la.DEFAULT_WEIGHTS, D=D, H=H)
        assert_same_round(got, ref, f"{mode} round {r}")
        D, H = Dg, Hg
    a.close()


@pytest.mark.parametrize("cfg,nets", [(2, 60000), (4, 20000), (5, 100000)])
def test_batched_equals_plain(la, cfg, nets):
    wl = fg.WORKLOADS[cfg].scaled(nets)
    grid, forest = fg.make_grid(wl, 6), fg.make_forest(wl, 6)
    a = _assigner(la, grid, forest)
    plain = _rounds(a, la, la.LA_MODE_PLAIN, 3, adjoint=True)
    batched = _rounds(a, la, la.LA_MODE_BATCHED, 3, adjoint=True)
    for r, (p, q) in enumerate(zip(plain, batched)):
        for k in ("layer", "b", "t", "D", "H", "J"):
            assert np.array_equal(p[k], q[k]), (cfg, r, k)
        assert p["stats"]["vias"] == q["stats"]["vias"] and p["stats"]["total_cost"] == q["stats"]["total_cost"]


def test_plain_after_batched(la):
    """The plain form recomputes every constant: after batched rounds have
    filled the constant caches of both weight sources, plain rounds on the
    same context still equal the batched ones (adjoint weights included)."""
    wl = fg.WORKLOADS[5].scaled(30000)
    grid, forest = fg.make_grid(wl, 8), fg.make_forest(wl, 8)
    a = _assigner(la, grid, forest)
    batched = _rounds(a, la, la.LA_MODE_BATCHED, 3, adjoint=True)
    plain = _rounds(a, la, la.LA_MODE_PLAIN, 3, adjoint=True)
    for r, (p, q) in enumerate(zip(batched, plain)):
        for k in ("layer", "b", "t", "D", "H", "J"):
            assert np.array_equal(p[k], q[k]), (r, k)


def test_batched_deep_trees_against_oracle(la):
    """Config 4 shape (Zipf pin counts up to 4096: deep trees handled by the
    persistent block-per-net kernels) against the oracle, two rounds."""
    wl = fg.WORKLOADS[4].scaled(8000)
    grid, forest = fg.make_grid(wl, 9), fg.make_forest(wl, 9)
    assert np.diff(forest["net_ptr"]).max() > 500
    a = _assigner(la, grid, forest)
    D = H = None
    for r in range(2):
        st = a.assign_round(mode=la.LA_MODE_BATCHED, reset=(r == 0), **la.DEFAULT_WEIGHTS)
        got = dict(zip(("layer", "b", "t"), (x.cpu().numpy() for x in a.get_assignment())))
        got["D"], got["H"] = (x.cpu().numpy() for x in a.get_state())
        got["J"] = a.get_net_cost().cpu().numpy()
        got["stats"] = st
        ref = ref_round(grid, forest, la.DEFAULT_WEIGHTS, D=D, H=H)
        assert_same_round(got, ref, f"round {r}")
        D, H = got["D"], got["H"]


def test_batched_reload_reuses_tuning(la):
    """A reload of a forest with the same bucket layout takes the tuned plan
    untimed (no trials) and gives the same round; another forest re-tunes."""
    wl = fg.WORKLOADS[4].scaled(6000)
    grid, forest = fg.make_grid(wl, 3), fg.make_forest(wl, 3)
    a = _assigner(la, grid, forest)
    first = _rounds(a, la, la.LA_MODE_BATCHED, 2)
    assert first[0]["stats"]["batch_trials"] > 0
    assert [q["stats"]["batch_graph_captured"] for q in first] == [1, 0]
    a.load_nets(forest)
    again = _rounds(a, la, la.LA_MODE_BATCHED, 2)
    assert again[0]["stats"]["batch_trials"] == 0
    assert again[0]["stats"]["batch_split"] == first[0]["stats"]["batch_split"]
    # the reloaded forest's arrays sit at the same addresses: the graph replays
    assert [q["stats"]["batch_graph_captured"] for q in again] == [0, 0]
    for p, q in zip(first, again):
        for k in ("layer", "b", "t", "D", "H", "J"):
            assert np.array_equal(p[k], q[k]), k
    # same trees, other caps and criticalities: the memo matches, the captured
    # rounds replay on the new values, and they still equal the plain form
    vals = dict(forest)
    vals["kappa"] = forest["kappa"] * 0.5
    vals["sink_cap"] = forest["sink_cap"] * 1.5
    a.load_nets(vals)
    rb = _rounds(a, la, la.LA_MODE_BATCHED, 2, adjoint=True)
    assert rb[0]["stats"]["batch_trials"] == 0
    assert rb[0]["stats"]["batch_graph_captured"] == 0
    rp = _rounds(a, la, la.LA_MODE_PLAIN, 2, adjoint=True)
    for p, q in zip(rb, rp):
        for k in ("layer", "b", "t", "D", "H", "J"):
            assert np.array_equal(p[k], q[k]), k
    assert not np.array_equal(rb[0]["J"], first[0]["J"])
    other = fg.make_forest(wl, 4)
    a.load_nets(other)
    st = a.assign_round(mode=la.LA_MODE_BATCHED, reset=True, **la.DEFAULT_WEIGHTS)
    assert st["batch_trials"] > 0
    got = dict(zip(("layer", "b", "t"), (x.cpu().numpy() for x in a.get_assignment())))
    a.assign_round(mode=la.LA_MODE_PLAIN, reset=True, **la.DEFAULT_WEIGHTS)
    for k, x in zip(("layer", "b", "t"), a.get_assignment()):
        assert np.array_equal(got[k], x.cpu().numpy()), k


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_without_look_ahead(la, mode):
    """The look-ahead ablation (r_est = 0, Table VII's "w/o ahead"): the oracle
    with rho = 0, for the Eq. 4 and the adjoint weight sources; the batched
    round's graph is re-captured when the switch changes and replayed after."""
    wl = fg.WORKLOADS[2].scaled(20000)
    grid, forest = fg.make_grid(wl, 11), fg.make_forest(wl, 11)
    a = _assigner(la, grid, forest)
    m = la.LA_MODE_PLAIN if mode == "plain" else la.LA_MODE_BATCHED
    zero = np.zeros(int(forest["num_nodes"]), np.float64)
    D = H = None
    got = None
    for r, (src, ahead) in enumerate([(0, False), (0, True), (0, False), (1, False), (1, False)]):
        if r == 3:
            a.reweight_adjoint()
        st = a.assign_round(mode=m, reset=(r == 0), weights=src, look_ahead=ahead, **la.DEFAULT_WEIGHTS)
        got = dict(zip(("layer", "b", "t"), (x.cpu().numpy() for x in a.get_assignment())))
        got["D"], got["H"] = (x.cpu().numpy() for x in a.get_state())
        got["J"] = a.get_net_cost().cpu().numpy()
        got["stats"] = st
        W, rho = (x.cpu().numpy() for x in a.get_weights(src))
        ref = ref_round(grid, forest, la.DEFAULT_WEIGHTS, D=D, H=H, W=W, rho=rho if ahead else zero)
        assert_same_round(got, ref, f"{mode} round {r} src {src} ahead {ahead}")
        D, H = got["D"], got["H"]


def test_nangate45_stack_against_oracle(la):
    """The Table I stack (10 layers, per-layer via R) on a scaled forest: two
    rounds against the oracle, plain and batched."""
    wl = fg.WORKLOADS[6].scaled(20000)
    grid, forest = fg.make_grid(wl, 12), fg.make_forest(wl, 12)
    a = _assigner(la, grid, forest)
    for mode in (la.LA_MODE_PLAIN, la.LA_MODE_BATCHED):
        D = H = None
        for r in range(2):
            st = a.assign_round(mode=mode, reset=(r == 0), **la.DEFAULT_WEIGHTS)
            got = dict(zip(("layer", "b", "t"), (x.cpu().numpy() for x in a.get_assignment())))
            got["D"], got["H"] = (x.cpu().numpy() for x in a.get_state())
            got["J"] = a.get_net_cost().cpu().numpy()
            got["stats"] = st
            ref = ref_round(grid, forest, la.DEFAULT_WEIGHTS, D=D, H=H)
            assert_same_round(got, ref, f"mode {mode} round {r}")
            D, H = got["D"], got["H"]


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_sequential_batches_against_oracle(la, mode):
    """Sequential batches (Sec. III-A): batch k sees the demand of batches < k
    with their new layers and every other net with its previous ones.  Two
    rounds against the oracle, plain and batched (level waves with the
    constant caches in one CUDA graph), batches from the GPU's Alg. 1
    partition of the nets' criticality, which must equal the oracle's; the
    Elmore passes walk every batch's levels."""
    wl = fg.WORKLOADS[2].scaled(12000)
    grid, forest = fg.make_grid(wl, 13), fg.make_forest(wl, 13)
    N = int(forest["num_nets"])
    net_of = np.repeat(np.arange(N), np.diff(forest["net_ptr"]))
    crit = np.zeros(N)
    np.maximum.at(crit, net_of, forest["kappa"])
    bt, nb = la.la_partition_batches(torch.from_numpy(crit).cuda(), critical_frac=0.6)
    batch = bt.cpu().numpy()
    ref_b, ref_nb = oracle.partition_batches(crit, None, critical_frac=0.6)
    assert np.array_equal(batch, ref_b) and nb == ref_nb >= 3
    m = la.LA_MODE_PLAIN if mode == "plain" else la.LA_MODE_BATCHED
    fb = dict(forest, batch=batch)
    a = _assigner(la, grid, fb)
    D = H = prev = None
    for r in range(2):
        st = a.assign_round(mode=m, reset=(r == 0), **la.DEFAULT_WEIGHTS)
        got = _read_round(a, st)
        ref = oracle.assign_round_batches(grid, forest, batch, la.DEFAULT_WEIGHTS, D=D, H=H, layer_prev=prev)
        assert_same_round(got, ref, f"{mode} round {r}")
        D, H, prev = got["D"], got["H"], got["layer"]
    if mode == "batched":
        assert st["batch_graph_captured"] == 0  # the second round replayed the first one's graph
        with pytest.raises(la.LaError) as e:
            a.assign_round(mode=m, local_demand=True, **la.DEFAULT_WEIGHTS)
        assert e.value.status == la.LA_ERR_INVALID
    R, C = a.rc_from_assignment()
    d = a.elmore(R, C).cpu().numpy()
    ref_d = oracle.elmore(grid, forest, prev, got["b"], got["t"], R.cpu().numpy(), C.cpu().numpy())
    assert np.allclose(d, ref_d, rtol=1e-10, atol=0.0)
    a.close()


def _chains(n, depth, X, Y, seed):
    """n zig-zag chains of `depth` nodes (deep trees with one node per level)."""
    from util_inputs import forest_from_rows
    rng = np.random.default_rng(seed)
    nets = []
    for i in range(n):
        x, y = int(rng.integers(0, X - depth // 2 - 2)), int(rng.integers(0, Y - depth // 2 - 2))
        rows = [(-1, x, y, 0, 0.0, 0.0)]
        for j in range(1, depth):
            if j % 2:
                x += 1
            else:
                y += 1
            pin = 0 if j % 7 == 0 or j == depth - 1 else -1
            rows.append((j - 1, x, y, pin, 1.0 if pin >= 0 else 0.0, float(rng.uniform(0.1, 1.0)) if pin >= 0 else 0.0))
        nets.append(forest_from_rows(rows, r_drv=100.0 + i))
    return nets


def test_batched_tail_kernels_equal_plain(la):
    """Deep trees (chains of 800 levels beside a Zipf forest): the top
    small-net levels in the one-block tail kernels (tail_threshold), with the
    tuner's own plan, and the plain form give the same rounds bit for bit."""
    wl = fg.WORKLOADS[4].scaled(4000)
    grid = fg.make_grid(wl, 21)
    forest = merge_forests([fg.make_forest(wl, 21)] + _chains(100, 800, wl.X, wl.Y, 21))
    a = _assigner(la, grid, forest)
    tail = _rounds(a, la, la.LA_MODE_BATCHED, 3, adjoint=True, tail_threshold=32768)
    for q in tail:
        assert q["stats"]["batch_tail_level"] < q["stats"]["batch_levels"], q["stats"]
    tuned = _rounds(a, la, la.LA_MODE_BATCHED, 3, adjoint=True)
    plain = _rounds(a, la, la.LA_MODE_PLAIN, 3, adjoint=True)
    for r, (p, q, u) in enumerate(zip(tail, plain, tuned)):
        for k in ("layer", "b", "t", "D", "H", "J"):
            assert np.array_equal(p[k], q[k]), (r, k)
            assert np.array_equal(u[k], q[k]), (r, k)
    with pytest.raises(RuntimeError, match="tail_threshold"):
        a.assign_round(mode=la.LA_MODE_BATCHED, reset=True, tail_threshold=-1, **la.DEFAULT_WEIGHTS)


def test_elmore_of_the_assignment(la):
    """la_elmore_assignment (R, C from the layers inside the passes, output in
    input order) equals la_elmore of la_rc_from_assignment bit for bit."""
    wl = fg.WORKLOADS[2].scaled(20000)
    grid, forest = fg.make_grid(wl, 14), fg.make_forest(wl, 14)
    a = _assigner(la, grid, forest)
    a.assign_round(reset=True, **la.DEFAULT_WEIGHTS)
    R, C = a.rc_from_assignment()
    ref = a.elmore(R, C).cpu().numpy()
    got = a.elmore_assignment().cpu().numpy()
    assert np.array_equal(got, ref)


# ---------------------------------------------------------------------------
# The headline shapes against the oracle, round by round, with the batched
# form's own tuned plan; forced splits through the persistent big-net kernels
# ---------------------------------------------------------------------------
def _read_round(a, st):
    got = dict(zip(("layer", "b", "t"), (x.cpu().numpy() for x in a.get_assignment())))
    got["D"], got["H"] = (x.cpu().numpy() for x in a.get_state())
    got["J"] = a.get_net_cost().cpu().numpy()
    got["stats"] = st
    return got


def _rounds_against_oracle(la, a, grid, forest, mode, rounds, label, force_split=0):
    """Round 0 with the Eq. 4 weights from D = H = 0, then rounds reweighted by
    the adjoint of the previous assignment; each round's oracle starts from
    the GPU's previous state (D, H) and the oracle's own adjoint weights of
    the GPU's previous assignment, which must equal the GPU's bit for bit."""
    D = H = W = rho = None
    out = []
    for r in range(rounds):
        src = la.LA_WEIGHTS_EQ4 if r == 0 else la.LA_WEIGHTS_ADJOINT
        st = a.assign_round(mode=mode, reset=(r == 0), weights=src, force_split=force_split, **la.DEFAULT_WEIGHTS)
        got = _read_round(a, st)
        ref = ref_round(grid, forest, la.DEFAULT_WEIGHTS, D=D, H=H, W=W, rho=rho)
        assert_same_round(got, ref, f"{label} round {r}")
        out.append(got)
        D, H = got["D"], got["H"]
        a.reweight_adjoint()
        W, rho = oracle.adjoint_weights(grid, forest, got["layer"], got["b"], got["t"])
        Wg, rhog = (x.cpu().numpy() for x in a.get_weights(la.LA_WEIGHTS_ADJOINT))
        assert np.array_equal(Wg, W) and np.array_equal(rhog, rho), f"{label} adjoint weights after round {r}"
    return out


def test_headline_grid_and_stack_against_oracle(la):
    """The full-scale workload's own grid and layer stack (2048 x 2048, 12
    layers with r_l = 8 x 10^(-l/11), capacities U{8..20} with 10% halved) and
    its net distribution, 1M nets, batched with the tuner's plan: an Eq. 4
    round and an adjoint-reweighted round, bit for bit against the oracle."""
    wl = fg.WORKLOADS[5].scaled(1_000_000)
    grid, forest = fg.make_grid(wl, 0), fg.make_forest(wl, 0)
    a = _assigner(la, grid, forest)
    out = _rounds_against_oracle(la, a, grid, forest, la.LA_MODE_BATCHED, 2, "2048x2048x12 1M")
    st = out[0]["stats"]
    assert st["batch_trials"] > 0 and st["batch_levels"] > 20
    a.close()


def test_uneven_sizes_against_oracle(la):
    """The uneven-batching workload (1024 x 1024 x 10, Zipf(1.6) pin counts on
    [2, 4096]) at 200k nets, batched with the tuner's plan: an Eq. 4 round and
    an adjoint-reweighted round against the oracle."""
    wl = fg.WORKLOADS[4].scaled(200_000)
    grid, forest = fg.make_grid(wl, 0), fg.make_forest(wl, 0)
    assert np.diff(forest["net_ptr"]).max() > 2000
    a = _assigner(la, grid, forest)
    _rounds_against_oracle(la, a, grid, forest, la.LA_MODE_BATCHED, 2, "zipf 200k")
    a.close()


@pytest.mark.parametrize("cfg,nets,split", [(4, 20000, 4), (4, 20000, 7), (5, 100000, 4), (5, 100000, 5)])
def test_forced_split_runs_the_persistent_kernels(la, cfg, nets, split):
    """force_split sends every net of more than 2^split nodes through the
    persistent block-per-net kernels (work queue, a block per net walking its
    levels): three adjoint rounds against the oracle, and equal to the plain
    form bit for bit."""
    wl = fg.WORKLOADS[cfg].scaled(nets)
    grid, forest = fg.make_grid(wl, 17), fg.make_forest(wl, 17)
    sizes = np.diff(forest["net_ptr"])
    a = _assigner(la, grid, forest)
    out = _rounds_against_oracle(la, a, grid, forest, la.LA_MODE_BATCHED, 3, f"cfg {cfg} split {split}",
                                 force_split=split)
    for q in out:
        assert q["stats"]["batch_split"] == split
        assert q["stats"]["batch_big_nets"] == int(np.sum(sizes > 2 ** split)) > 0
    plain = _rounds(a, la, la.LA_MODE_PLAIN, 3, adjoint=True)
    for r, (p, q) in enumerate(zip(plain, out)):
        for k in ("layer", "b", "t", "D", "H", "J"):
            assert np.array_equal(p[k], q[k]), (r, k)
    # back to the tuner's split on the same context
    st = a.assign_round(mode=la.LA_MODE_BATCHED, reset=True, **la.DEFAULT_WEIGHTS)
    assert st["batch_split"] == out[0]["stats"]["batch_split"] or st["batch_split"] != split
    with pytest.raises(la.LaError) as e:
        a.assign_round(mode=la.LA_MODE_BATCHED, force_split=3, **la.DEFAULT_WEIGHTS)
    assert e.value.status == la.LA_ERR_INVALID
    a.close()


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_exact_ties_follow_the_documented_rules(la, mode):
    """The exact-tie nets of the oracle's tie pins: the GPU takes the same
    documented choice (lowest tied son layer; fewest vias, then lowest bottom)."""
    from util_inputs import TIE_WEIGHTS, son_tie_case, stack_tie_case

    m = la.LA_MODE_PLAIN if mode == "plain" else la.LA_MODE_BATCHED
    for grid, forest, layers, stacks in (son_tie_case(), stack_tie_case()):
        a = _assigner(la, grid, forest)
        st = a.assign_round(mode=m, reset=True, **TIE_WEIGHTS)
        got = _read_round(a, st)
        ref = ref_round(grid, forest, TIE_WEIGHTS)
        assert_same_round(got, ref, mode)
        assert list(got["layer"]) == layers
        assert list(zip(got["b"], got["t"])) == stacks
        a.close()


# ---------------------------------------------------------------------------
# Failure paths: host-side fault injection (nothing faults on the GPU), input
# checks of la_set_assignment, and a clean device error word after rounds
# ---------------------------------------------------------------------------
def _small(la, seed=1):
    wl = fg.WORKLOADS[1].scaled(200)
    grid, forest = fg.make_grid(wl, seed), fg.make_forest(wl, seed)
    return grid, forest, _assigner(la, grid, forest)


@pytest.mark.parametrize("code", ["LA_ERR_DEVICE_CHECK", "LA_ERR_CUDA", "LA_ERR_TIMEOUT"])
def test_injected_device_failure_poisons_the_context(la, code):
    grid, forest, a = _small(la)
    a.assign_round(reset=True, **la.DEFAULT_WEIGHTS)
    la.la_check(a.ctx)  # clean after a normal round
    la.la_inject_fault(a.ctx, getattr(la, code))
    with pytest.raises(la.LaError) as e:
        a.assign_round(**la.DEFAULT_WEIGHTS)
    assert e.value.status == getattr(la, code)
    # poisoned: every later call but la_destroy / la_last_error is LA_ERR_STATE
    for call in (lambda: a.assign_round(**la.DEFAULT_WEIGHTS), lambda: la.la_check(a.ctx), a.get_assignment,
                 lambda: a.load_nets(forest), a.rc_from_assignment):
        with pytest.raises(la.LaError) as e2:
            call()
        assert e2.value.status == la.LA_ERR_STATE
    a.close()
    # a new context on the same device works and matches the oracle
    b = _assigner(la, grid, forest)
    got = gpu_round(b, la.DEFAULT_WEIGHTS, reset=True)
    assert_same_round(got, ref_round(grid, forest, la.DEFAULT_WEIGHTS))
    b.close()


def test_injected_allocation_failure_keeps_the_loaded_forest(la):
    """LA_ERR_OOM before the new forest has passed validation: the forest loaded
    before stays loaded and the context is not poisoned."""
    grid, forest, a = _small(la)
    first = gpu_round(a, la.DEFAULT_WEIGHTS, reset=True)
    other = fg.make_forest(fg.WORKLOADS[1].scaled(300), 2)
    la.la_inject_fault(a.ctx, la.LA_ERR_OOM)
    with pytest.raises(la.LaError) as e:
        a.load_nets(other)
    assert e.value.status == la.LA_ERR_OOM and "injected" in str(e.value)
    again = gpu_round(a, la.DEFAULT_WEIGHTS, reset=True)
    for k in ("layer", "b", "t", "D", "H", "J"):
        assert np.array_equal(first[k], again[k]), k
    a.load_nets(other)  # and the next load works
    got = gpu_round(a, la.DEFAULT_WEIGHTS, reset=True)
    assert_same_round(got, ref_round(grid, other, la.DEFAULT_WEIGHTS))
    la.la_inject_fault(a.ctx, la.LA_ERR_OOM)
    la.la_inject_fault(a.ctx, la.LA_OK)  # cleared: the next load allocates normally
    a.load_nets(forest)
    with pytest.raises(la.LaError) as e:
        la.la_inject_fault(a.ctx, la.LA_ERR_STATE)
    assert e.value.status == la.LA_ERR_INVALID
    a.close()


def test_set_assignment_checks_its_input(la):
    """la_set_assignment rejects a layer of the wrong direction, a stack that
    does not hold a son's layer, and a stack that does not hold the pin, with
    LA_ERR_INVALID naming the node; the assignment in place is unchanged and
    the context stays usable."""
    grid, forest, a = _small(la)
    a.assign_round(reset=True, **la.DEFAULT_WEIGHTS)
    layer, b, t = (x.clone() for x in a.get_assignment())
    lay_np, b_np, t_np = layer.cpu().numpy(), b.cpu().numpy(), t.cpu().numpy()
    par, ptr, pin = forest["parent"], forest["net_ptr"], forest["pin_layer"]
    net_of = np.repeat(np.arange(int(forest["num_nets"])), np.diff(ptr))
    gpar = np.where(par < 0, -1, ptr[net_of] + par)
    # a non-root node whose layer is moved to the other direction
    v = int(np.flatnonzero(gpar >= 0)[0])
    bad = lay_np.copy()
    bad[v] = lay_np[v] + 1 if lay_np[v] + 1 < grid["L"] else lay_np[v] - 1
    # a parent whose stack top is lowered below a son's layer (still holding
    # the parent's own layer and pin)
    u = next(int(x) for x in np.flatnonzero(gpar >= 0)
             if lay_np[x] > lay_np[gpar[x]] and pin[gpar[x]] < lay_np[x])
    p = int(gpar[u])
    bb, tt = b_np.copy(), t_np.copy()
    tt[p] = lay_np[u] - 1
    # a pin node whose stack no longer holds its pin layer
    w = next(int(x) for x in np.flatnonzero((pin >= 0) & (gpar >= 0)) if pin[x] != lay_np[x])
    b2, t2 = b_np.copy(), t_np.copy()
    if pin[w] < lay_np[w]:
        b2[w] = pin[w] + 1
    else:
        t2[w] = pin[w] - 1
    dev = layer.device
    for lay_, b_, t_ in ((bad, b_np, t_np), (lay_np, bb, tt), (lay_np, b2, t2)):
        with pytest.raises(la.LaError) as e:
            a.set_assignment(*(torch.from_numpy(x).to(dev) for x in (lay_, b_, t_)))
        assert e.value.status == la.LA_ERR_INVALID and "node" in str(e.value)
    now = [x.cpu().numpy() for x in a.get_assignment()]
    for x, y in zip(now, (lay_np, b_np, t_np)):
        assert np.array_equal(x, y)
    a.set_assignment(layer, b, t)
    la.la_check(a.ctx)
    a.close()


def test_elmore_small_and_large_nets(la):
    """The Elmore passes on the uneven workload (Zipf pin counts: nets from 2
    to thousands of nodes, so both the per-net kernel of small nets and the
    block-per-net kernel of large ones run): delays, gradients and the
    adjoint weights against the oracle, and la_elmore_assignment equal to
    la_elmore of la_rc_from_assignment bit for bit."""
    wl = fg.WORKLOADS[4].scaled(20000)
    grid, forest = fg.make_grid(wl, 23), fg.make_forest(wl, 23)
    sizes = np.diff(forest["net_ptr"])
    assert (sizes <= 32).sum() > 1000 and (sizes > 32).sum() > 100 and sizes.max() > 2000
    a = _assigner(la, grid, forest)
    a.assign_round(reset=True, **la.DEFAULT_WEIGHTS)
    layer, b, t = (x.cpu().numpy() for x in a.get_assignment())
    R, C = a.rc_from_assignment()
    Rn, Cn = R.cpu().numpy(), C.cpu().numpy()
    d = a.elmore(R, C)
    assert torch.equal(a.elmore_assignment(), d)
    np.testing.assert_allclose(d.cpu().numpy(), oracle.elmore(grid, forest, layer, b, t, Rn, Cn), rtol=1e-10, atol=0)
    rng = np.random.default_rng(5)
    g = rng.uniform(0.0, 1.0, len(Rn))
    dR, dC = a.elmore_backward(R, C, torch.from_numpy(g).cuda())
    dR_ref, dC_ref, _, _ = oracle.elmore_backward(grid, forest, layer, b, t, Rn, Cn, g)
    np.testing.assert_allclose(dR.cpu().numpy(), dR_ref, rtol=1e-10, atol=0)
    np.testing.assert_allclose(dC.cpu().numpy(), dC_ref, rtol=1e-10, atol=0)
    for _ in range(2):  # the first reweighting sums W, the second reuses it
        a.reweight_adjoint()
        W, rho = (x.cpu().numpy() for x in a.get_weights(la.LA_WEIGHTS_ADJOINT))
        Wr, rhor = oracle.adjoint_weights(grid, forest, layer, b, t)
        assert np.array_equal(W, Wr) and np.array_equal(rho, rhor)
    a.close()


# ---------------------------------------------------------------------------
# Net ordering and pin weights (Sec. III-A, Sec. III-C)
# ---------------------------------------------------------------------------
def test_logistic_pin_weight_against_oracle(la):
    """The GPU's logistic pin weights equal the oracle's within a few units in
    the last place (the two sides' exp() may round differently), exactly 1/2
    at slack / WNS = b, and 0 off the pins."""
    rng = np.random.default_rng(3)
    V = 300_000
    pin = np.where(rng.uniform(size=V) < 0.4, 0, -1).astype(np.int8)
    slack = rng.uniform(-200.0, 60.0, V)
    slack[:3] = [-60.0, -200.0, 0.0]  # x = b (WNS = -200), the worst slack, zero slack
    pin[:3] = 0
    wns = float(slack.min())
    got = la.la_logistic_pin_weight(torch.from_numpy(pin).cuda(), torch.from_numpy(slack).cuda(), wns).cpu().numpy()
    ref = oracle.logistic_pin_weight(pin, slack, wns)
    np.testing.assert_allclose(got, ref, rtol=4 * 2.0 ** -52, atol=0)
    assert got[0] == 0.5 and got[1] > 0.999 and np.all(got[pin < 0] == 0.0)
    with pytest.raises(la.LaError):
        la.la_logistic_pin_weight(torch.from_numpy(pin).cuda(), torch.from_numpy(slack).cuda(), 1.0)


def test_partition_against_oracle(la):
    """Alg. 1's partition on the GPU equals the oracle's net by net: random
    criticalities and slacks at several ratios, the interval-edge nets of the
    oracle's pin, and no slack at all; bad inputs are refused."""
    rng = np.random.default_rng(8)
    N = 500_000
    crit = rng.uniform(0, 10, N) ** 3
    slack = rng.uniform(-80, 30, N)
    for frac, ratio, sl in ((0.5, 0.7, slack), (0.05, 0.9, slack), (0.3, 0.7, None), (1.0, 1.0, slack)):
        g, nb = la.la_partition_batches(torch.from_numpy(crit).cuda(),
                                        None if sl is None else torch.from_numpy(sl).cuda(), frac, ratio)
        r, rnb = oracle.partition_batches(crit, sl, frac, ratio)
        assert np.array_equal(g.cpu().numpy(), r) and nb == rnb, (frac, ratio)
    ce = np.array([8, 4, 6, 2, 3.9999, 0.5, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0])
    se = np.array([-1, -1, -1, -1, -1, -100, -99, -99.5, -98.9, -96, -71, -69, 0.0, -100.0])
    g, nb = la.la_partition_batches(torch.from_numpy(ce).cuda(), torch.from_numpy(se).cuda(), 0.25, 0.7)
    r, rnb = oracle.partition_batches(ce, se, 0.25, 0.7)
    assert np.array_equal(g.cpu().numpy(), r) and nb == rnb == 8
    bad = crit.copy()
    bad[7] = -1.0
    with pytest.raises(la.LaError) as e:
        la.la_partition_batches(torch.from_numpy(bad).cuda())
    assert e.value.status == la.LA_ERR_INVALID


def test_slack_driven_ordering_end_to_end(la):
    """The paper's ordering on synthetic timing: per-pin slack from the
    Elmore delays of a first round against a required time, the logistic pin
    weights as the sinks' criticality (so Eq. 4 takes their maximum below
    each node), the nets partitioned by their largest weight and their worst
    slack, and two rounds in those sequential batches, batched, against the
    oracle given the same weights and batches."""
    wl = fg.WORKLOADS[2].scaled(20000)
    grid, forest = fg.make_grid(wl, 31), fg.make_forest(wl, 31)
    a = _assigner(la, grid, forest)
    a.assign_round(reset=True, **la.DEFAULT_WEIGHTS)
    delay = a.elmore_assignment().cpu().numpy()
    pin = forest["pin_layer"]
    sinks = pin >= 0
    req = np.quantile(delay[sinks], 0.8)
    slack = np.where(sinks, req - delay, 0.0)
    wns = float(slack[sinks].min())
    w = la.la_logistic_pin_weight(torch.from_numpy(pin).cuda(), torch.from_numpy(slack).cuda(), wns).cpu().numpy()
    N = int(forest["num_nets"])
    net_of = np.repeat(np.arange(N), np.diff(forest["net_ptr"]))
    crit = np.zeros(N)
    np.maximum.at(crit, net_of, w)
    nslack = np.full(N, np.inf)
    np.minimum.at(nslack, net_of[sinks], slack[sinks])
    nslack[~np.isfinite(nslack)] = 0.0
    bt, nb = la.la_partition_batches(torch.from_numpy(crit).cuda(), torch.from_numpy(nslack).cuda(), 0.9, 0.7)
    batch = bt.cpu().numpy()
    assert nb >= 3 and np.array_equal(batch, oracle.partition_batches(crit, nslack, 0.9, 0.7)[0])
    f2 = dict(forest, kappa=w, batch=batch)
    b = _assigner(la, grid, f2)
    ref_in = dict(forest, kappa=w)
    D = H = prev = None
    for r in range(2):
        st = b.assign_round(mode=la.LA_MODE_BATCHED, reset=(r == 0), **la.DEFAULT_WEIGHTS)
        got = _read_round(b, st)
        ref = oracle.assign_round_batches(grid, ref_in, batch, la.DEFAULT_WEIGHTS, D=D, H=H, layer_prev=prev)
        assert_same_round(got, ref, f"round {r}")
        D, H, prev = got["D"], got["H"], got["layer"]
    a.close()
    b.close()


def _adjoint_rounds(la, grid, forest, mode, fused, rounds=3, **kw):
    """Rounds with adjoint weights after the first; the weights come from the
    round itself (fused) or from la_reweight_adjoint after it."""
    a = _assigner(la, grid, forest)
    out = []
    for r in range(rounds):
        src = la.LA_WEIGHTS_ADJOINT if r > 0 else la.LA_WEIGHTS_EQ4
        st = a.assign_round(mode=mode, reset=(r == 0), weights=src, reweight_adjoint=fused, **kw,
                            **la.DEFAULT_WEIGHTS)
        if not fused:
            a.reweight_adjoint()
        W, rho = (x.cpu().numpy() for x in a.get_weights(la.LA_WEIGHTS_ADJOINT))
        got = dict(layer=a.get_assignment()[0].cpu().numpy(), J=a.get_net_cost().cpu().numpy(), W=W, rho=rho,
                   stats=st)
        out.append(got)
    a.close()
    return out


@pytest.mark.parametrize("case", ["plain", "batched", "batched_big_nets", "batched_tail", "plain_batches",
                                  "batched_batches"])
def test_reweighting_fused_into_the_backtrack(la, case):
    """reweight_adjoint = 1 leaves the same W and r_est, bit for bit, as
    la_reweight_adjoint after the round (the top-down pass done by every
    backtrack kernel: level waves, the tail kernel, the persistent big-net
    kernel, sequential batches), so the rounds that follow are the same too."""
    cfg, nets, kw = {"plain": (2, 20000, {}), "batched": (5, 100000, {}),
                     "batched_big_nets": (4, 20000, dict(force_split=4)),
                     "batched_tail": (2, 20000, dict(tail_threshold=8192)),
                     "plain_batches": (2, 12000, {}), "batched_batches": (2, 12000, {})}[case]
    wl = fg.WORKLOADS[cfg].scaled(nets)
    grid, forest = fg.make_grid(wl, 23), fg.make_forest(wl, 23)
    if case.endswith("batches"):
        N = int(forest["num_nets"])
        forest = dict(forest, batch=(np.arange(N) % 3).astype(np.int32))
    mode = la.LA_MODE_PLAIN if case.startswith("plain") else la.LA_MODE_BATCHED
    sep = _adjoint_rounds(la, grid, forest, mode, False, **kw)
    fus = _adjoint_rounds(la, grid, forest, mode, True, **kw)
    for r, (p, q) in enumerate(zip(sep, fus)):
        for k in ("W", "rho", "layer", "J"):
            assert np.array_equal(p[k], q[k]), (case, r, k)
    if case == "batched_big_nets":
        assert fus[0]["stats"]["batch_big_nets"] > 0
    if case == "batched_tail":
        assert fus[0]["stats"]["batch_tail_level"] < fus[0]["stats"]["batch_levels"]
    a = _assigner(la, grid, forest)
    with pytest.raises(la.LaError) as e:
        a.assign_round(mode=mode, reset=True, reweight_adjoint=2, **la.DEFAULT_WEIGHTS)
    assert e.value.status == la.LA_ERR_INVALID
    a.close()
