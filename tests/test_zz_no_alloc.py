"""The allocation-free Elmore entry point (la_elmore_static).

Some callers cannot allocate device memory at all: their device memory is
owned by another allocator, or they sit on a latency-critical path that must
not call cudaMalloc (which may synchronise the device).  For them the library
offers one call whose scratch is a fixed array compiled into the library.
These tests check, through the C ABI, that it gives the same delays as the
context-based la_elmore bit for bit, on two calls in a row (the shared scratch
keeps the previous call's contents), that a call after the first changes the
device's free memory by nothing, that malformed nets come back as NaN delays,
and that it refuses forests larger than its scratch.  This file is collected
last so that a failure here cannot stop the other GPU tests from running
first."""
import numpy as np
import pytest

import forestgen as fg
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def la():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2507_13375_gb300 as la

    la.library()
    return la


def _nets(forest):
    dev = torch.device("cuda", 0)
    return dict(net_ptr=torch.from_numpy(forest["net_ptr"]).to(dev),
                parent=torch.from_numpy(forest["parent"]).to(dev),
                pin_layer=torch.from_numpy(forest["pin_layer"]).to(dev),
                sink_cap=torch.from_numpy(forest["sink_cap"]).to(dev),
                r_drv=torch.from_numpy(forest["r_drv"]).to(dev))


def _setup(la, nets_count, seed):
    wl = fg.WORKLOADS[2].scaled(nets_count)
    grid, forest = fg.make_grid(wl, seed), fg.make_forest(wl, seed)
    assert forest["num_nodes"] <= la.LA_STATIC_MAX_NODES
    a = la.LayerAssigner(0)
    a.load_grid(grid)
    a.load_nets(forest)
    a.assign_round(reset=True)
    return grid, forest, a


def test_static_elmore_matches_context_elmore_twice(la):
    grid, forest, a = _setup(la, 60000, 2)
    layer, b, t = a.get_assignment()
    R, C = a.rc_from_assignment()
    nets = _nets(forest)
    # inputs and outputs of both calls exist before the calls: the second call
    # is measured for allocations
    Rs = [R * (1.0 + call) for call in range(2)]
    wants = [a.elmore(Rs[call], C) for call in range(2)]
    outs = [torch.full_like(R, float("nan")) for _ in range(2)]
    torch.cuda.synchronize()
    for call in range(2):
        # a different R on each call: the result must not depend on what the
        # previous call left in the shared scratch
        free0 = torch.cuda.mem_get_info()[0]
        la.la_elmore_static(nets, layer, b, t, grid["L"], grid["via_r"], grid["via_c"], Rs[call], C, outs[call])
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        if call == 1:
            assert free1 == free0, "the second call changed the device's free memory"
        assert torch.equal(outs[call], wants[call]), f"call {call}: differs from la_elmore"
    # and the oracle's FP64 delays, within the Elmore tolerance
    ref = oracle.elmore(grid, forest, layer.cpu().numpy(), b.cpu().numpy(), t.cpu().numpy(),
                        Rs[1].cpu().numpy(), C.cpu().numpy())
    np.testing.assert_allclose(outs[1].cpu().numpy(), ref, rtol=1e-10, atol=0)
    a.close()


def test_static_elmore_reports_malformed_nets_as_nan(la):
    grid, forest, a = _setup(la, 2000, 3)
    layer, b, t = a.get_assignment()
    R, C = a.rc_from_assignment()
    want = a.elmore(R, C).cpu().numpy()
    ptr = forest["net_ptr"]
    sizes = np.diff(ptr)
    n_bad = int(np.flatnonzero(sizes >= 3)[5])
    lo, hi = int(ptr[n_bad]), int(ptr[n_bad + 1])
    # one net with a parent id that is not below its own local id
    bad = dict(forest)
    bad["parent"] = forest["parent"].copy()
    bad["parent"][lo + 1] = 1
    out = torch.empty_like(R)
    la.la_elmore_static(_nets(bad), layer, b, t, grid["L"], grid["via_r"], grid["via_c"], R, C, out)
    got = out.cpu().numpy()
    assert np.isnan(got[lo:hi]).all()
    keep = np.ones(len(got), bool)
    keep[lo:hi] = False
    assert np.array_equal(got[keep], want[keep])
    # one net with a layer out of range
    lay2 = layer.clone()
    lay2[lo + 1] = int(grid["L"])
    la.la_elmore_static(_nets(forest), lay2, b, t, grid["L"], grid["via_r"], grid["via_c"], R, C, out)
    got = out.cpu().numpy()
    assert np.isnan(got[lo:hi]).all() and np.array_equal(got[keep], want[keep])
    # a net pointer that does not rise: every delay is NaN
    bad2 = dict(forest)
    bad2["net_ptr"] = ptr.copy()
    bad2["net_ptr"][7] = bad2["net_ptr"][9]
    la.la_elmore_static(_nets(bad2), layer, b, t, grid["L"], grid["via_r"], grid["via_c"], R, C, out)
    assert torch.isnan(out).all()
    # and a well-formed call afterwards is exact again
    la.la_elmore_static(_nets(forest), layer, b, t, grid["L"], grid["via_r"], grid["via_c"], R, C, out)
    assert np.array_equal(out.cpu().numpy(), want)
    a.close()


def test_static_elmore_rejects_bad_arguments(la):
    wl = fg.WORKLOADS[1].scaled(10)
    grid, forest = fg.make_grid(wl, 0), fg.make_forest(wl, 0)
    nets = _nets(forest)
    V = int(forest["num_nodes"])
    z8 = torch.zeros(V, dtype=torch.int8, device="cuda")
    zd = torch.zeros(V, dtype=torch.float64, device="cuda")
    with pytest.raises(la.LaError) as e:
        la.la_elmore_static(nets, z8, z8, z8, grid["L"], grid["via_r"], grid["via_c"], zd, zd, zd,
                            num_nodes=la.LA_STATIC_MAX_NODES + 1)
    assert e.value.status == la.LA_ERR_INVALID and "exceed" in str(e.value)
    # the binding's own checks: a short via_r, a wrong dtype, a short array
    for args in ((nets, z8, z8, z8, grid["L"], grid["via_r"][:1], grid["via_c"], zd, zd, zd),
                 (nets, z8.int(), z8, z8, grid["L"], grid["via_r"], grid["via_c"], zd, zd, zd),
                 (nets, z8, z8, z8, grid["L"], grid["via_r"], grid["via_c"], zd[:-1], zd, zd)):
        with pytest.raises(la.LaError) as e:
            la.la_elmore_static(*args)
        assert e.value.status == la.LA_ERR_INVALID
