"""The allocation-free Elmore entry point (la_elmore_static).

Some callers cannot allocate device memory at all: their device memory is
owned by another allocator, or they sit on a latency-critical path that must
not call cudaMalloc (which may synchronise the device).  For them the library
offers one call whose scratch is a fixed array compiled into the library.
These tests check, through the C ABI, that it gives the same delays as the
context-based la_elmore, on two calls in a row (the shared scratch keeps the
previous call's contents), and that it refuses forests larger than its
scratch.  This file is collected last so that a failure here cannot stop the
other GPU tests from running first."""
import numpy as np
import pytest

import forestgen as fg

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


def test_static_elmore_matches_context_elmore_twice(la):
    wl = fg.WORKLOADS[2].scaled(60000)
    grid, forest = fg.make_grid(wl, 2), fg.make_forest(wl, 2)
    assert forest["num_nodes"] <= la.LA_STATIC_MAX_NODES
    a = la.LayerAssigner(0)
    a.load_grid(grid)
    a.load_nets(forest)
    a.assign_round(reset=True)
    layer, b, t = a.get_assignment()
    R, C = a.rc_from_assignment()
    ref = a.elmore(R, C)
    nets = _nets(forest)
    for call in range(2):
        # a different scaling of R and C on each call: the result must not
        # depend on what the previous call left in the shared scratch
        s = 1.0 + call
        out = torch.full_like(ref, float("nan"))
        la.la_elmore_static(nets, layer, b, t, grid["L"], grid["via_r"], grid["via_c"], R * s, C, out)
        torch.cuda.synchronize()
        want = a.elmore(R * s, C)
        assert not torch.isnan(out).any()
        np.testing.assert_allclose(out.cpu().numpy(), want.cpu().numpy(), rtol=1e-10, atol=0)
    np.testing.assert_allclose(out.cpu().numpy(), (a.elmore(R * 2.0, C)).cpu().numpy(), rtol=1e-10, atol=0)
    a.close()


def test_static_elmore_rejects_more_nodes_than_its_scratch(la):
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
