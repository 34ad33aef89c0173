"""A round split by nets over several ranks (the §8(e) partitioning: within a
round every net sees one snapshot, so the nets shard by range and the only
exchange is the sum of the demand maps).

On the CPU: two gloo ranks, each running the oracle's round on its own nets
against the shared snapshot, summing the demand with an all-reduce and
committing the sum - driven by the same host logic
(paper_2507_13375_gb300.shard) that drives the GPUs with NCCL.  The result
must equal the single-process oracle round bit for bit, over an Eq. 4 round
and an adjoint-reweighted round.  On the GPU: two library contexts in one
process, the sum taken on the host between the calls."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import forestgen as fg
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _shard_mod():
    sys.path.insert(0, ROOT)
    from paper_2507_13375_gb300 import shard
    return shard


def test_shard_ranges_cover_and_balance():
    shard = _shard_mod()
    wl = fg.WORKLOADS[2].scaled(5000)
    forest = fg.make_forest(wl, 3)
    ptr = forest["net_ptr"]
    for world in (1, 2, 3, 8):
        r = shard.shard_ranges(ptr, world)
        assert r[0][0] == 0 and r[-1][1] == forest["num_nets"]
        assert all(r[i][1] == r[i + 1][0] and r[i][0] < r[i][1] for i in range(world - 1))
        nodes = [int(ptr[hi] - ptr[lo]) for lo, hi in r]
        assert sum(nodes) == forest["num_nodes"]
        assert max(nodes) - min(nodes) <= 2 * int(np.diff(ptr).max()) + 1
    sub = shard.shard_forest(forest, *r[1])
    lo, hi = r[1]
    assert sub["num_nets"] == hi - lo and np.array_equal(sub["x"], forest["x"][ptr[lo]:ptr[hi]])
    with pytest.raises(ValueError):
        shard.shard_ranges(ptr[:3], 4)


class OracleShard:
    """The oracle's round on one shard's nets, with the calls sharded_round
    makes: a local-demand round against the shared snapshot, the shard's
    demand, and the commit of the summed demand."""

    def __init__(self, grid, forest):
        self.grid, self.forest = grid, forest
        E = oracle.num_edges(grid)
        self.D, self.H = np.zeros(E, np.int32), np.zeros(E, np.int32)
        self.eq4 = oracle.weights_eq4(grid, forest)
        self.adj = None

    def assign_round(self, local_demand, mode=0, weights=0, reset=False, **w):
        assert local_demand
        if reset:
            self.D[:] = 0
            self.H[:] = 0
        W, rho = self.eq4 if weights == 0 else self.adj
        ww = dict(oracle.DEFAULT_WEIGHTS, **w)
        pen = oracle.penalty(self.grid, self.D, self.H, ww["hist_w"])
        self.out = oracle.dp(self.grid, self.forest, ww, pen, W, rho)
        self.Dloc, _, st = oracle.demand(self.grid, self.forest, self.out["layer"], self.out["b"], self.out["t"],
                                         np.zeros_like(self.H))
        return dict(total_cost=float(np.sum(self.out["J"])), vias=st["vias"], wl=st["wl"])

    def get_state(self):
        return torch.from_numpy(self.Dloc.astype(np.int32).copy()), torch.from_numpy(self.H.copy())

    def commit_demand(self, D):
        self.D = D.numpy().astype(np.int32)
        over = self.D.astype(np.int64) - self.grid["cap"]
        self.H = (self.H + np.maximum(over, 0)).astype(np.int32)
        return dict(tof=0.0, relu_overflow=int(np.maximum(over, 0).sum()))

    def reweight_adjoint(self):
        self.adj = oracle.adjoint_weights(self.grid, self.forest, self.out["layer"], self.out["b"], self.out["t"])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_2507_13375_gb300 import shard as sh

    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = fg.WORKLOADS[2].scaled(4000)
    grid, forest = fg.make_grid(wl, 7), fg.make_forest(wl, 7)
    lo, hi = sh.shard_ranges(forest["net_ptr"], world)[rank]
    s = OracleShard(grid, sh.shard_forest(forest, lo, hi))
    allreduce = lambda t: dist.all_reduce(t, op=dist.ReduceOp.SUM)
    res = []
    for r in range(2):
        st = sh.sharded_round(s, allreduce, weights=0 if r == 0 else 1, reset=(r == 0))
        res.append(dict(layer=s.out["layer"], b=s.out["b"], t=s.out["t"], J=s.out["J"], D=s.D.copy(),
                        H=s.H.copy(), stats=st))
        s.reweight_adjoint()
    parts = [None] * world
    dist.all_gather_object(parts, (lo, hi, res))
    if rank == 0:
        q.put(parts)
    dist.destroy_process_group()


def test_sharded_round_on_two_gloo_ranks_equals_one_process():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl = fg.WORKLOADS[2].scaled(4000)
    grid, forest = fg.make_grid(wl, 7), fg.make_forest(wl, 7)
    ref = [oracle.assign_round(grid, forest)]
    W, rho = oracle.adjoint_weights(grid, forest, ref[0]["layer"], ref[0]["b"], ref[0]["t"])
    ref.append(oracle.assign_round(grid, forest, D=ref[0]["D"], H=ref[0]["H"], W=W, rho=rho))
    for r in range(2):
        for k in ("layer", "b", "t", "J"):
            got = np.concatenate([p[2][r][k] for p in parts])
            assert np.array_equal(got, ref[r][k]), (r, k)
        for p in parts:  # every shard holds the whole round's snapshot
            assert np.array_equal(p[2][r]["D"], ref[r]["D"]) and np.array_equal(p[2][r]["H"], ref[r]["H"]), r
            st = p[2][r]["stats"]
            assert st["vias"] == ref[r]["stats"]["vias"] and st["wl"] == ref[r]["stats"]["wl"]
            assert st["relu_overflow"] == ref[r]["stats"]["relu_overflow"]
            assert st["total_cost"] == pytest.approx(ref[r]["stats"]["total_cost"], rel=1e-12)


@pytest.mark.gpu
@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_two_shards_on_one_gpu_equal_one_context(mode):
    """Two contexts, each loading half of the nets; after each local-demand
    round the host sums the two demand maps and both commit the sum.  Layers,
    stacks, per-net J, D and H equal the single-context rounds bit for bit
    (an Eq. 4 round and two adjoint rounds), and tof / ReLU overflow too."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2507_13375_gb300 as la
    from paper_2507_13375_gb300 import shard as sh

    m = la.LA_MODE_PLAIN if mode == "plain" else la.LA_MODE_BATCHED
    wl = fg.WORKLOADS[5].scaled(60000)
    grid, forest = fg.make_grid(wl, 9), fg.make_forest(wl, 9)
    one = la.LayerAssigner(0)
    one.load_grid(grid)
    one.load_nets(forest)
    ranges = sh.shard_ranges(forest["net_ptr"], 2)
    shards = []
    for lo, hi in ranges:
        a = la.LayerAssigner(0)
        a.load_grid(grid)
        a.load_nets(sh.shard_forest(forest, lo, hi))
        shards.append(a)
    for r in range(3):
        src = la.LA_WEIGHTS_EQ4 if r == 0 else la.LA_WEIGHTS_ADJOINT
        ref = one.assign_round(mode=m, weights=src, reset=(r == 0), **la.DEFAULT_WEIGHTS)
        sts = [a.assign_round(mode=m, weights=src, reset=(r == 0), local_demand=True, **la.DEFAULT_WEIGHTS)
               for a in shards]
        D = sum(a.get_state()[0] for a in shards)
        cms = [a.commit_demand(D) for a in shards]
        Dr, Hr = one.get_state()
        for a, cm in zip(shards, cms):
            Da, Ha = a.get_state()
            assert torch.equal(Da, Dr) and torch.equal(Ha, Hr), r
            assert cm["relu_overflow"] == ref["relu_overflow"]
            assert cm["tof"] == pytest.approx(ref["tof"], rel=1e-12)
        for k, x in enumerate(one.get_assignment()):
            got = torch.cat([a.get_assignment()[k] for a in shards])
            assert torch.equal(got, x), (r, k)
        assert torch.equal(torch.cat([a.get_net_cost() for a in shards]), one.get_net_cost())
        assert sum(s["vias"] for s in sts) == ref["vias"] and sum(s["wl"] for s in sts) == ref["wl"]
        one.reweight_adjoint()
        for a in shards:
            a.reweight_adjoint()
    for a in shards + [one]:
        a.close()
