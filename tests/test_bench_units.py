"""The bench's algorithmic DP flop count (the roofline's numerator) on a tree
counted by hand from the per-item costs its docstring lists."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _net(x0):
    # root (pin) at (x0, 0) -> bend (no pin) at (x0 + 5, 0) -> sink (pin) at (x0 + 5, 3)
    return dict(x=[x0, x0 + 5, x0 + 5], y=[0, 0, 3], parent=[-1, 0, 1], pin_layer=[0, -1, 0])


def _forest(nets):
    cat = {k: np.array(sum((n[k] for n in nets), []), dtype=np.int32 if k != "pin_layer" else np.int8)
           for k in ("x", "y", "parent", "pin_layer")}
    sizes = [len(n["x"]) for n in nets]
    cat["net_ptr"] = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    cat["num_nodes"], cat["num_nets"] = sum(sizes), len(nets)
    return cat


def test_dp_flops_by_hand():
    """Layers (H, V, H, V): two per direction.
      root: 1 candidate; one son on 2 layers, a pin:
            per layer 4 + 2 (son sum) + 4 (sink) + 2*2 (keys) + 2 (g) + 3 (f') = 19;
            per node 3 + 1 (pin) = 4                                 -> 23
      bend: 2 candidates (H); one son on 2 layers (V), no pin, not a root:
            per layer 4 + 2 + 4 + 2 + 3 + 9 (entry) = 24; per node 3 + 1 -> 52
      sink: 2 candidates (V); no son, a pin, not a root:
            per layer 4 + 4 + 2 + 9 = 19; per node 3 + 1 + 1 = 5     -> 43
    118 per net; a second net checks the per-net parent offsets."""
    dirs = (0, 1, 0, 1)
    assert bench.dp_algorithmic_flops(_forest([_net(0)]), dirs) == 118.0
    assert bench.dp_algorithmic_flops(_forest([_net(0), _net(20)]), dirs) == 236.0


def test_roofline_byte_rules():
    """The DP's compulsory bytes per segment, S (20 + 50 L_d) + 10 S: 320 B per
    segment at 12 layers (L_d = 6) and 270 B at 10, plus 10 B of backtrack; the
    Elmore passes 40 B (forward) and 48 B (adjoint) per RC node, two per
    segment."""
    assert bench.dp_method_bytes(1, 6.0) == 330.0
    assert bench.dp_method_bytes(1000, 5.0) == 280_000.0
    e = bench.elmore_method_bytes(10)
    assert e == {"rc_nodes": 20, "forward": 800.0, "adjoint": 960.0}
    # the batched form's own count (its constant caches included) is larger
    assert bench.dp_cache_bytes(V=7, S=6, N=1, LD=6) > bench.dp_method_bytes(6, 6.0)


def test_node_class_counts():
    """The DP's node classes of the hand-made net: the root (a pin, one son)
    is class 4, the bend (no pin, one son) class 7, the sink (a pin, no son)
    class 0; a second net doubles every count."""
    f = _forest([_net(0), _net(20)])
    f["pin_layer"] = f["pin_layer"].astype(np.int8)
    c = bench.node_class_counts(f)
    assert list(c) == [2, 0, 0, 0, 2, 0, 0, 2, 0]


def test_dp_capture_record_from_ncu_csv(tmp_path):
    """The capture record from an ncu CSV in ncu's own layout: launches grouped
    by ID, classes from the template arguments, nodes from the grid, units
    converted; a launch of another kernel is ignored."""
    hdr = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream", "Block Size",
           "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit", "Metric Value"]
    base = {"dram__bytes_read.sum": ("Mbyte", 1.0), "dram__bytes_write.sum": ("Kbyte", 500.0),
            "gpu__time_duration.sum": ("us", 10.0), "sm__inst_executed_pipe_fp64.sum": ("inst", 4200.0),
            "sm__inst_executed.sum": ("inst", 1e5), "launch__grid_size": ("", 100.0), "launch__block_size": ("", 256.0),
            "sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active": ("%", 40.0),
            "gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed": ("%", 30.0),
            "sm__warps_active.avg.pct_of_peak_sustained_active": ("%", 50.0),
            "smsp__issue_active.avg.pct_of_peak_sustained_active": ("%", 45.0),
            "smsp__average_warps_issue_stalled_long_scoreboard_per_issue_active.ratio": ("", 7.0)}
    lines = ['==PROF== Connected to process 1', ",".join(f'"{h}"' for h in hdr)]
    kernels = {"1": "void k_dp_level<12, 6, 1, 0, 1, 0>(LayerInfo, DPArgs)",   # bends: class 7
               "2": "void k_dp_level<12, 6, 2, 1, 1, 1>(LayerInfo, DPArgs)",   # root, several sons: class 5
               "3": "void k_scan_lines<6, 1>(const DevTables *, ScanArgs)"}
    for i, k in kernels.items():
        for name, (unit, val) in base.items():
            row = [i, "1", "python3", "h", k, "1", "7", "(256, 1, 1)", "(100, 1, 1)", "0", "10.3", "m", name, unit,
                   f"{val:,.1f}"]
            lines.append(",".join(f'"{x}"' for x in row))
    p = tmp_path / "dp.csv"
    p.write_text("\n".join(lines) + "\n")
    rec = bench.write_dp_record(str(p), "w", 6, "test", out_path=str(tmp_path / "rec.json"))
    assert sorted(rec["bytes_per_node"]) == ["5", "7"]
    # 1.5 MB over 100 blocks x 42 nodes (bends) and 100 x 256 roots
    assert abs(rec["bytes_per_node"]["7"] - 1.5e6 / 4200) < 0.01
    assert abs(rec["bytes_per_node"]["5"] - 1.5e6 / 25600) < 0.01
    assert rec["fp64_warp_inst_per_node"]["7"] == 1.0
    assert rec["captures"]["7"]["us"] == 10.0 and rec["captures"]["7"]["fp64_pipe_pct"] == 40.0
    assert rec["source_sha256"] == bench.dp_source_hash()
