"""bench.py's roofline.traffic field: DRAM bytes of a launch from a committed
ncu capture (profiles/traffic.json), scaled to the launch's algorithmic
bytes, and only while the kernel source is the one that was captured."""
import hashlib
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_entries_and_their_source_check():
    t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    assert {"phase1", "phase2", "tc_phase1", "tc_phase2", "tc_dense"} <= set(t["kernels"])
    for name, k in t["kernels"].items():
        assert os.path.exists(os.path.join(ROOT, k["capture"])), name
        # a launch reads at least the bytes it must (metadata and the vectors
        # come on top of the stored factors)
        assert k["dram_bytes"] >= 0.99 * k["algorithmic_bytes"] > 0, name
        with open(os.path.join(ROOT, "paper_2604_09147_gb300", "csrc", k["source"]), "rb") as f:
            current = hashlib.sha256(f.read()).hexdigest() == k["sha256"]
        got = bench.traffic_for(name, 2.0e9)
        if current:
            assert abs(got - k["dram_bytes"] / k["algorithmic_bytes"] * 2.0e9) <= 1e-6 * got
        else:
            assert got is None                  # a changed kernel reports no traffic until recaptured
    assert bench.traffic_for("no_such_kernel", 1.0) is None
