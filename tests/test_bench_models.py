"""bench.py's roofline inputs on CPU: the algorithmic byte models of the dominant kernels, and the
committed DRAM traffic record, which is reported only while the kernel's sources are unchanged."""
import json
import os
import shutil

import bench


def test_algorithmic_bytes_per_agent():
    # list kernel: 96 B of own state read and written (update fused) + 4 B per listed entry
    assert bench.KERNEL_BYTES["force_list"](7.0) == 124.0
    # the whole step as the method defines it: 4 passes over 32 B of agent state + 8 B per box
    assert bench.STEP_BYTES_PER_AGENT(1.0) == 136.0
    # neurite list kernel: 100 B per agent + 4 B per listed entry
    assert abs(bench.NEURITE_LIST_BYTES_PER_AGENT(15.4) - 161.6) < 1e-12


def test_traffic_record_follows_its_sources(tmp_path, monkeypatch):
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    kernel = "force_list"
    entry = rec[kernel]
    # a private copy of the record and of the sources it hashes
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(bench.ROOT, "profiles", "traffic.json"), tmp_path / "profiles")
    for src in entry["sources"]:
        dst = tmp_path / src
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, src), dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    current = bench.measured_traffic(kernel, 1000)
    if current is not None:  # the record matches the committed sources: per-agent bytes x agents
        assert abs(current - entry["dram_bytes_per_agent"] * 1000) < 1e-9
    # any edit of a source voids the record
    with open(tmp_path / entry["sources"][0], "a") as f:
        f.write("\n// edited\n")
    assert bench.measured_traffic(kernel, 1000) is None
    assert bench.measured_traffic("no_such_kernel", 1000) is None
