"""Host logic of bench.py (no GPU): the measured-traffic record is reported
only while the kernel sources match the capture; the algorithmic flop
table covers every scene the workloads use."""
import json
import os

import bench


def test_traffic_record_follows_the_kernel_sources(tmp_path):
    dig = bench.kernel_sources_digest()
    assert len(dig) == 64 and all(c in "0123456789abcdef" for c in dig)
    p = os.path.join(tmp_path, "traffic.json")
    with open(p, "w") as f:
        json.dump({"k": {"dram_bytes_per_launch": 123, "sources_sha256": dig},
                   "old": {"dram_bytes_per_launch": 456, "sources_sha256": "0" * 64}}, f)
    assert bench.measured_traffic("k", p) == 123
    assert bench.measured_traffic("old", p) is None     # kernels changed since the capture
    assert bench.measured_traffic("missing", p) is None
    assert bench.measured_traffic("k", os.path.join(tmp_path, "none.json")) is None


def test_flop_table_covers_the_workloads():
    for scene in ("quadruped", "biped", "pendulum", "arm_box"):
        fl = bench.alg_flops(scene)
        cats = fl["by_category_per_env_step"]
        assert abs(sum(cats.values()) - fl["flops_per_env_step"]) < 1e-6 * fl["flops_per_env_step"]
