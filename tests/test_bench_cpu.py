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
        json.dump({"k": {"dram_read_bytes": 123, "sources_sha256": dig},
                   "old": {"dram_read_bytes": 456, "sources_sha256": "0" * 64}}, f)
    assert bench.measured_traffic("k", p)["dram_read_bytes"] == 123
    assert bench.measured_traffic("old", p) is None     # kernels changed since the capture
    assert bench.measured_traffic("missing", p) is None
    assert bench.measured_traffic("k", os.path.join(tmp_path, "none.json")) is None


def test_traffic_scaling_arithmetic():
    """A 40-step capture (initial state + 40 steps of actions read) scaled to
    1,000 steps in 8 chunks: 1,000 steps of the per-step stream, plus the
    state read and written once per chunk."""
    state, act = 30_670_848, 2_097_152
    rec = {"steps": 40, "state_bytes": state, "dram_read_bytes": state + 40 * act, "dram_write_bytes": 0}
    assert bench.scaled_traffic(rec, 1000, 8, state) == 1000 * act + 16 * state
    assert bench.scaled_traffic(rec, 1000, 0, state) == 1000 * act + 2 * state  # static schedule: one chunk


def test_flop_table_covers_the_workloads():
    for scene in ("quadruped", "biped", "pendulum", "arm_box"):
        fl = bench.alg_flops(scene)
        cats = fl["by_category_per_env_step"]
        assert abs(sum(cats.values()) - fl["flops_per_env_step"]) < 1e-6 * fl["flops_per_env_step"]


def test_stream_chunks_cover_the_rollout_once():
    """Chunks of the streamed rollout (the e2e path): 16 steps first, then
    doubling up to the chunk length, covering every step once, in order."""
    from paper_2106_13281_gb300.system import stream_chunks
    assert stream_chunks(1000, 250, 16) == [(0, 16), (16, 48), (48, 112), (112, 240), (240, 490), (490, 740),
                                            (740, 990), (990, 1000)]
    assert stream_chunks(25, 10, 10) == [(0, 10), (10, 20), (20, 25)]
    assert stream_chunks(5, 100, 16) == [(0, 5)]
    for T, C, F in [(1, 1, 1), (7, 3, 1), (100, 100, 16), (999, 37, 5), (64, 8, 100)]:
        ch = stream_chunks(T, C, F)
        assert ch[0][0] == 0 and ch[-1][1] == T
        assert all(a[1] == b[0] for a, b in zip(ch, ch[1:]))
        assert all(0 < t1 - t0 <= max(1, min(C, T)) for t0, t1 in ch)
