"""Host-side pieces of bench.py (CPU only): the algorithmic bytes of the
push kernel, the DRAM traffic taken from the committed ncu summary (and
withheld once the kernel source changed), and the workload description."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_algorithmic_bytes():
    # 22-byte FP32 record read and written (44 B per particle) + E, B read
    # and J written once per cell (9 x 4 B); FP64: 42-byte record, 9 x 8 B
    assert bench.algorithmic_bytes(10, 3, 4) == 10 * 44 + 3 * 36
    assert bench.algorithmic_bytes(10, 3, 8) == 10 * 84 + 3 * 72
    n = 536870912
    assert bench.algorithmic_bytes(n, 2048 * 2048, 4) / n == pytest.approx(
        44.28, abs=0.01)


def test_traffic_follows_the_summary_of_the_same_kernel(tmp_path,
                                                        monkeypatch):
    n, cells = 1000, 10
    fake = tmp_path / "traffic.txt"
    fake.write_text("# comment\npush_deposit sha=%s precision=fp32 "
                    "dram_bytes_per_particle=43.3 source=x\n"
                    % bench.push_kernel_hash())
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(fake))
    assert bench.measured_traffic("fp32", n, cells) == pytest.approx(43.3 * n)
    assert bench.measured_traffic("fp64", n, cells) is None
    # a summary taken with another kernel source is not used
    fake.write_text("push_deposit sha=0000000000000000 precision=fp32 "
                    "dram_bytes_per_particle=43.3 source=x\n")
    assert bench.measured_traffic("fp32", n, cells) is None


def test_committed_traffic_summary_is_well_formed():
    # the committed line parses; it is used only while its sha matches
    with open(bench.TRAFFIC_PATH) as f:
        rows = [ln.split() for ln in f if ln.startswith("push_deposit ")]
    assert rows
    for r in rows:
        kv = dict(t.split("=", 1) for t in r[1:])
        assert len(kv["sha"]) == 16 and kv["precision"] in ("fp32", "fp64")
        assert 0 < float(kv["dram_bytes_per_particle"]) < 200


def test_sampled_config_names_the_box_it_ran():
    class A:
        nx = ny = 2048
        ppc = 8
        precision = "fp32"
    c = bench.sampled_config(A(), 256, 2 * 256 * 256 * 64)
    assert (c["nx"], c["ny"], c["sampled"]) == (256, 256, True)
    assert c["particles"] == 2 * 256 * 256 * 64
    assert "256x256" in c["workload"] and "2048x2048" in c["sampled_from"]


def test_workload_config_names_the_workload():
    class A:
        nx = ny = 2048
        ppc = 8
        precision = "fp32"
    c = bench.workload_config(A())
    assert c["particles"] == 2 * 2048 * 2048 * 64
    assert "2048x2048" in c["workload"]
    assert "L2" in c["l2"]


def test_aggregate_single_rank():
    value, ms, total = bench.aggregate(1000.0, 10.0, 1)
    assert (ms, total) == (10.0, 1000.0)
    assert value == pytest.approx(1e5)
