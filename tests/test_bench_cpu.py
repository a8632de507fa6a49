"""Host logic of bench.py (no GPU): the DRAM-traffic records behind
roofline.traffic, the split thresholds they are keyed to, and the JSON line
of the reference arm (the oracle timed on the host)."""
import json
import os
import sys

import pytest

sys.path.insert(0, os.path.join(os.path.dirname(__file__), ".."))
import bench  # noqa: E402


def _csv(path, rows):
    """An ncu --csv launch list with the two DRAM metrics (values in bytes)."""
    with open(path, "w") as f:
        f.write('"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n')
        for launch, kernel, rd, wr in rows:
            f.write(f'"{launch}","{kernel}(args)","dram__bytes_read.sum","byte","{rd}"\n')
            f.write(f'"{launch}","{kernel}(args)","dram__bytes_write.sum","byte","{wr}"\n')


def test_split_thresholds_follow_the_option_rounding():
    assert bench.split_thresholds(0.375, 0.0234375, 4096) == {"sparse": 1536, "uw_sparse": 96}
    assert bench.split_thresholds(0.375, 0.0, 4096) == {"sparse": 1536, "uw_sparse": 0}
    assert bench.split_thresholds(1e-9, 1e-9, 100) == {"sparse": 1, "uw_sparse": 1}


def test_traffic_records_are_keyed_to_workload_samples_split_and_sources(tmp_path, monkeypatch):
    """One record per (workload, samples, split): a second split adds a
    record, the same split replaces its record, and a lookup with any other
    key -- or after a kernel's sources change -- finds nothing."""
    path = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(path))
    csv1 = tmp_path / "a.csv"
    _csv(csv1, [("1", "void ufb::k_pairs_sparse<0>", 100, 20),
                ("2", "void ufb::k_pairs_sparse<0>", 300, 40),
                ("3", "ufb::k_pairs_tc", 1000, 10)])
    t96 = {"sparse": 1536, "uw_sparse": 96}
    t128 = {"sparse": 1536, "uw_sparse": 128}
    bench.record_traffic(str(csv1), "w", 4096, "cap", t96)
    # mean over launches of read + write
    assert bench.recorded_traffic("k_pairs_sparse<false>", "w", 4096, t96) == 230.0
    assert bench.recorded_traffic("k_pairs_tc", "w", 4096, t96) == 1010.0
    for key in (("w2", 4096, t96), ("w", 2048, t96), ("w", 4096, t128)):
        assert bench.recorded_traffic("k_pairs_tc", *key) is None
    csv2 = tmp_path / "b.csv"
    _csv(csv2, [("1", "ufb::k_pairs_tc", 500, 0)])
    bench.record_traffic(str(csv2), "w", 4096, "cap", t128)
    assert bench.recorded_traffic("k_pairs_tc", "w", 4096, t128) == 500.0
    assert bench.recorded_traffic("k_pairs_tc", "w", 4096, t96) == 1010.0
    bench.record_traffic(str(csv2), "w", 4096, "cap", t96)  # replaces the first record
    assert bench.recorded_traffic("k_pairs_tc", "w", 4096, t96) == 500.0
    assert len(json.load(open(path))["records"]) == 2
    # a changed source hash voids the record
    monkeypatch.setattr(bench, "kernel_source_hash", lambda kernel: "changed")
    assert bench.recorded_traffic("k_pairs_tc", "w", 4096, t96) is None


def test_traffic_records_read_the_unit_column(tmp_path, monkeypatch):
    """ncu prints large byte counts in Mbyte / Gbyte: the record is in bytes,
    and launches of separate captures (each numbered from 0) stay apart."""
    path = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(path))
    csv1 = tmp_path / "g.csv"
    with open(csv1, "w") as f:
        f.write('"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n')
        f.write('"0","ufb::k_pairs_tc(args)","dram__bytes_read.sum","Gbyte","2.5"\n')
        f.write('"0","ufb::k_pairs_tc(args)","dram__bytes_write.sum","Mbyte","500"\n')
        f.write('"0","void ufb::k_pairs_sparse<0>(args)","dram__bytes_read.sum","Kbyte","1"\n')
        f.write('"0","void ufb::k_pairs_sparse<0>(args)","dram__bytes_write.sum","byte","24"\n')
    t = {"sparse": 1, "uw_sparse": 2}
    bench.record_traffic(str(csv1), "w", 100, "cap", t)
    assert bench.recorded_traffic("k_pairs_tc", "w", 100, t) == 3.0e9
    assert bench.recorded_traffic("k_pairs_sparse<false>", "w", 100, t) == 1024.0


def test_kernel_hash_ignores_the_host_context_struct(tmp_path, monkeypatch):
    """The hash covers the kernel sources and the launch-planning functions,
    not the host-only context struct of the shared header."""
    h0 = bench.kernel_source_hash("k_pairs_sparse<false>")
    src = open(os.path.join(bench.ROOT, "paper_2107_05397_b300", "csrc", "ufb_internal.cuh")).read()
    assert "struct unifrac_ctx {" in src
    plan = bench.planning_source().decode()
    for sig in bench.PLANNING_FUNCTIONS:
        assert sig in plan
    assert h0 == bench.kernel_source_hash("k_pairs_sparse<true>")  # same sources
    assert h0 != bench.kernel_source_hash("k_pairs_tc")


def bench_workloads():
    from paper_2107_05397_b300 import synth
    return set(synth.WORKLOADS) | set(synth.BATCHED)


@pytest.mark.parametrize("kernel", sorted(bench.KERNEL_SOURCES))
def test_committed_traffic_has_every_pair_kernel(kernel):
    """profiles/traffic.json holds, for every pair kernel, records with bytes
    per launch and a source hash (null in the bench line once the sources
    move on, or for another workload, sample count or split)."""
    records = json.load(open(bench.TRAFFIC_PATH))["records"]
    mine = [r for r in records if kernel in r and r.get("workload") in bench_workloads()]
    assert mine
    for r in mine:
        assert r[kernel]["bytes_per_launch"] > 0 and len(r[kernel]["source_hash"]) == 16
        assert set(r["thresholds"]) == {"sparse", "uw_sparse"}


def test_traffic_hash_ignores_comments_only():
    """Records are keyed to the kernels' code: comments and blank lines do
    not change the key, code does (and a // inside a string is code)."""
    import bench
    base = 'int a = 1;  // one\n\n  const char *s = "x//y";\n// whole-line comment\n'
    same = 'int a = 1;\n  const char *s = "x//y";  // other words\n'
    assert bench.code_only(base) == bench.code_only(same)
    assert bench.code_only(base) != bench.code_only(base.replace("a = 1", "a = 2"))
    assert '"x//y"' in bench.code_only(base)


def _reference_line(env_extra=None):
    import subprocess
    env = dict(os.environ)
    env.update(env_extra or {})
    root = os.path.join(os.path.dirname(__file__), "..")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--workload", "tips1024_samples256", "--steps", "3", "--warmup", "1"],
                       capture_output=True, text=True, env=env, timeout=300, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


def test_reference_arm_prints_one_contract_line():
    """--impl reference times the oracle on the host and prints one JSON line
    with the arm's keys: impl, metric, value, unit, steps, a cpu_baseline
    describing the run and an e2e with no host-device bytes."""
    lines = _reference_line()
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["steps"] == 3 and line["warmup"] == 1 and line["value"] > 0
    assert line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"] == "tips1024_samples256"


def test_reference_arm_other_ranks_print_nothing():
    """Under torchrun only rank 0 runs the oracle; the other ranks exit 0
    without work or output."""
    assert _reference_line({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []
