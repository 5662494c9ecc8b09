"""DRAM-traffic records of bench.py, on CPU: an ncu launch list (--csv,
dram__bytes_{read,write}.sum) becomes per-unit bytes of the last build's
launches; a full-size capture of some kernels refines an existing record of
the same sources; a record of other sources is ignored."""
import argparse
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

HEADER = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
          '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n')


def _row(i, kernel, metric, unit, value):
    return (f'"{i}","1","python","h","void {kernel}(int)","1","7","(256, 1, 1)","(1, 1, 1)","0","10.3","",'
            f'"{metric}","{unit}","{value}"\n')


def _csv(path, builds):
    """builds: list of [(kernel, read_bytes, write_bytes)] in launch order."""
    lines = ["==PROF== Connected to process 1\n", HEADER]
    i = 0
    for b in builds:
        for kernel, rd, wr in b:
            lines.append(_row(i, kernel, "dram__bytes_read.sum", "byte", rd))
            lines.append(_row(i, kernel, "dram__bytes_write.sum", "byte", wr))
            i += 1
    path.write_text("".join(lines))


def _args(**kw):
    a = argparse.Namespace(workload="sift1m", precision="bf16", traffic_from=None, traffic_hash="abc",
                           traffic_command="cmd", traffic_full=False)
    for k, v in kw.items():
        setattr(a, k, v)
    return a


@pytest.fixture
def record(tmp_path, monkeypatch):
    out = tmp_path / "rec.json"
    monkeypatch.setattr(bench, "traffic_path", lambda w, p: str(out))
    return out


def test_last_build_per_unit_bytes(tmp_path, record):
    w = bench.WORKLOADS["sift1m"]
    n = bench.PROFILE_CASE["sift1m"]["n"]
    build = [("init_perm_kernel", 10, 10), ("project_bytes_tma_kernel", 1000, 0),
             ("leaf_tc_kernel", 8000, 800), ("merge_kernel", 500, 50),
             ("propagate_kernel", 300, 30), ("propagate_kernel", 200, 20)]
    warm = [(k, 10 * r, 10 * wr) for k, r, wr in build]  # the warm-up build must not count
    f = tmp_path / "t.csv"
    _csv(f, [warm, build])
    assert bench.traffic_from_csv(_args(traffic_from=str(f)), w) == 0
    rec = json.loads(record.read_text())
    pu = rec["per_unit"]
    assert rec["source_hash"] == "abc" and rec["case"]["n"] == n
    assert pu["propagate_kernel"]["bytes_per_unit"] == pytest.approx([330 / n, 220 / n])
    assert pu["leaf_tc_kernel"]["bytes_per_unit"] == pytest.approx(8800 / (n * w["T"]))
    assert pu["merge_kernel"]["bytes_per_unit"] == pytest.approx(550 / n)
    assert pu["project_bytes_tma_kernel"]["bytes_per_unit"] == pytest.approx(1000 / n)
    assert "init_perm_kernel" not in pu


def test_full_size_capture_refines_the_record(tmp_path, record):
    w = bench.WORKLOADS["sift1m"]
    f = tmp_path / "t.csv"
    _csv(f, [[("init_perm_kernel", 1, 1), ("merge_kernel", 500, 50), ("propagate_kernel", 300, 30),
              ("propagate_kernel", 200, 20)]])
    bench.traffic_from_csv(_args(traffic_from=str(f)), w)
    g = tmp_path / "full.csv"
    _csv(g, [[("propagate_kernel", 9000, 1000), ("propagate_kernel", 7000, 1000)]])
    bench.traffic_from_csv(_args(traffic_from=str(g), traffic_full=True), w)
    rec = json.loads(record.read_text())
    assert rec["full_size"] == ["propagate_kernel"]
    assert rec["per_unit"]["propagate_kernel"]["bytes_per_unit"] == pytest.approx([10000 / w["n"], 8000 / w["n"]])
    assert rec["per_unit"]["merge_kernel"]["bytes_per_unit"] == pytest.approx(550 / bench.PROFILE_CASE["sift1m"]["n"])


def test_record_of_other_sources_is_ignored(tmp_path, record, monkeypatch):
    record.write_text(json.dumps({"source_hash": "not-these-sources", "per_unit": {}}))
    assert bench.load_traffic("sift1m", "bf16") is None
    monkeypatch.setattr(bench, "source_hash", lambda: "not-these-sources")
    assert bench.load_traffic("sift1m", "bf16") is not None


def test_hash_is_required(tmp_path, record):
    f = tmp_path / "t.csv"
    _csv(f, [[("merge_kernel", 1, 1)]])
    with pytest.raises(SystemExit):
        bench.traffic_from_csv(_args(traffic_from=str(f), traffic_hash=None), bench.WORKLOADS["sift1m"])
