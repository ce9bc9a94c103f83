"""Host logic of bench.py, without a GPU: the child-process runner of the larger configurations
(its JSON line, a failing child, a child past its time limit) and the ncu traffic records tied
to a hash of the kernel's source."""
import hashlib
import json
import os
import subprocess

import pytest


@pytest.fixture
def bench():
    # imported here, not at collection: bench.py sets a CUDA start-up variable for its own process
    import bench as b
    return b


class _Done:
    def __init__(self, stdout, returncode=0, stderr=""):
        self.stdout, self.returncode, self.stderr = stdout, returncode, stderr


def test_child_line_returns_the_last_json_line(monkeypatch, bench):
    seen = {}

    def run(cmd, capture_output, text, timeout):
        seen["cmd"], seen["timeout"] = cmd, timeout
        return _Done("building...\n" + json.dumps({"value": 1.5}) + "\n" + json.dumps({"value": 2.5}) + "\n")

    monkeypatch.setattr(subprocess, "run", run)
    out = bench.child_line(["--workload", "serve"], timeout_s=7)
    assert out["value"] == 2.5 and out["child_wall_s"] >= 0
    assert seen["cmd"][-2:] == ["--workload", "serve"] and seen["timeout"] == 7
    assert os.path.basename(seen["cmd"][1]) == "bench.py"


def test_child_line_reports_a_failing_child(monkeypatch, bench):
    monkeypatch.setattr(subprocess, "run", lambda *a, **k: _Done("no line\n", 3, "Traceback: boom"))
    out = bench.child_line(["--workload", "batch512"], timeout_s=5)
    assert "error" in out and "exit status 3" in out["error"] and "boom" in out["error"]


def test_child_line_reports_a_child_past_its_limit(monkeypatch, bench):
    def run(cmd, capture_output, text, timeout):
        raise subprocess.TimeoutExpired(cmd, timeout)

    monkeypatch.setattr(subprocess, "run", run)
    out = bench.child_line(["--workload", "ellipsoid256"], timeout_s=3)
    assert out["error"] == "killed after 3 s" and out["args"] == ["--workload", "ellipsoid256"]


def test_traffic_records_carry_a_source_hash(bench):
    """Every traffic record in profiles/ names a source file and the hash it had when the
    capture was taken; the benchmark uses a record only while that hash still matches."""
    recs = bench.ncu_traffic()
    assert recs, "no traffic records in profiles/"
    for kernel, r in recs.items():
        assert r["bytes"] > 0 and isinstance(r["fresh"], bool), kernel
    # a record for a file whose contents changed is stale
    src = "paper_2503_22455_gb300/csrc/setup.cu"
    h = hashlib.sha256(open(os.path.join(bench.ROOT, src), "rb").read()).hexdigest()[:16]
    assert bench.source_sha(src) == h
    assert bench.source_sha("no/such/file.cu") is None
