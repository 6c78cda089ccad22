"""bench.py reports an ncu traffic record only while the kernel source it was
taken on is unchanged and the solver options match (host logic, CPU)."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _write(tmp, src_text, sha, options):
    src = tmp / "k.cu"
    src.write_text(src_text)
    rec = {"source_file": str(src), "source_section": ["// begin", "// end"], "source_sha1": sha,
           "options": options, "dram_bytes_per_launch": 123.0}
    (tmp / "profiles").mkdir(exist_ok=True)
    (tmp / "profiles" / "r.json").write_text(json.dumps(rec))


def test_record_follows_source_and_options(tmp_path, monkeypatch):
    body = "x\n// begin\nkernel body\n// end\ny\n"
    sha = hashlib.sha1("// begin\nkernel body\n".encode()).hexdigest()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _write(tmp_path, body, sha, {"theta_factor": 0.5, "hub_deg": 256, "piece": 1024})
    assert bench.traffic_for("r.json", {"theta_factor": 0.5, "hub_deg": 256, "piece": 1024}) == 123.0
    assert bench.traffic_for("r.json", None) == 123.0
    # other options: no record
    assert bench.traffic_for("r.json", {"theta_factor": 1.0}) is None
    assert bench.traffic_for("r.json", {"piece": 512}) is None
    # the kernel section changed: no record
    _write(tmp_path, body.replace("kernel body", "kernel body changed"), sha, {"theta_factor": 0.5})
    assert bench.traffic_for("r.json", {"theta_factor": 0.5}) is None
    # a change outside the section does not matter
    _write(tmp_path, "other\n" + body, sha, {"theta_factor": 0.5})
    assert bench.traffic_for("r.json", {"theta_factor": 0.5}) == 123.0
    # missing record or markers
    assert bench.traffic_for("absent.json", None) is None
    _write(tmp_path, "no markers here", sha, {})
    assert bench.traffic_for("r.json", None) is None


def test_committed_records_match_their_sources():
    """Every committed push/batch record names a source section that exists."""
    prof = os.path.join(ROOT, "profiles")
    names = [f for f in os.listdir(prof) if f.endswith("_traffic.json")]
    assert names
    for f in names:
        rec = json.load(open(os.path.join(prof, f)))
        src = open(os.path.join(ROOT, rec["source_file"])).read()
        a, b = rec["source_section"]
        assert a in src and b in src, f
        assert rec["dram_bytes_per_launch"] > 0
