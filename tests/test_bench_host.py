"""Host logic of bench.py that needs no GPU: the committed DRAM traffic of the
dominant kernel is reported only while the kernel's source is the one it was
measured on, and the roofline peak comes from the measured peaks file when
there is one."""
import json
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    import hashlib
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))["k_netsimplex"]
    same = hashlib.sha256(open(os.path.join(ROOT, d["source"]), "rb").read()).hexdigest() == d["source_sha256"]
    # the committed figure while the kernel is the one it was captured on, else none
    assert bench.load_traffic("k_netsimplex") == (d["dram_bytes_per_launch_full"] if same else None)
    # a copy of the tree whose kernel source differs by one byte: no traffic
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(ROOT, "profiles", "traffic.json"), tmp_path / "profiles" / "traffic.json")
    src = tmp_path / d["source"]
    src.parent.mkdir(parents=True)
    body = open(os.path.join(ROOT, d["source"]), "rb").read()
    src.write_bytes(body)
    d2 = dict(d, source_sha256=hashlib.sha256(body).hexdigest())
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"k_netsimplex": d2}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic("k_netsimplex") == d["dram_bytes_per_launch_full"]
    src.write_bytes(body + b" ")
    assert bench.load_traffic("k_netsimplex") is None
    assert bench.load_traffic("no_such_kernel") is None


def test_peaks_from_the_measured_file_else_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    pk, src = bench.peaks()
    assert src == "fallback" and pk["hbm_gbs"] == 6800.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 1234.5, "bf16_tflops": 1.0}))
    pk, src = bench.peaks()
    assert src == "measured" and pk["hbm_gbs"] == 1234.5
