"""Host logic of bench.py that needs no GPU: the DRAM-traffic record of the dominant kernel is
used only while the kernel's source is the one the counters were taken from (its SHA-256),
for the mixed path's fused kernel and the far field's leaf kernel alike; and the MUFU
roof's work count falls with twin pairs and with more nodes per unit."""
import hashlib
import json
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _tree(tmp_path, kernel, source, text, bytes_read, bytes_write, sha=None):
    src = tmp_path / "paper_1906_03938_gb300" / "csrc"
    src.mkdir(parents=True, exist_ok=True)
    (src / source).write_text(text)
    prof = tmp_path / "profiles"
    prof.mkdir(exist_ok=True)
    rec = {"dram_bytes_read": bytes_read, "dram_bytes_write": bytes_write,
           "source_sha256": sha or hashlib.sha256(text.encode()).hexdigest()}
    (prof / f"{kernel}_w1_traffic.json").write_text(json.dumps(rec))
    return src / source


@pytest.mark.parametrize("precision,kernel,source", [("mixed", "mixed_apply", "project_mixed.cu"),
                                                      ("hmatrix", "hm_leaf", "hmatrix.cu")])
def test_traffic_record_follows_the_source(tmp_path, monkeypatch, precision, kernel, source):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    path = _tree(tmp_path, kernel, source, "kernel v1\n", 1000, 234)
    assert bench.measured_traffic("w1", precision) == 1234
    path.write_text("kernel v2\n")                       # source changed since the capture
    assert bench.measured_traffic("w1", precision) is None
    assert bench.measured_traffic("other", precision) is None   # no record
    assert bench.measured_traffic("w1", "fp64") is None         # no dominant-kernel record


def test_mufu_work_count():
    rates = {"ex2": 1e13, "sin": 5e12, "cos": 5e12, "rsqrt": 5e12}
    base = bench.mufu_seconds_per_entry(rates, 32, 4, 0)
    twins = bench.mufu_seconds_per_entry(rates, 32, 4, 16)
    wider = bench.mufu_seconds_per_entry(rates, 32, 1, 0)
    assert twins < base < wider
    # every node still takes its own ex2 at every quadrature point
    assert twins > 7 * 32 / rates["ex2"]
