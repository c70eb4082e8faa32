"""Host logic of bench.py that needs no GPU: the DRAM-traffic record of the dominant kernel is
used only while the kernel's source is the one the counters were taken from (its SHA-256),
for the mixed path's fused kernel and the far field's leaf kernel alike; and the MUFU
roof's work count falls with twin pairs, with more nodes per unit and with twin pairs on
two-CTA clusters."""
import hashlib
import json
import os
import sys

import numpy as np
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
    # units of one node on two-CTA clusters: each twin pair shares its rsqrt, sine and
    # cosine, so 32 nodes in 16 pairs cost 16 (rsqrt, sin, cos) and 32 ex2 per point
    clus = bench.mufu_seconds_per_entry(rates, 32, 1, 16, clusters=True)
    expect = 7 * (32 / rates["ex2"] + 16 * (1 / rates["sin"] + 1 / rates["cos"] + 1 / rates["rsqrt"]))
    assert np.isclose(clus, expect) and clus < wider
    # unpaired nodes on clusters pay their own rsqrt, sine and cosine
    solo = bench.mufu_seconds_per_entry(rates, 5, 1, 2, clusters=True)
    assert np.isclose(solo, 7 * (5 / rates["ex2"] + 3 * (1 / rates["sin"] + 1 / rates["cos"] + 1 / rates["rsqrt"])))


def _fake_solve(values, mults, rng):
    """Eigenpairs as a solve returns them: each value repeated with independent vectors."""
    lam, cols = [], []
    for v, m in zip(values, mults):
        for _ in range(m):
            lam.append(v)
            cols.append(rng.normal(size=40) + 1j * rng.normal(size=40))
    return np.array(lam), np.stack(cols, axis=1), np.full(len(lam), 1e-13)


def test_method_count_roof():
    """The method's evaluation bound: at the measured GB300 rates (ex2 1e13/s, sin, cos,
    rsqrt 5e12/s) and 64 nodes, 7 x (ex2, sin, cos) per entry and node plus one rsqrt per
    quadrature point for all nodes gives 2.84e11 entries/s; one node alone pays the rsqrt."""
    rates = {"ex2": 1e13, "sin": 5e12, "cos": 5e12, "rsqrt": 5e12}
    peak = 64 / bench.mufu_seconds_method(rates, 64)
    assert abs(peak - 2.8369e11) / 2.8369e11 < 1e-3
    assert np.isclose(bench.mufu_seconds_method(rates, 1), 7 * (1e-13 + 2e-13 + 2e-13 + 2e-13))
    # the kernel's own count with twin clusters is below the method's (sin, cos shared)
    assert bench.mufu_seconds_per_entry(rates, 64, 1, 32, clusters=True) < \
        bench.mufu_seconds_method(rates, 64)


def test_eig_compare_flags_extras_missing_and_multiplicity():
    """The eigenvalue check used by the golden-solve tests and the bench: a clean solve
    passes; an extra converged value inside the contour, a missing golden value, a
    multiplicity short of vectors each fail; unconverged or near-contour values are left
    out of the extras."""
    import synth
    spec = synth.ContourSpec("ellipse", 6.5 + 0j, 1.5, 0.4)
    gold = [(5.44 - 3e-7j, 1), (7.6932 - 1e-6j, 2)]
    rng = np.random.default_rng(3)
    lam, X, rel = _fake_solve([g for g, _ in gold], [m for _, m in gold], rng)
    assert bench.eig_compare(lam, X, rel, gold, spec, 1e-10)["ok"]
    # an injected extra converged eigenvalue strictly inside the contour
    lam2 = np.append(lam, 6.1 + 0.01j)
    X2 = np.concatenate([X, rng.normal(size=(40, 1)) + 0j], axis=1)
    r = bench.eig_compare(lam2, X2, np.append(rel, 1e-12), gold, spec, 1e-10)
    assert not r["ok"] and len(r["extras"]) == 1 and not r["missing"]
    # the same value unconverged, or in the annulus next to the contour, is not an extra
    assert bench.eig_compare(lam2, X2, np.append(rel, 1e-3), gold, spec, 1e-10)["ok"]
    lam3 = np.append(lam, 7.99 + 0j)
    assert bench.eig_compare(lam3, X2, np.append(rel, 1e-12), gold, spec, 1e-10)["ok"]
    # a golden value missing from the solve (or the golden list short of a found value)
    r = bench.eig_compare(lam[1:], X[:, 1:], rel[1:], gold, spec, 1e-10)
    assert not r["ok"] and r["missing"][0][:2] == [5.44, -3e-7]
    r = bench.eig_compare(lam, X, rel, gold[1:], spec, 1e-10)
    assert not r["ok"] and len(r["extras"]) == 1
    # a double eigenvalue found twice with the same vector: multiplicity not met
    X4 = X.copy()
    X4[:, 2] = 2.0 * X4[:, 1]
    r = bench.eig_compare(lam, X4, rel, gold, spec, 1e-10)
    assert not r["ok"] and r["missing"] == [[7.6932, -1e-6, 2, 1]]
    # a value off by more than the tolerance is both missing and extra
    lam5 = lam.copy()
    lam5[0] *= 1 + 1e-8
    r = bench.eig_compare(lam5, X, rel, gold, spec, 1e-10)
    assert not r["ok"] and len(r["missing"]) == 1 and len(r["extras"]) == 1
