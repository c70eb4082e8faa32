"""The C-ABI library builds for sm_103a, loads, and exports every symbol the header
declares (no compute call: this runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bem_gb300.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bem_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1906_03938_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("bem_create", "bem_set_mesh", "bem_set_contour", "bem_project",
              "bem_cholqr2", "bem_residual"):
        assert s in syms


def test_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (bem_[a-z0-9_]+)\b", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing


def test_binding_knows_every_symbol(libpath):
    import paper_1906_03938_gb300 as bem
    assert set(bem.SIGNATURES) == set(declared_symbols())
    lib = bem.load()
    assert lib.bem_version().decode().startswith("bem_gb300")


def test_sm103a_only_and_no_oracle_in_product():
    """The package compiles for sm_103a only and never imports the oracle."""
    from paper_1906_03938_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    pkg = os.path.join(ROOT, "paper_1906_03938_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "bem_oracle" not in src, f
