"""The separation the parity claims rest on (CPU only):

* the product (the package and its CUDA / C++ sources) never imports, links or
  names the oracle, and has no CPU path: without its compiled library it
  raises;
* the oracle never includes, imports or links the product;
* the shared input generators (synth/) hold no transform arithmetic and import
  neither side.
"""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _files(*patterns):
    out = []
    for p in patterns:
        out += glob.glob(os.path.join(ROOT, p), recursive=True)
    return [f for f in out if "__pycache__" not in f and not f.endswith((".so", ".o"))]


def test_product_never_touches_the_oracle():
    files = _files("paper_1406_5597_gb300/*.py", "paper_1406_5597_gb300/csrc/*", "include/*.h", "bench.py")
    assert files
    for f in files:
        text = open(f, errors="replace").read()
        if f.endswith("bench.py"):
            # the one permitted use: the CPU-baseline / reference leg imports the oracle inside its own function
            for m in re.finditer(r"^(\s*)import oracle\b", text, flags=re.M):
                assert m.group(1), "bench.py imports the oracle at module level"
            continue
        assert not re.search(r"\boracle\b", text), f


def test_oracle_never_touches_the_product():
    for f in _files("oracle/*.c", "oracle/*.py"):
        text = open(f, errors="replace").read()
        assert not re.search(r"^\s*(import|from)\s+paper_1406_5597_gb300\b", text, flags=re.M), f
        assert not re.search(r'^\s*#\s*include\s*"', text, flags=re.M), f  # system headers only
        assert "csrc" not in text and "fft3d.h" not in text and "libfft3d" not in text, f


def test_shared_generators_hold_no_transform():
    for f in _files("synth/*.py"):
        text = open(f, errors="replace").read()
        assert not re.search(r"\bnp\.fft\b|numpy\.fft|\bscipy\.fft|\btorch\.fft|import oracle|paper_1406_5597_gb300", text), f


def test_product_fails_loudly_without_its_library(monkeypatch, tmp_path):
    import paper_1406_5597_gb300 as fft3d
    monkeypatch.setattr(fft3d, "_lib", None)
    monkeypatch.setattr(fft3d, "LIB_PATH", str(tmp_path / "missing_libfft3d.so"))
    with pytest.raises(RuntimeError, match="missing"):
        fft3d.load()
