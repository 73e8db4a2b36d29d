"""Host-side checks of the C ABI: the header, the built library and its
exports, and loud failure without a GPU.  No kernel runs here."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fastcat.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(fc_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2011_04736_gb300 import build
    return build.build()


def test_header_matches_binding():
    from paper_2011_04736_gb300 import fastcat
    assert _declared() == sorted(fastcat.ENTRY_POINTS)


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(fc_\w+)$", out, flags=re.M))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing


def test_library_loads_and_binds(libpath):
    from paper_2011_04736_gb300 import fastcat
    L = fastcat.load()
    for name in fastcat.ENTRY_POINTS:
        assert hasattr(L, name)
    assert fastcat.fc_last_error() == ""


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2011_04736_gb300 import fastcat
    monkeypatch.setattr(fastcat, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(fastcat, "_lib", None)
    with pytest.raises(RuntimeError, match="not found"):
        fastcat.load()


def test_create_without_gpu_is_an_error(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2011_04736_gb300 import fastcat
    with pytest.raises(fastcat.FastcatError) as ei:
        fastcat.fc_create(0)
    assert ei.value.code in (fastcat.FC_ECUDA, fastcat.FC_EINVAL)
