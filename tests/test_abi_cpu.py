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


class _FakeCudaTensor:
    """Stand-in with the attributes the argument checks read (no GPU needed)."""

    def __init__(self, n, dtype=None, device="cuda:0", contiguous=True):
        import torch
        self.n = n
        self.dtype = torch.float32 if dtype is None else dtype
        self.device = torch.device(device)
        self.is_cuda = True
        self._c = contiguous

    def numel(self):
        return self.n

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        raise AssertionError("the checks must not take a pointer")


def test_blur_static_argument_checks_on_host():
    import torch
    from paper_2011_04736_gb300 import fastcat
    n_img, n_v, n_u = 3, 10, 20
    n = n_img * n_v * n_u
    ok = _FakeCudaTensor(n)
    fastcat.check_blur_static_args(ok, _FakeCudaTensor(n + 5), n_img, n_v, n_u)
    bad = [(_FakeCudaTensor(n - 1), ok), (ok, _FakeCudaTensor(n - 1)),
           (_FakeCudaTensor(n, dtype=torch.bfloat16), ok),
           (ok, _FakeCudaTensor(n, dtype=torch.float64)),
           (_FakeCudaTensor(n, contiguous=False), ok),
           (ok, _FakeCudaTensor(n, device="cuda:1")),
           (torch.zeros(n), ok)]
    for T, I in bad:
        with pytest.raises(ValueError):
            fastcat.check_blur_static_args(T, I, n_img, n_v, n_u)
    with pytest.raises(ValueError):
        fastcat.check_blur_static_args(ok, ok, 0, n_v, n_u)


def test_fault_injection_arguments_checked_on_host(libpath):
    from paper_2011_04736_gb300 import fastcat
    fastcat.fc_inject_fault(fastcat.FC_FAULT_NONE)
    for kind, arg in ((7, 0), (fastcat.FC_FAULT_ALLOC, -1)):
        with pytest.raises(fastcat.FastcatError) as ei:
            fastcat.fc_inject_fault(kind, arg)
        assert ei.value.code == fastcat.FC_EINVAL
    fastcat.fc_inject_fault(fastcat.FC_FAULT_NONE)


def test_binding_constants_match_header():
    """Every FC_* integer constant the binding defines has the header's value."""
    from paper_2011_04736_gb300 import fastcat
    txt = open(HEADER).read()
    defs = {m.group(1): int(m.group(2)) for m in
            re.finditer(r"^#define\s+(FC_\w+)\s+(-?\d+)\s*(?:/\*.*)?$", txt, flags=re.M)}
    m = re.search(r"^#define\s+FC_STATIC_SCRATCH_FLOATS\s+\((\d+)u << (\d+)\)", txt, flags=re.M)
    defs["FC_STATIC_SCRATCH_FLOATS"] = int(m.group(1)) << int(m.group(2))
    names = [n for n in dir(fastcat) if n.startswith("FC_") and isinstance(getattr(fastcat, n), int)]
    checked = 0
    for n in names:
        if n in defs:
            assert getattr(fastcat, n) == defs[n], n
            checked += 1
    assert checked >= 20
    assert len(fastcat.FC_K_NAMES) == defs["FC_K_COUNT"]
