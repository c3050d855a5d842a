"""The C ABI library builds, loads and exports every symbol include/fstat.h
declares; the Python binding covers them all (CPU only, no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        with open(os.path.join(ROOT, "include", h)) as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        names |= set(re.findall(r"\b(fstat_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("fstat_create", "fstat_set_sfts", "fstat_set_templates", "fstat_compute", "fstat_get_toplist"):
        assert n in names


def test_library_builds_and_exports_every_symbol():
    import __graft_entry__ as ge
    path = ge._build_module().build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_covers_every_symbol():
    import paper_0904_1826_gb300 as fs
    assert sorted(fs.SIGNATURES) == _declared()
    assert fs.fstat_version().startswith("libfstat")


def test_no_device_is_an_error_code_not_a_crash():
    import paper_0904_1826_gb300 as fs
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(fs.FstatError) as e:
        fs.fstat_create(0)
    assert e.value.code == fs.FSTAT_ECUDA
    fs.fstat_destroy(None)
    assert fs.fstat_last_error(None) == ""
