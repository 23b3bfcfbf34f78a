"""The C-ABI library loads and exports every entry point include/slk.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "slk.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(slk_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1810_13044_gb300 import build
    return ctypes.CDLL(build.build())


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "slk_solve" in names and "slk_bound_iterate" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_1810_13044_gb300 import slk
    assert sorted(slk.EXPORTS) == _declared()


def test_binding_phase_names_follow_header_enum():
    """slk_profile_read fills one slot per SLK_PHASE_* value; the binding
    names them in the same order."""
    from paper_1810_13044_gb300 import slk
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"SLK_PHASE_KNN_PREP\s*=\s*0\s*,(.*?)SLK_PHASE_COUNT", src, flags=re.S)
    assert body is not None
    names = ["KNN_PREP"] + re.findall(r"SLK_PHASE_([A-Z_]+)", body.group(1))
    assert len(names) == len(slk.PHASES)
    assert [n.lower() for n in names] == [p.replace("mean_shift", "meanshift") for p in slk.PHASES]


def test_version_and_no_device_status(lib):
    lib.slk_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.slk_version()
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    h = ctypes.c_void_p()
    lib.slk_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p]
    assert lib.slk_create(ctypes.byref(h), 0, None) == -5  # SLK_ERR_NO_DEVICE
    assert not h.value


def test_product_path_fails_loudly_without_library(tmp_path):
    from paper_1810_13044_gb300 import slk
    with pytest.raises(RuntimeError, match="not built"):
        slk._lib = None
        try:
            slk.load(str(tmp_path / "missing.so"))
        finally:
            slk._lib = None
