"""Host-only checks of the C-ABI library: it builds for sm_103a, loads, and exports every
function that include/hfr.h declares (no compute calls: there may be no GPU here)."""

import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hfr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char|unsigned long long)\s*\**\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2401_16632_gb300.build import build

    path = build()
    return ctypes.CDLL(path)


def test_header_declares_the_stage_calls():
    names = _declared()
    for n in ["fr_residual", "hfr_local_jacobian", "hfr_condense", "hfr_trace_gmres", "hfr_backsolve", "imex_stage"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    import paper_2401_16632_gb300 as pkg

    names = _declared()
    assert sorted(pkg.ABI_SYMBOLS) == names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings_without_gpu(lib):
    lib.fr_status_string.restype = ctypes.c_char_p
    assert lib.fr_status_string(0) == b"ok"
    assert lib.fr_status_string(3) == b"singular block"


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_2401_16632_gb300 as pkg

    saved = pkg._lib
    pkg._lib = None
    try:
        with pytest.raises(RuntimeError, match="missing"):
            pkg.load_library(str(tmp_path / "nope.so"))
    finally:
        pkg._lib = saved


def test_binding_constants_match_the_header():
    import paper_2401_16632_gb300 as pkg

    src = open(os.path.join(ROOT, "include", "hfr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = dict((k, int(v)) for k, v in re.findall(r"\b(FR_[A-Z0-9_]+)\s*=\s*(\d+)", src))
    assert "FR_ERR_TIMEOUT" in consts and "FR_GMRES_FUSED" in consts
    for k, v in consts.items():
        assert getattr(pkg, k) == v, k
