"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/lgf.h declares; the oracle builds too."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lgf_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("lgf_create", "lgf_set_links", "lgf_fix", "lgf_get_links", "lgf_get_gauge", "lgf_destroy"):
        assert need in names


def test_library_exports_every_declared_symbol():
    from paper_1301_3460_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    from paper_1301_3460_gb300 import lgf

    lib = lgf.load()
    assert lib.lgf_strerror(0) == b"ok"
    assert b"SU(3)" in lib.lgf_strerror(lgf.LGF_ERR_NOT_SU3)


def test_oracle_builds():
    from oracle import oracle

    assert os.path.exists(oracle.build())
