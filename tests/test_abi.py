"""The C-ABI library builds, loads, and exports every entry point that
include/hsc.h declares (no GPU needed: nothing is computed)."""

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hsc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hsc_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("hsc_pca_one_band", "hsc_svm_probs", "hsc_knn_filter", "hsc_classify",
              "hsc_ctx_create", "hsc_ctx_destroy", "hsc_sync", "hsc_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2404_10631_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in declared_functions():
        assert hasattr(lib, n), n
    import paper_2404_10631_gb300 as pkg
    assert set(pkg.EXPORTED) == set(declared_functions())


def test_status_strings_without_gpu():
    import paper_2404_10631_gb300 as pkg
    L = pkg.lib()
    assert L.hsc_status_string(0) == b"HSC_OK"
    assert L.hsc_status_string(7) == b"HSC_ERR_NONFINITE"
    assert L.hsc_last_error(None) == b""


def test_package_import_does_not_load_the_library():
    import importlib
    import paper_2404_10631_gb300 as pkg
    importlib.reload(pkg)
    assert pkg._lib is None
