"""The C-ABI library builds, loads and exports every entry point that
include/curob.h declares; host-side argument checks run without a GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "curob.h")).read()
    return sorted(set(re.findall(r"\b(curob_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1407_7737_gb300 import binding
    return binding.load()


def test_header_declares_the_paper_interface():
    syms = declared_symbols()
    for s in ("curob_initialize", "curob_dispose", "curob_evaluate", "curob_evaluatef",
              "curob_h_evaluate", "curob_h_evaluatef"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_binding_names_match_header():
    from paper_1407_7737_gb300 import binding
    assert sorted(binding.EXPORTS) == declared_symbols()
    for s in declared_symbols():
        assert callable(getattr(binding, s))


def test_status_strings(lib):
    from paper_1407_7737_gb300 import binding
    for code in binding.STATUS:
        assert binding.curob_status_string(code)


def test_calls_before_initialize_fail_cleanly(lib):
    from paper_1407_7737_gb300 import binding as cu
    NI = cu.CODES["CUROB_ERR_NOT_INITIALIZED"]
    assert cu.curob_evaluate(0, 0, 1, 0, None, check=False) == NI
    assert cu.curob_evaluatef(0, 0, 1, 0, None, check=False) == NI
    assert cu.curob_dispose(check=False) == NI
    assert cu.curob_get_device_status(None, check=False) == NI
    assert cu.curob_set_precision(9, check=False) == cu.CODES["CUROB_ERR_INVALID_ARGUMENT"]


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1407_7737_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".hpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "curob_oracle" not in txt, f
