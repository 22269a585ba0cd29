"""The C-ABI library builds, loads and exports every symbol include/wr.h
declares (no GPU needed: nothing here launches device work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wr.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(wr_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_0704_2351_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["wr_create", "wr_matrix_load_csr", "wr_rank", "wr_rank_batch", "wr_result_rank",
                 "wr_result_sequence", "wr_result_generator", "wr_server_start", "wr_submit", "wr_wait",
                 "wr_server_stats", "wr_result_free", "wr_matrix_free", "wr_server_stop", "wr_destroy",
                 "wr_last_error"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_binding_names_match_the_header(lib):
    from paper_0704_2351_gb300 import wr
    for n in declared_functions():
        assert hasattr(wr, n), n


def test_null_arguments_are_rejected_without_device_work(lib):
    from paper_0704_2351_gb300 import wr
    lib.wr_rank.argtypes = [ctypes.c_void_p] * 4
    lib.wr_rank.restype = ctypes.c_int
    assert lib.wr_rank(None, None, None, None) == wr.WR_EINVAL
    assert "null" in wr.wr_last_error()
    lib.wr_matrix_info.restype = ctypes.c_int
    assert lib.wr_matrix_info(None, None, None, None, None, None) == wr.WR_EINVAL


def test_oracle_is_not_linked_into_the_library(lib):
    """The product path and the oracle share no code."""
    from paper_0704_2351_gb300 import _build
    data = open(_build.LIB, "rb").read()
    assert b"or_mbasis" not in data and b"or_sequence" not in data
    for src in _build.sources():
        text = open(src).read()
        assert "oracle" not in text.lower().replace("oracle's", "")
