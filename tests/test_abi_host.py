"""Host-only checks of the C ABI library (no GPU, no compute calls)."""
import os
import re

import pytest

from paper_1603_08390_gb300 import _build, genie

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "genie.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(genie_[a-z_0-9]+)\s*\(", text))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return genie.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    assert set(genie.EXPORTED) == _declared()


def test_version_and_error_text(lib):
    assert genie.genie_version() >= 100
    assert isinstance(genie.genie_last_error(), str)


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(genie, "_LIB", None)
    with pytest.raises(genie.GenieError):
        genie.load("/nonexistent/libgenie.so")


def test_product_code_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_1603_08390_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                with open(os.path.join(dirpath, f)) as fh:
                    src = fh.read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
                assert "mc_oracle" not in src and "liboracle" not in src, f


def test_opts_struct_layout_matches_header():
    # genie_search_opts: pointer, 4 x uint32, 2 pointers, host pointer, 2 events, flags (+pad)
    import ctypes
    assert ctypes.sizeof(genie.SearchOpts) == 8 + 4 * 4 + 8 * 3 + 8 * 2 + 8
    # genie_index_info: 2 x uint32, uint64, 4 x uint32, uint64, 2 x uint32, uint64
    assert ctypes.sizeof(genie.IndexInfo) == 56
    assert ctypes.sizeof(genie.IndexOpts) == 8
    assert ctypes.sizeof(genie.QueriesInfo) == 32
    # genie_server_opts / stats, genie_spq_opts / info, genie_calibration
    assert ctypes.sizeof(genie.ServerOpts) == 8 + 6 * 4
    assert ctypes.sizeof(genie.ServerStats) == 10 * 8
    assert ctypes.sizeof(genie.SpqOpts) == 16 and ctypes.sizeof(genie.SpqInfo) == 32
    assert ctypes.sizeof(genie.Calibration) == 8 + 8 + 8 * 4
