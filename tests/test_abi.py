"""The C-ABI library loads on a machine without a GPU and exports every entry
point include/fbcc.h declares (no compute call is made here)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fbcc.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2301_01356_gb300 import build, fbcc
    build.build_libfbcc()
    return fbcc.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fbcc_[a-z_0-9]+)\s*\(", text)))


def test_header_matches_binding():
    from paper_2301_01356_gb300 import fbcc
    assert declared_functions() == sorted(fbcc.EXPORTS)


def test_every_symbol_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} is declared in include/fbcc.h but not exported"


def test_host_only_calls(lib):
    from paper_2301_01356_gb300 import fbcc
    assert fbcc.load().fbcc_status_string(0) == b"ok"
    assert b"workspace" in fbcc.load().fbcc_status_string(6)
    # the workspace is O(n) plus a few bits per arc (section 4.3: O(n) auxiliary space)
    n, z = 1 << 20, 1 << 24
    b0 = fbcc.fbcc_workspace_bytes(n, z)
    b_arcs = fbcc.fbcc_workspace_bytes(n, 2 * z) - b0
    b_vert = fbcc.fbcc_workspace_bytes(2 * n, z) - b0
    assert b_arcs <= z * 0.5, "more than half a byte per arc of workspace"
    assert b_vert <= n * 240
    assert fbcc.fbcc_batch_workspace_bytes(n, z, 100) > b0


def test_no_cpu_fallback_without_library(tmp_path, monkeypatch):
    """The binding refuses to run when libfbcc is missing (no CPU path exists)."""
    import importlib
    from paper_2301_01356_gb300 import fbcc
    mod = importlib.reload(fbcc)
    with pytest.raises(RuntimeError, match="not built"):
        mod.load(str(tmp_path / "missing.so"))
    importlib.reload(fbcc)
