"""Host-only checks of the C ABI library (no GPU needed).

The CUDA library cross-compiles for sm_103a without a device; these tests
check that it builds, loads, exports every function include/bc_gb300.h
declares, and that the product path shares no code with the oracle.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bc_gb300.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bc_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["bc_init", "bc_shutdown", "bc_create_graph", "bc_destroy_graph", "bc_exact",
                     "bc_sources", "bc_submit", "bc_poll", "bc_debug_source", "bc_status_str"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_1409_7764_gb300 as bc
    from paper_1409_7764_gb300 import capi
    lib = bc.load()
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared but not exported"
    assert sorted(capi.EXPORTED) == declared_functions()


def test_status_strings_without_device():
    import paper_1409_7764_gb300 as bc
    lib = bc.load()
    assert lib.bc_status_str(0) == b"ok"
    assert b"2^64" in lib.bc_status_str(bc.BC_ERR_SIGMA_OVERFLOW)


def test_init_without_device_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    import paper_1409_7764_gb300 as bc
    with pytest.raises(bc.BCError) as ei:
        bc.Context(0)
    assert ei.value.status == bc.BC_ERR_CUDA


def test_product_path_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_1409_7764_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.lower(), f"{f} mentions the oracle"
                assert "bcgen" not in text, f"{f} imports the input generators"


def test_options_struct_matches_header():
    from paper_1409_7764_gb300 import capi
    assert ctypes.sizeof(capi.bc_opts) == 7 * 4
    # int64 x5, int32 x2, double, int64 x6, int32 x6
    assert ctypes.sizeof(capi.bc_stats) == 5 * 8 + 2 * 4 + 8 + 6 * 8 + 6 * 4
