"""Host-only checks of the C ABI library (no GPU needed).

The CUDA library cross-compiles for sm_103a without a device; these tests
check that it builds, loads, exports every function include/bc_gb300.h
declares, and that the product path shares no code with the oracle.
"""
import ctypes
import subprocess
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


def test_options_struct_matches_header(tmp_path):
    """The ctypes mirrors have the C structs' sizes and field offsets, as a C
    compiler lays them out from include/bc_gb300.h."""
    from paper_1409_7764_gb300 import capi
    fields = {"bc_opts": capi.bc_opts, "bc_stats": capi.bc_stats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "bc_gb300.h"',
             "int main(void) {"]
    for name, cls in fields.items():
        lines.append(f'  printf("%zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({name}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = []
    for cls in fields.values():
        want.append(ctypes.sizeof(cls))
        want += [getattr(cls, fname).offset for fname, _ in cls._fields_]
    assert got == want


def test_build_compiles_every_source_and_tracks_every_header():
    """Every translation unit under csrc/ is compiled into the library, and
    every header it includes makes the library stale when it changes."""
    from paper_1409_7764_gb300 import _build
    files = os.listdir(_build.CSRC)
    assert sorted(f for f in files if f.endswith(".cu")) == sorted(_build.SOURCES)
    assert sorted(f for f in files if f.endswith(".cuh")) == sorted(_build.HEADERS)
