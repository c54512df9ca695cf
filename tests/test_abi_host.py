"""The C-ABI library builds for sm_103a, loads, and exports every entry point declared in
include/*.h with the struct layouts the binding expects.  No GPU work is done here."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(sc_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("sc_create", "sc_destroy", "sc_build_scene", "sc_trace_camera", "sc_trace_lights",
                     "sc_resolve", "sc_sync_status", "sc_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2107_11008_gb300 import native as N

    lib = N.load()
    for name in _declared_functions():
        assert hasattr(lib, name), name
    assert set(N.SIGNATURES) >= _declared_functions()


def test_struct_layouts_and_version():
    from paper_2107_11008_gb300 import native as N

    lib = N.load()
    assert N.sc_abi_version() == 4
    sizes = (C.c_int32 * 16)()
    k = lib.sc_struct_sizes(sizes, 16)
    assert k == len(N.STRUCTS)
    assert list(sizes[:k]) == [C.sizeof(s) for s in N.STRUCTS]
    assert C.sizeof(N.sc_path_record) == 32 and C.sizeof(N.sc_light_record) == 48


def test_library_is_built_for_sm_103a():
    from paper_2107_11008_gb300 import build as B

    B.build_library()
    data = open(B.LIB, "rb").read()
    assert b"sm_103a" in data or b"sm_103" in data


def test_create_without_gpu_fails_cleanly():
    """Without a device sc_create reports an error instead of crashing."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2107_11008_gb300 import native as N

    with pytest.raises(N.ScError):
        N.sc_create(0, None)
    # a null context is rejected by every entry point
    assert N.load().sc_sync_status(None) == -1
    assert N.load().sc_trace_camera(None, None, None, None) == -1
