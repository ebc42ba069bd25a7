"""The C-ABI library loads and exports every symbol include/contact.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2401_10878_gb300 import build
from paper_2401_10878_gb300.contact import EXPORTS

HEADER = os.path.join(os.path.dirname(__file__), "..", "include", "contact.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(contact_[a-z0-9_]+)\s*\(", src)))


def test_header_declarations_match_binding():
    assert declared() == sorted(EXPORTS)


def test_library_exports_every_declared_symbol():
    try:
        path = build.build()
    except RuntimeError as e:
        pytest.skip(f"nvcc unavailable: {e}")
    lib = ctypes.CDLL(path)
    for name in declared():
        assert hasattr(lib, name), name
    # a pure host entry point can be called without a GPU
    lib.contact_damping_factor.restype = ctypes.c_double
    lib.contact_damping_factor.argtypes = [ctypes.c_double, ctypes.c_double]
    assert lib.contact_damping_factor(1.0, 2.0) == 0.0
    assert abs(lib.contact_damping_factor(0.0, 1.0) - 16.5) < 1e-15


def test_config_struct_layout():
    from paper_2401_10878_gb300.contact import Config
    # int32 + int32[3] (16), double dx (24), int32 + pad (32), 3 doubles (56),
    # 8 int32 (88), 4 doubles (120), 2 int32 (128), 3 pointers (152),
    # 2 int32 (160): 160 bytes
    assert ctypes.sizeof(Config) == 160
    assert Config.dx.offset == 16 and Config.smooth_width.offset == 32 and Config.precision.offset == 56
