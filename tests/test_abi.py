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


def test_init_refuses_domains_before_touching_the_device():
    """contact_init's domain checks run on the host before any CUDA call: a
    periodic box not above 4 R_max + 2 dx, and a particle whose node range could
    reach 2^16 nodes along an axis (the node sweep packs node offsets in 16
    bits), both return CONTACT_EDOMAIN with no context."""
    try:
        path = build.build()
    except RuntimeError as e:
        pytest.skip(f"nvcc unavailable: {e}")
    from paper_2401_10878_gb300.contact import EDOMAIN, Config
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.contact_config_default.argtypes = [ctypes.POINTER(Config), ctypes.c_int32, P, ctypes.c_double]
    lib.contact_config_default.restype = None
    lib.contact_init.argtypes = [ctypes.POINTER(Config), P, P, P, P, P, P, P, ctypes.POINTER(P)]
    lib.contact_init.restype = ctypes.c_int32
    import numpy as np

    def init(radius, cells):
        cfg = Config()
        nc = (ctypes.c_int32 * 3)(cells, cells, cells)
        lib.contact_config_default(ctypes.byref(cfg), 1, nc, 1.0)
        arrs = [np.zeros(1, np.int32), np.array([radius, 0.0, 0.0]), np.zeros(2, np.int32),
                np.zeros(4), np.full(1, 5e3), np.full(1, 0.3)]
        out = P(1)
        rc = lib.contact_init(ctypes.byref(cfg), *[a.ctypes.data_as(P) for a in arrs], None, ctypes.byref(out))
        return rc, out.value

    assert init(10.0, 41) == (EDOMAIN, None)          # L = 41 <= 4 * 10 + 2
    assert init(40000.0, 200000) == (EDOMAIN, None)   # 2 R / dx + 4 >= 65535
