"""CPU FP64 oracle of the contact hot path (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
(``bench.py``'s ``cpu_baseline`` and ``--impl reference``) may import this
package.  The CUDA library never does, and no product code path falls back to
it.  The C++ source is ``contact_oracle.cpp``; ``build()`` compiles it with g++.

Paper: Marquardt, Hafen, Krause, arXiv:2401.10878 -- Sec. 2.3 (force law,
Eq. contact_force_normal, E*, Eq. damping_factor), Sec. 3.3.1 (overlap sweep),
Sec. 3.3.2 (periodic images).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "contact_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

BAND_EPS = 1e-5   # lattice units: classification band of the parity checks


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (g++, OpenMP when available)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", _SRC]
    tmp = _LIB + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp], check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Law(ctypes.Structure):
    _fields_ = [("restitution", ctypes.c_double), ("mu_s", ctypes.c_double), ("mu_k", ctypes.c_double),
                ("u_k", ctypes.c_double), ("history", ctypes.c_int32), ("friction", ctypes.c_int32)]


class _Cfg(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int32 * 3), ("dx", ctypes.c_double), ("indicator", ctypes.c_int32),
                ("smooth_width", ctypes.c_double), ("inflate", ctypes.c_double),
                ("damping_c", ctypes.c_double), ("band_eps", ctypes.c_double),
                ("n_walls", ctypes.c_int32), ("walls", ctypes.c_void_p), ("wall_young", ctypes.c_void_p),
                ("wall_poisson", ctypes.c_void_p), ("box_mode", ctypes.c_int32),
                ("contact_resolution", ctypes.c_int32)]


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _configure(ctypes.CDLL(_LIB))
    return _lib


def _configure(lib):
    """Argument and return types of the oracle's C entry points on a loaded
    library (the tests that plant mistakes configure their variants with it)."""
    P = ctypes.c_void_p
    lib.oracle_contact_step.restype = ctypes.c_int64
    lib.oracle_contact_step.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int32] + [P] * 9 + \
        [ctypes.c_int64] + [P] * 7 + [ctypes.c_int64, P, P, ctypes.c_int32]
    lib.oracle_contact_step_ext.restype = ctypes.c_int64
    lib.oracle_contact_step_ext.argtypes = [ctypes.POINTER(_Cfg), ctypes.POINTER(_Law), ctypes.c_int32] + \
        [P] * 9 + [ctypes.c_int64] + [P] * 5 + [ctypes.c_int64, P, P, P, ctypes.c_int64, P, P, P, P, ctypes.c_int32]
    lib.oracle_gradient_ext.restype = ctypes.c_int64
    lib.oracle_gradient_ext.argtypes = [ctypes.POINTER(_Cfg), ctypes.POINTER(_Law), ctypes.c_int32] + \
        [P] * 9 + [ctypes.c_int64] + [P] * 6 + [ctypes.c_int32]
    lib.oracle_box_pipeline.restype = ctypes.c_int64
    lib.oracle_box_pipeline.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int32] + [P] * 8 + \
        [ctypes.c_int64, P, P, ctypes.c_int64] + [P] * 3
    lib.oracle_polytope_centroid.restype = ctypes.c_int32
    lib.oracle_polytope_centroid.argtypes = [P, ctypes.c_int32, P]
    lib.oracle_gradient.restype = ctypes.c_int64
    lib.oracle_gradient.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int32] + [P] * 13 + [ctypes.c_int32]
    lib.oracle_polytope_shift.restype = ctypes.c_int32
    lib.oracle_polytope_shift.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int32] + [P] * 9
    lib.oracle_aabb.restype = ctypes.c_int32
    lib.oracle_aabb.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int32] + [P] * 9
    lib.oracle_rotation.restype = None
    lib.oracle_rotation.argtypes = [P, P]
    lib.oracle_effective_modulus.restype = ctypes.c_double
    lib.oracle_effective_modulus.argtypes = [ctypes.c_double] * 4
    lib.oracle_damping_factor.restype = ctypes.c_double
    lib.oracle_damping_factor.argtypes = [ctypes.c_double] * 2
    lib.oracle_normal_force.restype = ctypes.c_double
    lib.oracle_normal_force.argtypes = [ctypes.c_double] * 5
    lib.oracle_polytope_vertices.restype = ctypes.c_int32
    lib.oracle_polytope_vertices.argtypes = [ctypes.c_int32, P, ctypes.c_double, ctypes.c_int32, P]
    lib.oracle_max_threads.restype = ctypes.c_int32
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _cfg(st, band_eps=BAND_EPS):
    c = _Cfg()
    for k in range(3):
        c.n_cells[k] = int(st.n_cells[k])
    c.dx, c.indicator, c.smooth_width = float(st.dx), int(st.indicator), float(st.smooth_width)
    c.inflate, c.damping_c, c.band_eps = float(st.inflate), float(st.damping_c), float(band_eps)
    c.box_mode = int(getattr(st, "box_mode", 0))
    c.contact_resolution = int(getattr(st, "contact_resolution", 8))
    walls = getattr(st, "walls", None)
    if walls is not None and len(walls):
        arrs = (_c(np.asarray(walls).reshape(-1, 4), np.float64), _c(st.wall_young, np.float64),
                _c(st.wall_poisson, np.float64))
        c.n_walls = len(arrs[0])
        c.walls, c.wall_young, c.wall_poisson = (a.ctypes.data for a in arrs)
        c._keep = arrs   # the arrays live as long as the struct
    return c


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle rejected the input (status {code})")
        self.code = code


def _shape_arrays(st):
    planes = st.planes if len(st.planes) else np.zeros((1, 4))
    return (_c(st.shape_type, np.int32), _c(st.shape_param, np.float64), _c(st.face_offset, np.int32),
            _c(planes, np.float64), _c(st.young, np.float64), _c(st.poisson, np.float64))


@dataclasses.dataclass
class Result:
    pair_ij: np.ndarray     # [P,2] int32, sorted by (i, j), i < j
    pair_shift: np.ndarray  # [P,3] int32 image index s of j (X_j' = X_j - s L)
    pair_box: np.ndarray    # [P,6] int32 node box lo, hi
    pair_out: np.ndarray    # [P,11] V, x_c[3], n[3], d, F[3] (force on j)
    pair_aux: np.ndarray    # [P,11] G[3], box cells, ambiguous cells, ambiguous normal cells, depth gap,
    #                         E*, sensitivities of V, moments, G to an eps change of every phi
    force: np.ndarray       # [N,3]
    torque: np.ndarray      # [N,3]
    seconds: float = 0.0
    threads: int = 1

    @property
    def n_pairs(self):
        return int(self.pair_ij.shape[0])

    @property
    def cells(self):
        return int(self.pair_aux[:, 3].sum())


def contact_step(st, pos=None, quat=None, vel=None, n_threads: int = 0, band_eps: float = BAND_EPS,
                 hist=None) -> Result:
    """Evaluate every candidate pair of the state (see contact_oracle.cpp);
    with the box pipeline, hist = (hist_ij, hist_c, hist_box) of the previous
    step gives the ongoing contacts' warm starts (the shared damping c stays)."""
    lib = _load()
    hij = np.zeros((0, 2), np.int32) if hist is None else _c(hist[0], np.int32)
    hb = None if hist is None or len(hist) < 3 or hist[2] is None else _c(hist[2], np.float64)
    pos = _c(st.pos if pos is None else pos, np.float64)
    quat = _c(st.quat if quat is None else quat, np.float64)
    vel = None if vel is None else _c(vel, np.float64)
    arrs = _shape_arrays(st)
    cfg = _cfg(st, band_eps)
    n = st.n
    cap = max(16, 16 * n)
    threads = n_threads if n_threads > 0 else lib.oracle_max_threads()
    while True:
        ij = np.zeros((cap, 2), np.int32)
        sh = np.zeros((cap, 3), np.int32)
        bx = np.zeros((cap, 6), np.int32)
        out = np.zeros((cap, 11))
        aux = np.zeros((cap, 11))
        f = np.zeros((n, 3))
        t = np.zeros((n, 3))
        t0 = time.perf_counter()
        P = lib.oracle_contact_step(ctypes.byref(cfg), n, *[_ptr(a) for a in arrs], _ptr(pos), _ptr(quat),
                                    _ptr(vel), cap, _ptr(ij), _ptr(sh), _ptr(bx), _ptr(out), _ptr(aux),
                                    _ptr(f), _ptr(t), len(hij), _ptr(hij), _ptr(hb), threads)
        dt = time.perf_counter() - t0
        if P < 0:
            raise OracleError(-P)
        if P <= cap:
            return Result(ij[:P], sh[:P], bx[:P], out[:P], aux[:P], f, t, dt, threads)
        cap = int(P)


@dataclasses.dataclass
class ContactLaw:
    """The contact law's extensions: contact history (each contact keeps the
    damping factor of Eq. (damping_factor) computed from its approach speed at
    its first step, with coefficient of restitution `restitution`) and the
    friction of Eq. (contact_force_tangential) with mu_s, mu_k and u_k."""
    restitution: float = 1.0
    mu_s: float = 0.0
    mu_k: float = 0.0
    u_k: float = 1.0
    history: bool = False
    friction: bool = False


@dataclasses.dataclass
class ExtResult:
    pair_ij: np.ndarray
    pair_out: np.ndarray
    pair_c: np.ndarray
    force: np.ndarray
    torque: np.ndarray
    hist_ij: np.ndarray     # this step's contacts (V > 0), sorted by (i, j)
    hist_c: np.ndarray
    hist_box: np.ndarray    # [H,6] their corrected boxes relative to X_i (box pipeline; zeros otherwise)

    @property
    def n_pairs(self):
        return len(self.pair_ij)


def contact_step_ext(st, law: ContactLaw, pos=None, quat=None, vel=None, hist=None, n_threads: int = 0) -> ExtResult:
    """The contact step with friction and the contact history; hist is the
    previous step's (hist_ij, hist_c) or (hist_ij, hist_c, hist_box), or None
    (no ongoing contact).  hist_box [H,6] (the box pipeline's warm start) is
    each contact's corrected box relative to the lower-ID particle's position."""
    lib = _load()
    pos = _c(st.pos if pos is None else pos, np.float64)
    quat = _c(st.quat if quat is None else quat, np.float64)
    vel = None if vel is None else _c(vel, np.float64)
    arrs = _shape_arrays(st)
    cfg = _cfg(st, BAND_EPS)
    lw = _Law(law.restitution, law.mu_s, law.mu_k, law.u_k, int(law.history), int(law.friction))
    hij = np.zeros((0, 2), np.int32) if hist is None else _c(hist[0], np.int32)
    hc = np.zeros(0) if hist is None else _c(hist[1], np.float64)
    hb = None if hist is None or len(hist) < 3 or hist[2] is None else _c(hist[2], np.float64)
    n = st.n
    cap = max(16, 16 * n)
    threads = n_threads if n_threads > 0 else lib.oracle_max_threads()
    while True:
        ij = np.zeros((cap, 2), np.int32)
        out = np.zeros((cap, 11))
        pc = np.zeros(cap)
        f = np.zeros((n, 3))
        t = np.zeros((n, 3))
        hij_o = np.zeros((cap, 2), np.int32)
        hc_o = np.zeros(cap)
        hb_o = np.zeros((cap, 6))
        nh = ctypes.c_int64(0)
        P = lib.oracle_contact_step_ext(ctypes.byref(cfg), ctypes.byref(lw), n, *[_ptr(a) for a in arrs],
                                        _ptr(pos), _ptr(quat), _ptr(vel), cap, _ptr(ij), _ptr(out), _ptr(pc),
                                        _ptr(f), _ptr(t), len(hc), _ptr(hij), _ptr(hc), _ptr(hb), cap, _ptr(hij_o),
                                        _ptr(hc_o), _ptr(hb_o), ctypes.byref(nh), threads)
        if P < 0:
            raise OracleError(-P)
        if P <= cap:
            H = nh.value
            return ExtResult(ij[:P], out[:P], pc[:P], f, t, hij_o[:H], hc_o[:H], hb_o[:H])
        cap = int(P)


def gradient(st, grad_force, grad_torque, pos=None, quat=None, vel=None, n_threads: int = 0):
    """Oracle FP64 gradient of sum_p (gF_p.F_p + gT_p.T_p) w.r.t. positions and raw quaternions."""
    lib = _load()
    pos = _c(st.pos if pos is None else pos, np.float64)
    quat = _c(st.quat if quat is None else quat, np.float64)
    vel = None if vel is None else _c(vel, np.float64)
    arrs = _shape_arrays(st)
    gp = np.zeros((st.n, 3))
    gq = np.zeros((st.n, 4))
    threads = n_threads if n_threads > 0 else lib.oracle_max_threads()
    P = lib.oracle_gradient(ctypes.byref(_cfg(st)), st.n, *[_ptr(a) for a in arrs], _ptr(pos), _ptr(quat),
                            _ptr(vel), _ptr(_c(grad_force, np.float64)), _ptr(_c(grad_torque, np.float64)),
                            _ptr(gp), _ptr(gq), threads)
    if P < 0:
        raise OracleError(-P)
    return gp, gq


def gradient_ext(st, law: ContactLaw, grad_force, grad_torque, pos=None, quat=None, vel=None, table=None,
                 n_threads: int = 0):
    """Oracle gradient with friction and, with the history on, each contact's
    damping factor from table = (ij [H,2] sorted, c [H]) held fixed."""
    lib = _load()
    pos = _c(st.pos if pos is None else pos, np.float64)
    quat = _c(st.quat if quat is None else quat, np.float64)
    vel = None if vel is None else _c(vel, np.float64)
    arrs = _shape_arrays(st)
    lw = _Law(law.restitution, law.mu_s, law.mu_k, law.u_k, int(law.history), int(law.friction))
    hij = np.zeros((0, 2), np.int32) if table is None else _c(table[0], np.int32)
    hc = np.zeros(0) if table is None else _c(table[1], np.float64)
    gp = np.zeros((st.n, 3))
    gq = np.zeros((st.n, 4))
    threads = n_threads if n_threads > 0 else lib.oracle_max_threads()
    P = lib.oracle_gradient_ext(ctypes.byref(_cfg(st)), ctypes.byref(lw), st.n, *[_ptr(a) for a in arrs], _ptr(pos),
                                _ptr(quat), _ptr(vel), len(hc), _ptr(hij), _ptr(hc),
                                _ptr(_c(grad_force, np.float64)), _ptr(_c(grad_torque, np.float64)), _ptr(gp),
                                _ptr(gq), threads)
    if P < 0:
        raise OracleError(-P)
    return gp, gq


def box_pipeline(st, pos=None, quat=None, hist=None):
    """The box pipeline's rough boxes [P,6] (node indices), corrected boxes
    [P,6] (physical) and flags [P,2] per candidate pair (st.box_mode = 1);
    hist = (hist_ij, hist_c, hist_box) of the previous step gives the warm
    starts of the ongoing contacts."""
    lib = _load()
    pos = _c(st.pos if pos is None else pos, np.float64)
    quat = _c(st.quat if quat is None else quat, np.float64)
    hij = np.zeros((0, 2), np.int32) if hist is None else _c(hist[0], np.int32)
    hb = None if hist is None or len(hist) < 3 or hist[2] is None else _c(hist[2], np.float64)
    cap = max(16, 16 * st.n)
    while True:
        rough = np.zeros((cap, 6), np.int32)
        box = np.zeros((cap, 6))
        flags = np.zeros((cap, 2))
        P = lib.oracle_box_pipeline(ctypes.byref(_cfg(st)), st.n, *[_ptr(a) for a in _shape_arrays(st)], _ptr(pos),
                                    _ptr(quat), len(hij), _ptr(hij), _ptr(hb), cap, _ptr(rough), _ptr(box),
                                    _ptr(flags))
        if P < 0:
            raise OracleError(-P)
        if P <= cap:
            return rough[:P], box[:P], flags[:P]
        cap = int(P)


def polytope_centroid(planes):
    """Volume centroid of the polytope n . y <= d (rows (n, d), origin inside)."""
    lib = _load()
    pl = _c(np.asarray(planes, float).reshape(-1, 4), np.float64)
    c = np.zeros(3)
    rc = lib.oracle_polytope_centroid(_ptr(pl), len(pl), _ptr(c))
    if rc != 0:
        raise OracleError(rc)
    return c


def polytope_shift(st):
    """Per particle [N,3]: the offset by which a polytope's body origin is
    moved to its volume centroid (zero where it already is, within 1e-6 x the
    smallest face offset); positions then name the centroid."""
    lib = _load()
    out = np.zeros((st.n, 3))
    rc = lib.oracle_polytope_shift(ctypes.byref(_cfg(st)), st.n, *[_ptr(a) for a in _shape_arrays(st)],
                                   _ptr(_c(st.pos, np.float64)), _ptr(_c(st.quat, np.float64)), _ptr(out))
    if rc != 0:
        raise OracleError(rc)
    return out


def aabb(st, pos=None, quat=None):
    """Per-particle node ranges [N,6] (lo, hi)."""
    lib = _load()
    pos = _c(st.pos if pos is None else pos, np.float64)
    quat = _c(st.quat if quat is None else quat, np.float64)
    out = np.zeros((st.n, 6), np.int32)
    rc = lib.oracle_aabb(ctypes.byref(_cfg(st)), st.n, *[_ptr(a) for a in _shape_arrays(st)], _ptr(pos),
                         _ptr(quat), _ptr(out))
    if rc != 0:
        raise OracleError(rc)
    return out


def rotation(q):
    R = np.zeros(9)
    _load().oracle_rotation(_ptr(_c(q, np.float64)), _ptr(R))
    return R.reshape(3, 3)


def effective_modulus(EA, nuA, EB, nuB):
    return _load().oracle_effective_modulus(EA, nuA, EB, nuB)


def damping_factor(e, u0):
    return _load().oracle_damping_factor(e, u0)


def normal_force(estar, V, d, c=0.0, ddot=0.0):
    return _load().oracle_normal_force(estar, V, d, c, ddot)


def polytope_vertices(planes, delta=0.0):
    planes = _c(planes, np.float64)
    cap = 4096
    out = np.zeros((cap, 3))
    nv = _load().oracle_polytope_vertices(len(planes), _ptr(planes), float(delta), cap, _ptr(out))
    if nv < 0:
        raise OracleError(1)
    return out[:nv]


def max_threads():
    return int(_load().oracle_max_threads())
