"""Python binding of libcontact (ctypes): argument marshalling only.

Every step of the contact path runs in the CUDA library; PyTorch only holds
device memory and provides the stream.  There is no CPU fallback: without the
compiled library or a GPU these calls raise.

    model = Contact.from_state(state)                  # contact_init
    out = model.step(pos, quat)                        # contact_step
    gpos, gquat = model.backward(gF, gT)               # contact_backward
    force, torque = contact_forces(model, pos, quat)   # torch.autograd.Function
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ECAPACITY, EDOMAIN, ETIMEOUT, ESTATE, EBOUNDS = range(9)
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ECAPACITY", 5: "EDOMAIN", 6: "ETIMEOUT",
          7: "ESTATE", 8: "EBOUNDS"}
SHARP, SMOOTH = 0, 1
FP32_TILE, FP64_PAIR = 0, 1
PAIR_OUT_COLS = 11

# every symbol the header declares (checked by the tests)
EXPORTS = ["contact_config_default", "contact_init", "contact_step", "contact_backward", "contact_check",
           "contact_clear_error", "contact_last_error", "contact_set_stream", "contact_stats",
           "contact_particle_boxes", "contact_narrow_time", "contact_damping_factor", "contact_kernels_per_step",
           "contact_kernels_per_backward", "contact_destroy", "contact_step_noalloc", "contact_step_host",
           "contact_history_get", "contact_history_set", "contact_history_reset", "contact_polytope_centroid",
           "contact_polytope_shift", "contact_fp32_ffma_rate", "contact_fp64_dfma_rate",
           "contact_adjoint_time", "contact_bounds_selftest"]


class Config(ctypes.Structure):
    _fields_ = [("n_particles", ctypes.c_int32), ("n_cells", ctypes.c_int32 * 3), ("dx", ctypes.c_double),
                ("indicator", ctypes.c_int32), ("smooth_width", ctypes.c_double),
                ("inflate", ctypes.c_double), ("damping_c", ctypes.c_double), ("precision", ctypes.c_int32),
                ("max_pairs", ctypes.c_int32), ("max_neighbors", ctypes.c_int32),
                ("max_tiles", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("narrow_events", ctypes.c_int32), ("history", ctypes.c_int32), ("friction", ctypes.c_int32),
                ("restitution", ctypes.c_double), ("mu_s", ctypes.c_double), ("mu_k", ctypes.c_double),
                ("u_k", ctypes.c_double), ("n_walls", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("walls", ctypes.c_void_p), ("wall_young", ctypes.c_void_p), ("wall_poisson", ctypes.c_void_p),
                ("box_mode", ctypes.c_int32), ("contact_resolution", ctypes.c_int32)]


class ContactError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"contact library error {STATUS.get(code, code)}: {msg}")
        self.code = code


_libs = {}


def library_path(checks: bool = False) -> str:
    return _build.LIB_CHECKS if checks else _build.LIB


def load_library(build_if_missing: bool = True, checks: bool = False):
    """Load libcontact.so, or with checks=True the checked build
    libcontact_checks.so (compiling it first when missing and nvcc exists)."""
    if checks in _libs:
        return _libs[checks]
    path = library_path(checks)
    if not os.path.exists(path):
        if not build_if_missing:
            raise ContactError(ECUDA, f"{path} not built (run __graft_entry__.build())")
        _build.build(checks=checks)
    lib = ctypes.CDLL(path)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.contact_config_default.argtypes = [ctypes.POINTER(Config), I32, P, D]
    lib.contact_config_default.restype = None
    lib.contact_init.argtypes = [ctypes.POINTER(Config), P, P, P, P, P, P, P, ctypes.POINTER(P)]
    lib.contact_init.restype = I32
    lib.contact_step.argtypes = [P] * 9
    lib.contact_step.restype = I32
    lib.contact_backward.argtypes = [P] * 5
    lib.contact_backward.restype = I32
    lib.contact_check.argtypes = [P]
    lib.contact_check.restype = I32
    lib.contact_clear_error.argtypes = [P]
    lib.contact_clear_error.restype = None
    lib.contact_last_error.argtypes = [P]
    lib.contact_last_error.restype = ctypes.c_char_p
    lib.contact_set_stream.argtypes = [P, P]
    lib.contact_set_stream.restype = I32
    lib.contact_stats.argtypes = [P, P]
    lib.contact_stats.restype = I32
    lib.contact_narrow_time.argtypes = [P, P]
    lib.contact_narrow_time.restype = I32
    lib.contact_adjoint_time.argtypes = [P, P]
    lib.contact_adjoint_time.restype = I32
    lib.contact_bounds_selftest.argtypes = [P]
    lib.contact_bounds_selftest.restype = I32
    lib.contact_particle_boxes.argtypes = [P, P]
    lib.contact_particle_boxes.restype = I32
    lib.contact_damping_factor.argtypes = [D, D]
    lib.contact_damping_factor.restype = D
    lib.contact_kernels_per_step.argtypes = [P]
    lib.contact_kernels_per_step.restype = I32
    lib.contact_kernels_per_backward.argtypes = [P]
    lib.contact_kernels_per_backward.restype = I32
    lib.contact_destroy.argtypes = [P]
    lib.contact_destroy.restype = None
    lib.contact_step_noalloc.argtypes = [ctypes.POINTER(Config)] + [P] * 12
    lib.contact_step_noalloc.restype = I32
    lib.contact_step_host.argtypes = [P] * 9
    lib.contact_step_host.restype = I32
    lib.contact_polytope_centroid.argtypes = [P, I32, P]
    lib.contact_polytope_centroid.restype = I32
    lib.contact_polytope_shift.argtypes = [P, P]
    lib.contact_polytope_shift.restype = I32
    lib.contact_fp32_ffma_rate.argtypes = [I32, P]
    lib.contact_fp32_ffma_rate.restype = I32
    lib.contact_fp64_dfma_rate.argtypes = [I32, P]
    lib.contact_fp64_dfma_rate.restype = I32
    lib.contact_history_get.argtypes = [P, ctypes.c_int64, P, P, P, P]
    lib.contact_history_get.restype = I32
    lib.contact_history_set.argtypes = [P, ctypes.c_int64, P, P, P]
    lib.contact_history_set.restype = I32
    lib.contact_history_reset.argtypes = [P]
    lib.contact_history_reset.restype = I32
    _libs[checks] = lib
    return lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return ctypes.c_void_p(t.data_ptr())
    return t.ctypes.data_as(ctypes.c_void_p)


def damping_factor(restitution: float, u0: float) -> float:
    """Eq. (damping_factor) through the library."""
    return float(load_library().contact_damping_factor(restitution, u0))


class Contact:
    """One contact context (contact_init ... contact_destroy) on a CUDA device."""

    def __init__(self, shape_type, shape_param, face_offset, planes, young, poisson, n_cells, dx,
                 indicator=SHARP, smooth_width=1.0, inflate=0.0, damping_c=0.0, precision=FP32_TILE,
                 max_pairs=None, max_neighbors=64, max_tiles=0, use_graph=True, narrow_events=False,
                 history=False, restitution=1.0, friction=False, mu_s=0.0, mu_k=0.0, u_k=1.0,
                 walls=None, wall_young=None, wall_poisson=None, box_mode=0, contact_resolution=8,
                 device=None, stream=None, checks=False):
        if not torch.cuda.is_available():
            raise ContactError(ECUDA, "no CUDA device: the contact path has no CPU fallback")
        self.lib = load_library(checks=checks)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        n = int(len(shape_type))
        cfg = Config()
        nc = (ctypes.c_int32 * 3)(*[int(v) for v in n_cells])
        self.lib.contact_config_default(ctypes.byref(cfg), n, nc, float(dx))
        cfg.indicator, cfg.smooth_width, cfg.inflate = int(indicator), float(smooth_width), float(inflate)
        cfg.damping_c, cfg.precision = float(damping_c), int(precision)
        cfg.history, cfg.restitution = int(bool(history)), float(restitution)
        cfg.friction, cfg.mu_s, cfg.mu_k, cfg.u_k = int(bool(friction)), float(mu_s), float(mu_k), float(u_k)
        wall_arrs = ()
        if walls is not None and len(walls):
            # fixed walls (m, h): read by contact_init only, alive until it returns
            wall_arrs = (np.ascontiguousarray(walls, dtype=np.float64).reshape(-1, 4),
                         np.ascontiguousarray(wall_young, dtype=np.float64).reshape(-1),
                         np.ascontiguousarray(wall_poisson, dtype=np.float64).reshape(-1))
            if not (len(wall_arrs[1]) == len(wall_arrs[2]) == len(wall_arrs[0])):
                raise ContactError(EINVAL, "walls, wall_young and wall_poisson differ in length")
            cfg.n_walls = len(wall_arrs[0])
            cfg.walls, cfg.wall_young, cfg.wall_poisson = (a.ctypes.data for a in wall_arrs)
        self.n_walls = int(cfg.n_walls)
        cfg.box_mode, cfg.contact_resolution = int(box_mode), int(contact_resolution)
        if max_pairs is not None:
            cfg.max_pairs = int(max_pairs)
        cfg.max_neighbors, cfg.max_tiles, cfg.use_graph = int(max_neighbors), int(max_tiles), int(bool(use_graph))
        cfg.narrow_events = int(narrow_events)   # False/True, or K > 1 back-to-back node sweeps
        self.cfg = cfg
        self.n = n
        self.steps = 0   # contact_step calls so far (the adjoint differentiates the last)
        self.max_pairs = int(cfg.max_pairs)
        arrs = [np.ascontiguousarray(shape_type, np.int32), np.ascontiguousarray(shape_param, np.float64),
                np.ascontiguousarray(face_offset, np.int32),
                np.ascontiguousarray(planes if len(planes) else np.zeros((1, 4)), np.float64),
                np.ascontiguousarray(young, np.float64), np.ascontiguousarray(poisson, np.float64)]
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            handle = ctypes.c_void_p()
            rc = self.lib.contact_init(ctypes.byref(cfg), *[_ptr(a) for a in arrs],
                                       ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(handle))
        if rc != OK:
            raise ContactError(rc, "contact_init rejected the configuration or shapes")
        self.ctx = handle
        dev = self.device
        self.pair_ij = torch.zeros((self.max_pairs, 2), dtype=torch.int32, device=dev)
        self.pair_out = torch.zeros((self.max_pairs, PAIR_OUT_COLS), dtype=torch.float64, device=dev)
        self.n_pairs = torch.zeros(1, dtype=torch.int32, device=dev)
        self.force = torch.zeros((n, 3), dtype=torch.float64, device=dev)
        self.torque = torch.zeros((n, 3), dtype=torch.float64, device=dev)

    @classmethod
    def from_state(cls, st, **kw):
        """Context for a workloads.State (shapes, material, lattice, indicator)."""
        args = dict(indicator=st.indicator, smooth_width=st.smooth_width, inflate=st.inflate,
                    damping_c=st.damping_c, walls=getattr(st, "walls", None),
                    wall_young=getattr(st, "wall_young", None), wall_poisson=getattr(st, "wall_poisson", None),
                    box_mode=getattr(st, "box_mode", 0), contact_resolution=getattr(st, "contact_resolution", 8))
        args.update(kw)
        return cls(st.shape_type, st.shape_param, st.face_offset, st.planes, st.young, st.poisson, st.n_cells,
                   st.dx, **args)

    # ------------------------------------------------------------------ calls
    def _raise(self, rc, what):
        msg = self.lib.contact_last_error(self.ctx).decode()
        raise ContactError(rc, f"{what}: {msg}")

    def step_host(self, pos, quat, vel=None, force=None, torque=None, pairs=False):
        """contact_step_host: host (CPU) float64 arrays in, host forces and
        torques out; returns when the results are in host memory.  Page-locked
        torch CPU tensors (pin_memory) are read and written by the step's
        kernels in place, in one captured graph.  With pairs=True the pair ids
        and outputs are copied too.  A call with the same tensor objects as the
        previous one (the usual loop over reused buffers) skips their checks."""
        fast = getattr(self, "_host_fast", None)
        if fast is not None and not pairs and fast[0] == (id(pos), id(quat), id(vel), id(force), id(torque)) \
                and fast[1] == (pos.data_ptr(), quat.data_ptr(), force.data_ptr(), torque.data_ptr()):
            rc = self.lib.contact_step_host(self.ctx, *fast[2])
            self.steps += 1
            if rc != OK:
                self._raise(rc, "contact_step_host")
            return dict(force=force, torque=torque, n_pairs=int(fast[3][0]))
        out = self._step_host_checked(pos, quat, vel, force, torque, pairs)
        return out

    def _step_host_checked(self, pos, quat, vel, force, torque, pairs):
        given = (pos, quat, vel, force, torque)

        def host(t, shape):
            if not isinstance(t, torch.Tensor) or t.dtype != torch.float64:
                t = torch.as_tensor(t, dtype=torch.float64)
            if t.is_cuda or t.shape != shape or not t.is_contiguous():
                raise ContactError(EINVAL, f"step_host: expected a contiguous CPU float64 array of shape {shape}")
            return t
        s3, s4, s6 = torch.Size((self.n, 3)), torch.Size((self.n, 4)), torch.Size((self.n, 6))
        pos = host(pos, s3)
        quat = host(quat, s4)
        vel = host(vel, s6) if vel is not None else None
        force = torch.empty(s3, dtype=torch.float64) if force is None else host(force, s3)
        torque = torch.empty(s3, dtype=torch.float64) if torque is None else host(torque, s3)
        pin = force.is_pinned()
        if getattr(self, "_host_np", {}).get(pin) is None:   # reused across calls (a pinned allocation is slow)
            self._host_np = dict(getattr(self, "_host_np", {}))
            self._host_np[pin] = torch.zeros(1, dtype=torch.int32, pin_memory=pin)
        n_pairs = self._host_np[pin]
        pij = torch.empty((self.max_pairs, 2), dtype=torch.int32) if pairs else None
        pout = torch.empty((self.max_pairs, 11), dtype=torch.float64) if pairs else None
        args = (ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(quat.data_ptr()),
                ctypes.c_void_p(vel.data_ptr() if vel is not None else 0),
                ctypes.c_void_p(n_pairs.data_ptr()), ctypes.c_void_p(force.data_ptr()),
                ctypes.c_void_p(torque.data_ptr()),
                ctypes.c_void_p(pij.data_ptr() if pairs else 0),
                ctypes.c_void_p(pout.data_ptr() if pairs else 0))
        rc = self.lib.contact_step_host(self.ctx, *args)
        self.steps += 1
        if rc != OK:
            self._raise(rc, "contact_step_host")
        # the same tensor objects next time: reuse the checked arguments (the
        # cache holds the tensors, so their ids stay theirs)
        if not pairs and all(a is b for a, b in zip((pos, quat, vel, force, torque), given)):
            self._host_fast = ((id(pos), id(quat), id(vel), id(force), id(torque)),
                               (pos.data_ptr(), quat.data_ptr(), force.data_ptr(), torque.data_ptr()), args,
                               n_pairs.numpy(), given)
        else:
            self._host_fast = None
        out = dict(force=force, torque=torque, n_pairs=int(n_pairs.item()))
        if pairs:
            P = min(out["n_pairs"], self.max_pairs)
            out.update(pair_ij=pij[:P], pair_out=pout[:P])
        return out

    def step_async(self, pos, quat, vel=None):
        """Enqueue contact_step on the context stream (outputs in self.*)."""
        for t in (pos, quat) + ((vel,) if vel is not None else ()):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise ContactError(EINVAL, "pos/quat/vel must be contiguous float64 CUDA tensors")
        if pos.shape != (self.n, 3) or quat.shape != (self.n, 4):
            raise ContactError(EINVAL, "pos must be [N,3] and quat [N,4]")
        rc = self.lib.contact_step(self.ctx, _ptr(pos), _ptr(quat), _ptr(vel), _ptr(self.pair_ij),
                                   _ptr(self.pair_out), _ptr(self.n_pairs), _ptr(self.force), _ptr(self.torque))
        self.steps += 1
        if rc != OK:
            self._raise(rc, "contact_step")

    def step(self, pos, quat, vel=None, check=True):
        """contact_step; waits for the result when check is True."""
        cur = torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cur)
        self.step_async(pos, quat, vel)
        cur.wait_stream(self.stream)
        if check:
            self.check()
        P = int(self.n_pairs.item())
        P = min(P, self.max_pairs)
        return dict(pair_ij=self.pair_ij[:P], pair_out=self.pair_out[:P], force=self.force, torque=self.torque,
                    n_pairs=P)

    def backward(self, grad_force, grad_torque, check=True):
        gp = torch.zeros((self.n, 3), dtype=torch.float64, device=self.device)
        gq = torch.zeros((self.n, 4), dtype=torch.float64, device=self.device)
        cur = torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cur)
        rc = self.lib.contact_backward(self.ctx, _ptr(grad_force.contiguous()), _ptr(grad_torque.contiguous()),
                                       _ptr(gp), _ptr(gq))
        if rc != OK:
            self._raise(rc, "contact_backward")
        cur.wait_stream(self.stream)
        if check:
            self.check()
        return gp, gq

    def check(self):
        rc = self.lib.contact_check(self.ctx)
        if rc != OK:
            self._raise(rc, "device error")

    def clear_error(self):
        self.lib.contact_clear_error(self.ctx)

    def stats(self):
        s = (ctypes.c_int64 * 10)()
        rc = self.lib.contact_stats(self.ctx, s)
        if rc != OK:
            self._raise(rc, "contact_stats")
        keys = ["pairs", "cells", "tiles", "overlapping", "kernels", "narrow_grid", "bins_x", "replayed",
                "nominal_ops", "max_tiles"]
        return dict(zip(keys, [int(v) for v in s]))

    def adjoint_time_ms(self) -> float:
        """Device time of the last backward's cell-sweep kernel (CUDA events)."""
        ms = ctypes.c_float()
        rc = self.lib.contact_adjoint_time(self.ctx, ctypes.byref(ms))
        if rc != OK:
            self._raise(rc, "contact_adjoint_time")
        return float(ms.value)

    def narrow_time_ms(self) -> float:
        """Device time of the last step's node-sweep kernel (CUDA events)."""
        ms = ctypes.c_float()
        rc = self.lib.contact_narrow_time(self.ctx, ctypes.byref(ms))
        if rc != OK:
            self._raise(rc, "contact_narrow_time")
        return float(ms.value)

    def particle_boxes(self):
        out = torch.zeros((self.n, 6), dtype=torch.int32, device=self.device)
        rc = self.lib.contact_particle_boxes(self.ctx, _ptr(out))
        if rc != OK:
            self._raise(rc, "contact_particle_boxes")
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return out

    def polytope_shift(self):
        """[N,3] float64 host: the offset by which each polytope's body origin
        was moved to its volume centroid (zero where it already was);
        positions name the centroid."""
        out = np.zeros((self.n, 3))
        rc = self.lib.contact_polytope_shift(self.ctx, out.ctypes.data)
        if rc != OK:
            self._raise(rc, "contact_polytope_shift")
        return out

    def history(self, boxes: bool = False):
        """Contact history after the last step: (ij [H,2] int32, c [H] float64)
        host arrays sorted by (i, j); with boxes=True also box [H,6] float64,
        each contact's corrected box minus X_i (the box pipeline's warm start;
        zeros in the default sample set)."""
        n = ctypes.c_int64()
        rc = self.lib.contact_history_get(self.ctx, 0, None, None, None, ctypes.byref(n))
        if rc != OK:
            self._raise(rc, "contact_history_get")
        ij = np.zeros((n.value, 2), dtype=np.int32)
        c = np.zeros(n.value, dtype=np.float64)
        box = np.zeros((n.value, 6), dtype=np.float64)
        rc = self.lib.contact_history_get(self.ctx, n.value, ij.ctypes.data, c.ctypes.data, box.ctypes.data,
                                          ctypes.byref(n))
        if rc != OK:
            self._raise(rc, "contact_history_get")
        return (ij, c, box) if boxes else (ij, c)

    def set_history(self, ij, c, box=None):
        """Replace the contact history (e.g. from a checkpoint); box [H,6] is
        required with the box pipeline."""
        ij = np.ascontiguousarray(ij, dtype=np.int32).reshape(-1, 2)
        c = np.ascontiguousarray(c, dtype=np.float64).reshape(-1)
        if len(c) != len(ij):
            raise ContactError(EINVAL, "ij and c differ in length")
        bp = None
        if box is not None:
            box = np.ascontiguousarray(box, dtype=np.float64).reshape(-1, 6)
            if len(box) != len(ij):
                raise ContactError(EINVAL, "ij and box differ in length")
            bp = box.ctypes.data
        rc = self.lib.contact_history_set(self.ctx, len(c), ij.ctypes.data, c.ctypes.data, bp)
        if rc != OK:
            self._raise(rc, "contact_history_set")

    def reset_history(self):
        rc = self.lib.contact_history_reset(self.ctx)
        if rc != OK:
            self._raise(rc, "contact_history_reset")

    def kernels_per_step(self):
        return int(self.lib.contact_kernels_per_step(self.ctx))

    def kernels_per_backward(self):
        return int(self.lib.contact_kernels_per_backward(self.ctx))

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.contact_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def polytope_centroid(planes) -> np.ndarray:
    """Volume centroid of the polytope n . y <= d (rows (n, d), unit n, d > 0).
    Poses refer to the centre of mass: contact_init moves a polytope whose
    centroid is off its body origin there (d -= n . centroid; see
    Contact.polytope_shift), so positions name the centroid."""
    lib = load_library()
    pl = np.ascontiguousarray(planes, dtype=np.float64).reshape(-1, 4)
    c = np.zeros(3)
    rc = lib.contact_polytope_centroid(pl.ctypes.data, len(pl), c.ctypes.data)
    if rc != OK:
        raise ContactError(rc, "contact_polytope_centroid: invalid planes")
    return c


class ContactFunction(torch.autograd.Function):
    """(pos, quat, vel) -> (force, torque, pair_ij, pair_out) with the
    library's adjoint as backward.  vel (or None) enters the damping and the
    friction and is not differentiated; the pair outputs carry no gradient."""

    @staticmethod
    def forward(ctx, model, pos, quat, vel):
        v = None if vel is None else vel.detach().to(torch.float64).contiguous()
        out = model.step(pos.detach().to(torch.float64).contiguous(), quat.detach().to(torch.float64).contiguous(), v)
        ctx.model = model
        ctx.step_id = model.steps
        ctx.vel = v   # the adjoint reads the step's velocities: they stay alive until backward
        pij, pout = out["pair_ij"].clone(), out["pair_out"].clone()
        ctx.mark_non_differentiable(pij, pout)
        return out["force"].clone(), out["torque"].clone(), pij, pout

    @staticmethod
    def backward(ctx, gF, gT, _g_ij, _g_out):
        if ctx.model.steps != ctx.step_id:
            raise RuntimeError("contact_forces: the model stepped again after this forward; the adjoint "
                               "differentiates the model's last step only")
        gp, gq = ctx.model.backward(gF.to(torch.float64).contiguous(), gT.to(torch.float64).contiguous())
        return None, gp, gq, None


def contact_forces(model: Contact, pos: torch.Tensor, quat: torch.Tensor, vel: torch.Tensor = None,
                   pairs: bool = False):
    """Per-particle contact force and torque [N,3], differentiable w.r.t. pos
    and quat (smoothed indicator).  vel [N,6] (v, omega), if given, drives the
    damping and friction (not differentiated).  With pairs=True also returns
    dict(pair_ij [P,2], pair_out [P,11]) of the step.  A backward must come
    before the model's next step."""
    force, torque, pij, pout = ContactFunction.apply(model, pos, quat, vel)
    if pairs:
        return force, torque, dict(pair_ij=pij, pair_out=pout)
    return force, torque


def fp32_ffma_rate(iters: int = 2000) -> float:
    """Measured FP32 FFMA lane-operations per second of the current device
    (contact_fp32_ffma_rate): the counterpart of the roofline's derived peak."""
    lib = load_library()
    out = ctypes.c_double()
    rc = lib.contact_fp32_ffma_rate(int(iters), ctypes.byref(out))
    if rc != OK:
        raise ContactError(rc, "contact_fp32_ffma_rate")
    return out.value


def fp64_dfma_rate(iters: int = 50) -> float:
    """Measured FP64 DFMA lane-operations per second of the current device
    (contact_fp64_dfma_rate): the peak of the all-FP64 comparison form."""
    lib = load_library()
    out = ctypes.c_double()
    rc = lib.contact_fp64_dfma_rate(int(iters), ctypes.byref(out))
    if rc != OK:
        raise ContactError(rc, "contact_fp64_dfma_rate")
    return out.value
