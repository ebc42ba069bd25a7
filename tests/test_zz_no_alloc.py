"""contact_step_noalloc (needs a GB300): the context-free entry point for
callers that cannot allocate device memory -- e.g. a host program whose own
pool allocator owns all device memory, or a loop that may not call the
driver's allocator between steps.  Its scratch is a static device array, so
two calls in a row must each match contact_step on the same inputs.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2401_10878_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(lib, model, st, pos, quat):
    from paper_2401_10878_gb300.contact import Config
    cfg = Config()
    ctypes.memmove(ctypes.byref(cfg), ctypes.byref(model.cfg), ctypes.sizeof(Config))
    dev = model.device
    out = dict(pair_ij=torch.zeros((model.max_pairs, 2), dtype=torch.int32, device=dev),
               pair_out=torch.zeros((model.max_pairs, 11), dtype=torch.float64, device=dev),
               n_pairs=torch.zeros(1, dtype=torch.int32, device=dev),
               force=torch.zeros((st.n, 3), dtype=torch.float64, device=dev),
               torque=torch.zeros((st.n, 3), dtype=torch.float64, device=dev))
    host = [np.ascontiguousarray(st.shape_type, np.int32), np.ascontiguousarray(st.shape_param, np.float64),
            np.ascontiguousarray(st.young, np.float64), np.ascontiguousarray(st.poisson, np.float64)]
    s = torch.cuda.current_stream(dev)
    rc = lib.contact_step_noalloc(ctypes.byref(cfg), *[a.ctypes.data_as(ctypes.c_void_p) for a in host],
                                  ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(quat.data_ptr()),
                                  *[ctypes.c_void_p(out[k].data_ptr()) for k in
                                    ("pair_ij", "pair_out", "n_pairs", "force", "torque")],
                                  ctypes.c_void_p(s.cuda_stream))
    return rc, out


@pytest.mark.parametrize("name", ["mixed27", "cubes1934"])
def test_noalloc_matches_contact_step_twice(name):
    from paper_2401_10878_gb300.contact import Contact
    st = W.mixed_grid_27() if name == "mixed27" else W.settling_cubes_dense()
    st.indicator = 0
    model = Contact.from_state(st, max_pairs=8192)
    seq_p, seq_q = W.pose_sequence(st, 2)
    for call in range(2):      # two calls in a row share the static scratch
        pos = torch.tensor(seq_p[call], device="cuda")
        quat = torch.tensor(seq_q[call], device="cuda")
        ref = model.step(pos, quat)
        rc, out = _noalloc(model.lib, model, st, pos, quat)
        assert rc == 0, rc
        P = int(out["n_pairs"].item())
        assert P == ref["n_pairs"] > 0
        assert torch.equal(out["pair_ij"][:P], ref["pair_ij"])
        # tolerance of the FP32-tile parity tests (1e-5 relative on forces and
        # torques, 1e-6 on volumes); both paths run the same deterministic kernels
        po, pr = out["pair_out"][:P].cpu().numpy(), ref["pair_out"].cpu().numpy()
        assert np.allclose(po[:, 0], pr[:, 0], rtol=1e-6, atol=0)
        scale = np.abs(pr[:, 8:11]).max()
        assert np.abs(po - pr).max() <= 1e-5 * max(scale, 1.0)
        for k in ("force", "torque"):
            a, b = out[k].cpu().numpy(), ref[k].cpu().numpy()
            assert np.abs(a - b).max() <= 1e-5 * max(np.abs(b).max(), 1.0)
    model.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2401_10878_gb300.contact import Config, EINVAL, load_library
    lib = load_library()
    st = W.mixed_grid_27()
    cfg = Config()
    nc = (ctypes.c_int32 * 3)(*st.n_cells)
    lib.contact_config_default(ctypes.byref(cfg), 4096, nc, 1.0)   # more particles than the maximum
    dummy = torch.zeros(4096 * 11, dtype=torch.float64, device="cuda")
    host = np.zeros(4096 * 3)
    types = np.zeros(4096, np.int32)
    rc = lib.contact_step_noalloc(ctypes.byref(cfg), types.ctypes.data_as(ctypes.c_void_p),
                                  host.ctypes.data_as(ctypes.c_void_p), host.ctypes.data_as(ctypes.c_void_p),
                                  host.ctypes.data_as(ctypes.c_void_p), *[ctypes.c_void_p(dummy.data_ptr())] * 7,
                                  None)
    assert rc == EINVAL
    lib.contact_config_default(ctypes.byref(cfg), st.n, nc, 1.0)
    cfg.max_pairs = 1 << 20                                        # pair capacity beyond the maximum
    rc = lib.contact_step_noalloc(ctypes.byref(cfg), types.ctypes.data_as(ctypes.c_void_p),
                                  host.ctypes.data_as(ctypes.c_void_p), host.ctypes.data_as(ctypes.c_void_p),
                                  host.ctypes.data_as(ctypes.c_void_p), *[ctypes.c_void_p(dummy.data_ptr())] * 7,
                                  None)
    assert rc == EINVAL


def test_noalloc_matches_contact_step_at_a_spacing_that_is_not_a_power_of_two():
    """dx = 0.7: the per-particle tables (sizes in lattice units, compliance)
    are formed with the same rounded operations on both paths, so the node
    classification and the pair volumes agree exactly."""
    from paper_2401_10878_gb300.contact import Contact
    st = W.mixed_grid_27()
    st.indicator = 0
    st.dx = 0.7
    st.pos = st.pos * 0.7
    st.shape_param = st.shape_param * 0.7
    model = Contact.from_state(st, max_pairs=8192)
    pos = torch.tensor(st.pos, device="cuda")
    quat = torch.tensor(st.quat, device="cuda")
    ref = model.step(pos, quat)
    rc, out = _noalloc(model.lib, model, st, pos, quat)
    assert rc == 0, rc
    P = int(out["n_pairs"].item())
    assert P == ref["n_pairs"] > 0
    assert torch.equal(out["pair_ij"][:P], ref["pair_ij"])
    po, pr = out["pair_out"][:P].cpu().numpy(), ref["pair_out"].cpu().numpy()
    assert np.array_equal(po[:, 0], pr[:, 0])
    scale = np.abs(pr[:, 8:11]).max()
    assert np.abs(po - pr).max() <= 1e-5 * max(scale, 1.0)
    model.close()


def test_noalloc_capacity_limits():
    """Fewer pair slots than pairs, or a tile budget below the pairs' tiles,
    return CONTACT_ECAPACITY with n_pairs holding the pairs needed; the next
    call with room succeeds."""
    from paper_2401_10878_gb300.contact import Contact, ECAPACITY
    st = W.mixed_grid_27()
    st.indicator = 0
    model = Contact.from_state(st, max_pairs=8192)
    pos = torch.tensor(st.pos, device="cuda")
    quat = torch.tensor(st.quat, device="cuda")
    need = model.step(pos, quat)["n_pairs"]
    for field, value in (("max_pairs", 8), ("max_tiles", 4)):
        saved = getattr(model.cfg, field)
        setattr(model.cfg, field, value)
        rc, out = _noalloc(model.lib, model, st, pos, quat)
        setattr(model.cfg, field, saved)
        assert rc == ECAPACITY, (field, rc)
        assert int(out["n_pairs"].item()) == need
    rc, out = _noalloc(model.lib, model, st, pos, quat)
    assert rc == 0 and int(out["n_pairs"].item()) == need
    model.close()
