"""CUDA box pipeline (the paper's rough detection, box correction and N_c^3
sampling, Sec. 3.3.1) vs the oracle's (needs a GB300).

The rough box and the corrected box are reproduced exactly unless the oracle
reports a node within eps of the rough threshold or two nearest lines of a
face within 1e-4 dx (those pairs are flagged); the sample counts are then
exact and the sample volume agrees to FP64 rounding, so the tolerances are
the lattice path's (tests/parity.py) with the sample volume as the unit.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2401_10878_gb300 import workloads as W
from tests.parity import compare, gpu_step

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def boxed(st, nc=8):
    st = dataclasses.replace(st)
    st.box_mode, st.contact_resolution = 1, nc
    return st


def run(st, vel=None):
    from paper_2401_10878_gb300.contact import Contact
    m = Contact.from_state(st)
    g = gpu_step(m, st, vel=vel)
    r = oracle.contact_step(st, vel=vel)
    rough, box, flags = oracle.box_pipeline(st)
    nc = st.contact_resolution
    dV = np.prod((box[:, 3:] - box[:, :3]) / nc, axis=1)
    ext = (box[:, 3:] - box[:, :3]).min(axis=1)
    rep = compare(st, g, r, fp64=False, smooth=st.indicator == 1,
                  box=(dV, (flags[:, 0] > 0) | (flags[:, 1] > 0), ext))
    m.close()
    return rep, r


@pytest.mark.parametrize("nc", [4, 8, 16])
def test_mixed27_box_pipeline(nc):
    rep, r = run(boxed(W.mixed_grid_27(), nc))
    print("mixed27 box", nc, rep)
    assert np.count_nonzero(r.pair_out[:, 0]) > 20


def test_cubes400_box_pipeline():
    rep, _ = run(boxed(W.settling_cubes()))
    print("cubes400 box", rep)


def test_mixed1934_box_pipeline_full_size():
    rep, r = run(boxed(W.mixed_settling()))
    print("mixed1934 box", rep)
    assert np.count_nonzero(r.pair_out[:, 0]) > 300


def test_cubes1934_walls_box_pipeline():
    st = boxed(W.floor_and_ceiling(W.settling_cubes_dense()))
    rep, r = run(st)
    print("cubes1934 + walls box", rep)
    assert (r.pair_ij[:, 1] >= st.n).sum() > 50


def test_smoothed_box_pipeline_with_damping():
    st = boxed(W.mixed_grid_27())
    st.indicator, st.smooth_width, st.damping_c = 1, 1.0, 0.3
    rng = np.random.default_rng(2)
    vel = np.concatenate([rng.normal(size=(st.n, 3)) * 0.05, rng.normal(size=(st.n, 3)) * 0.01], axis=1)
    rep, _ = run(st, vel)
    print("mixed27 smooth box + damping", rep)


def test_box_pipeline_refuses_backward_and_history():
    from paper_2401_10878_gb300.contact import ESTATE, Contact, ContactError
    st = boxed(W.mixed_grid_27())
    st.indicator = 1
    m = Contact.from_state(st)
    gpu_step(m, st)
    z = torch.zeros((st.n, 3), dtype=torch.float64, device=m.device)
    with pytest.raises(ContactError) as e:
        m.backward(z, z)
    assert e.value.code == ESTATE
    m.close()
    with pytest.raises(ContactError):
        Contact.from_state(st, history=True)
