"""CUDA contact step vs the FP64 oracle, element by element (needs a GB300).

Workloads: the 27-particle mixed grid (FP64 on both sides), the 400-cube
settling box, the 1934-particle mixed-shape box at full size, the 1934-cube
box in smoothed mode, the resolution sweep; plus edge cases (no pairs, one
pair, periodic corners, > 20-face polytopes, inflation, damping, capacity and
input errors, graph replay).
"""
import numpy as np
import pytest

import oracle
from paper_2401_10878_gb300 import workloads as W
from tests.helpers import cube_planes, state
from tests.parity import assert_flat, compare, gpu_step

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def model_for(st, **kw):
    from paper_2401_10878_gb300.contact import Contact
    return Contact.from_state(st, **kw)


def run_parity(st, precision=0, **kw):
    m = model_for(st, precision=precision, **kw)
    g = gpu_step(m, st)
    r = oracle.contact_step(st)
    rep = compare(st, g, r, fp64=precision == 1, smooth=st.indicator == 1)
    boxes = m.particle_boxes().cpu().numpy()
    assert np.array_equal(boxes, oracle.aabb(st)), "particle node ranges differ"
    m.close()
    return rep


@pytest.fixture(scope="module")
def states():
    return {
        "c1": W.mixed_grid_27(),
        "c2": W.settling_cubes(),
        "c3": W.mixed_settling(),
        "c4": W.settling_cubes_dense(),
    }


@pytest.mark.parametrize("precision", [1, 0])
def test_mixed27_grid(states, precision):
    rep = run_parity(states["c1"], precision)
    print("mixed27", precision, rep)
    assert rep.pairs > 40


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("smooth", [False, True])
def test_mixed27_elongated_cuboids(precision, smooth):
    """Spheres and cuboids of unequal half extents (7, 5, 4): the sphere /
    cuboid kernel variant with per-axis slabs (every other workload's cuboids
    are cubes)."""
    st = W.mixed_grid_27(cuboid_half=(7.0, 5.0, 4.0))
    if smooth:
        st.indicator, st.smooth_width = 1, 1.0
    rep = run_parity(st, precision)
    print("mixed27 cuboids", precision, smooth, rep)
    assert rep.pairs > 40


@pytest.mark.parametrize("precision", [0, 1])
def test_cubes400_settling(states, precision):
    print("cubes400", precision, run_parity(states["c2"], precision))


def test_mixed1934_full_size(states):
    rep = run_parity(states["c3"], 0)
    print("mixed1934", rep)
    assert rep.flagged <= 0.01 * rep.pairs


def test_mixed1934_fp64_form(states):
    print("mixed1934 fp64", run_parity(states["c3"], 1))


def test_cubes1934_sharp_and_smooth(states):
    """The headline configuration: sharp mode meets the benchmark spec's flat
    bounds directly (V and first moments 1e-6 relative, force and torque 1e-5
    relative, on every unflagged pair and particle)."""
    st = states["c4"]
    sharp = W.State(**{**st.__dict__, "indicator": 0})
    rep = run_parity(sharp, 0)
    print("cubes1934 sharp", rep)
    assert_flat(rep)
    print("cubes1934 smooth", run_parity(st, 0))


@pytest.mark.parametrize("edge", [8, 12, 16, 24])
def test_resolution_sweep_and_exact_box_volume(edge):
    st = W.resolution_sweep(edge)
    print("sweep", edge, run_parity(st, 0))
    m = model_for(st)
    g = gpu_step(m, st)
    # face-aligned pairs (both axis-aligned, faces on half-integer nodes): exact box overlap
    al = st.info["aligned"]
    ij = g["pair_ij"]
    both = al[ij[:, 0]] & al[ij[:, 1]]
    assert both.sum() > 10
    h = st.shape_param[0, 0]
    for p in np.nonzero(both)[0]:
        i, j = ij[p]
        d = W.min_image(st.pos[j] - st.pos[i], st.box)
        ov = np.clip(2 * h - np.abs(d), 0, None)
        assert g["pair_out"][p, 0] == np.prod(ov)
    m.close()


def test_smoothed_fp64_form(states):
    st = W.mixed_grid_27()
    st.indicator = 1
    print("mixed27 smooth fp64", run_parity(st, 1))
    print("mixed27 smooth fp32", run_parity(st, 0))


# ----------------------------------------------------------------- edge cases

def test_no_pairs_and_single_pair():
    far = state([0, 1], [[5, 0, 0], [4, 4, 4]], [[10, 10, 10], [40, 40, 40]])
    m = model_for(far)
    g = gpu_step(m, far)
    assert g["n_pairs"] == 0 and np.all(g["force"] == 0) and np.all(g["torque"] == 0)
    m.close()
    one = state([0, 1], [[6, 0, 0], [4, 4, 4]], [[20.3, 20.1, 20.7], [29.0, 21.0, 19.5]],
                quat=[[1, 0, 0, 0], list(W.random_quaternions(np.random.default_rng(1), 1)[0])])
    print("single", run_parity(one, 0), run_parity(one, 1))


def test_periodic_corner_pairs():
    rng = np.random.default_rng(2)
    q = W.random_quaternions(rng, 8)
    pos = []
    for c in range(4):
        base = np.array([63.6, 0.4, 63.2]) if c == 0 else rng.random(3) * 64
        pos += [base, np.mod(base + rng.normal(size=3) * 2 + [8, 0, 0], 64)]
    types = [1, 0, 1, 1, 0, 0, 1, 0]
    st = state(types, [[5, 5, 5] if t == 1 else [6, 0, 0] for t in types], pos, q)
    print("periodic", run_parity(st, 0))


def test_positions_on_the_periodic_boundary():
    """Centres at x = 0, y = -0.0 and z = the largest double below L, each
    touching a partner across the boundary: the pairs, their images and the
    node ranges bit for bit, the outputs with the usual tolerances (both
    forms); a centre at exactly L is refused on both sides."""
    from paper_2401_10878_gb300.contact import ContactError, EINVAL
    top = np.nextafter(64.0, 0.0)
    pos = [[0.0, 20.0, 20.0], [59.0, 20.5, 20.0], [30.0, -0.0, 30.0], [31.0, 55.0, 30.5],
           [40.0, 40.0, top], [41.0, 40.5, 6.0]]
    types = [1, 0, 0, 1, 1, 0]
    params = [[5, 5, 5], [5.5, 0, 0], [6, 0, 0], [4.5, 4.5, 4.5], [3, 4, 5], [5, 0, 0]]
    st = state(types, params, pos, W.random_quaternions(np.random.default_rng(3), 6))
    r = oracle.contact_step(st)
    assert r.n_pairs == 3 and np.all(r.pair_out[:, 0] > 0) and np.abs(r.pair_shift).sum() == 3
    print("boundary", run_parity(st, 0), run_parity(st, 1))
    m = model_for(st)
    gpu_step(m, st)
    assert np.array_equal(m.particle_boxes().cpu().numpy(), oracle.aabb(st))
    bad = st.pos.copy()
    bad[4, 2] = 64.0
    with pytest.raises(ContactError) as e:
        gpu_step(m, st, pos=bad)
    assert e.value.code == EINVAL
    with pytest.raises(oracle.OracleError):
        oracle.contact_step(st, pos=bad)
    m.close()


def test_concentric_shapes_degenerate_normal():
    """Concentric shapes centred on a node: G vanishes by symmetry, so the
    normal is undefined (the oracle's FP64 sums cancel below the fallback
    threshold and its centre-line fallback is zero; the FP32 partial sums
    leave rounding noise).  What the method does define is compared: V bit for
    bit, d, and a finite normal of unit or zero length with F along it."""
    cases = [state([0, 0], [[6, 0, 0], [4, 0, 0]], [[30.0, 30.0, 30.0]] * 2),
             state([1, 1], [[4, 4, 4], [4, 4, 4]], [[30.0, 30.0, 30.0]] * 2)]
    for st in cases:
        r = oracle.contact_step(st)
        m = model_for(st)
        g = gpu_step(m, st)
        o, ro = g["pair_out"][0], r.pair_out[0]
        assert g["n_pairs"] == 1 and o[0] == ro[0] and abs(o[7] - ro[7]) <= 1e-6
        nn = np.linalg.norm(o[4:7])
        assert np.all(np.isfinite(o)) and (nn == 0.0 or abs(nn - 1.0) < 1e-12)
        if nn > 0:
            assert np.linalg.norm(np.cross(o[8:11], o[4:7])) <= 1e-9 * np.linalg.norm(o[8:11])
        print("concentric", st.shape_type.tolist(), "V", o[0], "d", o[7], "|n|", nn, "oracle |n|",
              np.linalg.norm(ro[4:7]))
        m.close()


def test_many_face_polytopes_and_inflation():
    rng = np.random.default_rng(3)
    polys = [W.random_polytope(rng, f, 9.0)[0] for f in (24, 32, 8, 20)]
    pos = [[20, 20, 20], [35, 21, 19], [20, 36, 21], [34, 36, 20]]
    q = W.random_quaternions(rng, 4)
    st = state([2, 2, 2, 2], np.zeros((4, 3)), pos, q, planes=polys, inflate=0.2)
    print("polytopes", run_parity(st, 0), run_parity(st, 1))


def test_velocities_and_damping():
    st = W.mixed_grid_27()
    st.damping_c = W.YOUNG and 0.3
    rng = np.random.default_rng(4)
    vel = rng.normal(size=(st.n, 6)) * 0.1
    m = model_for(st)
    g = gpu_step(m, st, vel=vel)
    r = oracle.contact_step(st, vel=vel)
    print("damped", compare(st, g, r, fp64=False, smooth=False))
    m.close()


def test_graph_replay_and_repeat():
    st = W.mixed_settling(n=300, L=120)
    m = model_for(st)
    a = gpu_step(m, st)
    seq_p, seq_q = W.pose_sequence(st, 3)
    for s in range(3):
        g = gpu_step(m, st, seq_p[s], seq_q[s])
        r = oracle.contact_step(st, pos=seq_p[s], quat=seq_q[s])
        compare(st.with_poses(seq_p[s], seq_q[s]), g, r, fp64=False, smooth=False)
    b = gpu_step(m, st)
    assert np.array_equal(a["pair_out"], b["pair_out"]) and np.array_equal(a["force"], b["force"])
    m.close()


def test_repeated_node_sweep_for_timing():
    """narrow_events = K > 1 runs the node sweep K times between the timing
    events; every run recomputes the same outputs from the same tiles (a pair
    of several tiles resets its counter when it completes), so the step's
    results are those of a plain step bit for bit, in both forms and both
    indicators; box_mode 1 refuses it."""
    from paper_2401_10878_gb300.contact import ContactError, EINVAL
    for st in (W.mixed_settling(n=300, L=120), W.settling_cubes()):
        for ind in (0, 1):
            st.indicator = ind
            for prec in (0, 1):
                m = model_for(st, precision=prec)
                a = gpu_step(m, st)
                m.close()
                m = model_for(st, precision=prec, narrow_events=3)
                b = gpu_step(m, st)
                assert m.narrow_time_ms() > 0.0
                m.close()
                for k in ("pair_ij", "pair_out", "force", "torque"):
                    assert np.array_equal(a[k], b[k]), (st.name, ind, prec, k)
    st = W.mixed_grid_27()
    st.box_mode = 1
    with pytest.raises(ContactError) as e:
        model_for(st, narrow_events=2)
    assert e.value.code == EINVAL


def test_capacity_and_input_errors():
    from paper_2401_10878_gb300.contact import ContactError, ECAPACITY, EINVAL
    st = W.mixed_settling(n=300, L=120)
    m = model_for(st, max_pairs=8)
    with pytest.raises(ContactError) as e:
        gpu_step(m, st)
    assert e.value.code == ECAPACITY
    assert int(m.n_pairs.item()) == oracle.contact_step(st).n_pairs
    m.close()
    m = model_for(st)
    bad = st.pos.copy()
    bad[5, 1] = st.box[1] + 3.0
    with pytest.raises(ContactError) as e:
        gpu_step(m, st, pos=bad)
    assert e.value.code == EINVAL
    m.clear_error()
    gpu_step(m, st)   # the context is usable again
    # NaN position, NaN and zero quaternions: the same sticky error, then recovery
    for field, row, value in (("pos", 7, np.nan), ("quat", 3, np.nan), ("quat", 4, 0.0)):
        p, q = st.pos.copy(), st.quat.copy()
        if field == "pos":
            p[row, 0] = value
        else:
            q[row, :] = value
        with pytest.raises(ContactError) as e:
            gpu_step(m, st, pos=p, quat=q)
        assert e.value.code == EINVAL, field
        m.clear_error()
    gpu_step(m, st)
    m.close()


def test_cell_list_bin_capacity():
    """30 sphere centres inside one cell-list bin whose capacity is 17
    (twice the bin volume over the inscribed-ball volume, plus 8): the step
    reports ECAPACITY; after clear_error the context steps a spread-out state."""
    from paper_2401_10878_gb300.contact import ContactError, ECAPACITY
    rng = np.random.default_rng(5)
    k = 30
    crowded = 6.0 + rng.uniform(-1.0, 1.0, size=(k, 3))
    st = state([0] * k, [[5.0, 0, 0]] * k, crowded, n=64)
    m = model_for(st)
    with pytest.raises(ContactError) as e:
        gpu_step(m, st)
    assert e.value.code == ECAPACITY
    m.clear_error()
    g = np.stack(np.meshgrid(*[np.arange(4)] * 3, indexing="ij"), -1).reshape(-1, 3)[:k]
    spread = 8.0 + 14.0 * g + rng.uniform(-0.5, 0.5, size=(k, 3))
    r = oracle.contact_step(st, pos=spread, quat=st.quat)
    out = gpu_step(m, st, pos=spread)
    compare(st.with_poses(spread, st.quat), out, r, fp64=False, smooth=False)
    m.close()


def test_graph_update_for_new_buffers():
    """New input buffers on the same stream update the captured graph in place
    (stats 'replayed' = 2) instead of instantiating it again; the results stay
    those of a fresh context, and the same buffers replay it (= 1)."""
    st = W.mixed_grid_27()
    m = model_for(st)
    tp = torch.tensor(st.pos, device="cuda")
    tq = torch.tensor(st.quat, device="cuda")
    m.step(tp, tq)
    assert m.stats()["replayed"] == 0
    ref_f, ref_p = m.force.clone(), m.pair_out.clone()
    tp2, tq2 = tp.clone(), tq.clone()
    m.step(tp2, tq2)
    assert m.stats()["replayed"] == 2
    assert torch.equal(m.force, ref_f) and torch.equal(m.pair_out, ref_p)
    m.step(tp2, tq2)
    assert m.stats()["replayed"] == 1
    assert torch.equal(m.force, ref_f)
    m.close()


def test_step_host_buffers():
    """contact_step_host: pinned CPU tensors (copies inside the graph) and
    pageable numpy arrays both give the device-pointer step's results bit for
    bit, pair outputs included; a backward after it uses its tape."""
    st = W.mixed_grid_27()
    m = model_for(st)
    dev = m.step(torch.tensor(st.pos, device="cuda"), torch.tensor(st.quat, device="cuda"))
    ref_f, ref_t = dev["force"].cpu(), dev["torque"].cpu()
    ref_ij, ref_out, P = dev["pair_ij"].cpu(), dev["pair_out"].cpu(), dev["n_pairs"]
    hp = torch.tensor(st.pos).pin_memory()
    hq = torch.tensor(st.quat).pin_memory()
    hf = torch.empty((st.n, 3), dtype=torch.float64).pin_memory()
    ht = torch.empty((st.n, 3), dtype=torch.float64).pin_memory()
    for _ in range(2):   # capture, then replay
        out = m.step_host(hp, hq, force=hf, torque=ht, pairs=True)
        assert out["n_pairs"] == P
        assert torch.equal(out["force"], ref_f) and torch.equal(out["torque"], ref_t)
        assert torch.equal(out["pair_ij"], ref_ij) and torch.equal(out["pair_out"], ref_out)
    out = m.step_host(np.ascontiguousarray(st.pos), np.ascontiguousarray(st.quat))   # pageable
    assert torch.equal(out["force"], ref_f) and torch.equal(out["torque"], ref_t)
    m.close()


def test_step_host_mapped_buffers_with_velocities():
    """Pinned host poses, forces and torques are read and written by the
    step's kernels in place; the velocities are still copied: with damping
    the results equal the device-pointer step's bit for bit, over several
    calls with changing inputs."""
    st = W.mixed_grid_27()
    st.damping_c = 0.3
    m = model_for(st)
    rng = np.random.default_rng(8)
    hp = torch.empty((st.n, 3), dtype=torch.float64).pin_memory()
    hq = torch.empty((st.n, 4), dtype=torch.float64).pin_memory()
    hv = torch.empty((st.n, 6), dtype=torch.float64).pin_memory()
    hf = torch.empty((st.n, 3), dtype=torch.float64).pin_memory()
    ht = torch.empty((st.n, 3), dtype=torch.float64).pin_memory()
    pos, quat = W.pose_sequence(st, 3, seed=9, sigma_x=0.3, sigma_rot=0.02)
    for s in range(3):
        vel = rng.normal(size=(st.n, 6)) * 0.1
        dev = m.step(torch.tensor(pos[s], device="cuda"), torch.tensor(quat[s], device="cuda"),
                     torch.tensor(vel, device="cuda"))
        ref_f, ref_t, P = dev["force"].cpu(), dev["torque"].cpu(), dev["n_pairs"]
        hp.copy_(torch.from_numpy(pos[s]))
        hq.copy_(torch.from_numpy(quat[s]))
        hv.copy_(torch.from_numpy(vel))
        out = m.step_host(hp, hq, hv, force=hf, torque=ht)
        assert out["n_pairs"] == P
        assert torch.equal(hf, ref_f) and torch.equal(ht, ref_t)
    m.close()


def test_step_host_waits_for_its_own_step():
    """contact_step_host returns once its own step's results are in host
    memory: with in-place host buffers and an idle stream it waits for the
    token its step publishes at the end.  A loop of calls with changing poses
    gives the device-pointer steps' forces and torques bit for bit, and a call
    right after an asynchronous step (work still queued on the stream)
    synchronises instead and is exact too."""
    st = W.settling_cubes()
    m = model_for(st)
    pos, quat = W.pose_sequence(st, 6, seed=5, sigma_x=0.3, sigma_rot=0.02)
    refs = []
    for k in range(6):
        dev = m.step(torch.tensor(pos[k], device="cuda"), torch.tensor(quat[k], device="cuda"))
        refs.append((dev["force"].cpu(), dev["torque"].cpu()))
    hp = torch.empty((st.n, 3), dtype=torch.float64).pin_memory()
    hq = torch.empty((st.n, 4), dtype=torch.float64).pin_memory()
    hf = torch.empty((st.n, 3), dtype=torch.float64).pin_memory()
    ht = torch.empty((st.n, 3), dtype=torch.float64).pin_memory()
    for rnd in range(2):
        for k in range(6):
            hp.copy_(torch.from_numpy(pos[k]))
            hq.copy_(torch.from_numpy(quat[k]))
            m.step_host(hp, hq, force=hf, torque=ht)
            assert torch.equal(hf, refs[k][0]) and torch.equal(ht, refs[k][1]), (rnd, k)
    tp, tq = torch.tensor(pos[0], device="cuda"), torch.tensor(quat[0], device="cuda")
    m.step_async(tp, tq)   # queued, not waited for
    hp.copy_(torch.from_numpy(pos[3]))
    hq.copy_(torch.from_numpy(quat[3]))
    m.step_host(hp, hq, force=hf, torque=ht)
    assert torch.equal(hf, refs[3][0]) and torch.equal(ht, refs[3][1])
    m.close()


def test_fp32_ffma_rate_against_the_derived_peak():
    """The measured FFMA rate lies between half and 105 % of SMs x 128 lanes x
    the maximum SM clock (the node sweep's roofline peak)."""
    from paper_2401_10878_gb300.contact import fp32_ffma_rate
    props = torch.cuda.get_device_properties(0)
    rate = fp32_ffma_rate()
    derived = props.multi_processor_count * 128 * 2070e6
    print("FFMA rate", rate / 1e12, "T/s; derived peak at 2070 MHz", derived / 1e12)
    assert 0.5 * derived <= rate <= 1.05 * derived


def test_fp64_dfma_rate_probe():
    """The measured DFMA rate is positive and far below the FFMA rate (the
    FP64 pipe of this GPU is narrow): the peak the all-FP64 form is held to."""
    from paper_2401_10878_gb300.contact import fp32_ffma_rate, fp64_dfma_rate
    d, f = fp64_dfma_rate(), fp32_ffma_rate()
    print("DFMA rate", d / 1e12, "T/s; FFMA rate", f / 1e12, "T/s")
    assert 1e10 <= d <= 0.5 * f


def test_user_stream_capture():
    st = W.mixed_grid_27()
    m = model_for(st, use_graph=False)
    tp = torch.tensor(st.pos, device="cuda")
    tq = torch.tensor(st.quat, device="cuda")
    m.step(tp, tq)
    ref = m.force.clone()
    m.force.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        m.lib.contact_set_stream(m.ctx, __import__("ctypes").c_void_p(s.cuda_stream))
        with torch.cuda.graph(g, stream=s):
            m.step_async(tp, tq)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(m.force, ref)
    m.close()
