"""The pins catch plausible mistakes: each case compiles the oracle with one
mistake planted in its source (a dropped term, a wrong sign or factor, a
transposed index, a wrong rounding rule), swaps it in for the oracle, and
requires the pin that guards that step to fail.  CPU only; the mistakes live
in temporary copies, never in the oracle itself."""
import concurrent.futures
import ctypes
import os
import shutil
import subprocess

import pytest

import oracle
from tests import test_centroid as TC
from tests import test_oracle_box_pipeline as TB
from tests import test_oracle_contact_law as TL
from tests import test_oracle_diagnostics as TD
from tests import test_oracle_pins as TP
from tests import test_oracle_walls as TW

# (name, text in the oracle, planted replacement, pin that must fail)
CASES = [
    ("centroid pyramid factor", "mom[k] += vf * 0.75 * (ac[k] / area);", "mom[k] += vf * 0.70 * (ac[k] / area);",
     TC.test_pyramid_centroid_at_a_quarter_height),
    ("force prefactor", "if (val(vd) > 0.0) fmag = (4.0 / (3.0 * M_PI)) * estar * sqrt_s(vd) * damp;",
     "if (val(vd) > 0.0) fmag = (4.0 / (3.0 * std::sqrt(M_PI))) * estar * sqrt_s(vd) * damp;",
     TP.test_lens_worked_example_force_and_depth),
    ("normal: sign of A's band term", "SG[k] = SG[k] + (-(HpA * HB)) * gA[k] + (HA * HpB) * gB[k];",
     "SG[k] = SG[k] + (HpA * HB) * gA[k] + (HA * HpB) * gB[k];", TP.test_swap_labels_flips_normal_and_force),
    ("first moments: transposed index", "SM[k] = SM[k] + W * c[k];", "SM[k] = SM[k] + W * c[(k + 1) % 3];",
     TP.test_lens_centroid_and_normal),
    ("depth: dropped term", "S f = -phA - phB;", "S f = -phA;", TP.test_depth_of_a_deep_sphere_pair),
    ("effective modulus: nu not squared", "return 1.0 / ((1.0 - nuA * nuA) / EA + (1.0 - nuB * nuB) / EB);",
     "return 1.0 / ((1.0 - nuA) / EA + (1.0 - nuB) / EB);", TP.test_effective_modulus_special_cases),
    ("periodic image: floor for round", "std::nearbyint((pos[3 * j + k] - pos[3 * i + k]) / L)",
     "std::floor((pos[3 * j + k] - pos[3 * i + k]) / L)", TP.test_periodic_pairs_across_faces_edges_corners),
    ("warm start: box not relative to X_i",
     "const double wl = (XA[a] + warm[a]) - srough, wh = (XA[a] + warm[3 + a]) + srough;",
     "const double wl = warm[a] - srough, wh = warm[3 + a] + srough;",
     lambda: TB.test_warm_start_follows_particle_i_across_the_periodic_boundary(0.6875, 33.0, 0)),
    ("warm start: no widening",
     "const double wl = (XA[a] + warm[a]) - srough, wh = (XA[a] + warm[3 + a]) + srough;",
     "const double wl = (XA[a] + warm[a]), wh = (XA[a] + warm[3 + a]);",
     TB.test_stored_box_bounds_the_correction),
    ("rotation: sign of w z in R[0][1]", "R[1] = s * (x * y - w * z);", "R[1] = s * (x * y + w * z);",
     TP.test_rotation_known_quaternions),
    ("smoothed indicator: wrong smoothstep", "if (smooth) *H = t * t * (3.0 - 2.0 * t);",
     "if (smooth) *H = t * (3.0 - 2.0 * t);", TP.test_smoothed_band_weights_of_mirrored_faces_sum_to_sharp),
    ("damping: no clamp at zero", "if (val(damp) < 0.0) damp = S(0.0);", "",
     TL.test_shared_damping_clamped_when_separating_fast),
    ("friction: wrong direction", "res.F[k] = res.F[k] + coef * fmag * ut[k] / utn;",
     "res.F[k] = res.F[k] - coef * fmag * ut[k] / utn;", TL.test_friction_opposes_sliding_and_dissipates),
    ("history: c of an ongoing contact dropped", "        law.c = hist_c[row];", "        law.c = 0.0;",
     TL.test_history_keeps_c_until_the_contact_ends),
    ("box correction skipped", "shift[k][side] = std::isfinite(best) ? best : 0.0;", "shift[k][side] = 0.0;",
     TB.test_face_aligned_boxes_exact),
    ("wall: half-space inverted", "return S(((e[0] * x[0] + e[1] * x[1]) + e[2] * x[2]) - e[3] - inflate);",
     "return S(e[3] - ((e[0] * x[0] + e[1] * x[1]) + e[2] * x[2]) - inflate);",
     lambda: TW.test_face_aligned_cube_on_floor_exact(17.5, 1)),
    ("rough detection: half the cell for the half diagonal", "const double srough = std::sqrt(0.75) * dx;",
     "const double srough = 0.5 * dx;", TB.test_rough_box_equals_brute_force_scan),
    ("quaternion not normalised", "const S s = 2.0 / nn;", "const S s = 2.0;",
     TP.test_rotation_orthonormal_and_scale_free),
    ("dual numbers: derivative of the square root", "r.g[i] = (r.v > 0.0) ? a.g[i] / (2.0 * r.v) : 0.0;",
     "r.g[i] = (r.v > 0.0) ? a.g[i] / r.v : 0.0;", TP.test_dual_gradient_matches_central_differences),
    ("wall candidate test too strict", "if (!(((t[0] + t[1]) + t[2]) <= H)) return false;",
     "if (!(((t[0] + t[1]) + t[2]) <= H - 1.0)) return false;", TW.test_brute_force_scan_near_oblique_walls),
    ("box correction: sphere entry point", "*t0 = -b - sq;", "*t0 = -b;",
     lambda: TB.test_sphere_lens_box_inside_and_volume(8)),
    ("friction: mu_s* coefficient", "law.mu_s * (1.0 - 0.09 * ratio * ratio * ratio * ratio);",
     "law.mu_s * (1.0 - 0.9 * ratio * ratio * ratio * ratio);", TL.test_friction_worked_values),
    ("box pipeline: samples at cell corners", "s_lo[k] += 0.5 * s_step[k];   // cell centres",
     "s_lo[k] += 0.0 * s_step[k];", TB.test_face_aligned_boxes_exact),
    ("contact point: box origin dropped", "res.xc[k] = o[k] + (dx3 * SM[k]) / V;", "res.xc[k] = (dx3 * SM[k]) / V;",
     TP.test_contact_point_inside_both_shapes),
    ("torque on A: one component's sign", "res.TA[2] = ra[0] * FA[1] - ra[1] * FA[0];",
     "res.TA[2] = ra[1] * FA[0] - ra[0] * FA[1];", TP.test_momentum_balance),
    ("torque on B: lever arm from A's centre",
     "centre of mass (Sec. 2.2)\n  S ra[3] = {res.xc[0] - XA[0], res.xc[1] - XA[1], res.xc[2] - XA[2]};\n"
     "  S rb[3] = {res.xc[0] - XB[0], res.xc[1] - XB[1], res.xc[2] - XB[2]};",
     "centre of mass (Sec. 2.2)\n  S ra[3] = {res.xc[0] - XA[0], res.xc[1] - XA[1], res.xc[2] - XA[2]};\n"
     "  S rb[3] = {res.xc[0] - XA[0], res.xc[1] - XA[1], res.xc[2] - XA[2]};", TP.test_momentum_balance),
    # the parity checks' diagnostics
    ("band count: eps band ten times too wide", "const bool loose = pa <= eps && pb <= eps;",
     "const bool loose = pa <= 10.0 * eps && pb <= 10.0 * eps;", TD.test_band_count_nodes_just_outside_a_sphere),
    ("face ties: gap threshold", "const bool tieA = gapA < eps || (!smooth && std::fabs(pb) <= eps);",
     "const bool tieA = gapA < 0.5 || (!smooth && std::fabs(pb) <= eps);", TD.test_face_tie_count_on_a_cube_edge),
    ("depth gap: sign", "(top1 - top2) / dx", "(top2 - top1) / dx", TD.test_depth_gap_closed_form_and_symmetric_tie),
    ("volume sensitivity: B's term dropped", "const double dw = hpa * hb + ha * hpb;", "const double dw = hpa * hb;",
     TD.test_sensitivities_of_a_smoothed_slab),
    ("moment sensitivity: a lever-arm component dropped",
     "m_sens += dw * eps * std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);",
     "m_sens += dw * eps * std::sqrt(c[0] * c[0] + c[1] * c[1]);", TD.test_sensitivities_of_a_smoothed_slab),
    ("normal sensitivity: the product term dropped", "g_sens += (dhpa * hb + 2.0 * hpa * hpb + ha * dhpb) * eps;",
     "g_sens += (dhpa * hb + ha * dhpb) * eps;", TD.test_sensitivities_of_a_smoothed_slab),
    ("normal sensitivity (sharp): B's term dropped", "g_sens += (dhpa * hb + ha * dhpb) * eps;",
     "g_sens += (dhpa * hb) * eps;", TD.test_sensitivities_of_a_sharp_slab),
    ("rough band: eps ten times too wide", "const bool loose = pa < srough + eps && pb < srough + eps;",
     "const bool loose = pa < srough + 10.0 * eps && pb < srough + 10.0 * eps;",
     TD.test_rough_band_nodes_around_a_sphere),
    ("box face ties: exact ties counted", "second - best < 1e-4 * dx && second != best", "second - best < 1e-4 * dx",
     TD.test_face_ties_of_face_aligned_boxes_are_exact),
    ("box face ties: threshold", "second - best < 1e-4 * dx && second != best",
     "second - best < 1e-2 * dx && second != best", TD.test_face_ties_of_slightly_tilted_boxes),
]


def _compile(i, old, new, tmp):
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, f"planted text not unique or missing: {old}"
    path = os.path.join(tmp, f"planted_{i}.cpp")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = os.path.join(tmp, f"planted_{i}.so")
    subprocess.run(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", path, "-o", so],
                   check=True, capture_output=True)
    return so


@pytest.fixture(scope="module")
def planted_libs(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    tmp = str(tmp_path_factory.mktemp("planted"))
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        futs = [ex.submit(_compile, i, old, new, tmp) for i, (_, old, new, _) in enumerate(CASES)]
        return [f.result() for f in futs]


@pytest.mark.parametrize("case", range(len(CASES)), ids=[c[0] for c in CASES])
def test_pin_catches_planted_mistake(case, planted_libs):
    name, _, _, pin = CASES[case]
    saved = oracle._lib
    oracle._lib = oracle._configure(ctypes.CDLL(planted_libs[case]))
    try:
        with pytest.raises(Exception):   # an assertion, or an index or oracle error from missing pairs
            pin()
    finally:
        oracle._lib = saved


def test_unplanted_oracle_passes_the_same_pins():
    for _, _, _, pin in CASES:
        pin()
