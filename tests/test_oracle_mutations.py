"""The oracle's pins catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign or index, a
transposed operand, an off-by-one border) in a copy of the oracle's C source
(built into a separate library) or of its Python orchestration (loaded as a
separate module), and runs the pins against it: at least one pin must fail.
The oracle itself is never modified."""
import os
import subprocess
import sys
import tempfile
import types

import pytest

import test_oracle_pins as P
from oracle import oracle as O

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "stab_oracle.c")

# (name, original text, planted mistake)
MUTATIONS = [
    ("pyramid weight", "static const int k5[5] = {1, 4, 6, 4, 1};", "static const int k5[5] = {1, 4, 6, 4, 2};"),
    ("reflect-101 off by one", "if (i >= n) i = 2 * n - 2 - i;", "if (i >= n) i = 2 * n - 1 - i;"),
    ("pyramid rounding", "dst[(size_t)y * dp + x] = (uint8_t)((s + 128) >> 8);", "dst[(size_t)y * dp + x] = (uint8_t)(s >> 8);"),
    ("luma weight swap", "(77 * p[0] + 150 * p[1] + 29 * p[2] + 128)", "(29 * p[0] + 150 * p[1] + 77 * p[2] + 128)"),
    ("eigenvalue sign", "float den = (float)tr + sqrtf((float)disc);", "float den = (float)tr - sqrtf((float)disc);"),
    ("tensor cross term dropped", "b += gx * gy;", "b += 0;"),
    ("NMS tie rule", "if (!(v > u || (v == u && idx < uidx)))", "if (!(v > u || (v == u && idx > uidx)))"),
    ("threshold not strict", "if (!(v > thr)) continue;", "if (!(v >= thr)) continue;"),
    ("gradient scale", "static double gx_at(const plane_t *P, int x, int y) { return 0.5 * (", "static double gx_at(const plane_t *P, int x, int y) { return 1.0 * ("),
    ("LK update sign", "nx += ex; ny += ey;", "nx -= ex; ny += ey;"),
    ("LK 2x2 solve transposed", "double ex = (Gyy * bx - Gxy * by) / D;", "double ex = (Gxx * bx - Gxy * by) / D;"),
    ("bilinear weight", "(1 - ax) * ay * f(P, x0, y0 + 1)", "ax * ay * f(P, x0, y0 + 1)"),
    ("level scaling", "double px = ldexp(ux, -l), py = ldexp(uy, -l);", "double px = ldexp(ux, -l), py = ldexp(uy, 1 - l);"),
    ("reported min eigenvalue not normalised", "if (lam_min && lam / n < lam_min[0]) { lam_min[0] = lam / n;",
     "if (lam_min && lam < lam_min[0]) { lam_min[0] = lam;"),
    ("backward check skipped", "status[k] = (uint8_t)(s1 && s2 && e <= fb_thresh);", "status[k] = (uint8_t)(s1);"),
    ("splitmix constant", "z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;", "z = (z ^ (z >> 27)) * 0x94D049BB133111EAULL;"),
    ("rotation cross sign", "B += x0 * y1 - x1 * y0;", "B += x1 * y0 - x0 * y1;"),
    ("scale without sqrt", "double sc = rigid ? 1.0 : sqrt(A * A + B * B) / Sxx;", "double sc = rigid ? 1.0 : (A * A + B * B) / Sxx;"),
    ("translation uses dst mean twice", "double tx = mud[0] - sc * (c * mus[0] - sn * mus[1]);", "double tx = mud[0] - sc * (c * mud[0] - sn * mus[1]);"),
    ("smoothing window alignment", "int before = (W - 1) / 2, after = W / 2;", "int before = W / 2, after = (W - 1) / 2;"),
    ("correction sign", "mp[4 * t + c] = m[4 * t + c] + (S[4 * t + c] - C[4 * t + c]);", "mp[4 * t + c] = m[4 * t + c] - (S[4 * t + c] - C[4 * t + c]);"),
    ("warp matrix transposed", "float qx = fmaf(M[0], xf, fmaf(M[1], yf, M[2]));", "float qx = fmaf(M[0], xf, fmaf(M[3], yf, M[2]));"),
    ("warp rounding", "float r = floorf(v + 0.5f);", "float r = floorf(v);"),
    ("inverse warp rotation sign", "double a00 = is * c, a01 = is * sn, a10 = -is * sn, a11 = is * c;", "double a00 = is * c, a01 = -is * sn, a10 = is * sn, a11 = is * c;"),
    ("adjoint rotation term sign", "s * (-ry * gxv + rx * gyv)", "s * (ry * gxv + rx * gyv)"),
    ("crop zoom inverted", "double iz = 1.0 / zoom;", "double iz = zoom;"),
    ("crop composed before the compensation", "P[i][j] += W[i][k] * Zi[k][j];", "P[i][j] += Zi[i][k] * W[k][j];"),
    ("crop zoom about the origin", "double Zi[3][3] = {{iz, 0, cx - iz * cx}, {0, iz, cy - iz * cy}, {0, 0, 1}};",
     "double Zi[3][3] = {{iz, 0, 0}, {0, iz, 0}, {0, 0, 1}};"),
    ("affine determinant sign", "float det = fmaf(u1x, u2y, -(u1y * u2x));", "float det = fmaf(u1x, u2y, (u1y * u2x));"),
    ("affine minimal solve column swap", "m[1] = fmaf(v2x, u1x, -(v1x * u2x)) / det;", "m[1] = fmaf(v1x, u1x, -(v2x * u2x)) / det;"),
    ("affine third index skip order", "    if (c >= lo) c += 1;\n    if (c >= hi) c += 1;", "    if (c >= hi) c += 1;\n    if (c >= lo) c += 1;"),
    ("affine normal equations transposed", "Syx[r][c] += y[r] * x[c];", "Syx[r][c] += y[c] * x[r];"),
    ("affine translation from the source mean", "double ty = mud[1] - (A[1][0] * mus[0] + A[1][1] * mus[1]);",
     "double ty = mud[1] - (A[1][0] * mus[0] + A[1][1] * mud[1]);"),
    ("adjoint image weight", "double wt[4] = {(1 - ax) * (1 - ay), ax * (1 - ay), (1 - ax) * ay, ax * ay};", "double wt[4] = {(1 - ax) * (1 - ay), (1 - ax) * ay, ax * (1 - ay), ax * ay};"),
]

# Mistakes planted in the oracle's Python orchestration (oracle.py).
PY_MUTATIONS = [
    ("hybrid tie goes to rigid", "return e_rigid < e_sim", "return e_rigid <= e_sim"),
    ("hybrid comparison reversed", "return e_rigid < e_sim", "return e_rigid > e_sim"),
    ("hybrid may choose a failed fit", "    if ok_rigid:\n        return True", "    if ok_sim:\n        return True"),
    ("hybrid schedule off by one", "if p.hybrid and (t - 1) % p.dwell == 0:", "if p.hybrid and t % p.dwell == 0:"),
    ("hybrid motion from the other model", "f = fr if rigid else fs", "f = fs if rigid else fr"),
    ("hybrid choice not held", "rigid = cur_rigid if p.hybrid else p.rigid", "rigid = False if p.hybrid else p.rigid"),
    ("detection phase ignored", "(t - 1 + p.redetect_phase) % p.redetect_period == 0", "(t - 1) % p.redetect_period == 0"),
    ("detection phase sign", "(t - 1 + p.redetect_phase) % p.redetect_period == 0",
     "(t - 1 - p.redetect_phase) % p.redetect_period == 0"),
]

PINS = [
    (P.test_luma_hand_values, {}), (P.test_luma_vs_textbook_weights, {}),
    (P.test_pyramid_hand_4x4, {}), (P.test_pyramid_impulse, {}),
    (P.test_pyramid_vs_library_convolution, dict(h=33, w=17)), (P.test_pyramid_vs_library_convolution, dict(h=5, w=7)),
    (P.test_pyramid_constant_and_range, {}),
    (P.test_structure_tensor_vs_scipy, {}), (P.test_lambda_vs_exact_and_eigvalsh, {}),
    (P.test_lambda_edge_flat_and_rotation, {}),
    (P.test_detect_vs_brute_force, dict(seed=0, plateau=False)), (P.test_detect_vs_brute_force, dict(seed=1, plateau=True)),
    (P.test_detect_tie_rule_on_symmetric_blocks, {}), (P.test_detect_threshold_is_strict, {}),
    (P.test_grad_planes_vs_numpy_gradient, {}),
    (P.test_lk_zero_motion_is_exact, {}), (P.test_lk_integer_translation, dict(dx=-7, dy=5)),
    (P.test_lk_subpixel_translation_of_smooth_texture, {}), (P.test_lk_first_iteration_is_the_newton_step, {}),
    (P.test_lk_backward_check_rejects_inconsistent_track, {}),
    (P.test_lk_reported_min_eigenvalue_is_that_of_the_window_tensor, {}),
    (P.test_splitmix64_published_outputs, {}),
    (P.test_ls_closed_form_exact_pairs, dict(rigid=False)), (P.test_ls_matches_svd_procrustes, dict(rigid=False)),
    (P.test_fit_recovers_model_with_outliers, dict(rigid=False)),
    (P.test_smoothing_hand_values, {}), (P.test_smoothing_constant_velocity_and_window_one, {}),
    (P.test_warp_identity_and_integer_shift, {}), (P.test_warp_inverse_of_rotation_is_rot90, {}),
    (P.test_warp_vs_scipy_bilinear, {}), (P.test_warp_inverse_maps_points_back, {}),
    (P.test_charbonnier_gradient_vs_finite_differences, {}),
    (P.test_hybrid_choice_rule, {}), (P.test_hybrid_prefers_similarity_under_a_scale_change, {}),
    (P.test_hybrid_prefers_rigid_when_similarity_buys_inliers_with_error, {}),
    (P.test_crop_zoom_is_a_zoom_about_the_centre, {}), (P.test_crop_zoom_composes_after_the_compensation, {}),
    (P.test_crop_zoom_of_linear_ramp, {}), (P.test_crop_zoom_hides_the_unfilled_border, {}),
    (P.test_sample_triples_distinct_and_uniform, {}), (P.test_affine_exact_pairs_recovered, {}),
    (P.test_affine_refit_is_least_squares_on_inliers, {}), (P.test_affine_of_a_similarity_is_the_similarity, {}),
    (P.test_affine_collinear_points_are_skipped, {}),
    (P.test_hybrid_transitions_on_scripted_pairs, {}), (P.test_hybrid_dwell_schedule_and_bookkeeping, {}),
    (P.test_detection_cycle_and_its_phase, dict(phase=2)),
]


@pytest.fixture(scope="module")
def tmpdir_mod():
    with tempfile.TemporaryDirectory() as d:
        yield d


@pytest.mark.parametrize("name,orig,bad", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(name, orig, bad, tmpdir_mod):
    src = open(SRC).read()
    assert src.count(orig) >= 1, f"mutation site not found: {orig}"
    path_c = os.path.join(tmpdir_mod, f"m{abs(hash(name))}.c")
    path_so = path_c[:-2] + ".so"
    open(path_c, "w").write(src.replace(orig, bad))
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", path_so, path_c,
                           "-lm"])
    prev = O.use_library(path_so)
    caught = None
    try:
        for fn, kw in PINS:
            try:
                fn(**kw)
            except Exception as e:           # a pin failed (assertion or error): mistake caught
                caught = f"{fn.__name__}: {type(e).__name__}"
                break
    finally:
        O.restore_library(prev)
    assert caught is not None, f"no pin caught the planted mistake '{name}'"


def _first_failing_pin():
    for fn, kw in PINS:
        try:
            fn(**kw)
        except Exception as e:               # a pin failed (assertion or error): mistake caught
            return f"{fn.__name__}: {type(e).__name__}"
    return None


@pytest.mark.parametrize("name,orig,bad", PY_MUTATIONS, ids=[m[0] for m in PY_MUTATIONS])
def test_planted_python_mistake_is_caught(name, orig, bad):
    src = open(O.__file__).read()
    assert src.count(orig) >= 1, f"mutation site not found: {orig}"
    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = O.__file__
    sys.modules["oracle_mutant"] = mod
    try:
        exec(compile(src.replace(orig, bad), O.__file__, "exec"), mod.__dict__)
        P.O = mod
        caught = _first_failing_pin()
    finally:
        P.O = O
        del sys.modules["oracle_mutant"]
    assert caught is not None, f"no pin caught the planted mistake '{name}'"
