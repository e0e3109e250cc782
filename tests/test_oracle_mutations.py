"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a temporary copy of the oracle's C source (a
dropped rounding term, a flipped sign, a transposed operand, an off-by-one
comparison ...), builds it, points the oracle wrapper at the broken build and
runs the pin battery of test_oracle_pins.py.  At least one pin must fail for
every planted mistake.  The cross-check against the Python restatement is
left out of the battery on purpose: the pins alone must catch each mistake.
Everything here runs on the CPU.
"""
import os
import subprocess

import pytest

import oracle

from . import test_oracle_lk as lk_pins
from . import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "evsim_oracle.c")

MUTATIONS = {
    "offset_sign": ("(int64_t)x * 65536 - offx", "(int64_t)x * 65536 + offx"),
    "flow_components_swapped": ("p1x = p0x + Fx[p], p1y = p0y + Fy[p]",
                                "p1x = p0x + Fy[p], p1y = p0y + Fx[p]"),
    "rounding_term_dropped": ("(b - a) * w + 2048, 4096", "(b - a) * w, 4096"),
    "accum_strict_compare": ("if (D >= cp) {", "if (D > cp) {"),
    "weight_floor_not_rounded": ("((int64_t)k * 8192 + N) / (2 * (int64_t)N)",
                                 "((int64_t)k * 4096) / (int64_t)N - (k < N ? 0 : 0) + 0 * N"),
    "taps_transposed": ("int64_t l00 = L[iy * W + ix], l01 = L[iy * W + x1];",
                        "int64_t l00 = L[iy * W + ix], l01 = L[y1 * W + ix];"),
    "time_rounded_not_floored": ("floordiv((int64_t)k * dt, N)", "(((int64_t)k * dt + N / 2) / N)"),
    "fraction_before_clamp": [("  if (px < 0) px = 0;", "  int64_t fx0 = (px & 0xFFFF) >> 4;\n  if (px < 0) px = 0;"),
                              ("int64_t fx = (px & 0xFFFF) >> 4,", "int64_t fx = fx0,")],
    "offset_truncated": ("floordiv((int64_t)Fx[p] * k, N)", "(((int64_t)Fx[p] * k) / N)"),
    "reset_non_strict": ("            if (D > cp)\n              emit(out, cap, &n, crossing",
                         "            if (D >= cp)\n              emit(out, cap, &n, crossing"),
    "log_base_2": ("65536.0 * log((double)v + 1.0)", "65536.0 * log2((double)v + 1.0)"),
    "luma_weights_swapped": ("77 * r + 150 * g + 29 * b", "29 * r + 150 * g + 77 * b"),
    "reference_moves_one_step": ("R[p] = (int32_t)(R[p] + m * cp);", "R[p] = (int32_t)(R[p] + cp);"),
    "activity_strict": ("a = d >= cact;", "a = d > cact;"),
    "adaptive_off_by_one": ("(int64_t)n * n * 4294967296LL < max_f2",
                            "(int64_t)n * n * 4294967296LL <= max_f2"),
    "y_fraction_from_x": ("fy = (py & 0xFFFF) >> 4", "fy = (px & 0xFFFF) >> 4"),
    "column_major_order": ("for (int32_t y = y0; y < y1; ++y) {\n        for (int32_t x = 0; x < W; ++x) {",
                           "for (int32_t x = 0; x < W; ++x) {\n        for (int32_t y = y0; y < y1; ++y) {"),
    "polarity_bit_inverted": ("(y << 1) | (pos ? 1 : 0)", "(y << 1) | (pos ? 0 : 1)"),
    "flow_floored": ("(int32_t)nearbyint(d * 65536.0)", "(int32_t)floor(d * 65536.0)"),
    "reset_starts_from_new_frame": ("if (c->ref_mode == ORC_RESET) memcpy(R, Lprev,",
                                    "if (c->ref_mode == ORC_RESET) memcpy(R, Lcur,"),
    "negative_reference_step": ("R[p] = (int32_t)(R[p] - m * cn);", "R[p] = (int32_t)(R[p] - m * cp);"),
    "clamp_y_one_row_short": ("maxy = (int64_t)(H - 1) * 65536", "maxy = (int64_t)(H - 2) * 65536"),
    "time_base_from_current_frame": ("int64_t t_prev = t_us[i - 1] - t_us[0];",
                                     "int64_t t_prev = t_us[i] - t_us[0] - (t_us[1] - t_us[0]);"),
    # difference-frame interpolation (orc_run_diff)
    "diff_planes_swapped": [("int64_t s0 = orc_bilinear(Dp, W, H, p0x, p0y);",
                             "int64_t s0 = orc_bilinear(Dc, W, H, p0x, p0y);"),
                            ("int64_t s1 = orc_bilinear(Dc, W, H, p1x, p1y);",
                             "int64_t s1 = orc_bilinear(Dp, W, H, p1x, p1y);")],
    "diff_current_plane_sign": ("Dc[p] = L0[p] - L1[p];", "Dc[p] = L1[p] - L0[p];"),
    "diff_previous_plane_skips_a_frame": ("Dp[p] = L1[p] - L2[p];", "Dp[p] = L0[p] - L2[p];"),
    "diff_non_strict_threshold": ("if (I > cp) emit(out, cap, &n, tk, x, y, 1);",
                                  "if (I >= cp) emit(out, cap, &n, tk, x, y, 1);"),
    "diff_offset_sign": ("int64_t s0 = orc_bilinear(Dp, W, H, p0x, p0y);",
                         "int64_t s0 = orc_bilinear(Dp, W, H, p0x + 2 * offx, p0y);"),
    "accumulate_polarity_inverted": ("frame[(int64_t)y * W + x] += (ev[i].yp & 1) ? 1 : -1;",
                                     "frame[(int64_t)y * W + x] += (ev[i].yp & 1) ? -1 : 1;"),
    "accumulate_window_end_inclusive": ("if (t < t_begin || t >= t_end) continue;",
                                        "if (t < t_begin || t > t_end) continue;"),
    "accumulate_transposed": ("frame[(int64_t)y * W + x] +=", "frame[(int64_t)x * H + y] +="),
    "activity_default_uses_the_larger_threshold": ("(cp < cn ? cp : cn);", "(cp > cn ? cp : cn);"),
    "no_horizontal_neighbour": ("int64_t x1 = ix + 1 < W ? ix + 1 : W - 1;", "int64_t x1 = ix;"),
    "threshold_maps_swapped": ("          int32_t cp = pixel_threshold(cpos_map, c->c_pos_q16, p);\n"
                               "          int32_t cn = pixel_threshold(cneg_map, c->c_neg_q16, p);\n"
                               "          int64_t D = I - R[p];",
                               "          int32_t cp = pixel_threshold(cneg_map, c->c_pos_q16, p);\n"
                               "          int32_t cn = pixel_threshold(cpos_map, c->c_neg_q16, p);\n"
                               "          int64_t D = I - R[p];"),
    "luma_rounding_dropped": ("(77 * r + 150 * g + 29 * b + 128) >> 8", "(77 * r + 150 * g + 29 * b) >> 8"),
    "linear_table_scale": ("lut[v] = v * 65536;", "lut[v] = v * 65535;"),
    "nan_flow_not_zeroed": ("  if (d != d) return 0;\n", "\n"),
    "activity_against_the_reference": ("int64_t d = (int64_t)Lcur[p] - Lprev[p];",
                                       "int64_t d = (int64_t)Lcur[p] - R[p];"),
    "adaptive_n_over_inactive_pixels": ("        if (!act[p]) continue;\n        int64_t f2",
                                        "        int64_t f2"),
    "accum_negative_strict": ("} else if (-D >= cn) {", "} else if (-D > cn) {"),
    "reset_negative_non_strict": ("else if (D < -(int64_t)cn)", "else if (D <= -(int64_t)cn)"),
    "accumulate_window_start_exclusive": ("if (t < t_begin || t >= t_end) continue;",
                                          "if (t <= t_begin || t >= t_end) continue;"),
    "diff_starts_at_the_second_frame": ("    if (i < 2) continue;", "    if (i < 1) continue;"),
    "diff_flow_of_the_previous_frame": ("    const float* fl = flows + (int64_t)i * P * 2;\n    int64_t m = 0;",
                                        "    const float* fl = flows + (int64_t)(i - 1) * P * 2;\n    int64_t m = 0;"),
    "diff_negative_threshold_uses_cp": ("else if (I < -(int64_t)cn) emit(", "else if (I < -(int64_t)cp) emit("),
    "diff_time_from_the_frame_before_last": ("    int64_t t_prev = t_us[i - 1] - t_us[0];\n    int64_t dt = t_us[i] - t_us[i - 1];\n    for (int32_t k = 1; k <= N; ++k) {\n      int64_t w = ((int64_t)k * 8192 + N) / (2 * (int64_t)N);\n      uint32_t tk = (uint32_t)(t_prev + floordiv((int64_t)k * dt, N));\n      for (int32_t y = 0; y < H; ++y) {\n        for (int32_t x = 0; x < W; ++x) {\n          int64_t p = (int64_t)y * W + x;\n          /* interpolated difference",
                                             "    int64_t t_prev = t_us[i - 2] - t_us[0];\n    int64_t dt = t_us[i] - t_us[i - 1];\n    for (int32_t k = 1; k <= N; ++k) {\n      int64_t w = ((int64_t)k * 8192 + N) / (2 * (int64_t)N);\n      uint32_t tk = (uint32_t)(t_prev + floordiv((int64_t)k * dt, N));\n      for (int32_t y = 0; y < H; ++y) {\n        for (int32_t x = 0; x < W; ++x) {\n          int64_t p = (int64_t)y * W + x;\n          /* interpolated difference"),
    "fraction_has_thirteen_bits": ("int64_t fx = (px & 0xFFFF) >> 4,", "int64_t fx = (px & 0xFFFF) >> 3,"),
    "interval_from_the_first_frame": ("    int64_t dt = t_us[i] - t_us[i - 1];\n    if (dt <= 0)",
                                      "    int64_t dt = t_us[i] - t_us[0];\n    if (dt <= 0)"),
    "sparse_inactive_pixels_simulated": ("          if (!act[p]) continue;\n          /* Interpolated frame",
                                         "          /* Interpolated frame"),
    # per-crossing event times (orc_crossing_time and its callers)
    "crossing_level_counted_from_zero": ("orc_crossing_time(tk1, tk, ip, I, Rb + j * cp, 1)",
                                         "orc_crossing_time(tk1, tk, ip, I, Rb + (j - 1) * cp, 1)"),
    "crossing_from_substep_end_time": ("int64_t tk1 = t_prev + floordiv((int64_t)(k - 1) * dt, N);",
                                       "int64_t tk1 = t_prev + floordiv((int64_t)k * dt, N);"),
    "crossing_previous_value_kept_at_frame": ("          Iprev[p] = (int32_t)I;\n", "\n"),
    "crossing_falling_measured_as_rising": ("int64_t num = rising ? level - i_prev : i_prev - level;",
                                            "int64_t num = level - i_prev;"),
    "crossing_time_rounded": ("return t_prev + floordiv((t_cur - t_prev) * num, den);",
                              "return t_prev + ((t_cur - t_prev) * num + den / 2) / den;"),
    "crossing_negative_level_uses_cp": ("orc_crossing_time(tk1, tk, ip, I, Rb - j * cn, 0)",
                                        "orc_crossing_time(tk1, tk, ip, I, Rb - j * cp, 0)"),
    "diff_blend_reversed": ("int64_t I = lerp_q12(s0, s1, w);\n          int32_t cp = pixel_threshold(cpos_map, c->c_pos_q16, p);\n          int32_t cn = pixel_threshold(cneg_map, c->c_neg_q16, p);\n          if (I > cp)",
                            "int64_t I = lerp_q12(s1, s0, w);\n          int32_t cp = pixel_threshold(cpos_map, c->c_pos_q16, p);\n          int32_t cn = pixel_threshold(cneg_map, c->c_neg_q16, p);\n          if (I > cp)"),
    # pyramidal Lucas-Kanade flow (orc_flow_lk)
    "lk_gradient_sign_in_the_window_matrix": (
        "const int64_t ix = (int64_t)lk_at(Il, w, h, qx + 1, qy) - lk_at(Il, w, h, qx - 1, qy);",
        "const int64_t ix = (int64_t)lk_at(Il, w, h, qx - 1, qy) - lk_at(Il, w, h, qx + 1, qy);"),
    "lk_guess_not_doubled": [("gx = 2 * Dp[2 * pp];", "gx = Dp[2 * pp];"),
                             ("gy = 2 * Dp[2 * pp + 1];", "gy = Dp[2 * pp + 1];")],
    "lk_update_sign": ("const double scale = -131072.0 / det;",
                       "const double scale = 131072.0 / det;"),
    "lk_components_swapped": [("vx += (int64_t)nearbyint(nx * scale);",
                               "vx += (int64_t)nearbyint(ny * scale);"),
                              ("vy += (int64_t)nearbyint(ny * scale);",
                               "vy += (int64_t)nearbyint(nx * scale);")],
    "lk_window_short_by_one": ("          for (int j = -r; j <= r; ++j)\n            for (int i = -r; i <= r; ++i) {",
                               "          for (int j = -r; j < r; ++j)\n            for (int i = -r; i <= r; ++i) {"),
    "lk_temporal_difference_sign": ("const int64_t it = jv - lk_at(Il, w, h, qx, qy);",
                                    "const int64_t it = lk_at(Il, w, h, qx, qy) - jv;"),
    "lk_eigenvalue_test_dropped": ("if (lmin / area >= c->min_eig && det > 0.0) {", "if (det > 0.0) {"),
    "lk_second_frame_not_sampled": ("lk_bilinear(Jl, w, h, qx * 65536 + gx + vx, qy * 65536 + gy + vy);",
                                    "lk_bilinear(Il, w, h, qx * 65536 + gx + vx, qy * 65536 + gy + vy);"),
}


def battery():
    """The pins, each with fixed arguments."""
    yield pins.test_lut_log_closed_form
    yield pins.test_lut_linear
    yield pins.test_luma_bt601
    yield pins.test_flow_q16
    for a, b, c in [(20, 1, 2), (200, -1, -1), (40, 2, 1), (100, 0, -2)]:
        yield lambda a=a, b=b, c=c: pins.test_bilinear_of_a_plane(a, b, c)
    yield pins.test_bilinear_at_integer_positions_is_indexing
    yield pins.test_adaptive_substeps_is_ceil_of_max_flow
    yield lambda: pins.test_identical_frames_zero_flow_no_events(oracle.SPARSE, oracle.ACCUM, oracle.LOG)
    yield lambda: pins.test_identical_frames_zero_flow_no_events(oracle.DENSE, oracle.RESET, oracle.LINEAR)
    for N in (1, 5, 8):
        yield lambda N=N: pins.test_uniform_step_gives_floor_of_difference_over_C(N, 9000, 17000)
    yield pins.test_alternating_steps_give_alternating_bursts
    yield lambda: pins.test_exhaustive_one_pixel_pairs(7, oracle.LOG, 3001)
    yield lambda: pins.test_exhaustive_one_pixel_pairs(1, oracle.LINEAR, 7 * 65536 + 5)
    for m, N in [((1, 0), 3), ((0, -1), 4), ((1, -1), 2), ((-2, 1), 3)]:
        for ref in (oracle.ACCUM, oracle.RESET):
            yield lambda m=m, N=N, ref=ref: pins.test_integer_translation_reproduces_shifted_samples(m, N, ref)
    for N in (3, 8):
        yield lambda N=N: pins.test_plane_images_with_fractional_flow(N)
    for N in (2, 5, 8):
        yield lambda N=N: pins.test_plane_with_subpixel_flow_at_unit_resolution(N)
    yield pins.test_blend_is_within_half_a_unit_of_the_exact_line
    yield pins.test_conservation_and_band_invariant
    yield pins.test_kaiser_difference_frame_special_case
    yield pins.test_sparse_with_zero_activity_threshold_equals_dense
    yield pins.test_sparse_misses_pixels_just_under_the_activity_threshold
    yield pins.test_time_order_and_raster_order
    yield pins.test_rgb_input_uses_bt601_luma
    yield pins.test_per_pixel_threshold_maps
    yield pins.test_adaptive_substeps_per_frame
    yield pins.test_diff_one_substep_is_the_kaiser_difference_frame
    for N in (4, 10):
        for v in [(40, 120, 30), (200, 90, 210), (128, 130, 250)]:
            yield lambda N=N, v=v: pins.test_diff_uniform_frames_follow_the_exact_line(N, v)
    for s_, N in [((1, 0), 3), ((0, -1), 4), ((1, 1), 2), ((-2, 1), 2)]:
        yield lambda s_=s_, N=N: pins.test_diff_translation_reproduces_shifted_difference_samples(s_, N)
    for v0, v1 in [(60, 200), (220, 35), (128, 128)]:
        yield lambda v0=v0, v1=v1: pins.test_accumulated_frame_of_a_uniform_step(v0, v1)
    yield pins.test_accumulated_frame_positions_polarity_and_window
    for N in (1, 4):
        for cp, cn in [(40000, 40000), (70001, 123457)]:
            yield lambda N=N, cp=cp, cn=cn: \
                pins.test_crossing_times_of_monotone_ramps_follow_the_exact_line(N, cp, cn)
    yield lambda: pins.test_crossing_times_reset_one_substep(5 * 65536 + 123)
    yield pins.test_crossing_time_primitive_properties
    yield pins.test_sparse_default_activity_threshold_is_the_smaller_threshold
    yield pins.test_sparse_disregards_slow_drift_below_the_activity_threshold
    yield pins.test_sparse_adaptive_substeps_follow_the_active_pixels_only
    yield lambda: pins.test_crossing_times_keep_events_and_stay_inside_their_substep(
        oracle.SPARSE, oracle.ACCUM)
    # Lucas-Kanade flow
    yield lk_pins.test_identical_frames_give_zero_flow
    yield lk_pins.test_untextured_frames_are_not_tracked
    for u, v in [(2, 0), (0, -2), (2, -2), (-4, 2)]:
        yield lambda u=u, v=v: lk_pins.test_exactly_linear_motion_is_recovered_exactly(u, v)
    yield lk_pins.test_transposed_frames_give_the_transposed_flow_at_one_step
    yield lk_pins.test_mirrored_frames_give_the_mirrored_flow_at_one_step
    yield lk_pins.test_one_dimensional_texture_is_not_tracked
    yield lk_pins.test_translation_is_recovered_to_a_fraction_of_a_pixel
    yield lk_pins.test_motion_beyond_the_window_needs_the_pyramid
    yield lk_pins.test_rgb_frames_give_the_flow_of_their_luma
    yield lk_pins.test_no_window_passes_an_unreachable_eigenvalue_threshold


def test_battery_passes_on_the_real_oracle():
    for pin in battery():
        pin()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    subs = MUTATIONS[name]
    if isinstance(subs, tuple):
        subs = [subs]
    bad = open(SRC).read()
    for old, new in subs:
        assert bad.count(old) >= 1, f"mutation anchor missing: {name}"
        bad = bad.replace(old, new, 1)
    c_path = tmp_path / "mutant.c"
    c_path.write_text(bad)
    so = tmp_path / "libmutant.so"
    inc = os.path.dirname(SRC)
    subprocess.run(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                    "-I", inc, "-o", str(so), str(c_path), "-lm"], check=True)
    oracle.use_library(str(so))
    caught = []
    try:
        for pin in battery():
            try:
                pin()
            except (AssertionError, ValueError):
                caught.append(getattr(pin, "__name__", "pin"))
                break
    finally:
        oracle.use_library(None)
    assert caught, f"no pin caught the planted mistake '{name}'"
