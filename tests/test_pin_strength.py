"""Strength of the oracle's pins.  Each mutant plants one plausible mistake (a
dropped term, a wrong sign, bound, index, operand or rounding) in a copy of
the oracle's C source, on the CPU; the pin files (tests/test_oracle_*.py,
which check the oracle against the paper's worked examples, closed forms,
invariants, library routines and brute force -- never against the CUDA path)
must then report failing tests.  The unmutated copy must pass them, so a
mutant counts as caught only by a genuine test failure (pytest exit code 1),
not by a crash or a collection error."""
import glob
import os
import re
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "jslam_oracle.c")
# unit pins first: a mutant that breaks the level geometry or the culling
# cap then fails there, before the whole-image pipeline can overrun a buffer
_FIRST = ("pyramid", "fast", "pyca", "orb")
PINS = sorted(glob.glob(os.path.join(ROOT, "tests", "test_oracle_*.py")),
              key=lambda f: (next((i for i, k in enumerate(_FIRST) if f.endswith(f"_{k}.py")), len(_FIRST)), f))

# (name, text in the source, replacement, which occurrence (0 = first))
MUTANTS = [
    # geometry and pyramid (Sec. III; reading of the resampling)
    ("scale_power_off_by_one", "for (int32_t i = 0; i < n; ++i) s = s * (double)scale;",
     "for (int32_t i = 0; i <= n; ++i) s = s * (double)scale;", 0),
    ("level_width_truncated", "W[n] = (int32_t)floor((double)W0 / s + 0.5);",
     "W[n] = (int32_t)floor((double)W0 / s);", 0),
    ("cell_size_rounded", "int32_t cn = (int32_t)floor((double)cell / s);",
     "int32_t cn = (int32_t)floor((double)cell / s + 0.5);", 0),
    ("cell_size_may_reach_zero", "c[n] = cn < 1 ? 1 : cn;", "c[n] = cn;", 0),
    ("bilinear_corner_aligned", "double u = ((double)x + 0.5) * s - 0.5;", "double u = (double)x * s;", 0),
    ("bilinear_weight_truncated", "int32_t w = (int32_t)floor((u - (double)i) * 256.0 + 0.5);",
     "int32_t w = (int32_t)floor((u - (double)i) * 256.0);", 0),
    ("bilinear_vertical_uses_x_weight", "uint32_t v = (256u - (uint32_t)b) * top + (uint32_t)b * bot;",
     "uint32_t v = (256u - (uint32_t)a) * top + (uint32_t)a * bot;", 0),
    ("bilinear_weights_swapped", "uint32_t top = (256u - (uint32_t)a) * p00 + (uint32_t)a * p01;",
     "uint32_t top = (uint32_t)a * p00 + (256u - (uint32_t)a) * p01;", 0),
    ("bilinear_no_rounding", "out[(size_t)y * pitch_out + x] = (uint8_t)((v + 32768u) >> 16);",
     "out[(size_t)y * pitch_out + x] = (uint8_t)(v >> 16);", 0),
    ("pyramid_rounds_ties_down", "out[(size_t)y * pitch_out + x] = (uint8_t)((v + 32768u) >> 16);",
     "out[(size_t)y * pitch_out + x] = (uint8_t)((v + 32767u) >> 16);", 0),
    ("bilinear_shift_at_255", "if (w == 256) { i += 1; w = 0; }", "if (w == 255) { i += 1; w = 0; }", 0),
    # Gaussian (Sec. III; reading 2)
    ("blur_sigma_sqrt2", "g[i + 3] = exp(-(double)(i * i) / (2.0 * 2.0 * 2.0));",
     "g[i + 3] = exp(-(double)(i * i) / (2.0 * 2.0));", 0),
    ("blur_rounding_to_edge_tap", "w[3] += 256 - total;", "w[0] += 256 - total;", 0),
    ("clamp_low_to_high", "return v < lo ? lo : (v > hi ? hi : v);", "return v < lo ? hi : (v > hi ? hi : v);", 0),
    ("blur_border_shifted", "acc += (uint32_t)w[i + 3] * in[(size_t)y * pitch_in + clampi(x + i, 0, W - 1)];",
     "acc += (uint32_t)w[i + 3] * in[(size_t)y * pitch_in + clampi(x + i, 1, W - 1)];", 0),
    ("blur_no_rounding", "out[(size_t)y * pitch_out + x] = (uint8_t)((acc + 32768u) >> 16);",
     "out[(size_t)y * pitch_out + x] = (uint8_t)(acc >> 16);", 0),
    ("blur_vertical_border", "acc += (uint32_t)w[j + 3] * h[(size_t)clampi(y + j, 0, H - 1) * W + x];",
     "acc += (uint32_t)w[j + 3] * h[(size_t)clampi(y + j, 0, H - 2) * W + x];", 0),
    ("blur_rounds_ties_down", "out[(size_t)y * pitch_out + x] = (uint8_t)((acc + 32768u) >> 16);",
     "out[(size_t)y * pitch_out + x] = (uint8_t)((acc + 32767u) >> 16);", 0),
    ("blur_rounds_just_below_half_up", "out[(size_t)y * pitch_out + x] = (uint8_t)((acc + 32768u) >> 16);",
     "out[(size_t)y * pitch_out + x] = (uint8_t)((acc + 32769u) >> 16);", 0),
    # FAST with Bounded Rectification (Sec. II-A, Eq. 1-3)
    ("ring_mirrored", "static const int32_t RING_DY[16] = { 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1, 0, 1, 2, 3 };",
     "static const int32_t RING_DY[16] = { -3, -3, -2, -1, 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3 };", 0),
    ("ring_axes_swapped", "dx[k] = RING_DX[k]; dy[k] = RING_DY[k];", "dx[k] = RING_DY[k]; dy[k] = RING_DX[k];", 0),
    ("bright_not_strict", "if (d > eps) Bb |= 1u << k;", "if (d >= eps) Bb |= 1u << k;", 0),
    ("dark_not_strict", "if (d < -eps) Bd |= 1u << k;", "if (d <= -eps) Bd |= 1u << k;", 0),
    ("response_over_arc_only", "r += d < 0 ? -d : d;", "r += (d > eps || d < -eps) ? (d < 0 ? -d : d) : 0;", 0),
    ("run_without_wraparound", "while (len < 16 && ((mask >> ((start + len) % 16)) & 1u)) ++len;",
     "while (start + len < 16 && ((mask >> (start + len)) & 1u)) ++len;", 0),
    ("eq3_conjunctive", "return (nb >= p_min && nb <= p_max) || (nd >= p_min && nd <= p_max);",
     "return (nb >= p_min && nb <= p_max) && (nd >= p_min && nd <= p_max);", 0),
    ("eq3_upper_bound_exclusive", "return (nb >= p_min && nb <= p_max) || (nd >= p_min && nd <= p_max);",
     "return (nb >= p_min && nb < p_max) || (nd >= p_min && nd < p_max);", 0),
    ("eq3_dark_polarity_dropped", "return (nb >= p_min && nb <= p_max) || (nd >= p_min && nd <= p_max);",
     "return (nb >= p_min && nb <= p_max);", 0),
    ("border_one_row_short", "for (int32_t y = border; y < H - border; ++y)",
     "for (int32_t y = border; y <= H - border; ++y)", 0),
    # Feature Culling (Sec. II-C-1)
    ("cull_fallback_replaces", "            if (!any_hi) {\n                if (!corner_lo) continue;",
     "            if (!any_hi || corner_lo) {\n                if (!corner_lo) continue;", 0),
    # Feature Culling (Sec. II-C-1)
    ("cull_weakest_first", "if (a->r != b->r) return a->r > b->r ? -1 : 1;",
     "if (a->r != b->r) return a->r < b->r ? -1 : 1;", 0),
    ("cull_tie_x_before_y", "    if (a->y != b->y) return a->y < b->y ? -1 : 1;\n    if (a->x != b->x) return a->x < b->x ? -1 : 1;\n    return 0;\n}\n\nint32_t or_cull_level",
     "    if (a->x != b->x) return a->x < b->x ? -1 : 1;\n    if (a->y != b->y) return a->y < b->y ? -1 : 1;\n    return 0;\n}\n\nint32_t or_cull_level", 0),
    ("cull_no_fallback", "if (!corner_lo) continue;", "continue;", 0),
    ("cull_partial_cells_dropped", "int32_t cells_x = (W + c - 1) / c, cells_y = (H + c - 1) / c;",
     "int32_t cells_x = W / c, cells_y = H / c;", 0),
    ("cull_k_plus_one", "for (int32_t i = 0; i < m && i < k; ++i) {", "for (int32_t i = 0; i < m && i <= k; ++i) {", 0),
    # Pyramidal Feature Aggregation (Sec. II-C-2)
    ("pfa_rule1_equal_scores_dominate", ": (Kl[qp] > kl || (Kl[qp] == kl && Kr[qp] > kr));",
     ": (Kl[qp] > kl || (Kl[qp] == kl && Kr[qp] >= kr));", 0),
    ("projection_truncated", "int32_t X = (int32_t)floor((double)x * s + 0.5);",
     "int32_t X = (int32_t)floor((double)x * s);", 0),
    ("kl_counts_every_scale", "Kl[p] += occ[(size_t)n * plane + p];", "Kl[p] += 1;", 0),
    ("kr_counts_instead_of_sums", "M[at] = r[i];", "M[at] = 1;", 0),
    ("nms_window_too_wide", "int32_t rad = (q - 1) / 2;", "int32_t rad = q - 1;", 0),
    ("nms_kl_not_strict", "int32_t dom = rule == 0 ? (Kl[qp] > kl && Kr[qp] > kr)",
     "int32_t dom = rule == 0 ? (Kl[qp] >= kl && Kr[qp] > kr)", 0),
    ("nms_either_score", "int32_t dom = rule == 0 ? (Kl[qp] > kl && Kr[qp] > kr)",
     "int32_t dom = rule == 0 ? (Kl[qp] > kl || Kr[qp] > kr)", 0),
    ("nms_lexicographic_reversed", ": (Kl[qp] > kl || (Kl[qp] == kl && Kr[qp] > kr));",
     ": (Kr[qp] > kr || (Kr[qp] == kr && Kl[qp] > kl));", 0),
    # orientation (Sec. III, ORB)
    ("moments_swapped", "m10 += dx * v;\n            m01 += dy * v;", "m10 += dy * v;\n            m01 += dx * v;", 0),
    ("disk_boundary_excluded", "if (dx * dx + dy * dy > OR_DISK_R * OR_DISK_R) continue;",
     "if (dx * dx + dy * dy >= OR_DISK_R * OR_DISK_R) continue;", 0),
    ("atan2_arguments_swapped", "*theta = atan2((double)m01, (double)m10);",
     "*theta = atan2((double)m10, (double)m01);", 0),
    ("sector_tables_swapped", "cosb[b] = cos(phi);\n        sinb[b] = sin(phi);", "cosb[b] = sin(phi);\n        sinb[b] = cos(phi);", 0),
    ("sector_test_sign", "double t = t1 - t2;", "double t = t1 + t2;", 0),
    ("sector_boundary_open", "return t >= 0.0;", "return t > 0.0;", 0),
    # steered BRIEF (Sec. III)
    ("splitmix_shift", "z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;", "z = (z ^ (z >> 28)) * 0x94D049BB133111EBull;", 0),
    ("uniform_scale_doubled", "double u1 = (double)((or_splitmix64_next(state) >> 11) + 1) * (1.0 / 9007199254740992.0);",
     "double u1 = (double)((or_splitmix64_next(state) >> 11) + 1) * (2.0 / 9007199254740992.0);", 0),
    ("pattern_sigma_31_4", "const double sigma = 31.0 / 5.0;", "const double sigma = 31.0 / 4.0;", 0),
    ("pattern_radius_14", "if (v[0] * v[0] + v[1] * v[1] > 169) continue;",
     "if (v[0] * v[0] + v[1] * v[1] > 196) continue;", 0),
    ("pattern_rejects_shared_y", "if (v[0] == v[2] && v[1] == v[3]) continue;",
     "if (v[0] != v[2] && v[1] == v[3]) continue;", 0),
    ("pattern_rejects_shared_x", "if (v[0] == v[2] && v[1] == v[3]) continue;",
     "if (v[0] == v[2] && v[1] != v[3]) continue;", 0),
    ("pattern_rotated_backwards", "double xr = cx - sy;\n                double yr = sx + cy;",
     "double xr = cx + sy;\n                double yr = cy - sx;", 0),
    ("descriptor_comparison_reversed", "if (a < b) desc[i / 32] |= 1u << (i % 32);",
     "if (a > b) desc[i / 32] |= 1u << (i % 32);", 0),
    ("descriptor_bit_order_reversed", "if (a < b) desc[i / 32] |= 1u << (i % 32);",
     "if (a < b) desc[i / 32] |= 1u << (31 - i % 32);", 0),
    ("descriptor_xy_swapped", "int32_t a = blur[(size_t)(y + py) * pitch + (x + px)];",
     "int32_t a = blur[(size_t)(y + px) * pitch + (x + py)];", 0),
    ("pattern_rotation_truncated", "out[((size_t)b * OR_NPAIRS + i) * 4 + pt * 2 + 0] = (int8_t)lround(xr);",
     "out[((size_t)b * OR_NPAIRS + i) * 4 + pt * 2 + 0] = (int8_t)xr;", 0),
    # whole-image pipeline (cap, order, levels used)
    ("cap_kr_before_kl", "    if (a->kl != b->kl) return a->kl > b->kl ? -1 : 1;\n    if (a->kr != b->kr) return a->kr > b->kr ? -1 : 1;",
     "    if (a->kr != b->kr) return a->kr > b->kr ? -1 : 1;\n    if (a->kl != b->kl) return a->kl > b->kl ? -1 : 1;", 0),
    ("canonical_x_before_y", "    if (a->y != b->y) return a->y < b->y ? -1 : 1;\n    if (a->x != b->x) return a->x < b->x ? -1 : 1;\n    return 0;\n}\n\nint32_t or_check_params",
     "    if (a->x != b->x) return a->x < b->x ? -1 : 1;\n    if (a->y != b->y) return a->y < b->y ? -1 : 1;\n    return 0;\n}\n\nint32_t or_check_params", 0),
    ("cap_tie_skips_y", "    if (a->y != b->y) return a->y < b->y ? -1 : 1;\n    if (a->x != b->x) return a->x < b->x ? -1 : 1;\n    return 0;\n}\n\nstatic int cmp_canonical",
     "    if (a->y == b->y) return a->y < b->y ? -1 : 1;\n    if (a->x != b->x) return a->x < b->x ? -1 : 1;\n    return 0;\n}\n\nstatic int cmp_canonical", 0),
    ("fallback_needs_eps_lo_2", "if (p->fast_thresh_lo > 0) {", "if (p->fast_thresh_lo > 1) {", 0),
    ("params_pfa_rule_unchecked", "if (p->pfa_rule < 0 || p->pfa_rule > 1) return -1;",
     "if (p->pfa_rule < 0 || p->pfa_rule > 1) return 0;", 0),
    ("extract_ignores_invalid_params", "if (or_check_params(W0, H0, p) != 0) return -1;",
     "if (or_check_params(W0, H0, p) != 0) return 0;", 0),
    ("params_nms_q_parity_bit", "(p->nms_q & 1) == 0", "(p->nms_q & 2) == 0", 0),
    ("params_levels_from_2", "if (p->levels < 1 || p->levels > OR_MAX_LEVELS) return -1;",
     "if (p->levels < 2 || p->levels > OR_MAX_LEVELS) return -1;", 0),
    ("fallback_runs_at_eps_0", "if (p->fast_thresh_lo > 0) {", "if (p->fast_thresh_lo >= 0) {", 0),
    ("params_threshold_254_rejected", "p->fast_thresh > 254) return -1;", "p->fast_thresh >= 254) return -1;", 0),
    ("params_cell_128_rejected", "if (p->cell < 1 || p->cell > 128) return -1;",
     "if (p->cell < 1 || p->cell >= 128) return -1;", 0),
    ("params_border_16_rejected", "if (p->border < 16) return -1;", "if (p->border <= 16) return -1;", 0),
    ("params_size_4096_rejected", "W0 > 4096 || H0 > 4096) return -1;", "W0 >= 4096 || H0 > 4096) return -1;", 0),
    ("params_level_size_39_rejected", "if (W[n] < 2 * p->border + 1 || H[n] < 2 * p->border + 1) return -1;",
     "if (W[n] <= 2 * p->border + 1 || H[n] < 2 * p->border + 1) return -1;", 0),
    ("cap_ignores_summed_response", "    if (a->kl != b->kl) return a->kl > b->kl ? -1 : 1;\n    if (a->kr != b->kr) return a->kr > b->kr ? -1 : 1;\n",
     "    if (a->kl != b->kl) return a->kl > b->kl ? -1 : 1;\n", 0),
    ("angle_bin_not_stored", "out->angle_bin[i] = (uint8_t)bin;", ";", 0),
    ("descriptor_uses_sector_0", "rot + (size_t)bin * OR_NPAIRS * 4", "rot + (size_t)0 * OR_NPAIRS * 4", 0),
    ("fallback_uses_primary_threshold",
     "or_fast(raw[n], W[n], H[n], W[n], p->fast_thresh_lo, p->p_min, p->p_max, p->border, lo, resp_lo);",
     "or_fast(raw[n], W[n], H[n], W[n], p->fast_thresh, p->p_min, p->p_max, p->border, lo, resp_lo);", 0),
    ("pipeline_ignores_pfa_rule", "or_pfa_core(n_cand, lev, X, Y, R, W0, H0, L, p->nms_q, p->pfa_rule, Kl, Kr, alive);",
     "or_pfa_core(n_cand, lev, X, Y, R, W0, H0, L, p->nms_q, 0, Kl, Kr, alive);", 0),
    ("pipeline_pyramid_width_as_height", "or_pyramid_level(L0, W0, H0, pitch0, p->scale, n, raw[n], W[n], H[n], W[n]);",
     "or_pyramid_level(L0, H0, H0, pitch0, p->scale, n, raw[n], W[n], H[n], W[n]);", 0),
    ("pipeline_pfa_width_as_height", "or_pfa_core(n_cand, lev, X, Y, R, W0, H0, L, p->nms_q, p->pfa_rule, Kl, Kr, alive);",
     "or_pfa_core(n_cand, lev, X, Y, R, H0, H0, L, p->nms_q, p->pfa_rule, Kl, Kr, alive);", 0),
    ("orientation_on_blurred_level", "or_orient(raw[k->level], W[k->level], k->x, k->y, &m10, &m01, &theta, &bin);",
     "or_orient(blur[k->level], W[k->level], k->x, k->y, &m10, &m01, &theta, &bin);", 0),
    ("descriptor_on_raw_level", "or_describe(blur[k->level], W[k->level], k->x, k->y,",
     "or_describe(raw[k->level], W[k->level], k->x, k->y,", 0),
    ("cap_deeper_level_first", "if (a->level != b->level) return a->level < b->level ? -1 : 1;",
     "if (a->level != b->level) return a->level > b->level ? -1 : 1;", 0),
    ("response_stores_kr", "out->response[i] = (uint16_t)k->r;", "out->response[i] = (uint16_t)k->kr;", 0),
    # stereo matching (Sec. III middle-end)
    ("match_band_floor", "return (int32_t)ceil((double)row_band_px * s);", "return (int32_t)floor((double)row_band_px * s);", 0),
    ("match_same_level_only", "if (nr < nl - 1 || nr > nl + 1) continue;", "if (nr != nl) continue;", 0),
    ("match_disparity_sign", "int32_t disp = (int32_t)Lk->X[i] - (int32_t)Rk->X[j];",
     "int32_t disp = (int32_t)Rk->X[j] - (int32_t)Lk->X[i];", 0),
    ("match_tie_larger_disparity", "if (d < best_d || (d == best_d && disp < best_disp)) {",
     "if (d < best_d || (d == best_d && disp > best_disp)) {", 0),
    ("match_none_reports_distance_0", "right_idx[i] = -1; disparity[i] = 0; dist[i] = 0xFFFF;",
     "right_idx[i] = -1; disparity[i] = 0; dist[i] = 0;", 0),
    ("match_max_disparity_exclusive", "if (disp < 0 || disp > p->max_disp) continue;",
     "if (disp < 0 || disp >= p->max_disp) continue;", 0),
    ("match_index_0_lost", "if (best_j < 0) {", "if (best_j <= 0) {", 0),
    ("match_loops_over_left_count", "for (int32_t j = 0; j < Rk->count; ++j) {", "for (int32_t j = 0; j < Lk->count; ++j) {", 0),
    ("match_right_level_from_left", "int32_t nr = Rk->level[j];", "int32_t nr = Lk->level[j];", 0),
    ("match_threshold_exclusive", "} else if (best_d <= p->match_max_dist) {", "} else if (best_d < p->match_max_dist) {", 0),
    ("popcount_skips_bits", "while (v) { c += (int32_t)(v & 1u); v >>= 1; }", "while (v) { c += (int32_t)(v & 1u); v >>= 2; }", 0),
    ("match_and_instead_of_xor", "d += popcount32(Lk->desc[(size_t)i * 8 + w] ^ Rk->desc[(size_t)j * 8 + w]);",
     "d += popcount32(Lk->desc[(size_t)i * 8 + w] & Rk->desc[(size_t)j * 8 + w]);", 0),
    # correlation minimisation (NEXT-1)
    ("subpixel_xr0_truncated", "int32_t xr0 = (int32_t)floor((double)Rk->X[j] / s + 0.5);",
     "int32_t xr0 = (int32_t)floor((double)Rk->X[j] / s);", 0),
    ("subpixel_window_off_by_one", "if (xi - w < 0 || xi + w >= W || yi - w < 0 || yi + w >= H",
     "if (xi - w < 0 || xi + w > W || yi - w < 0 || yi + w > H", 0),
    ("subpixel_no_centre_normalisation", "int32_t a = (int32_t)A[(size_t)(yi + dy) * W + xi + dx] - lc;",
     "int32_t a = (int32_t)A[(size_t)(yi + dy) * W + xi + dx];", 0),
    ("subpixel_right_centre_unshifted", "int32_t rc = B[(size_t)yi * W + xr0 + t];",
     "int32_t rc = B[(size_t)yi * W + xr0];", 0),
    ("subpixel_lower_median", "uint64_t median = kept[n_kept / 2];", "uint64_t median = kept[(n_kept - 1) / 2];", 0),
    ("subpixel_window_last_row_dropped", "for (int32_t dy = -w; dy <= w; ++dy)", "for (int32_t dy = -w; dy < w; ++dy)", 0),
    ("subpixel_window_last_column_dropped", "for (int32_t dx = -w; dx <= w; ++dx) {", "for (int32_t dx = -w; dx < w; ++dx) {", 0),
    ("subpixel_zero_disparity_rejected", "if (q * den < num) continue;", "if (q * den <= num) continue;", 0),
    ("subpixel_max_disparity_rejected", "if (s * (double)(q * den - num) > (double)p->max_disp * (double)den) continue;",
     "if (s * (double)(q * den - num) >= (double)p->max_disp * (double)den) continue;", 0),
    ("subpixel_max_disparity_on_q_plus_delta", "if (s * (double)(q * den - num) > (double)p->max_disp * (double)den) continue;",
     "if (s * (double)(q * den + num) > (double)p->max_disp * (double)den) continue;", 0),
    ("parabola_denominator_3", "int64_t num = d1 - d3, den = 2 * (d1 + d3 - 2 * d2);",
     "int64_t num = d1 - d3, den = 3 * (d1 + d3 - 2 * d2);", 0),
    ("parabola_centre_weight_3", "int64_t num = d1 - d3, den = 2 * (d1 + d3 - 2 * d2);",
     "int64_t num = d1 - d3, den = 2 * (d1 + d3 - 3 * d2);", 0),
    ("subpixel_left_x_by_match_index", "int32_t n = Lk->level[i], xi = Lk->x[i], yi = Lk->y[i];",
     "int32_t n = Lk->level[i], xi = Lk->x[j], yi = Lk->y[i];", 0),
    ("subpixel_level_from_right", "int32_t n = Lk->level[i], xi = Lk->x[i], yi = Lk->y[i];",
     "int32_t n = Rk->level[i], xi = Lk->x[i], yi = Lk->y[i];", 0),
    ("subpixel_outlier_loop_over_right", "for (int32_t i = 0; i < Lk->count; ++i)\n            if (disp_out[i] >= 0.0f",
     "for (int32_t i = 0; i < Rk->count; ++i)\n            if (disp_out[i] >= 0.0f", 0),
    ("negative_disparity_kept", "if (q * den < num) continue;", ";", 0),
    ("median_of_unsorted_sads", "qsort(kept, (size_t)n_kept, sizeof(uint32_t), cmp_u32);", ";", 0),
    ("median_of_descending_sads", "return x < y ? -1 : (x > y ? 1 : 0);", "return x > y ? -1 : (x < y ? 1 : 0);", 0),
    ("subpixel_levels_one_scale_short", "or_pyramid_level(L0, W0, H0, pitch0, p->scale, n, lev[n], Wn[n], Hn[n], Wn[n]);",
     "or_pyramid_level(L0, W0, H0, pitch0, p->scale, n - 1, lev[n], Wn[n], Hn[n], Wn[n]);", 0),
    ("subpixel_last_minimum", "if (acc < sad[best]) best = t + L;", "if (acc <= sad[best]) best = t + L;", 0),
    ("subpixel_parabola_sign", "int64_t num = d1 - d3, den = 2 * (d1 + d3 - 2 * d2);",
     "int64_t num = d3 - d1, den = 2 * (d1 + d3 - 2 * d2);", 0),
    ("subpixel_parabola_half", "int64_t num = d1 - d3, den = 2 * (d1 + d3 - 2 * d2);",
     "int64_t num = d1 - d3, den = (d1 + d3 - 2 * d2);", 0),
    ("subpixel_outlier_factor_2", "10u * (uint64_t)sad_out[i] > 21u * median", "10u * (uint64_t)sad_out[i] > 20u * median", 0),
    ("subpixel_depth_not_inverse", "depth_out[i] = bf > 0.0 ? (float)(bf / (disp > 0.01 ? disp : 0.01)) : 0.0f;",
     "depth_out[i] = bf > 0.0 ? (float)(bf * (disp > 0.01 ? disp : 0.01)) : 0.0f;", 0),
    ("subpixel_minimum_at_minus_L_kept", "if (ts == -L || ts == L) continue;", "if (ts == L) continue;", 0),
    # tracking (NEXT-2)
    ("track_stops_at_level_8", "float zf = (float)or_level_scale(scale, lvl[q]);",
     "if (lvl[q] >= OR_MAX_LEVELS) { idx_out[q] = -1; dist_out[q] = 0xFFFF; continue; }\n        "
     "float zf = (float)or_level_scale(scale, lvl[q]);", 0),
    ("track_band_two_levels_up", "if (m < (int32_t)lvl[q] - 1 || m > (int32_t)lvl[q] + 1) continue;",
     "if (m < (int32_t)lvl[q] - 1 || m > (int32_t)lvl[q] + 2) continue;", 0),
    ("track_same_level_only", "if (m < (int32_t)lvl[q] - 1 || m > (int32_t)lvl[q] + 1) continue;",
     "if (m != (int32_t)lvl[q]) continue;", 0),
    ("track_lower_level_dropped", "if (m < (int32_t)lvl[q] - 1 || m > (int32_t)lvl[q] + 1) continue;",
     "if (m <= (int32_t)lvl[q] - 1 || m > (int32_t)lvl[q] + 1) continue;", 0),
    ("track_dy_window_exclusive", "if (fabsf(dx) > r || fabsf(dy) > r) continue;",
     "if (fabsf(dx) > r || fabsf(dy) >= r) continue;", 0),
    ("track_max_dist_exclusive", "int ok = bd <= max_dist &&", "int ok = bd < max_dist &&", 0),
    ("track_hamming_7_words", "for (int32_t w = 0; w < 8; ++w)\n                d += popcount32(desc[(size_t)q * 8 + w]",
     "for (int32_t w = 0; w < 7; ++w)\n                d += popcount32(desc[(size_t)q * 8 + w]", 0),
    ("track_ratio_08", "int ok = bd <= max_dist && (sd == 0x7fffffff || 10 * bd <= 9 * sd);",
     "int ok = bd <= max_dist && (sd == 0x7fffffff || 10 * bd <= 8 * sd);", 0),
    ("track_second_not_updated", "if (d < bd) { sd = bd; bd = d; best = k; }", "if (d < bd) { bd = d; best = k; }", 0),
    ("track_window_unscaled", "volatile float r = radius * zf;", "volatile float r = radius;", 0),
    # the arc response (alternative reading of the Sec. III response)
    ("arc_positions_shorter_runs", "while (len < n && ((mask >> ((start + len) % 16)) & 1u)) ++len;",
     "while (len < n - 1 && ((mask >> ((start + len) % 16)) & 1u)) ++len;", 0),
    ("arc_positions_skip_wrap", "for (int32_t j = 0; j < n; ++j) on |= 1u << ((start + j) % 16);",
     "for (int32_t j = 0; j < n; ++j) on |= 1u << ((start + j) & 7);", 0),
    ("arc_response_no_eps", "if ((on >> k) & 1u) sum += (d[k] < 0 ? -d[k] : d[k]) - eps;",
     "if ((on >> k) & 1u) sum += (d[k] < 0 ? -d[k] : d[k]);", 0),
    ("arc_response_sums_polarities", "if (sum > best) best = sum;", "best += sum;", 0),
    ("arc_response_ignores_p_max", "if (n < p_min || n > p_max) continue;", "if (n < p_min) continue;", 0),
    ("fast_arc_dark_not_strict", "if (d[k] < -eps) Bd |= 1u << k;", "if (d[k] <= -eps) Bd |= 1u << k;", 0),
    ("fast_arc_centre_shifted", "int32_t ic = img[(size_t)y * pitch + x];",
     "int32_t ic = img[(size_t)y * pitch + x + 1];", 1),
    ("arc_fallback_ranked_by_primary", "if (!hi[q]) resp[q] = resp_arc[q];", "if (hi[q]) resp[q] = resp_arc[q];", 0),
    ("arc_mode_keeps_circle_sad",
     "or_fast_arc(raw[n], W[n], H[n], W[n], p->fast_thresh, p->p_min, p->p_max, p->border, hi, resp);",
     "or_fast(raw[n], W[n], H[n], W[n], p->fast_thresh, p->p_min, p->p_max, p->border, hi, resp);", 0),
    # the cascaded pyramid (alternative reading of the resampling)
    ("cascade_from_level_zero",
     "or_pyramid_level(raw[n - 1], W[n - 1], H[n - 1], W[n - 1], p->scale, 1, raw[n], W[n], H[n], W[n]);",
     "or_pyramid_level(raw[0], W[0], H[0], W[0], p->scale, 1, raw[n], W[n], H[n], W[n]);", 0),
    ("cascade_by_zeta_n",
     "or_pyramid_level(raw[n - 1], W[n - 1], H[n - 1], W[n - 1], p->scale, 1, raw[n], W[n], H[n], W[n]);",
     "or_pyramid_level(raw[n - 1], W[n - 1], H[n - 1], W[n - 1], p->scale, n, raw[n], W[n], H[n], W[n]);", 0),
    ("mode_check_accepts_2", "if (p->response_mode < 0 || p->response_mode > 1 || p->pyramid_mode < 0 || p->pyramid_mode > 1) return -1;",
     "if (p->response_mode < 0 || p->response_mode > 2 || p->pyramid_mode < 0 || p->pyramid_mode > 2) return -1;", 0),
]

# Mutants that change no output over the oracle's domain (checked below):
# the p = q redraw never fires for the seed's first 256 accepted pairs; the
# projection's clamp to W0 - 1 never binds for a level pixel, since
# x <= W_n - 1 <= W0 / zeta^n - 1/2 gives x zeta^n + 1/2 <= W0 - zeta^n / 2 + 1/2
# < W0.
EQUIVALENT = [("pattern_allows_p_equal_q", "if (v[0] == v[2] && v[1] == v[3]) continue;", ""),
              ("projection_unclamped", "return X < W0 - 1 ? X : W0 - 1;", "return X;")]
# A mutant that changes only a choice the paper leaves open: the Box-Muller
# sine branch draws an equally valid Gaussian, i.e. another of this build's
# own BRIEF patterns (the CUDA path is held to the oracle's table in full).
SPEC_FREE = [("box_muller_sine_branch", "return radius * cos(ang);", "return radius * sin(ang);")]

_PROBE = r"""
import sys, hashlib
sys.path.insert(0, {root!r})
from oracle import oracle as O
O._SRC, O._LIB = {src!r}, {lib!r}
import numpy as np
h = hashlib.sha256(O.pattern_base().tobytes())
for W0 in (64, 377, 752, 1241, 1920, 4096):
    W, _, _ = O.level_geometry(W0, W0, 8, 1.2, 32)
    for n in range(8):
        h.update(np.array([O.project(x, n, 1.2, W0) for x in range(int(W[n]))], np.int32).tobytes())
print(h.hexdigest())
"""


_DRIVER = r"""
import sys
sys.path.insert(0, {root!r})
from oracle import oracle as O
O._SRC, O._LIB = {src!r}, {lib!r}
import pytest
sys.exit(pytest.main({pins!r} + ["-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]))
"""


def _mutate(text, old, new, occ):
    at = -1
    for _ in range(occ + 1):
        at = text.find(old, at + 1)
        assert at >= 0, f"mutation site not found: {old[:60]!r}"
    return text[:at] + new + text[at + len(old):]


def _run(tmp, name, text):
    d = os.path.join(tmp, name)
    os.makedirs(d)
    src, lib = os.path.join(d, "jslam_oracle.c"), os.path.join(d, "libjslam_oracle.so")
    with open(src, "w") as f:
        f.write(text)
    code = _DRIVER.format(root=ROOT, src=src, lib=lib, pins=PINS)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, cwd=ROOT)
    return r.returncode, r.stdout[-1500:] + r.stderr[-1500:]


def test_mutation_sites_exist():
    text = open(SRC).read()
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)
    for name, old, new, occ in MUTANTS + [e + (0,) for e in EQUIVALENT + SPEC_FREE]:
        assert text.count(old) > occ and old != new, name


@pytest.fixture(scope="module")
def outcomes():
    text = open(SRC).read()
    jobs = [("unmutated", text)] + [(n, _mutate(text, o, w, k)) for n, o, w, k in MUTANTS]
    with tempfile.TemporaryDirectory() as tmp, ThreadPoolExecutor(max(2, min(8, os.cpu_count() or 2))) as ex:
        futs = {n: ex.submit(_run, tmp, n, t) for n, t in jobs}
        return {n: f.result() for n, f in futs.items()}


def test_unmutated_oracle_passes_the_pins(outcomes):
    rc, log = outcomes["unmutated"]
    assert rc == 0, log


def test_every_mutant_fails_a_pin(outcomes):
    survivors = [n for n, _, _, _ in MUTANTS if outcomes[n][0] == 0]
    broken = {n: outcomes[n] for n, _, _, _ in MUTANTS if outcomes[n][0] not in (0, 1)}
    assert not broken, {n: (rc, log[-600:]) for n, (rc, log) in broken.items()}
    assert not survivors, survivors


def test_listed_equivalent_mutants_change_no_output():
    """The pattern and every level pixel's s0 projection (six widths, eight
    levels) are the same with each mutant listed as equivalent."""
    text = open(SRC).read()
    jobs = [("unmutated", text)] + [(n, _mutate(text, o, w, 0)) for n, o, w in EQUIVALENT]
    out = {}
    with tempfile.TemporaryDirectory() as tmp:
        for name, t in jobs:
            d = os.path.join(tmp, name)
            os.makedirs(d)
            src, lib = os.path.join(d, "jslam_oracle.c"), os.path.join(d, "libjslam_oracle.so")
            with open(src, "w") as f:
                f.write(t)
            r = subprocess.run([sys.executable, "-c", _PROBE.format(root=ROOT, src=src, lib=lib)],
                               capture_output=True, text=True, timeout=600, cwd=ROOT)
            assert r.returncode == 0, r.stderr[-1500:]
            out[name] = r.stdout.strip()
    assert all(v == out["unmutated"] for v in out.values()), out


def _functions(text):
    """(name, start, end) of every function defined at column 0."""
    out = []
    for m in re.finditer(r"^(?=[A-Za-z_])[\w \*]*?\b(\w+)\s*\([^;{}]*\)\s*\{", text, flags=re.M):
        out.append((m.group(1), m.start(), text.find("\n}\n", m.end())))
    return out


def test_every_oracle_function_hosts_a_mutant():
    """Each function of the oracle carries at least one named mutant, so that a
    function added later without pins that catch a mistake in it is noticed."""
    text = open(SRC).read()
    funcs = _functions(text)
    assert len(funcs) > 30
    hosted = {name: 0 for name, _, _ in funcs}
    for _, old, _, occ in MUTANTS:
        at = -1
        for _ in range(occ + 1):
            at = text.find(old, at + 1)
        for name, a, b in funcs:
            if a <= at < b:
                hosted[name] += 1
    assert not [n for n, c in hosted.items() if c == 0], hosted
