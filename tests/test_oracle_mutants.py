"""Every plausible mistake planted in the oracle fails at least one pin.

Each mutant is a copy of ``oracle/rcp_oracle.c`` with one textual change (a
dropped term, a flipped sign, a swapped operand, an off-by-half index), built
into a temporary library. The pins in ``oracle_pins`` must reject it. This shows
that the pins are not retyped formulas: they constrain every part of the oracle.
"""
import os
import subprocess
import tempfile

import pytest

import oracle
import oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "rcp_oracle.c")

MUTANTS = {
    "colour_sign": ("2.0 * c[0] - 1.0", "1.0 - 2.0 * c[0]"),
    "colour_axes_swapped": ("dr * R[a] + dg * U[a]", "dg * R[a] + dr * U[a]"),
    "blue_axis_dropped": ("db * F[a]", "0.0 * F[a]"),
    "rows_bottom_up": ("(1.0 - 2.0 * v) * tn", "(2.0 * v - 1.0) * tn"),
    "aspect_dropped": ("* tn * aspect", "* tn"),
    "no_half_pixel": ("(double)x + 0.5, (double)y + 0.5", "(double)x, (double)y"),
    "eye_not_reaimed": ("Pe2[a] = Pe[a] + V[a]; Pp2[a] = Pp[a]; }", "Pe2[a] = Pe[a] + V[a]; Pp2[a] = Pp[a] + V[a]; }"),
    "target_moves_eye": ("Pe2[a] = Pe[a]; Pp2[a] = Pp[a] + V[a]; }", "Pe2[a] = Pe[a] + V[a]; Pp2[a] = Pp[a] + V[a]; }"),
    "up_axis_flipped": ("cross3(R, F, U);", "cross3(F, R, U);"),
    "depth_plus": ("fabs(z - z0)", "fabs(z + z0)"),
    "mt_open_edge": ("uu >= 0.0 && vv >= 0.0 && uu + vv <= 1.0", "uu > 0.0 && vv > 0.0 && uu + vv < 1.0"),
    "mt_loose_bound": ("uu >= 0.0 && vv >= 0.0", "uu >= 0.0 && vv >= -0.1"),
    "mt_t_from_wrong_edge": ("*t = dot3(e2, Q) * inv;", "*t = dot3(e1, Q) * inv;"),
    "sphere_far_root_first": ("*t0 = -b - q;", "*t0 = -b + q;"),
    "lambert_no_ambient_split": ("s->ambient + (1.0 - s->ambient) * vis * lam", "s->ambient + vis * lam"),
    "shadow_ignored": ("vis = occ ? 0.0 : 1.0;", "vis = 1.0;"),
    "shadow_offset_inward": ("ps[a] = p[a] + eps * N[a]", "ps[a] = p[a] - eps * N[a]"),
    "shadow_past_light": ("tmax = norm3(ls);", "tmax = INFINITY; norm3(ls);"),
    "point_light_reversed": ("sub3(s->light, p, L);", "sub3(p, s->light, L);"),
    "one_sided": ("if (dot3(N, d) > 0.0) {", "if (0) {"),
    "sky_reversed": ("rgbz[0] = (1.0 - sv) + sv * 0.5;", "rgbz[0] = sv + (1.0 - sv) * 0.5;"),
    "tie_to_higher_id": ("t > tmin && t < best) { best = t; best_id = i; }", "t > tmin && t <= best) { best = t; best_id = i; }"),
    "no_clamp": ("rgbz[a] = rgbz[a] < 0.0 ? 0.0 : (rgbz[a] > 1.0 ? 1.0 : rgbz[a]);", "(void)0;"),
    "no_recursion": ("memcpy(c, rgbt, sizeof(double) * 3);", "(void)rgbt;"),
    "sphere_id_offset": ("best_id = s->T + j;", "best_id = j;"),
    "flag_dropped": ("    *flag = fl;\n    return 0;\n}\n\n/*\n * Any hit", "    *flag = 0;\n    return 0;\n}\n\n/*\n * Any hit"),
    "point_flag_dropped": ("if (ill) fl |= ORC_FLAG_ID | ORC_FLAG_POINT;", "if (ill) fl |= ORC_FLAG_ID;"),
    "shadow_flag_as_id": ("if (samb) amb |= ORC_FLAG_SHADOW;", "if (samb) amb |= ORC_FLAG_ID;"),
    "image_green_sign": ("const double sy = (double)y - k_px", "const double sy = (double)y + k_px"),
    "image_uses_blue": ("(2.0 * (double)c[1] - 1.0)", "(2.0 * (double)c[2] - 1.0)"),
    "image_round_down": ("(int64_t)floor(sx + 0.5)", "(int64_t)floor(sx)"),
    "mirror_repeats_edge": ("return m < n ? m : period - 1 - m;", "return m < n ? m : period - m;"),
    "image_no_centering": ("k_px * (2.0 * (double)c[0] - 1.0)", "k_px * (double)c[0]"),
    "image_band_dropped": ("return fabs(frac - 0.5) <= band;", "return fabs(frac - 0.5) < 0.0 * band;"),
    "image_band_at_integers": ("return fabs(frac - 0.5) <= band;", "return frac <= band || 1.0 - frac <= band;"),
    "image_band_row_uses_x": ("near_half(sy, ORC_IMG_TOL * ((double)y + k_px + 1.0))",
                              "near_half(sx, ORC_IMG_TOL * ((double)y + k_px + 1.0))"),
    "normal_cross_swapped": ("cross3(C, N, X);", "cross3(N, C, X);"),
    "normal_not_carried": ("orc_shade_ray(J->s, o, d, rgbt, nrm, &id, &amb);",
                           "orc_shade_ray(J->s, o, d, rgbt, NULL, &id, &amb);"),
    "normal_ms_wrong_pixel": ("orc_nearest_pixel(J->W, J->H, px, py) : NULL;",
                              "orc_nearest_pixel(J->W, J->H, px + 1.0, py) : NULL;"),
    "nearest_pixel_half_shift": ("int64_t nx = (int64_t)floor(px), ny = (int64_t)floor(py);",
                                 "int64_t nx = (int64_t)floor(px - 0.5), ny = (int64_t)floor(py - 0.5);"),
    "normal_not_output": ("        if (nrm) memcpy(nrm, N, sizeof(N));\n", "\n"),
    "depth_along_ray": ("return id < 0 ? 0.0 : t * dot3(d, F);", "return id < 0 ? 0.0 : t;"),
    "depth_wrong_axis": ("    sub3(cam + 3, cam, F);\n    normalize3(F);\n}", "    sub3(cam + 6, cam, F);\n    normalize3(F);\n}"),
    "jitter_sign": ("const double px = (double)x + (double)J->jitter[2 * s]", "const double px = (double)x - (double)J->jitter[2 * s]"),
    "bilinear_weights_swapped": ("{{(1.0 - wx) * (1.0 - wy), wx * (1.0 - wy)}", "{{wx * (1.0 - wy), (1.0 - wx) * (1.0 - wy)}"),
    "ms_mean_wrong": ("J->out[4 * i + a] = acc[a] / (double)J->spp;", "J->out[4 * i + a] = acc[a] / (double)(J->spp + 1);"),
    "bilinear_no_half_shift": ("const double qx = px - 0.5, qy = py - 0.5;", "const double qx = px, qy = py;"),
    "tmin_ignored": ("if (mt_raw(s->v + 9 * i, s->n + 3 * i, o, d, &t) && t > tmin && t < best)",
                     "if (mt_raw(s->v + 9 * i, s->n + 3 * i, o, d, &t) && t > 0.0 && t < best)"),
    "any_hit_closed_end": ("if (t > tmin && t < tmax) {", "if (t > tmin && t <= tmax) {"),
    "any_hit_sphere_closed_end": ("if (ts[r] > tmin && ts[r] < tmax) {", "if (ts[r] > tmin && ts[r] <= tmax) {"),
    "diam_ignores_radius": ("if (c[a] - c[3] < lo[a]) lo[a] = c[a] - c[3];", "if (c[a] < lo[a]) lo[a] = c[a];"),
}


def _build_mutant(name, find, repl, tmpdir):
    src = open(SRC).read()
    assert src.count(find) >= 1, f"mutant {name}: pattern not found"
    mut = src.replace(find, repl, 1)
    cpath = os.path.join(tmpdir, f"{name}.c")
    open(cpath, "w").write(mut)
    hdr = os.path.join(os.path.dirname(SRC), "rcp_oracle.h")
    open(os.path.join(tmpdir, "rcp_oracle.h"), "w").write(open(hdr).read())
    out = os.path.join(tmpdir, f"lib{name}.so")
    subprocess.run(["gcc", "-O1", "-std=gnu99", "-fPIC", "-shared", "-pthread", "-ffp-contract=off", cpath,
                    "-o", out, "-lm"], check=True)
    return out


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    find, repl = MUTANTS[name]
    with tempfile.TemporaryDirectory() as td:
        lp = _build_mutant(name, find, repl, td)
        caught = []
        for check in P.ALL_CHECKS:
            try:
                check(lp)
            except Exception:  # any failure of a pin rejects the mutant
                caught.append(check.__name__)
        assert caught, f"no pin rejects mutant {name}"


def test_unmutated_copy_passes():
    with tempfile.TemporaryDirectory() as td:
        lp = _build_mutant("identity", "#include <math.h>", "#include <math.h>", td)
        for check in P.ALL_CHECKS:
            check(lp)
