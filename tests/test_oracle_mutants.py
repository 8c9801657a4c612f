"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of one oracle source (on the CPU, in a
temporary directory), builds the oracle library from the copies, and runs the
pin suites of that source against it through TSDF_ORACLE_LIB; the suites must
fail. The real oracle is untouched.
"""

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
SOURCES = ("tsdf_oracle.c", "raycast_oracle.c", "icp_oracle.c")
PINS = {
    "tsdf_oracle.c": ("test_oracle_golden.py", "test_oracle_pins.py", "test_oracle_colour.py"),
    "raycast_oracle.c": ("test_raycast_oracle.py",),
    "icp_oracle.c": ("test_icp_oracle.py",),
}

# fusion (Sections 3.1-4.3), planted in tsdf_oracle.c
MUTANTS = {
    "divisor_uses_capped_weight": (
        "((double)w * (*F) + f) / (double)(w + 1));",
        "((double)w * (*F) + f) / (double)(w + 1 > p->max_weight ? p->max_weight : w + 1));"),
    "pixel_floor_instead_of_nearest": (
        "*ix = (int)floor(u[0] + 0.5);",
        "*ix = (int)floor(u[0]);"),
    "rotation_transposed": (
        "out[r] = M[4 * r + 0] * p[0] + M[4 * r + 1] * p[1] +\n                 M[4 * r + 2] * p[2] + M[4 * r + 3];",
        "out[r] = M[r] * p[0] + M[4 + r] * p[1] +\n                 M[8 + r] * p[2] + M[4 * r + 3];"),
    "eta_sign_flipped": (
        "truncated_sdf(p, (double)fc->depth[pix] - pc[2], &f, flag)",
        "truncated_sdf(p, pc[2] - (double)fc->depth[pix], &f, flag)"),
    "band_edge_excluded": (
        "if (eta < -p->mu) return 0;",
        "if (eta <= -p->mu) return 0;"),
    "border_off_by_one": (
        "const double hi[2] = { fc->width - 2, fc->height - 2 };",
        "const double hi[2] = { fc->width - 1, fc->height - 1 };"),
    "band_half_width": (
        "qa[i] = (d - mu) * r[i];",
        "qa[i] = (d - 0.5 * mu) * r[i];"),
    "fixed_point_rounds": (
        "return (int16_t)(x * 32767.0);",
        "return (int16_t)lrint(x * 32767.0);"),
    "no_clamp_to_one": (
        "*f = fmin(eta / p->mu, 1.0);",
        "*f = eta / p->mu;"),
    "block_box_too_big": (
        "hi[i] = (double)BLOCK * (key[i] + 1) * s + grow;",
        "hi[i] = (double)BLOCK * (key[i] + 2) * s + grow;"),
    "weight_not_capped": (
        "*W = w + 1 < p->max_weight ? w + 1 : p->max_weight;",
        "*W = w + 1;"),
    "voxel_at_cell_centre": (
        "const double pm[3] = { (double)v[0] * s, (double)v[1] * s, (double)v[2] * s };",
        "const double pm[3] = { (v[0] + 0.5) * s, (v[1] + 0.5) * s, (v[2] + 0.5) * s };"),
    "initial_sdf_zero": (
        "static const double SDF_INITIAL = 1.0;",
        "static const double SDF_INITIAL = 0.0;"),
    "colour_truncates": (
        "rgbw[c] = (uint8_t)floorf(x + 0.5f);",
        "rgbw[c] = (uint8_t)x;"),
    "colour_weight_uncapped": (
        "rgbw[3] = (uint8_t)(wc + 1 > p->max_weight ? p->max_weight : wc + 1);",
        "rgbw[3] = (uint8_t)(wc + 1);"),
    "colour_channels_swapped": (
        "const float num = (float)wc * (float)rgbw[c] + (float)obs[c];",
        "const float num = (float)wc * (float)rgbw[c] + (float)obs[2 - c];"),
    "colour_neighbour_pixel": (
        "update_colour(p, fc->rgb + 4 * pix, rgbw);",
        "update_colour(p, fc->rgb + 4 * (pix + 1), rgbw);"),
    "colour_divisor_capped": (
        "const float den = (float)(wc + 1);",
        "const float den = (float)(wc + 1 > p->max_weight ? p->max_weight : wc + 1);"),
}
MUTANTS = {k: ("tsdf_oracle.c",) + v for k, v in MUTANTS.items()}

# raycast (Section 4.4), planted in raycast_oracle.c
RAYCAST_MUTANTS = {
    "ray_no_step_back": (
        "t -= BLOCK; /* one step back, then the finer search */",
        "/* no step back */"),
    "ray_one_refinement_step": (
        "B = grow(B, mu_v, grad, r->D, edge);\n                t += sdf * mu_v;\n            }",
        "}"),
    "ray_refinement_wrong_sign": (
        "t += sdf * mu_v;\n            at(r, t, P);",
        "t -= sdf * mu_v;\n            at(r, t, P);"),
    "ray_no_wrong_side": (
        "if (state == SEARCH_BLOCK_FINE && sdf < 0.0)\n            return 0;",
        "(void)0;"),
    "ray_range_starts_at_far_corner": (
        "fill_rect(ex_lo, ex_hi, W, u0, u1, v0, v1, zmin, zmax);",
        "fill_rect(ex_lo, ex_hi, W, u0, u1, v0, v1, zmax, zmax);"),
    "ray_coverage_rounding_outward": (
        "const double lo = ceil(a), hi = floor(b);",
        "const double lo = floor(a), hi = ceil(b);"),
    "ray_steps_in_metres": (
        "const double mu_v = p->mu / p->voxel_size, dv = p->delta_v;",
        "const double mu_v = p->mu, dv = p->delta_v;"),
    "ray_interp_weights_swapped": (
        "const double x00 = (1.0 - f[0]) * val[0] + f[0] * val[1];",
        "const double x00 = f[0] * val[0] + (1.0 - f[0]) * val[1];"),
    "ray_direction_not_rotated": (
        "E[i] = Li[3 * i] * rc[0] + Li[3 * i + 1] * rc[1] + Li[3 * i + 2] * rc[2];",
        "E[i] = rc[i];"),
    "ray_near_clip_by_far_corner": (
        "if (zmin < zn - dz)\n            continue; /* a corner nearer than the near plane: clipped */",
        "if (zmax < zn - dz)\n            continue;"),
    "ray_block_of_sample_truncated": (
        "const long b[3] = {(long)floor(P[0] / BLOCK), (long)floor(P[1] / BLOCK),\n                               (long)floor(P[2] / BLOCK)};",
        "const long b[3] = {(long)(P[0] / BLOCK), (long)(P[1] / BLOCK), (long)(P[2] / BLOCK)};"),
}
MUTANTS.update({k: ("raycast_oracle.c",) + v for k, v in RAYCAST_MUTANTS.items()})

# depth tracker terms (Section 4.1), planted in icp_oracle.c
ICP_MUTANTS = {
    "icp_jacobian_sign": (
        "const double J[6] = {P[1] * N[2] - P[2] * N[1], P[2] * N[0] - P[0] * N[2],\n                         P[0] * N[1] - P[1] * N[0], N[0], N[1], N[2]};",
        "const double J[6] = {P[2] * N[1] - P[1] * N[2], P[0] * N[2] - P[2] * N[0],\n                         P[1] * N[0] - P[0] * N[1], N[0], N[1], N[2]};"),
    "icp_residual_sign": (
        "const double diff[3] = {P[0] - V[0], P[1] - V[1], P[2] - V[2]};",
        "const double diff[3] = {V[0] - P[0], V[1] - P[1], V[2] - P[2]};"),
    "icp_pose_not_inverted": (
        "affine(c.Tinv, p, P);",
        "for (int r = 0; r < 3; ++r) P[r] = M[4 * r] * p[0] + M[4 * r + 1] * p[1] + M[4 * r + 2] * p[2] + M[4 * r + 3];"),
    "icp_threshold_unsquared": (
        "if (dist2 > m2)\n        return 0;",
        "if (dist2 > c->max_dist)\n        return 0;"),
    "icp_hessian_diagonal_only": (
        "out[t++] = J[a] * J[b];",
        "out[t++] = a == b ? J[a] * J[b] : 0.0;"),
    "icp_normals_not_normalised": (
        "n[0] = x[0] / len;\n            n[1] = x[1] / len;\n            n[2] = x[2] / len;",
        "n[0] = x[0];\n            n[1] = x[1];\n            n[2] = x[2];"),
}
MUTANTS.update({k: ("icp_oracle.c",) + v for k, v in ICP_MUTANTS.items()})

# swapping (Section 5), planted in tsdf_oracle.c, caught by the swapping pins
SWAP_MUTANTS = {
    "swap_merge_floor_division": (
        "*Fd = or_i16_to_float((int16_t)((wh * qh + (long)*wd * qd) / w));",
        "*Fd = or_i16_to_float((int16_t)floor((double)(wh * qh + (long)*wd * qd) / w));"),
    "swap_merge_host_weight_only": (
        "((double)wh * Fh + (double)*wd * *Fd) / (double)w);",
        "((double)wh * Fh + (double)*wd * *Fd) / (double)wh);"),
    "swap_merge_weight_uncapped": (
        "*wd = (uint8_t)(w > p->max_weight ? p->max_weight : w);",
        "*wd = (uint8_t)w;"),
    "swap_colour_merge_truncates": (
        "d[c] = (uint8_t)((2 * num + w) / (2 * w));",
        "d[c] = (uint8_t)(num / w);"),
    "swap_margin_ignored": (
        "const double lo_u = -0.5 - margin, hi_u = fc->width - 0.5 + margin;",
        "const double lo_u = -0.5, hi_u = fc->width - 0.5;"),
    "swap_straddle_invisible": (
        "if (n_front < 8) return 1;",
        "if (n_front < 8) return 0;"),
    "swap_capacity_ignored": (
        "if (n_own < capacity) sel[k++] = c[i].b;",
        "sel[k++] = c[i].b;"),
    "swap_prefetch_ignores_room": (
        "prefetch = s->p.pool_blocks - s->n_alloc >= capacity;",
        "prefetch = 1;"),
    "swap_out_takes_pending": (
        "const int resident = b->allocated && !b->on_host;",
        "const int resident = b->allocated;"),
}
MUTANTS.update({k: ("tsdf_oracle.c",) + v + (("test_oracle_swap.py",),)
                for k, v in SWAP_MUTANTS.items()})


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    target, old, new = MUTANTS[name][:3]
    pins = MUTANTS[name][3] if len(MUTANTS[name]) > 3 else PINS[target]
    srcs = []
    for f in SOURCES:
        text = open(os.path.join(ORACLE, f)).read()
        if f == target:
            assert text.count(old) == 1, f"mutation site for {name} not unique / not found"
            text = text.replace(old, new)
        (tmp_path / f).write_text(text)
        srcs.append(str(tmp_path / f))
    (tmp_path / "tsdf_oracle.h").write_text(open(os.path.join(ORACLE, "tsdf_oracle.h")).read())
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-o", str(lib)] + srcs +
                          ["-lm"])
    env = dict(os.environ, TSDF_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] +
                       [os.path.join(ROOT, "tests", t) for t in pins],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
