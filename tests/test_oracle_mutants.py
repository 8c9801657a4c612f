"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of oracle/tsdf_oracle.c (on the CPU,
in a temporary directory), builds it, and runs the pin suites against it
through TSDF_ORACLE_LIB; the suites must fail. The real oracle is untouched.
"""

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "tsdf_oracle.c")

MUTANTS = {
    "divisor_uses_capped_weight": (
        "double Fn = ((double)w0 * (*F) + f) / (double)(w0 + 1);",
        "double Fn = ((double)w0 * (*F) + f) / (double)(w0 + 1 > p->max_weight ? p->max_weight : w0 + 1);"),
    "pixel_floor_instead_of_nearest": (
        "int ix = (int)(x + 0.5), iy = (int)(y + 0.5);",
        "int ix = (int)(x), iy = (int)(y);"),
    "rotation_transposed": (
        "out[r] = M[4 * r + 0] * p[0] + M[4 * r + 1] * p[1] +\n                 M[4 * r + 2] * p[2] + M[4 * r + 3];",
        "out[r] = M[r] * p[0] + M[4 + r] * p[1] +\n                 M[8 + r] * p[2] + M[4 * r + 3];"),
    "eta_sign_flipped": (
        "double eta = (double)dm - pc[2];\n    if (near_value(eta, -mu, p->delta_eta)) *flag = 1;",
        "double eta = pc[2] - (double)dm;\n    if (near_value(eta, -mu, p->delta_eta)) *flag = 1;"),
    "band_edge_excluded": (
        "if (eta < -mu) return 0;",
        "if (eta <= -mu) return 0;"),
    "border_off_by_one": (
        "const double xmax = fc->width - 2, ymax = fc->height - 2;\n    if (near_value(x, 1.0",
        "const double xmax = fc->width - 1, ymax = fc->height - 1;\n    if (near_value(x, 1.0"),
    "band_half_width": (
        "qa[i] = (d - mu) * r[i];",
        "qa[i] = (d - 0.5 * mu) * r[i];"),
    "fixed_point_rounds": (
        "return (int16_t)(x * 32767.0);",
        "return (int16_t)lrint(x * 32767.0);"),
    "no_clamp_to_one": (
        "    double f = eta / mu;\n    if (f > 1.0) f = 1.0;\n    int w0 = *W;",
        "    double f = eta / mu;\n    int w0 = *W;"),
    "block_box_too_big": (
        "hi[i] = (double)BLOCK * (key[i] + 1) * s + grow;",
        "hi[i] = (double)BLOCK * (key[i] + 2) * s + grow;"),
    "weight_not_capped": (
        "    if (wn > p->max_weight) wn = p->max_weight;\n    *F = store_value",
        "    *F = store_value"),
    "voxel_at_cell_centre": (
        "double pm[3] = { (double)v[0] * s, (double)v[1] * s, (double)v[2] * s };\n    double pc[3];\n    apply_affine(fc->M, pm, pc);                   /* pt_camera = M_d pt */",
        "double pm[3] = { (v[0] + 0.5) * s, (v[1] + 0.5) * s, (v[2] + 0.5) * s };\n    double pc[3];\n    apply_affine(fc->M, pm, pc);                   /* pt_camera = M_d pt */"),
    "initial_sdf_zero": (
        "static const double SDF_INITIAL = 1.0;",
        "static const double SDF_INITIAL = 0.0;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique / not found"
    mutated = src.replace(old, new)
    c = tmp_path / "tsdf_oracle.c"
    c.write_text(mutated)
    (tmp_path / "tsdf_oracle.h").write_text(open(SRC.replace(".c", ".h")).read())
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-o", str(lib),
                           str(c), "-lm"])
    env = dict(os.environ, TSDF_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_golden.py"),
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
