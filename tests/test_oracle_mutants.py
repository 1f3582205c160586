"""The oracle's pins have teeth: each plausible mistake planted in a copy of
oracle.c (built on the CPU into a temporary directory) makes at least one pin
of tests/test_oracle.py fail."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "u_v_swapped": ("*u_out = V / det;\n  *v_out = W / det;", "*u_out = W / det;\n  *v_out = V / det;"),
    "T_drops_a_term": ("fmaf(W, Cz, fmaf(V, Bz, UAz))", "fmaf(W, Cz, UAz)"),
    "single_sided": ("if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return 0;",
                     "if (U < 0.0f || V < 0.0f || W < 0.0f) return 0;"),
    "origin_minus_vertex": ("A[k] = p[k] - o[k];", "A[k] = o[k] - p[k];"),
    "tie_to_highest_id": ("return t < bt || (t == bt && id < bid);", "return t < bt || (t == bt && id > bid);"),
    "tmin_not_clamped": ("const float tlo = tmin > 0.0f ? tmin : 0.0f;", "const float tlo = tmin;"),
    "tmax_open_interval": ("if (!(t >= tlo && t <= tmax)) return 0;", "if (!(t >= tlo && t < tmax)) return 0;"),
    "edge_fma": ("float U = CxBy - CyBx;", "float U = fmaf(Cx, By, -CyBx);"),
    "grad_weight_p0": ("const double w[3] = {1.0 - u - v, u, v};", "const double w[3] = {1.0 - u, u, v};"),
    "grad_lambda_sign": ("gr[k] = -lam[k];", "gr[k] = lam[k];"),
    "grad_ray_t_scale": ("gr[3 + k] = -t * lam[k];", "gr[3 + k] = -lam[k];"),
    "bvh_visits_right_only": ("  visit(q, nd->left);\n  if (q->any && q->found) return;\n",
                              "  if (q->any && q->found) return;\n"),
    "cpq_edge_bc_weights_swapped": ("u = 1.0f - s; v = s;", "u = s; v = 1.0f - s;"),
    "cpq_vertex_b_region": ("if (d3 >= 0.0f && d4 <= d3) {", "if (d3 >= 0.0f && d4 >= d3) {"),
    "cpq_dot_drops_z": ("return (x[0] * y[0] + x[1] * y[1]) + x[2] * y[2];", "return x[0] * y[0] + x[1] * y[1];"),
    "cpq_radius_open": ("if (d2 <= p[3] && better(", "if (d2 < p[3] && better("),
    "cpq_face_weights_swapped": ("u = fv; v = fw;", "u = fw; v = fv;"),
}

PINS = ["tests/test_oracle.py"]


def _run_pins_against(src_text, tmp_path):
    mdir = tmp_path / "oracle"
    mdir.mkdir()
    (mdir / "oracle.c").write_text(src_text)
    (mdir / "oracle.h").write_text(open(os.path.join(ROOT, "oracle", "oracle.h")).read())
    lib = mdir / "liboracle.so"
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                    "-shared", str(mdir / "oracle.c"), "-o", str(lib), "-lm"], check=True)
    # run the pins in a child process against the mutant library
    code = (
        "import sys, pytest, oracle\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        f"oracle.use_library({str(lib)!r})\n"
        "oracle.build = lambda force=False: oracle.LIB_PATH\n"
        f"sys.exit(pytest.main(['-x', '-q', '-p', 'no:cacheprovider', {os.path.join(ROOT, PINS[0])!r}]))\n")
    return subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600)


def test_unmutated_copy_passes_the_pins(tmp_path):
    r = _run_pins_against(open(SRC).read(), tmp_path)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found once: {name}"
    r = _run_pins_against(src.replace(old, new), tmp_path)
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
