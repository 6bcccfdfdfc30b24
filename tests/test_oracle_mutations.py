"""The oracle's pins have teeth: each plausible slip planted in a copy of the
oracle (on the CPU) makes at least one pin fail.

Each case copies oracle/ to a temporary directory, applies one textual
mutation to oracle.c, and runs the named pin tests against the mutated copy
in a subprocess; the test passes when those pins fail."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [
    ("gouy phase sign", "  double phase = -0.5 * k * r2 * invR + gouy;",
     "  double phase = -0.5 * k * r2 * invR - gouy;", "solve_paraxial_equation"),
    ("wavefront curvature sign", "  double phase = -0.5 * k * r2 * invR + gouy;",
     "  double phase = 0.5 * k * r2 * invR + gouy;", "solve_paraxial_equation"),
    ("transposed cross product in the Boris rotation",
     "  double uprime[3] = {um[0] + (um[1] * tau[2] - um[2] * tau[1]),",
     "  double uprime[3] = {um[0] + (um[2] * tau[1] - um[1] * tau[2]),", "gyration"),
    ("dropped half electric kick", "  for (int a = 0; a < 3; ++a) u[a] = up[a] + h * E[a];",
     "  for (int a = 0; a < 3; ++a) u[a] = up[a];", "plane_wave_exact or pure_electric"),
    ("dropped longitudinal E_z", "      EB[2] = creal((-I * s->vphi / p->omega) * (px * DX + py * DY));",
     "      EB[2] = 0.0;", "maxwell_residual_scaling"),
    ("Gaussian envelope width", "      return exp(-2.0 * log(2.0) * eta * eta / (p->env_len * p->env_len));",
     "      return exp(-4.0 * log(2.0) * eta * eta / (p->env_len * p->env_len));", "envelope_widths"),
    ("flying-focus group-delay sign",
     "      s->fphi[j] = s->fphi[j - 1] + 0.5 * (tau_j + tau_m) * (s->fw[j] - s->fw[j - 1]);",
     "      s->fphi[j] = s->fphi[j - 1] - 0.5 * (tau_j + tau_m) * (s->fw[j] - s->fw[j - 1]);",
     "flying_focus_peak or flying_focus_table"),
    ("trilinear weight swapped", "          double wt = (cx ? w[0] : 1.0 - w[0]) * (cy ? w[1] : 1.0 - w[1]) *",
     "          double wt = (cx ? 1.0 - w[0] : w[0]) * (cy ? w[1] : 1.0 - w[1]) *", "trilinear"),
    ("Laguerre sign", "    sum += (i % 2 == 0) ? term : -term;", "    sum += term;", "scipy_laguerre"),
    ("LG extra Gouy order", "    phase += (double)(2 * p->lg_p + al) * gouy + (double)p->lg_l * atan2(y, x);",
     "    phase += (double)(p->lg_p + al) * gouy + (double)p->lg_l * atan2(y, x);", "solve_paraxial_equation"),
    ("Yee phase-velocity coefficient", "    s->vphi = 1.0 - (1.0 / 24.0) * (1.0 - cr * cr) * wdx * wdx;",
     "    s->vphi = 1.0 - (1.0 / 12.0) * (1.0 - cr * cr) * wdx * wdx;", "yee"),
    ("flying-focus profile wavenumber", "    k = (1.0 - p->beta_f) * s->k;", "    k = s->k;",
     "reduced_paraxial"),
    ("Yee E update with a full-step B difference swapped",
     "    for (int64_t k = 1; k < nz; ++k) E[k] -= r * (B[k] - B[k - 1]);",
     "    for (int64_t k = 1; k < nz; ++k) E[k] += r * (B[k] - B[k - 1]);", "yee1d_scheme"),
    ("Yee B half step taken as a full step",
     "E[k] -= r * (B[k] - B[k - 1]);\n    for (int64_t k = 0; k + 1 < nz; ++k) B[k] -= 0.5 * r * (E[k + 1] - E[k]);",
     "E[k] -= r * (B[k] - B[k - 1]);\n    for (int64_t k = 0; k + 1 < nz; ++k) B[k] -= r * (E[k + 1] - E[k]);",
     "yee1d_scheme"),
    ("Ex sampled on the cell node instead of the x edge", "    {0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5},",
     "    {0.0, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5},", "staggering"),
    ("1D-3V push moves the transverse position",
     "      for (int a = s->p.one_d ? 2 : 0; a < 3; ++a) pos[a] += dt * u[a] / g;",
     "      for (int a = 0; a < 3; ++a) pos[a] += dt * u[a] / g;", "one_d"),
    ("Bx sampled at the By position", "    {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0},",
     "    {0.5, 0.0, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0},", "staggering"),
]

PLASMA = "tests/test_oracle_pins_plasma.py"
MUTATIONS += [
    ("current without the phase-velocity factor zeta", "  s->jamp = wp * wp * s->zeta / w;",
     "  s->jamp = wp * wp / w;", "cw_is_carried", PLASMA),
    ("current phase shift with the wrong sign", "  double th = L1 / p->omega;", "  double th = -L1 / p->omega;",
     "finite_duration", PLASMA),
    ("B finite-duration terms without the 1 - v_phi/v_g weight", "      double th = s->fdc * L1 / p->omega;",
     "      double th = L1 / p->omega;", "finite_duration", PLASMA),
    ("current amplitude second-derivative sign",
     "  double A = 1.0 - L2 / (p->omega * p->omega) + 0.5 * th * th;",
     "  double A = 1.0 + L2 / (p->omega * p->omega) + 0.5 * th * th;", "finite_duration", PLASMA),
    ("plasma B0/E0 without the plasma factor",
     "    s->bratio = cw * sqrt(1.0 - (wp * wp) / (w * w) * s->zeta * h / sw);", "    s->bratio = cw;",
     "cw_is_carried", PLASMA),
    ("fluid current driven by the updated E",
     "    for (int64_t k = 0; k < nz; ++k) J[k] += dt * wp2[k] * E[k];\n"
     "    for (int64_t k = 1; k < nz; ++k) E[k] = (E[k] - r * (B[k] - B[k - 1])) - dt * J[k];",
     "    for (int64_t k = 1; k < nz; ++k) E[k] = (E[k] - r * (B[k] - B[k - 1])) - dt * J[k];\n"
     "    for (int64_t k = 0; k < nz; ++k) J[k] += dt * wp2[k] * E[k];", "cw_is_carried", PLASMA),
    ("Ampere current sign", "E[k] = (E[k] - r * (B[k] - B[k - 1])) - dt * J[k];",
     "E[k] = (E[k] - r * (B[k] - B[k - 1])) + dt * J[k];", "cw_is_carried", PLASMA),
    ("plasma group velocity without cos(omega dt/2)",
     "    s->vg = r * r * sk * ck * p->yee_dx / (sw * cw * p->yee_dt);",
     "    s->vg = r * r * sk * ck * p->yee_dx / (sw * p->yee_dt);", "domega_dk", PLASMA),
    ("split line E2 source sign", "- dt * (J[k] - J1[0]);", "- dt * (J[k] + J1[0]);",
     "split_line_keeps", PLASMA),
    ("Gaussian L2 without the L1^2 term", "      *L2 = (*L1) * (*L1) - 2.0 * a;", "      *L2 = -2.0 * a;",
     "log_derivatives", PLASMA),
    ("split line current driven by E2 only", "      J[k] += dt * wp2[k] * (EB[0] + E2[k]);",
     "      J[k] += dt * wp2[k] * E2[k];", "split_line_keeps", PLASMA),
    ("split line J1 at t_n instead of t_n + dt/2",
     "      or_current(s, 0.0, 0.0, z0 + (double)k * dz, t + 0.5 * dt, J1);",
     "      or_current(s, 0.0, 0.0, z0 + (double)k * dz, t, J1);", "split_line_keeps", PLASMA),
]


@pytest.mark.parametrize("mutation", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, mutation):
    name, old, new, selector = mutation[:4]
    pins = mutation[4] if len(mutation) > 4 else "tests/test_oracle_pins.py"
    work = tmp_path / "w"
    work.mkdir()
    shutil.copytree(os.path.join(ROOT, "oracle"), work / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "tests"), work / "tests", ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copytree(os.path.join(ROOT, "paper_2307_04843_gb300"), work / "paper_2307_04843_gb300",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__", "_build"))
    src = (work / "oracle" / "oracle.c").read_text()
    assert src.count(old) == 1, "mutation anchor not found: " + name
    (work / "oracle" / "oracle.c").write_text(src.replace(old, new))
    env = dict(os.environ, PYTHONPATH=str(work))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        pins, "-k", selector],
                       cwd=str(work), env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, "pins did not catch: %s\n%s" % (name, r.stdout[-2000:])
