"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake (a dropped term, a sign, a wrong index or factor) in a
scratch copy of the oracle's C source, rebuilds that copy, and runs the pin suite
against it: the suite must fail.  Nothing here touches the real oracle or a GPU.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    # refraction metric terms (Eq. eikonal-sphere:1-3)
    "metric_sign": ("F[3] = -G[0] / hX - k * cg[2] / r + k * tphi * cg[1] / r;",
                    "F[3] = -G[0] / hX - k * cg[2] / r - k * tphi * cg[1] / r;"),
    "metric_dropped": ("F[5] = -G[2] + k * cg[0] / r + l * cg[1] / r;", "F[5] = -G[2] + k * cg[0] / r;"),
    "gamma_term_dropped": ("(dN2[q] - d.D / d.K2 * dG2[q])", "(dN2[q])"),
    "coriolis_gradient": ("*df2 = 8.0 * m->G.omega * m->G.omega * sin(Y) * cos(Y);",
                          "*df2 = 4.0 * m->G.omega * m->G.omega * sin(Y) * cos(Y);"),
    # group velocity and integrator
    "cg_vertical_sign": ("d->ch[2] = -mm * d->D", "d->ch[2] = mm * d->D"),
    "rk3_coefficient": ("{1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0}", "{1.0 / 3.0, 15.0 / 16.0, 7.0 / 15.0}"),
    "one_face_carrier": ("F[q] = 0.5 * (vel[0] + vel[1]);", "F[q] = vel[0];"),
    "gather_wrong_spacing": ("- A[node(m, k, j - 1, i)]) / (2.0 * dY);", "- A[node(m, k, j - 1, i)]) / (2.0 * dX);"),
    # saturation
    "kappa_factor": ("double fac = fmax(0.0, 1.0 - 2.0 * kappa * K2 * dt);",
                     "double fac = fmax(0.0, 1.0 - kappa * K2 * dt);"),
    "threshold_integrand": ("*pj = s[SM] * s[SM] * d.kh2 / (d.w * d.K2) * A * alpha;",
                            "*pj = s[SM] * s[SM] * d.kh2 / (d.w * d.K2 * d.K2) * A * alpha;"),
    # projection and tendencies
    "coriolis_flux_sign": ("out[0] = (d->w2 * ch[0] * kk + f2 * ch[1] * ll) / den * A;",
                           "out[0] = (d->w2 * ch[0] * kk - f2 * ch[1] * ll) / den * A;"),
    "elastic_sign": ("out[4] = -f2 * n2 * ch[2] / den * kk * A;", "out[4] = f2 * n2 * ch[2] / den * kk * A;"),
    "vertical_overlap": ("double w = w_h * ov / dz;", "double w = w_h * ov / s[SEZ];"),
    "volume_share": ("rp->alpha = physical_volume(m, s) / cell_volume(m, rp->j, rp->k);", "rp->alpha = 1.0;"),
    "divergence_cos": ("double dp_u = (cn * pl_n - cs * pl_s) / (2.0 * dY);",
                       "double dp_u = (pl_n - pl_s) / (2.0 * dY);"),
    # bookkeeping
    "split_id_reuse": ("oid[1] = m->next_id++;", "oid[1] = m->next_id;"),
    # potential-temperature flux and tendency
    "theta_flux_sign": ("out[8] = -f * n2 * ch[2] / den * ll * A;", "out[8] = f * n2 * ch[2] / den * ll * A;"),
    "theta_flux_component": ("out[9] = f * n2 * ch[2] / den * kk * A;", "out[9] = f * n2 * ch[2] / den * ll * A;"),
    "theta_div_cos": ("if (j + 1 < ny) yn = cos(row_lat(m, j + 1)) * THF(tp, node(m, k, j + 1, i));",
                      "if (j + 1 < ny) yn = THF(tp, node(m, k, j + 1, i));"),
    # columnar mode (single-column approximation)
    "columnar_metric_term": ("        F[5] = -G[2];\n    } else if (is_sphere(m)) {",
                             "        F[5] = -G[2] + k * cg[0] / r;\n    } else if (is_sphere(m)) {"),
    "columnar_horizontal_divergence": ("                    div_u = (fz_top_l - fz_bot_l) / dz;\n",
                                       "                    div_u = div_u;\n"),
    # smoothing (App. B.4 reading), edge gradients and values (App. B.1 reading), cap ties, exits
    "smooth_box_weights": ("double w = (di == 0 ? 2.0 : 1.0) * (dj == 0 ? 2.0 : 1.0);", "double w = 16.0 / 9.0;"),
    "smooth_x_only": ("double w = (di == 0 ? 2.0 : 1.0) * (dj == 0 ? 2.0 : 1.0);",
                      "double w = (di == 0 ? 2.0 : 1.0) * (dj == 0 ? 4.0 : 0.0);"),
    "smooth_pole_mirror": ("if (is_sphere(m)) jj = clampl(jj, 0, ny - 1);",
                           "if (is_sphere(m)) jj = jj < 0 ? 1 : (jj > ny - 1 ? ny - 2 : jj);"),
    "pole_gradient_halved": ("m->grad[f][1][c] = (A[node(m, k, 1, i)] - A[node(m, k, 0, i)]) / dY;",
                             "m->grad[f][1][c] = (A[node(m, k, 1, i)] - A[node(m, k, 0, i)]) / (2.0 * dY);"),
    "top_gradient_halved": ("m->grad[f][2][c] = (A[node(m, nz - 1, j, i)] - A[node(m, nz - 2, j, i)]) / dz;",
                            "m->grad[f][2][c] = (A[node(m, nz - 1, j, i)] - A[node(m, nz - 2, j, i)]) / (2.0 * dz);"),
    "edge_value_extrapolated": ("*q0 = n - 2; *q1 = n - 1; *t = 1.0;",
                                "*q0 = n - 2; *q1 = n - 1; *t = s - (double)(n - 2);"),
    "cap_tie_smaller_id_removed": ("if (x->id != y->id) return x->id > y->id ? -1 : 1;",
                                   "if (x->id != y->id) return x->id < y->id ? -1 : 1;"),
    "exit_at_the_pole": ("double phimax = 0.5 * M_PI - 0.5 * cell_y(m);", "double phimax = 0.5 * M_PI;"),
    # ghost-layer launch
    "ghost_pz_unscaled": ("e[SPZ] = s[SPZ] * e[SEZ] / y[SEZ];", "e[SPZ] = s[SPZ];"),
    "ghost_propagates_in_3d": ("rk3_mode(m, y, dt, 1);", "rk3_mode(m, y, dt, m->P.columnar);"),
    "ghost_keeps_reflected": ("    if (!(y[SM] < 0.0)) {\n        m->st.n_filtered++;",
                              "    if (0) {\n        m->st.n_filtered++;"),
    "ghost_extent_from_bottom": ("double lo = bot > layer_top ? bot : layer_top;", "double lo = bot;"),
}


def _run(name, tmp_root):
    a, b = MUTATIONS[name]
    src = open(os.path.join(ROOT, "oracle", "gwam_oracle.c")).read()
    assert a in src, name
    d = os.path.join(tmp_root, name)
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(d, "oracle"),
                    ignore=shutil.ignore_patterns("*.so", "__pycache__", "*.tmp*"))
    with open(os.path.join(d, "oracle", "gwam_oracle.c"), "w") as fh:
        fh.write(src.replace(a, b))
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(d, "tests"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copytree(os.path.join(ROOT, "paper_2309_11257_gb300"), os.path.join(d, "paper_2309_11257_gb300"),
                    ignore=shutil.ignore_patterns("__pycache__", "*.so", "csrc", "_build"))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "tests/test_oracle_pins.py"], cwd=d, capture_output=True, text=True, timeout=600)
    return name, r.returncode, r.stdout[-400:]


def test_pins_catch_planted_mistakes(tmp_path):
    names = sorted(MUTATIONS)
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        results = list(ex.map(lambda n: _run(n, str(tmp_path)), names))
    survivors = [(n, out) for n, rc, out in results if rc == 0]
    assert not survivors, survivors
    for n, rc, out in results:
        assert rc == 1, (n, out)   # failed tests, not a crash or a collection error
