"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of the oracle source (on the CPU,
in a temporary directory), builds it, and runs the pin suite against the
mutated library in a subprocess.  The suite must fail for every mutant: a
mutant that passes would mean that part of the oracle is not pinned.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mppi_oracle.c")
PIN_FILES = ["tests/test_oracle_noise.py", "tests/test_oracle_model.py", "tests/test_oracle_cost.py",
             "tests/test_oracle_softmin.py", "tests/test_golden_paper.py"]

# (name, [(original text, mutated text), ...])
MUTANTS = [
    ("philox-word", [("uint32_t n0 = hi1 ^ c1 ^ k0;", "uint32_t n0 = hi0 ^ c1 ^ k0;")]),
    ("philox-key-bump", [("k1 += W1;", "k1 += W0;")]),
    ("uniform-offset", [("(2.0 * (double)(r >> 9) + 1.0)", "(2.0 * (double)(r >> 9) + 0.5)")]),
    ("box-muller-pair", [("*z1 = radius * sin(two_pi * u1);", "*z1 = radius * cos(two_pi * u1);")]),
    ("quat-product-order", [("out[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];",
                             "out[1] = a[0] * b[1] + a[1] * b[0] - a[2] * b[3] + a[3] * b[2];")]),
    ("quat-rate-half", [("xdot[3 + i] = 0.5 * qw[i];", "xdot[3 + i] = qw[i];")]),
    ("rotation-entry", [("Rm[2] = 2.0 * (x * z + w * y);", "Rm[2] = 2.0 * (x * z - w * y);")]),
    ("gravity-sign", [("double gravity[3] = {0.0, 0.0, -Mdl->g};", "double gravity[3] = {0.0, 0.0, Mdl->g};")]),
    ("gyro-sign", [("xdot[10 + i] = (tau[i] - wxJw[i]) / Mdl->J[i];",
                    "xdot[10 + i] = (tau[i] + wxJw[i]) / Mdl->J[i];")]),
    ("rk4-weights", [("k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]", "k1[i] + 2.0 * k2[i] + k3[i] + 2.0 * k4[i]")]),
    ("rk4-stage", [("xs[i] = x[i] + h * k3[i];", "xs[i] = x[i] + 0.5 * h * k3[i];")]),
    ("no-renormalise", [("for (int i = 3; i < 7; ++i) x_next[i] /= n;", "(void)n;")]),
    ("rate-demand-sign", [("w_dot_d[i] = (u_d[1 + i] - w[i]) / dt;", "w_dot_d[i] = (u_d[1 + i] + w[i]) / dt;")]),
    ("gyro-in-torque", [("tau_d[i] = Mdl->J[i] * w_dot_d[i] + wxJw[i];", "tau_d[i] = Mdl->J[i] * w_dot_d[i];")]),
    ("clip-bound", [("if (T > Mdl->T_max) T = Mdl->T_max;", "if (T > Mdl->T_max) T = Mdl->T_min;")]),
    ("allocation-yaw-row", [("-c,  -c,  c,   c};", "-c,  c,  -c,   c};")]),
    ("omega-clip-step", [("w_clip[i] = w[i] + w_dot_clip * dt;", "w_clip[i] = w_dot_clip * dt;")]),
    ("rho-weights-swapped", [("P->c_v * dv + P->c_w * dw", "P->c_w * dv + P->c_v * dw")]),
    ("quat-term-unsquared", [("P->c_q * dq * dq", "P->c_q * dq")]),
    ("rate-term-range", [("if (j > 0) S += orc_rate_cost(P, u_prev, u);", "S += orc_rate_cost(P, u_prev, u);")]),
    ("input-cost-unclamped", [("S += orc_input_cost(P, u);", "S += orc_input_cost(P, u_raw);")]),
    ("tracking-j0-dropped", [("double S = orc_rho_ref(P, x, &ref[0]) + orc_obstacle_cost",
                              "double S = 0.0 * orc_rho_ref(P, x, &ref[0]) + orc_obstacle_cost")]),
    ("reference-index", [("orc_rho_ref(P, x, &ref[13 * (j + 1)])", "orc_rho_ref(P, x, &ref[13 * j])")]),
    ("indicator-per-obstacle", [("if (s <= 0.0) in_collision = 1;", "if (s <= 0.0) in_collision += 1;"),
                                ("(in_collision ? P->c_obs : 0.0)", "(in_collision * P->c_obs)")]),
    ("cylinder-uses-z", [("double d2 = o[3] < 0.0 ? dx * dx + dy * dy : dx * dx + dy * dy + dz * dz;",
                          "double d2 = dx * dx + dy * dy + dz * dz;")]),
    ("barrier-inside", [("exp(-P->beta * (s > 0.0 ? s : 0.0))", "exp(-P->beta * s)")]),
    ("weights-temperature", [("w[k] = isfinite(S[k]) ? exp(-(S[k] - rho) / lambda) / eta : 0.0;",
                              "w[k] = isfinite(S[k]) ? exp(-(S[k] - rho) * lambda) / eta : 0.0;"),
                             ("eta += isfinite(S[k]) ? exp(-(S[k] - rho) / lambda) : 0.0;",
                              "eta += isfinite(S[k]) ? exp(-(S[k] - rho) * lambda) : 0.0;")]),
    ("update-sign", [("acc[c] += w[k] * delta[c];", "acc[c] -= w[k] * delta[c];")]),
    ("shift-tail", [("else later = P->tail_mode == 1 ? u[4 * (N - 1) + c] : u_init[c];",
                     "else later = u_init[c];")]),
    ("apply-old-nominal", [("orc_clamp_input(Mdl, &u_new[0], u0);", "orc_clamp_input(Mdl, &u_nom[0], u0);")]),
    ("delay-ignored", [("orc_rk4_step(Mdl, x_hat, F, tau, P->delay, x0);", "(void)0;")]),
    ("grid-index-order", [("int occ = inside ? P->grid[((size_t)idx[2] * P->gy + idx[1]) * P->gx + idx[0]] != 0 : 0;",
                           "int occ = inside ? P->grid[((size_t)idx[0] * P->gy + idx[1]) * P->gx + idx[2]] != 0 : 0;")]),
    ("grid-rounding", [("double f = floor(c);", "double f = round(c);")]),
    ("grid-ignored", [("if (orc_grid_occupied(P, x, &face)) in_collision = 1;", "orc_grid_occupied(P, x, &face);")]),
]


def _run_mutant(tmpdir, name, edits):
    src = open(SRC).read()
    for old, new in edits:
        assert src.count(old) == 1, (name, old)
        src = src.replace(old, new)
    cpath = os.path.join(tmpdir, f"{name}.c")
    lpath = os.path.join(tmpdir, f"lib{name}.so")
    with open(cpath, "w") as f:
        f.write(src)
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    O.build(force=True, src=cpath, out=lpath)
    env = dict(os.environ, MPPI_ORACLE_LIB=lpath)
    # Philox's bit pattern is pinned by the independent library check only.
    select = [] if name.startswith("philox") else ["-k", "not independent_library"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        *select, *PIN_FILES],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return name, r.returncode, r.stdout[-400:]


def test_every_planted_mistake_is_caught(tmp_path):
    pytest.importorskip("triton")
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda m: _run_mutant(str(tmp_path), *m), MUTANTS))
    survivors = [(n, out) for n, rc, out in results if rc == 0]
    assert not survivors, "pins do not catch: " + ", ".join(n for n, _ in survivors)
    # Sanity: the unmutated oracle passes the same suite.
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-k", "not independent_library", *PIN_FILES], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-800:]
