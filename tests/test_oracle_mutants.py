"""The oracle's pins must catch plausible mistakes (CPU).

Each mutant is a copy of the oracle's C source with one deliberate slip -- a
dropped term, a flipped sign, a wrong index, direction or weight, a link that
should not count -- built into its own library. The pin suite
(test_oracle_pins.py) runs against it and must fail; a mutant that survives
is a mistake the pins would let through. The oracle's own source is never
changed. Mutants that cannot change any result are not listed: counting the
fluid-to-fluid (or solid-to-solid) links in the momentum exchange, for
instance, adds pairs of opposite links that cancel exactly.
"""
import concurrent.futures
import os
import re
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "vplbm_oracle.c")
HDR = os.path.join(ROOT, "oracle", "vplbm_oracle.h")

# (name, text in the source, replacement); each text occurs exactly once
MUTANTS = [
    ("velocity set: diagonals rotated", "(double)(2 * a - 9) * M_PI / 4.0", "(double)(2 * a - 7) * M_PI / 4.0"),
    ("weights: diagonal weight doubled", "for (int a = 5; a <= 8; ++a) w[a] = 1.0 / 36.0;",
     "for (int a = 5; a <= 8; ++a) w[a] = 1.0 / 18.0;"),
    ("moment matrix: one entry", "{0, 1, -1, 1, -1, 0, 0, 0, 0},", "{0, 1, -1, 1, -1, 0, 0, 0, 1},"),
    ("equilibrium: sign of the u.u term", "double contraction = xu * xu - CS2 * uu;",
     "double contraction = xu * xu + CS2 * uu;"),
    ("equilibrium: linear term scaled", "(1.0 + xu / CS2 + contraction", "(1.0 + xu * CS2 + contraction"),
    ("forcing: sign of u in (xi - u)", "double vx = (m->xi[a][0] - ux) / CS2", "double vx = (m->xi[a][0] + ux) / CS2"),
    ("MRT: s_q from Lambda", "double sq = 1.0 / (0.5 + c->lambda / (1.0 / sn - 0.5));",
     "double sq = 1.0 / (0.5 + c->lambda * (1.0 / sn - 0.5));"),
    ("MRT: energy-square moment relaxed at s_q", "S[2] = sn;", "S[2] = sq;"),
    ("MRT: sign of the forcing moments", "- (1.0 - m->S[k] / 2.0) * MF[k];", "+ (1.0 - m->S[k] / 2.0) * MF[k];"),
    ("SRT: forcing prefactor dropped", "double pre = 1.0 - 1.0 / (2.0 * c->tau);", "double pre = 1.0;"),
    ("velocity: half force dropped", "double bx = jx + 0.5 * r * c->g[0];", "double bx = jx + r * c->g[0];"),
    ("penalization: kappa denominator", "double kappa = ce / (1.0 + half);", "double kappa = ce / (1.0 + ce);"),
    ("body motion: velocity phase", "*vy = b->amp_y * rate * co;", "*vy = b->amp_y * rate * s;"),
    ("rotation: sign of omega x r", "sx = st[4 * b + 2] - bd->omega * dy;", "sx = st[4 * b + 2] + bd->omega * dy;"),
    ("mask: boundary node excluded", "int in = bd->outside ? (r2 >= R2) : (r2 <= R2);",
     "int in = bd->outside ? (r2 > R2) : (r2 < R2);"),
    ("free slip: no mirror", "as = m->mirror_y[a];", "as = a;"),
    ("inlet: speed dropped", "equilibrium(m, 1.0, c->u_in[0], c->u_in[1], m->feq_in);",
     "equilibrium(m, 1.0, 0.0, c->u_in[1], m->feq_in);"),
    ("outlet: copies the wrong column", "xs = nx - 1;", "xs = nx - 2;"),
    ("periodic y: off by one", "if (c->bc_y == ORC_BC_PERIODIC) {\n      ys = (ys + ny) % ny;",
     "if (c->bc_y == ORC_BC_PERIODIC) {\n      ys = (ys + ny + 1) % ny;"),
    ("momentum exchange: sign of the solid side", "const double flow = f[(size_t)a * plane + (size_t)y * nx + x] +",
     "const double flow = f[(size_t)a * plane + (size_t)y * nx + x] -"),
    ("momentum exchange: solid side not reversed", "f[(size_t)abar * plane + (size_t)ys * nx + xs];",
     "f[(size_t)a * plane + (size_t)ys * nx + xs];"),
    ("momentum exchange: links through walls", "if (c->bc_y != ORC_BC_PERIODIC) continue;", ""),
    ("momentum exchange: diagonal links dropped",
     "for (int a = 1; a < 9; ++a) {\n        int xs = x + m.xi[a][0], ys = y + m.xi[a][1];",
     "for (int a = 1; a < 5; ++a) {\n        int xs = x + m.xi[a][0], ys = y + m.xi[a][1];"),
    ("convective outlet: weights swapped",
     "ghost[(size_t)a * ny + y] = (g_old + c->u_conv * f_last) / (1.0 + c->u_conv);",
     "ghost[(size_t)a * ny + y] = (c->u_conv * g_old + f_last) / (1.0 + c->u_conv);"),
    ("convective outlet: state rows swapped", "static const int OUTLET_DIRS[3] = {3, 6, 7};",
     "static const int OUTLET_DIRS[3] = {3, 7, 6};"),
    ("convective outlet: wrong neighbour column",
     "const double f_last = src[(size_t)a * plane + (size_t)y * nx + (nx - 1)];",
     "const double f_last = src[(size_t)a * plane + (size_t)y * nx + (nx - 2)];"),
    ("convective outlet: row of the ghost", "return ghost[(size_t)as * ny + ys];", "return ghost[(size_t)as * ny + y];"),
    ("SRT: relaxation times tau instead of over it",
     "fout[a] = f[a] - (f[a] - feq[a]) / c->tau + pre * F[a];",
     "fout[a] = f[a] - (f[a] - feq[a]) * c->tau + pre * F[a];"),
    ("force record: sign of the reaction", "sfx -= px;", "sfx += px;"),
    ("mass record: rest population dropped", "for (int a = 0; a < 9; ++a) smass += fl[a];",
     "for (int a = 1; a < 9; ++a) smass += fl[a];"),
    ("node-by-node step: bodies of the next step",
     "double* st = body_states(c, t);\n  double* ghost = (double*)calloc(9 * (size_t)ny, sizeof(double));",
     "double* st = body_states(c, t + 1);\n  double* ghost = (double*)calloc(9 * (size_t)ny, sizeof(double));"),
    ("node-by-node step: outlet state not advanced",
     "if (outlet_advance(c, f, ghost) != 0) { /* the state itself is not advanced */\n    free(st);\n"
     "    free(ghost);\n    return 1;\n  }\n  for (int64_t k = 0; k < n; ++k) {",
     "if (0) {\n    free(st);\n    free(ghost);\n    return 1;\n  }\n  for (int64_t k = 0; k < n; ++k) {"),
    ("moments: mask of the next time",
     "orc_mask(c, t, chi, us);\n  if (outlet_advance(c, f, ghost) != 0) { /* the state itself is not advanced */\n"
     "    free(chi);",
     "orc_mask(c, t + 1, chi, us);\n  if (outlet_advance(c, f, ghost) != 0) { /* the state itself is not advanced */\n"
     "    free(chi);"),
]


def _run_mutant(tmp, idx, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique: {old!r}"
    d = os.path.join(tmp, f"m{idx}")
    os.makedirs(d, exist_ok=True)
    shutil.copy(HDR, d)
    with open(os.path.join(d, "vplbm_oracle.c"), "w") as fh:
        fh.write(src.replace(old, new))
    lib = os.path.join(d, "liboracle.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-o", lib, os.path.join(d, "vplbm_oracle.c"), "-lm"], check=True)
    env = dict(os.environ, VPLBM_ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-x", "-q", "-p", "no:cacheprovider"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    caught = re.findall(r"FAILED (\S+)", r.stdout)
    return r.returncode, caught[0] if caught else None


def test_pins_catch_every_mutant(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        futs = {name: ex.submit(_run_mutant, str(tmp_path), i, old, new)
                for i, (name, old, new) in enumerate(MUTANTS)}
        results = {name: f.result() for name, f in futs.items()}
    for name, (rc, caught) in results.items():
        print(f"{name:48s} caught by {caught}")
    survivors = [name for name, (rc, _) in results.items() if rc == 0]
    assert not survivors, f"mutants the pins let through: {survivors}"
