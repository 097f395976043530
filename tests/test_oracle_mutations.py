"""Checks that the oracle's pins are sharp: each plausible mistake below (a
dropped term, a wrong sign, index or offset, a swapped operand) is planted in a
copy of the oracle's C source on the CPU, built, and the pin suite must fail
against that build.  Nothing here touches a GPU."""
import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pic_oracle.c")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

MUTATIONS = [
    ("boris: gamma dropped from t", "t[a] = k * eb[3 + a] / gm;", "t[a] = k * eb[3 + a];"),
    ("boris: u- x t sign", "ud[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);",
     "ud[0] = um[0] + (um[2] * t[1] - um[1] * t[2]);"),
    ("boris: s without factor 2", "sv[a] = 2.0 * t[a] / (1.0 + t2);", "sv[a] = t[a] / (1.0 + t2);"),
    ("boris: second half kick dropped", "u[a] = up[a] + k * eb[a];", "u[a] = up[a];"),
    ("push: non-relativistic position update", "np_[a] = pos[a] + s->dt * u[a] / g;",
     "np_[a] = pos[a] + s->dt * u[a];"),
    ("staggering: Bx at a cell centre", "{0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}", "{0.5, 0.5, 0.5}, {0.5, 0.0, 0.5}"),
    ("staggering: Ez at a node", "{0.0, 0.0, 0.5}, /* E */", "{0.0, 0.0, 0.0}, /* E */"),
    ("esirkepov: 1/3 term as 1/2", "0.5 * S0[1][m] * DS[2][n] + DS[1][m] * DS[2][n] / 3.0);",
     "0.5 * S0[1][m] * DS[2][n] + DS[1][m] * DS[2][n] / 2.0);"),
    ("esirkepov: half term without 1/2", "double W = DS[0][l] * (S0[1][m] * S0[2][n] + 0.5 * DS[1][m] * S0[2][n] +",
     "double W = DS[0][l] * (S0[1][m] * S0[2][n] + DS[1][m] * S0[2][n] +"),
    ("esirkepov: current sign", "const double cx = -qw / (dy * dz * dt);", "const double cx = qw / (dy * dz * dt);"),
    ("esirkepov 2D: out-of-plane 1/3 term", "DSx[l] * DSz[n] / 3.0;", "DSx[l] * DSz[n] / 2.0;"),
    ("esirkepov 2D: Jz weight", "acc += DSz[n] * (S0x[l] + 0.5 * DSx[l]);", "acc += DSz[n] * (S0x[l] + DSx[l]);"),
    ("esirkepov: quadratic window from floor(x)", "return (int64_t)floor(X0 + 0.5) - 2;",
     "return (int64_t)floor(X0) - 2;\n    if (0) return 0;"),
    ("esirkepov: cubic window one node short", "    return (int64_t)floor(X0) - 2;\n}",
     "    return (int64_t)floor(X0) - 1;\n}"),
    ("shape: cubic outer piece", "if (a < 2.0) return (2.0 - a) * (2.0 - a) * (2.0 - a) / 6.0;",
     "if (a < 2.0) return (2.0 - a) * (2.0 - a) / 6.0;"),
    ("shape: cubic inner piece sign", "if (a < 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;",
     "if (a < 1.0) return 2.0 / 3.0 - a * a - 0.5 * a * a * a;"),
    ("gather: cubic support from the nearest node", "    return (int64_t)floor(xi) - 1;\n}",
     "    return (int64_t)floor(xi + 0.5) - 1;\n}"),
    ("ampere: J sign", "F(ORC_EX, i, j, k) += dt * (cBx - F(ORC_JX, i, j, k));",
     "F(ORC_EX, i, j, k) += dt * (cBx + F(ORC_JX, i, j, k));"),
    ("faraday: backward instead of forward difference",
     "double cEx = (F(ORC_EZ, i, j + 1, k) - F(ORC_EZ, i, j, k)) * iy -",
     "double cEx = (F(ORC_EZ, i, j, k) - F(ORC_EZ, i, j - 1, k)) * iy -"),
    ("ampere: forward instead of backward difference",
     "double cBz = (F(ORC_BY, i, j, k) - F(ORC_BY, i - 1, j, k)) * ix -",
     "double cBz = (F(ORC_BY, i + 1, j, k) - F(ORC_BY, i, j, k)) * ix -"),
    ("faraday: full instead of half step", "const double h = 0.5 * s->dt;", "const double h = s->dt;"),
    ("shape: quadratic centre value", "if (a < 0.5) return 0.75 - a * a;", "if (a < 0.5) return 0.75 - 0.5 * a * a;"),
    ("gather: linear support from the nearest node", "if (order == 1) return (int64_t)floor(xi);",
     "if (order == 1) return (int64_t)floor(xi + 0.5);"),
    ("knapsack: ties to the highest worker", "if (best < 0 || load[w] < load[best]) best = w;",
     "if (best < 0 || load[w] <= load[best]) best = w;"),
    ("knapsack: ascending instead of descending", "while (j >= 0 && costs[order[j]] < costs[v])",
     "while (j >= 0 && costs[order[j]] > costs[v])"),
    ("morton: y and z bits swapped", "key |= (uint64_t)((by >> i) & 1) << (3 * i + 1);",
     "key |= (uint64_t)((by >> i) & 1) << (3 * i + 2);"),
    ("sfc: strict threshold off by one worker", "if (prefix * (double)n_workers >= (double)(w + 1) * total && w < n_workers - 1) w++;",
     "if (prefix * (double)n_workers >= (double)(w) * total && w < n_workers - 1) w++;"),
    ("efficiency: total instead of average", "return (total / (double)n_workers) / mx;", "return total / mx;"),
    ("threshold: strict improvement", "return e_new >= (1.0 + theta) * e_old;", "return e_new > (1.0 + theta) * e_old;"),
    ("antenna: sheet amplitude without factor 2", "double amp = 2.0 * s->las_a0 / s->d[2] * env;",
     "double amp = s->las_a0 / s->d[2] * env;"),
    ("damping: profile linear in the depth", "    return 1.0 - 0.5 * r * r;\n}", "    return 1.0 - 0.5 * r;\n}"),
    ("damping: factor 1/2 dropped", "    return 1.0 - 0.5 * r * r;\n}", "    return 1.0 - r * r;\n}"),
    ("damping: depth counted from 0",
     "if (k < A) p = A - k;\n    else if (k > s->n[2] - 1 - A) p = k - (s->n[2] - 1 - A);",
     "if (k < A) p = A - 1 - k;\n    else if (k > s->n[2] - 1 - A) p = k - (s->n[2] - A);"),
    ("damping layer disabled", "if (s->absorb <= 0) return;\n    for (int64_t k = 0;", "return;\n    for (int64_t k = 0;"),
    ("particles: upper absorbing boundary ignored", "if (np_[2] < zlo || np_[2] >= zhi) drop[ndrop++] = p;",
     "if (np_[2] < zlo) drop[ndrop++] = p;"),
    ("speedup model: exponent dropped", "return pow(1.0 / e0, x);", "return 1.0 / e0;"),
    ("energy-conserving gather: lower order along node directions",
     "int o = (s->ec && STAG[comp][a] == 0.5) ? s->order - 1 : s->order;",
     "int o = (s->ec && STAG[comp][a] == 0.0) ? s->order - 1 : s->order;"),
    ("energy-conserving gather: box shape from floor instead of the nearest node",
     "if (order == 0) return (int64_t)floor(xi + 0.5);", "if (order == 0) return (int64_t)floor(xi);"),
    ("energy-conserving gather: flag ignored", "    s->ec = energy_conserving;\n", "    s->ec = 0;\n"),
    ("boris: rotation from u- instead of u'", "up[0] = um[0] + (ud[1] * sv[2] - ud[2] * sv[1]);",
     "up[0] = um[0] + (um[1] * sv[2] - um[2] * sv[1]);"),
    ("morton 2D: x and z bits swapped",
     "key |= (uint64_t)((bx >> i) & 1) << (2 * i);\n            key |= (uint64_t)((bz >> i) & 1) << (2 * i + 1);",
     "key |= (uint64_t)((bx >> i) & 1) << (2 * i + 1);\n            key |= (uint64_t)((bz >> i) & 1) << (2 * i);"),
    ("esirkepov 2D: out-of-plane current with u_y instead of v_y", "else deposit2d(s, qw, X0, X1, u[1] / g);",
     "else deposit2d(s, qw, X0, X1, u[1]);"),
    ("ampere: Jz sign", "F(ORC_EZ, i, j, k) += dt * (cBz - F(ORC_JZ, i, j, k));",
     "F(ORC_EZ, i, j, k) += dt * (cBz + F(ORC_JZ, i, j, k));"),
    ("knapsack: box cap ignored", "if (cnt[w] >= cap) continue;", "if (0 && cnt[w] >= cap) continue;"),
    ("gather: quadratic support from floor(x)", "if (order == 2) return (int64_t)floor(xi + 0.5) - 1;",
     "if (order == 2) return (int64_t)floor(xi) - 1;"),
    ("shape: quadratic outer piece without 1/2", "if (a < 1.5) return 0.5 * (1.5 - a) * (1.5 - a);",
     "if (a < 1.5) return (1.5 - a) * (1.5 - a);"),
    ("faraday: d(Ey)/dz term dropped from curl_x E",
     "double cEx = (F(ORC_EZ, i, j + 1, k) - F(ORC_EZ, i, j, k)) * iy -\n"
     "                             (F(ORC_EY, i, j, k + 1) - F(ORC_EY, i, j, k)) * iz;",
     "double cEx = (F(ORC_EZ, i, j + 1, k) - F(ORC_EZ, i, j, k)) * iy;"),
    ("bin: positions outside the domain not wrapped", "c[a] = wrap((int64_t)floor(pos[a] / dd), n[a]) / bsize[a];",
     "c[a] = ((int64_t)floor(pos[a] / dd) < 0 ? 0 : (int64_t)floor(pos[a] / dd) % n[a]) / bsize[a];"),
    ("bin: box index with z fastest", "box[p] = (c[2] * nb[1] + c[1]) * nb[0] + c[0];",
     "box[p] = (c[0] * nb[1] + c[1]) * nb[2] + c[2];"),
    ("boris: gamma of u^{n-1/2} instead of u-",
     "double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);",
     "double gm = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);"),
    ("field update: E before the first B half step", "    add_antenna(s);\n    push_b_half(s);\n    push_e(s);\n",
     "    add_antenna(s);\n    push_e(s);\n    push_b_half(s);\n"),
    ("field update: second B half step dropped", "    push_e(s);\n    push_b_half(s);\n    damp_fields(s);",
     "    push_e(s);\n    damp_fields(s);"),
    ("esirkepov: dz for dy in the Jz prefactor", "const double cz = -qw / (dx * dy * dt);",
     "const double cz = -qw / (dx * dz * dt);"),
    ("positions: no wrap at the upper end", "    if (x >= L) x -= L;\n    return x;", "    return x;"),
    ("box counts: positions not wrapped", "c[a] = wrap((int64_t)floor(pos[a] / s->d[a]), s->n[a]) / bsize[a];",
     "c[a] = ((int64_t)floor(pos[a] / s->d[a]) < 0 ? 0 : (int64_t)floor(pos[a] / s->d[a]) % s->n[a]) / bsize[a];"),
    ("box counts: x and y box indices swapped", "counts[(c[2] * nb[1] + c[1]) * nb[0] + c[0]]++;",
     "counts[(c[2] * nb[1] + c[0]) * nb[0] + c[1]]++;"),
    ("rho: charge density without the cell volume", "double qw = sp->q * sp->w[p] / vol;", "double qw = sp->q * sp->w[p];"),
    ("rho: shape one order low", "for (int l = 0; l < np1; l++) wt[a][l] = orc_shape(o, X[a] - (double)(b[a] + l));",
     "for (int l = 0; l < np1; l++) wt[a][l] = orc_shape(o > 1 ? o - 1 : o, X[a] - (double)(b[a] + l));"),
    ("antenna: cosine carrier", "double env = exp(-tt * tt) * sin(s->las_omega * (t - s->las_tpeak));",
     "double env = exp(-tt * tt) * cos(s->las_omega * (t - s->las_tpeak));"),
    ("antenna: envelope twice as long", "double tt = (t - s->las_tpeak) / s->las_tau;",
     "double tt = (t - s->las_tpeak) / (2.0 * s->las_tau);"),
    ("antenna: waist read as the Gaussian's sigma", "exp(-r2 / (s->las_w0 * s->las_w0));",
     "exp(-r2 / (2.0 * s->las_w0 * s->las_w0));"),
    ("antenna: source at t = n dt instead of (n + 1/2) dt", "double t = ((double)s->step + 0.5) * s->dt;",
     "double t = ((double)s->step) * s->dt;"),
]


def _run_mutant(idx, desc, old, new, tmpdir):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique or missing: {desc}"
    mpath = os.path.join(tmpdir, f"m{idx}.c")
    lpath = os.path.join(tmpdir, f"libm{idx}.so")
    with open(mpath, "w") as f:
        f.write(src.replace(old, new))
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-I", os.path.join(ROOT, "oracle"), "-o", lpath, mpath, "-lm"])
    env = dict(os.environ, PIC_ORACLE_LIB=lpath)
    r = subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return desc, r.returncode


def test_every_planted_mistake_fails_a_pin():
    with tempfile.TemporaryDirectory() as tmp:
        with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
            futs = [ex.submit(_run_mutant, i, *m, tmp) for i, m in enumerate(MUTATIONS)]
            results = [f.result() for f in futs]
    survivors = [d for d, rc in results if rc == 0]
    assert not survivors, f"pins did not catch: {survivors}"
