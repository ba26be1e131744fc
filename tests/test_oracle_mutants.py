"""Mutation tests of the oracle's pins: each plausible mistake below is
planted in a copy of the oracle's C source (on the CPU), compiled, and the pin
suite (test_oracle_pins.py) must fail against it.  A surviving mutant would
mean a part of the oracle no pin fixes."""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, original text, mutated text): one plausible mistake each
MUTANTS = [
    ("shear strain without 1/2", "e12[g] = 0.5 * (uy + vx);", "e12[g] = (uy + vx);"),
    ("divergence sign", "loc[(size_t)K * 18 + j] = -fx;", "loc[(size_t)K * 18 + j] = fx;"),
    ("Jacobian transposed", "E->dx[g][j] = (J11 * M->q2x[g][j] - J10 * M->q2e[g][j]) / det;",
     "E->dx[g][j] = (J11 * M->q2x[g][j] - J01 * M->q2e[g][j]) / det;"),
    ("Gauss weights halved", "ws[i] = 2.0 / ((1.0 - x * x) * dpn * dpn);",
     "ws[i] = 1.0 / ((1.0 - x * x) * dpn * dpn);"),
    ("Delta cross term", "k_mix * e11 * e22", "k_mix * e11 * e11"),
    ("s22 uses e22 twice", "s22[g] = alphaInv * (PD * (c_a * e22 + c_b * e11) - 0.5 * P);",
     "s22[g] = alphaInv * (PD * (c_a * e22 + c_b * e22) - 0.5 * P);"),
    ("no relaxation of S11", "*q11 = fac * *q11 + a;", "*q11 = *q11 + a;"),
    ("ice strength exponent", "exp(-p->C * (1.0 - a))", "exp(-p->C * a)"),
    ("h not clamped", "double h = fmax(0.0, hg);\n      double a = fmin", "double h = hg;\n      double a = fmin"),
    ("Coriolis sign", "vout[j] = (a * rx + b * ry) / det;", "vout[j] = (a * rx - b * ry) / det;"),
    ("drag without rho_w", "double c = l[j] * p->Cw * p->rho_water *", "double c = l[j] * p->Cw *"),
    ("mass without rho_ice", "m[G.node[j]] += p->rho_ice * G.wdet[g] * h * M->q2[g][j];",
     "m[G.node[j]] += G.wdet[g] * h * M->q2[g][j];"),
    ("local node index transposed", "E->node[a + 3 * b] = (2 * ky + b) * nw + 2 * kx + a;",
     "E->node[a + 3 * b] = (2 * ky + a) * nw + 2 * kx + b;"),
    ("no beta relaxation", "mdt * (p->beta * vprev[j] + vn[j])", "mdt * (vprev[j] + vn[j])"),
    ("DG basis constant", "all[3] = xh * xh - 1.0 / 12.0;", "all[3] = xh * xh - 1.0 / 6.0;"),
    ("Q2 node moved", "q2_nodes[3] = {0.0, 0.5, 1.0};", "q2_nodes[3] = {0.0, 0.4, 1.0};"),
    ("inverse mass skipped", "acc += mass[s * n_s + t] * E->wdet[g] * M->psi_s[t][g];",
     "acc += (s == t) * E->wdet[g] * M->psi_s[t][g];"),
    ("north boundary not Dirichlet", "ix == nw - 1 || iy == nh - 1)", "ix == nw - 1)"),
    ("velocity uses v^n for drag", "double dvx = ox - vprev[j], dvy = oy - vprev[nn + j];",
     "double dvx = ox - vn[j], dvy = oy - vn[nn + j];"),
    ("stress 12 coefficient", "s12[g] = alphaInv * (PD * c_s * e12);",
     "s12[g] = alphaInv * (PD * c_a * e12);"),
    ("isoparametric dx/deta from the xi-derivative", "J01 += xn[0] * M->q2e[g][j];",
     "J01 += xn[0] * M->q2x[g][j];"),
    ("isoparametric map reads y for x", "J00 += xn[0] * M->q2x[g][j];",
     "J00 += xn[1] * M->q2x[g][j];"),
    ("ocean drag takes the y current in x", "l[j] * tau[j] + c * ox;", "l[j] * tau[j] + c * oy;"),
    ("drag relative velocity ignores the ocean",
     "double dvx = ox - vprev[j], dvy = oy - vprev[nn + j];",
     "double dvx = -vprev[j], dvy = -vprev[nn + j];"),
    ("ice height evaluated with the stress basis",
     "hg += H[(size_t)K * n_a + t] * M->psi_a[t][g];\n        ag",
     "hg += H[(size_t)K * n_a + t] * M->psi_s[t][g];\n        ag"),
    ("ice concentration evaluated with the stress basis",
     "ag += A[(size_t)K * n_a + t] * M->psi_a[t][g];",
     "ag += A[(size_t)K * n_a + t] * M->psi_s[t][g];"),
    ("lumped mass from the constant ice coefficient only",
     "for (int t = 0; t < n_a; ++t) hg += H", "for (int t = 0; t < 1; ++t) hg += H"),
    ("concentration not clamped above", "double a = fmin(1.0, fmax(0.0, ag));",
     "double a = fmax(0.0, ag);"),
    ("per-element P* ignored", "double Pst = PstarK ? PstarK[K] : p->Pstar;",
     "double Pst = p->Pstar;"),
    ("P* of the neighbouring element", "PstarK ? PstarK[K] :",
     "PstarK ? PstarK[(K + 1) % (M->nx * M->ny)] :"),
    ("singular node: y component not written",
     "if (det == 0.0) {\n      vout[j] = 0.0;\n      vout[nn + j] = 0.0;",
     "if (det == 0.0) {\n      vout[j] = 0.0;\n      vout[j] = 0.0;"),
    ("singular node: y written to another node",
     "if (det == 0.0) {\n      vout[j] = 0.0;\n      vout[nn + j] = 0.0;",
     "if (det == 0.0) {\n      vout[j] = 0.0;\n      vout[nn - j] = 0.0;"),
]


# mistakes in the transport (advection) part, against its own pins
ADVECTION_MUTANTS = [
    ("volume term sign", "RH[i] += w * h * g;", "RH[i] -= w * h * g;"),
    ("east flux sign", "else if (e == 1) f = J[3] * vx - J[1] * vy;",
     "else if (e == 1) f = -(J[3] * vx - J[1] * vy);"),
    ("downwind instead of upwind", "if (f >= 0.0 || nb < 0) {", "if (f < 0.0 || nb < 0) {"),
    ("contravariant velocity transposed", "double vt_xi = J[3] * vx - J[1] * vy,",
     "double vt_xi = J[3] * vx - J[2] * vy,"),
    ("west neighbour trace on the wrong edge",
     "if (e == 0) { xi = 0.0; eta = t; nxi = 1.0; neta = t; }",
     "if (e == 0) { xi = 0.0; eta = t; nxi = 0.0; neta = t; }"),
    ("Heun weights", "H[k] = 0.5 * H[k] + 0.5 * (H1[k] + dt * LH[k]);",
     "H[k] = 0.25 * H[k] + 0.75 * (H1[k] + dt * LH[k]);"),
    ("RK3 second stage weights", "H2[k] = 0.75 * H[k] + 0.25 * (H1[k] + dt * LH[k]);",
     "H2[k] = 0.5 * H[k] + 0.5 * (H1[k] + dt * LH[k]);"),
    ("mass matrix without det J", "mass[i * n_a + j] += w * det * psi[i] * psi[j];",
     "mass[i * n_a + j] += w * psi[i] * psi[j];"),
    ("product rule of the basis gradient", "deta[i] = px[kxs[i]] * dpy[kys[i]];",
     "deta[i] = dpx[kxs[i]] * py[kys[i]];"),
    ("edge weight dropped", "RH[i] -= w * f * hh * psi[i];", "RH[i] -= f * hh * psi[i];"),
    ("DG2 rule too low", "static int adv_nq(int n_a) { return n_a == 6 ? 4 : 3; }",
     "static int adv_nq(int n_a) { return n_a == 6 ? 3 : 3; }"),
    ("Euler step sign", "H1[k] = H[k] + dt * LH[k];", "H1[k] = H[k] - dt * LH[k];"),
    ("isoparametric transport Jacobian transposed", "J[2 * c + 1] += xn[c] * deta[j];",
     "J[2 * c + 1] += xn[c] * dxi[j];"),
    ('Euler step of A sign', 'A1[k] = A[k] + dt * LA[k]; }',
     'A1[k] = A[k] - dt * LA[k]; }'),
    ('Heun weights of A', 'A[k] = 0.5 * A[k] + 0.5 * (A1[k] + dt * LA[k]);',
     'A[k] = 0.25 * A[k] + 0.5 * (A1[k] + dt * LA[k]);'),
    ('RK3 second stage of A', 'A2[k] = 0.75 * A[k] + 0.25 * (A1[k] + dt * LA[k]);',
     'A2[k] = 0.75 * A[k] + 0.25 * (A1[k] - dt * LA[k]);'),
    ('RK3 last stage of A', 'A[k] = A[k] / 3.0 + 2.0 * (A2[k] + dt * LA[k]) / 3.0;',
     'A[k] = A[k] / 3.0 + 2.0 * (A2[k] - dt * LA[k]) / 3.0;'),
    ('forward Euler leaves A unchanged', 'memcpy(A, A1, sizeof(double) * n);',
     'memcpy(A, A1, sizeof(double) / n);'),
    ('one-element-wide meshes refused', 'if (nx < 1 || ny < 1 || !xy || !vel || !H || !A || n_steps < 0)',
     'if (nx <= 1 || ny < 1 || !xy || !vel || !H || !A || n_steps < 0)'),
]


def _run_pins_against(src, tmp_path, pins):
    mut = tmp_path / "mutant.c"
    mut.write_text(src)
    so = tmp_path / "mutant.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                    "-D_POSIX_C_SOURCE=199309L", "-o", str(so), str(mut), "-lm"], check=True)
    env = dict(os.environ, MEVP_ORACLE_LIB=str(so))
    return subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", pins),
                           "-x", "-q", "-p", "no:cacheprovider"], env=env, cwd=ROOT,
                          capture_output=True, text=True, timeout=600)


@pytest.mark.parametrize("name,old,new", ADVECTION_MUTANTS, ids=[m[0] for m in ADVECTION_MUTANTS])
def test_advection_mutant_is_caught_by_the_pins(name, old, new, tmp_path):
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, f"mutation site not unique/found: {name}"
    r = _run_pins_against(src.replace(old, new), tmp_path, "test_oracle_advection_pins.py")
    assert r.returncode != 0, f"mutant survived the pins: {name}\n{r.stdout[-2000:]}"


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught_by_the_pins(name, old, new, tmp_path):
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, f"mutation site not unique/found: {name}"
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "mutant.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                    "-D_POSIX_C_SOURCE=199309L", "-o", str(so), str(mut), "-lm"], check=True)
    env = dict(os.environ, MEVP_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests",
                                                                     "test_oracle_pins.py"),
                        "-x", "-q", "-p", "no:cacheprovider"], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant survived the pins: {name}\n{r.stdout[-2000:]}"
