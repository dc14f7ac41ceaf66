"""The oracle's pins must catch plausible mistakes. Each case plants one
mistake in a copy of pg_oracle.c (on the CPU), builds it, and runs the pin
suite against it: the suite has to fail."""

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pg_oracle.c")
SRC_TREE = os.path.join(ROOT, "oracle", "pg_tree.c")
PINS = ["tests/test_oracle_newton.py", "tests/test_oracle_table.py", "tests/test_oracle_grad.py",
        "tests/test_oracle_ext.py", "tests/test_oracle_tree.py"]

MUTATIONS = {
    "potential sign": ("nadd(&ph, -m / rh);", "nadd(&ph, m / rh);", 0),
    "list-mode potential sign": ("nadd(&ph, -m / rh);", "nadd(&ph, m / rh);", 1),
    "softening dropped": ("dz * dz + e2;        /* r^2 + eps_i^2 */", "dz * dz;"),
    "list-mode softening dropped": ("double rh2 = dx * dx + dy * dy + dz * dz + c->eps2;",
                                    "double rh2 = dx * dx + dy * dy + dz * dz;"),
    "per-i softening not squared": ("double e2 = c->eps_i ? c->eps_i[i] * c->eps_i[i] : c->eps2;",
                                    "double e2 = c->eps_i ? c->eps_i[i] : c->eps2;"),
    "softening of the j-particle": ("double e2 = c->eps_i ? c->eps_i[i] * c->eps_i[i] : c->eps2;",
                                    "double e2 = c->eps_i && c->nj > 1 ? c->eps_i[1 - (i & 1)] * "
                                    "c->eps_i[1 - (i & 1)] : c->eps2;"),
    "table potential sign": ("nadd(&ph, m * table_eval_s(c->E, c->F, c->smax, c->G0, c->G1, s, NULL));",
                             "nadd(&ph, -m * table_eval_s(c->E, c->F, c->smax, c->G0, c->G1, s, NULL));"),
    "table potential of r, not s": ("double s = (dx * dx + dy * dy + dz * dz) * c->sc2 + 2.0;",
                                    "double s = sqrt(dx * dx + dy * dy + dz * dz) * c->sc2 + 2.0;"),
    "difference transposed": ("double dx = c->xj[3 * j] - xi;", "double dx = xi - c->xj[3 * j];", 0),
    "list-mode difference transposed": ("double dx = c->xj[3 * j] - xi;",
                                        "double dx = xi - c->xj[3 * j];", 1),
    "kernel exponent": ("double k3 = m / (rh2 * rh);                           /* m / r_hat^3 */",
                        "double k3 = m / rh2;"),
    "self not skipped": ("            if (j == sk) continue;\n            double dx = c->xj[3 * j] - xi;",
                         "            double dx = c->xj[3 * j] - xi;"),
    "bin exponent off by one": ("int bE = e - 2;", "int bE = e - 1;"),
    "knot exponent": ("return ldexp(1.0 + (double)bF / (double)nF, (int)bE + 1);",
                      "return ldexp(1.0 + (double)bF / (double)nF, (int)bE);"),
    "s_max fraction": ("(2.0 - ldexp(1.0, -F))", "(2.0 - ldexp(1.0, -F - 1))"),
    "cutoff entry kept": ("            G0[k] = 0.0f;\n            G1[k] = 0.0f;",
                          "            G0[k] = v[k];\n            G1[k] = 0.0f;"),
    "interpolation anchor": ("return (double)G0[k] + (s - orc_knot(E, F, k)) * (double)G1[k];",
                             "return (double)G0[k] + (s - orc_knot(E, F, k + 1)) * (double)G1[k];"),
    "S2 denominator": ("70.0 * x4 - 48.0 * x5 + 7.0 * x6) / (35.0 * a * a);",
                       "70.0 * x4 - 48.0 * x5 + 7.0 * x6) / (35.0 * a * a * a);"),
    "Gaussian term dropped": ("double w = erfc(u) + (r / (rs * sqrt(M_PI))) * exp(-u * u);",
                              "double w = erfc(u);"),
    "periodic image": ("if (box > 0.0) d -= box * nearbyint(d / box);",
                       "if (box > 0.0) d -= box * floor(d / box);"),
    "gradient second sum sign": ("nadd(&gx[q], -M->m[o] * (K * wk[q]", "nadd(&gx[q], M->m[o] * (K * wk[q]"),
    "kernel derivative": ("*Kp = -1.5 * (*K) / rh2;", "*Kp = -0.5 * (*K) / rh2;"),
    "hat weight": ("acc[kb] += pw * (1.0 - t);", "acc[kb] += pw * t;"),
}


# mistakes planted in the tree oracle (pg_tree.c)
TREE_MUTATIONS = {
    "tree opening compares side, not its square": ("if (!holds && side2 < lim) {",
                                                   "if (!holds && side < lim) {"),
    "tree node holding the group accepted": ("if (!holds && side2 < lim) {", "if (side2 < lim) {"),
    "tree centre of mass undivided": ("for (int a = 0; a < 3; ++a) c[a] = t->nS[3 * k + a] / t->nM[k];",
                                      "for (int a = 0; a < 3; ++a) c[a] = t->nS[3 * k + a];"),
    "tree leaf drops its last particle": (
        "for (long long j = t->nfirst[k]; j < t->nfirst[k] + t->ncount[k]; ++j) {\n                if (out)",
        "for (long long j = t->nfirst[k]; j < t->nfirst[k] + t->ncount[k] - 1; ++j) {\n                if (out)"),
    "tree pseudo-particle mass halved": ("            ps[3] = M;\n", "            ps[3] = 0.5 * M;\n"),
    "quadrupole spread without the factor 2": ("double al = sqrt(2.0 * (d13 > 0.0 ? d13 : 0.0) / M);",
                                               "double al = sqrt((d13 > 0.0 ? d13 : 0.0) / M);"),
    "quadrupole pseudo-particle mass M / 4": ("ps[3] = ps[7] = ps[11] = M / 3.0;",
                                              "ps[3] = ps[7] = ps[11] = M / 4.0;"),
    "quadrupole triangle half-height": ("double h = sqrt(3.0) / 2.0;", "double h = 0.5;"),
    "quadrupole spread from the middle eigenvalue": ("d23 = lam[i2] - lam[i3];", "d23 = lam[i1] - lam[i3];"),
    "quadrupole moments about the origin": ("y[a] = t->xs[3 * i + a] - c[a];", "y[a] = t->xs[3 * i + a];"),
    "quadrupole rotation sign": ("A[k][p] = c * akp - sn * akq;", "A[k][p] = c * akp + sn * akq;"),
    "quadrupole eigenvectors transposed": ("e1[a] = V[a][i1]; e2[a] = V[a][i2];", "e1[a] = V[i1][a]; e2[a] = V[i2][a];"),
    "quadrupole sign convention dropped": ("        if (e1[big] < 0.0)\n", "        if (0)\n"),
    "tree finest-level moment skips mass": ("            M = M + t->ms[i];\n", "\n"),
    "tree own particle kept": ("if (j == i) continue;\n                double xj[3], mj;",
                               "double xj[3], mj;"),
}


# mistakes planted in the PM oracle (pm.py), caught by its own pins
PM_SRC = os.path.join(ROOT, "oracle", "pm.py")
PM_MUTATIONS = {
    "TSC centre weight": ("0.75 - d * d", "0.75 - d"),
    "nearest mesh point floored": ("j0 = np.floor(u + 0.5)", "j0 = np.floor(u)"),
    "assignment window not divided out": ("phik = rk * green / tsc_window(N)", "phik = rk * green"),
    "gradient sign": ("np.fft.irfftn(-1j * kk * phik", "np.fft.irfftn(1j * kk * phik"),
    "Green's function without 4 pi": ("-4.0 * np.pi * split_factor(np.sqrt(k2)", "-1.0 * split_factor(np.sqrt(k2)"),
    "Gaussian split halved exponent": ("return np.exp(-(k * scale) ** 2)", "return np.exp(-(k * scale) ** 2 / 2)"),
    "S2 form factor not squared": ("        return out ** 2", "        return out"),
    "density not per cell volume": ("return rho.reshape(N, N, N) / h ** 3", "return rho.reshape(N, N, N)"),
    "k-space sum sign": ("c = -4.0 * np.pi / L ** 3", "c = 4.0 * np.pi / L ** 3"),
    "S2 series second term": ("qs ** 2 / 15.0", "qs ** 2 / 10.0"),
}


@pytest.mark.parametrize("name", sorted(PM_MUTATIONS))
def test_pins_catch_pm_mutation(name, tmp_path):
    old, new = PM_MUTATIONS[name]
    src = open(PM_SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique for {name}"
    mut = tmp_path / "pm_mut.py"
    mut.write_text(src.replace(old, new))
    env = dict(os.environ, PG_ORACLE_PM=str(mut))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "tests/test_oracle_pm.py"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode != 0, f"pins did not catch: {name}\n{r.stdout[-2000:]}"


def _run_pins(tmp_path, name, oracle_src, tree_src):
    mut = tmp_path / "pg_oracle_mut.c"
    mut.write_text(oracle_src)
    mtree = tmp_path / "pg_tree_mut.c"
    mtree.write_text(tree_src)
    so = tmp_path / "liborc_mut.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so), str(mut),
                    str(mtree), "-lm", "-lpthread"], check=True)
    env = dict(os.environ, PG_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch: {name}\n{r.stdout[-2000:]}"


@pytest.mark.parametrize("name", sorted(TREE_MUTATIONS))
def test_pins_catch_tree_mutation(name, tmp_path):
    old, new = TREE_MUTATIONS[name]
    src = open(SRC_TREE).read()
    assert src.count(old) == 1, f"mutation anchor not unique for {name}"
    _run_pins(tmp_path, name, open(SRC).read(), src.replace(old, new))


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name, tmp_path):
    old, new, *which = MUTATIONS[name]
    src = open(SRC).read()
    if which:       # the anchor recurs: plant the mistake in one occurrence
        parts = src.split(old)
        k = which[0]
        assert len(parts) > k + 1, f"mutation anchor missing for {name}"
        src = old.join(parts[:k + 1]) + new + old.join(parts[k + 1:])
    else:
        assert src.count(old) == 1, f"mutation anchor not unique for {name}"
        src = src.replace(old, new)
    _run_pins(tmp_path, name, src, open(SRC_TREE).read())
