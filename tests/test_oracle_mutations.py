"""Plants plausible mistakes in a copy of the oracle (a dropped term, a wrong
sign, a transposed operand, a wrong index or factor) and checks that the pins of
test_oracle_pins.py catch every one of them.  CPU only."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gd_oracle.c")

# (name, original text, mutated text)
MUTATIONS = [
    ("gradient energy factor", "hscale(gCg, 0.5 * m->c_d)", "hscale(gCg, m->c_d)"),
    ("penalty sign", "hd dk = hsub(phi, kappa);", "hd dk = hadd(phi, kappa);"),
    ("dropped det H in J-1", "x[2] = hadd(hadd(trH, hscale(hsub(hsq(trH), HH), 0.5)), det3(H));",
     "x[2] = hadd(trH, hscale(hsub(hsq(trH), HH), 0.5));"),
    ("I2 factor", "x[1] = hadd(hscale(a, 2.0), hscale(hsub(hsq(a), AA), 0.5));",
     "x[1] = hadd(hscale(a, 2.0), hscale(hsub(hsq(a), AA), 0.25));"),
    ("normalising coefficient", "m->psi_n = 2.0 * dN[0] + 4.0 * dN[1] + dN[2];",
     "m->psi_n = 2.0 * dN[0] + 2.0 * dN[1] + dN[2];"),
    ("dropped H^T H in C - I", "for (int k = 0; k < 3; ++k) s = hadd(s, hmul(H[k][i], H[k][j]));",
     "for (int k = 0; k < 3; ++k) s = hadd(s, hc(0.0));"),
    ("C for C^-1 in the gradient energy", "gCg = hadd(gCg, hmul(hmul(g[i], adj[i][j]), g[j]));",
     "gCg = hadd(gCg, hmul(hmul(g[i], C[i][j]), g[j]));"),
    ("q_nloc sign", "q = hadd(q, hscale(hdiv(hsub(phi, kappa), degradation(m, kappa)), c));",
     "q = hadd(q, hscale(hdiv(hsub(kappa, phi), degradation(m, kappa)), c));"),
    ("degradation threshold", "if (kappa.v > m->kappa_d) return hexp", "if (kappa.v > 0.0) return hexp"),
    ("transposed Jacobian inverse", "for (int k = 0; k < dim; ++k) s += dNr[a][k] * inv[k][J];",
     "for (int k = 0; k < dim; ++k) s += dNr[a][k] * inv[J][k];"),
    ("coupling sign in the tangent", "D[c * nz + e] += mixed[c] * dkdz[e];", "D[c * nz + e] -= mixed[c] * dkdz[e];"),
    ("quadrature weight", "*Jw = det;", "*Jw = 1.0;"),
    ("loading test", "if (r0 > 0.0) {\n        inf->loading = 1;", "if (r0 > 0.05) {\n        inf->loading = 1;"),
    ("yield normalisation", "m->y_s = 1.0 / N.a;", "m->y_s = 1.0;"),
    ("volumetric term", "return hadd(hscale(iso, m->mu_e), hscale(hsq(t), m->lambda_e));",
     "return hadd(hscale(iso, m->mu_e), hscale(t, m->lambda_e));"),
    ("adjoint: history coupling of the weight sensitivity", "v[c] = Psi(&m, zz, hc(kap)).ab + mixed[c] * dk;",
     "v[c] = Psi(&m, zz, hc(kap)).ab;"),
    ("adjoint: unloading history sensitivity", "if (dk_dkp) dk_dkp[q] = inf.loading ? 0.0 : 1.0;",
     "if (dk_dkp) dk_dkp[q] = 0.0;"),
    ("adjoint: weight derivative of the yield normalisation", "m->c_ys = hinv(Np);", "m->c_ys = hc(1.0 / Np.v);"),
    ("staggered: the nodal solve updates the history", "    if (m->frozen) {\n        memset(inf, 0, sizeof(*inf));",
     "    if (0) {\n        memset(inf, 0, sizeof(*inf));"),
    ("staggered: frozen tangent keeps the implicit-function term", "    if (inf->loading) {\n        double drk",
     "    if (inf->loading || m->frozen) {\n        double drk"),
]

# the pins that run against each mutant (the fast ones)
PINS = ("stress_free or dd1 or closed_form_chain or objectivity or neo_hooke or small_strain or "
        "residual_is_energy or tangent_is or homogeneous_patch or mullins or kkt or single_hex8 or "
        "yield_function or degradation or local_equals or patch_test or nonlocal_field or adjoint or staggered")


@pytest.mark.parametrize("name,orig,mut", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(name, orig, mut):
    src = open(SRC).read()
    assert src.count(orig) == 1, f"mutation anchor not found once: {orig!r}"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "mut.c")
        so = os.path.join(d, "mut.so")
        open(c, "w").write(src.replace(orig, mut))
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", so, c, "-lm"])
        env = dict(os.environ, GD_ORACLE_SO=so)
        r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                            "-x", "-q", "-k", PINS, "-p", "no:cacheprovider"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode != 0, f"no pin caught the planted mistake '{name}'"
