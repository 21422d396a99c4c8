"""Mutation check of the oracle pins.

Each case plants one plausible mistake (a dropped conjugate, a flipped sign,
a wrong index, a wrong factor) in a private copy of the oracle source, builds
it into a temporary directory and runs the pin suite against it in a child
process.  Every mutant must make at least one pin fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "opo_oracle.c")

MUTANTS = [
    ("pump exponent sign", "A[1] * A[2] * conj(e);", "A[1] * A[2] * e;"),
    ("signal drops conjugate", "A[0] * conj(A[2]) * e;", "A[0] * A[2] * e;"),
    ("idler uses signal kappa", "f[2] = I * kap[2]", "f[2] = I * kap[1]"),
    ("degenerate pump without 1/2", "I * (kap[0] / 2.0)", "I * (kap[0])"),
    ("GVM sign", "double phase = -p->dbeta1[x] * om", "double phase = p->dbeta1[x] * om"),
    ("GVD sign", "+ p->beta2[x] * om * om / 2.0", "- p->beta2[x] * om * om / 2.0"),
    ("TOD factor 1/3", "om * om * om / p->tod_div", "om * om * om / 3.0"),
    ("field loss instead of power loss", "exp(-p->alpha[x] * dz / 2.0)", "exp(-p->alpha[x] * dz)"),
    ("RK4 stage 4 from k2", "t[x] = y[x] + h * k3[x];", "t[x] = y[x] + h * k2[x];"),
    ("RK4 stage 4 position", "nl_rhs(p, kap, t, z0 + h, k4);", "nl_rhs(p, kap, t, z0 + h / 2.0, k4);"),
    ("second half-step z", "orc_rk4_step(p, fields, zj + dz / 2.0, dz / 2.0);",
     "orc_rk4_step(p, fields, zj, dz / 2.0);"),
    ("delay sign", "om * om / 2.0 - om * p->delay;", "om * om / 2.0 + om * p->delay;"),
    ("time origin", "return (double)(idx - p->n / 2) * dt;", "return (double)idx * dt;"),
    ("EOM ignores round trip", "(tau_of(p, j) + (double)m * p->t_rt)", "(tau_of(p, j) + 0.0 * (double)m)"),
    ("output coupling", "? sqrt(1.0 - p->R[x]) : 1.0;", "? 1.0 : 1.0;"),
    ("centroid uses FFT index", "num += ((double)kk / p->t_window) * pk;",
     "num += ((double)k / p->t_window) * pk + 0.0 * kk;"),
    ("sech width", "fwhm / (2.0 * acosh(sqrt(2.0)))", "fwhm / 1.665"),
    ("idler not dumped", "memset(a, 0, sizeof(double) * fsz);", "(void)a;"),
    ("resonant pump not injected", "a[i] += pump[i];", "a[i] += 0.0 * pump[i];"),
    ("ns pulse field FWHM", "exp(-2.0 * log(2.0) * t * t", "exp(-4.0 * log(2.0) * t * t"),
    ("ns slice ignores round trip", "double t = (double)m * p->t_rt + tau_of(p, j)",
     "double t = 0.0 * (double)m * p->t_rt + tau_of(p, j)"),
    ("beta4 factor 1/12", "om * om * om * om / 24.0", "om * om * om * om / 12.0"),
    ("beta4 sign", "+ p->beta4[x] * om", "- p->beta4[x] * om"),
    ("XPM counted once", "itot += 2.0 * inten[y];", "itot += 1.0 * inten[y];"),
    ("Kerr k0 of the signal", "double k0 = 2.0 * ORC_PI / p->lambda[x];",
     "double k0 = 2.0 * ORC_PI / p->lambda[1];"),
    ("extra crystals skipped", "for (int32_t k = 0; k <= p->nextra; k++) {",
     "for (int32_t k = 0; k <= 0 * p->nextra; k++) {"),
    ("extra crystal keeps the first one's dispersion", "q->beta2[x] = c->beta2[x];",
     "q->beta2[x] = p->beta2[x];"),
    ("extra crystal keeps the first one's indices", "q->nidx[x] = c->nidx[x];",
     "q->nidx[x] = p->nidx[x];"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_kill_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not found: " + name
    mut = tmp_path / "opo_oracle.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-I", os.path.join(ROOT, "oracle"), "-o", str(lib), str(mut), "-lm"])
    env = dict(os.environ, OPO_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "mutant survived the pins: " + name
