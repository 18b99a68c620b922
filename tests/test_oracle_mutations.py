"""The oracle pins catch plausible mistakes.

Each case plants one mistake (a dropped term, a flipped sign, transposed
operands, an off-by-one level) in a temporary copy of ``oracle/oracle.c``,
builds it on the CPU, and runs the pin suite against it in a subprocess;
the suite must fail.  The committed oracle is never touched.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "jerk_sign": ("ki[c] += m[j] * (dv[c] * r3inv - 3.0 * xv", "ki[c] += m[j] * (dv[c] * r3inv + 3.0 * xv"),
    "jerk_drop_dv": ("(dv[c] * r3inv - 3.0", "(0.0 * r3inv - 3.0"),
    "acc_sign": ("ai[c] += m[j] * dx[c] * r3inv;", "ai[c] -= m[j] * dx[c] * r3inv;"),
    "no_softening": ("const double r2 = eps2 + dx[0]", "const double r2 = 0.0 * eps2 + dx[0]"),
    "jerk_r5_power": ("const double r5inv = r3inv * rinv * rinv;", "const double r5inv = r3inv * rinv;"),
    "predict_k_coeff": ("k[e] * dt3 / 6.0", "k[e] * dt3 / 2.0"),
    "predict_v_order": ("vp[e] = v[e] + a[e] * dt + k[e] * dt2 / 2.0;", "vp[e] = v[e] + a[e] * dt;"),
    "corr_transposed": ("(4.0 * k[e] + 2.0 * kp[c])", "(2.0 * k[e] + 4.0 * kp[c])"),
    "corr_a3_sign": ("a3[c] = 12.0 * da / dt3", "a3[c] = -12.0 * da / dt3"),
    "corr_x_coeff": ("a3[c] / 120.0 * dt5", "a3[c] / 24.0 * dt5"),
    "criterion_inverted": ("return sqrt(eta * num / den);", "return sqrt(eta * den / num);"),
    "criterion_a2_begin": ("a2e[c] = a2[c] + a3[c] * dt;", "a2e[c] = a2[c];"),
    "level_off_by_one": ("int L = 1 - e;", "int L = -e;"),
    "grow_unchecked": ("if (l_old - 1 >= lmin && t_new % two_dt_old == 0) return l_old - 1;",
                       "if (l_old - 1 >= lmin) return l_old - 1;"),
    "schedule_tie": ("if (tn == tmin) active[na++]", "if (tn <= tmin + 1) active[na++]"),
    "energy_half": ("ep += 0.5 * m[i] * phi[i];", "ep += m[i] * phi[i];"),
    "self_term": ("if (j == i) continue;\n            double dx[3]", "double dx[3]"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor missing: {old!r}"
    d = tmp_path / name
    d.mkdir()
    shutil.copy(os.path.join(ROOT, "oracle", "oracle.h"), d / "oracle.h")
    (d / "oracle.c").write_text(src.replace(old, new, 1))
    so = d / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                    str(d / "oracle.c"), "-o", str(so), "-lm"], check=True)
    env = dict(os.environ, NBODY_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
