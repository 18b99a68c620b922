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
    # the start of a run: Eq. (initTimestep) wired into the first levels
    "init_level_off_by_one": ("level[i] = (int8_t)L;", "level[i] = (int8_t)(L + 1);"),
    "init_other_row_jerk": ("orc_dt_initial(a + 3 * i, k + 3 * i, eta_init)", "orc_dt_initial(a + 3 * i, k, eta_init)"),
    # the summation-check and sorted-summation oracles
    "rsqrt_cmp_flip": ("return P < one ? -1 : (P > one ? 1 : 0);", "return P < one ? 1 : (P > one ? -1 : 0);"),
    "rsqrt_exp_off": ("const int K = 2 * (e0 - 1) + er;", "const int K = 2 * e0 + er;"),
    "terms_jerk_sign": ("mr3 * fmaf(-w, dx[c], dv[c])", "mr3 * fmaf(w, dx[c], dv[c])"),
    "terms_lo_dropped": ("dx[c] = (hj - hi_i[c]) + (lj - lo_i[c]);", "dx[c] = (hj - hi_i[c]);"),
    "terms_xv_order": ("const float xv = fmaf(dx[2], dv[2], fmaf(dx[1], dv[1], dx[0] * dv[0]));",
                       "const float xv = dx[0] * dv[0] + dx[1] * dv[1] + dx[2] * dv[2];"),
    "sorted_by_value": ("const uint32_t ma = a & 0x7fffffffu, mb = b & 0x7fffffffu;", "const uint32_t ma = a, mb = b;"),
    "sorted_largest_first": ("if (ma != mb) return ma < mb ? -1 : 1;", "if (ma != mb) return ma < mb ? 1 : -1;"),
}

# pin suite that must catch each mutant (default: the FP64 oracle's pins)
PINS = {name: "test_oracle_sumcheck.py" for name in MUTANTS
        if name.startswith(("rsqrt_", "terms_", "sorted_"))}


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
                        os.path.join(ROOT, "tests", PINS.get(name, "test_oracle_pins.py"))],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"


ADJ_SRC = os.path.join(ROOT, "oracle", "adjoint.py")
ADJ_MUTANTS = {
    "vjp_r5_sign": ("gd = mj * (R3[..., None] * ga[:, None, :] - 3.0", "gd = mj * (R3[..., None] * ga[:, None, :] + 3.0"),
    "vjp_drop_r7": ("+ 15.0 * (R7 * de * dgk)", "+ 0.0 * (R7 * de * dgk)"),
    "vjp_roles_swapped": ("gx = gd.sum(0) - gd.sum(1)", "gx = gd.sum(1) - gd.sum(0)"),
    "vjp_mass_drop_egk": ("gm = (R3 * dga + R3 * egk", "gm = (R3 * dga + 0.0 * egk"),
    "loss_grad_no_pot": ("gx = 2.0 * x - m[:, None]", "gx = 2.0 * x - 0.0 * m[:, None]"),
    "vjp_seed_drops_velocity": ("gv = np.array(g_vT, float).reshape(-1, 3)", "gv = 0.0 * np.array(g_vT, float).reshape(-1, 3)"),
    "reverse_predictor_dt2": ("ga = g_a + g_xp * dt ** 2 / 2.0 + g_vp * dt", "ga = g_a + g_xp * dt ** 2 + g_vp * dt"),
}


@pytest.mark.parametrize("name", sorted(ADJ_MUTANTS))
def test_adjoint_pins_catch_mutant(tmp_path, name):
    """The same for the numpy reverse-mode oracle: the mutated module replaces oracle.adjoint in a
    subprocess that runs its pins."""
    old, new = ADJ_MUTANTS[name]
    src = open(ADJ_SRC).read()
    assert src.count(old) >= 1, f"mutation anchor missing: {old!r}"
    mod = tmp_path / "adjoint_mutant.py"
    mod.write_text(src.replace(old, new, 1))
    boot = ("import sys, importlib.util; sys.path.insert(0, %r); import oracle; "
            "spec = importlib.util.spec_from_file_location('oracle.adjoint', %r); "
            "m = importlib.util.module_from_spec(spec); spec.loader.exec_module(m); "
            "sys.modules['oracle.adjoint'] = m; oracle.adjoint = m; import pytest; "
            "sys.exit(pytest.main(['-q', '-x', '-p', 'no:cacheprovider', %r]))"
            % (ROOT, str(mod), os.path.join(ROOT, "tests", "test_oracle_adjoint.py")))
    r = subprocess.run([sys.executable, "-c", boot], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode not in (0, 4, 5), r.stdout[-2000:] + r.stderr[-2000:]
    assert "failed" in r.stdout, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"


PKG_SRC = os.path.join(ROOT, "oracle", "__init__.py")
PKG_MUTANTS = {
    # the wrapper hands eta to the start of a run where eta_init belongs
    "init_eta_for_eta_init": ("self.n, m, x, v, self.eps2, self.eta_init, self.lmin",
                              "self.n, m, x, v, self.eps2, self.eta, self.lmin"),
}


@pytest.mark.parametrize("name", sorted(PKG_MUTANTS))
def test_wrapper_pins_catch_mutant(tmp_path, name):
    """The same for the oracle's Python wrapper: a copy of the oracle package with one mistake in
    __init__.py (its C source unchanged) is imported in place of the real one before the pins run."""
    old, new = PKG_MUTANTS[name]
    src = open(PKG_SRC).read()
    assert src.count(old) == 1, f"mutation anchor missing or ambiguous: {old!r}"
    pkg = tmp_path / "oracle"
    pkg.mkdir()
    for f in ("oracle.c", "oracle.h", "adjoint.py"):
        shutil.copy(os.path.join(ROOT, "oracle", f), pkg / f)
    (pkg / "__init__.py").write_text(src.replace(old, new, 1))
    boot = ("import sys; sys.path.insert(0, %r); import oracle; assert oracle.__file__.startswith(%r); "
            "sys.path.insert(1, %r); import pytest; "
            "sys.exit(pytest.main(['-q', '-x', '-p', 'no:cacheprovider', %r]))"
            % (str(tmp_path), str(tmp_path), ROOT, os.path.join(ROOT, "tests", "test_oracle_pins.py")))
    r = subprocess.run([sys.executable, "-c", boot], cwd=str(tmp_path), capture_output=True, text=True, timeout=600)
    assert r.returncode not in (0, 4, 5), r.stdout[-2000:] + r.stderr[-2000:]
    assert "failed" in r.stdout, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
