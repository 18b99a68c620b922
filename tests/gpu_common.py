"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest

from tests.fp32_bounds import bounds

EPS2 = (1.0 / 256) ** 2

# Tolerances against the FP64 oracle:
#  - every row, acc and jerk as vectors and pot: |error| <= the a-priori FP32
#    bound of tests/fp32_bounds.py (position/velocity rounding, pair arithmetic,
#    summation);
#  - the stated per-particle thresholds, 1e-5 relative for plain FP32 pair math
#    and 1e-6 for the compensated form (its literal 1e-10 lies below the
#    rounding of one FP32 pair term and is checked on the summation alone, by
#    the summation-check mode), on the quantities the statement names, |acc|
#    and |jerk| (and the potential), and also on the acc and jerk vectors: the
#    relative error of each key must be <= REL for at least FRAC[mode][key] of
#    the rows whenever >= 100 rows are compared.  The fractions below 1 come
#    from rows with a close neighbour: FP32 positions resolve a separation r
#    only to u |x| / r, and the jerk, with its r^-3 and r^-5 terms, feels this
#    most.  Those rows stay inside their FP32 bound.
REL = {"plain": 1e-5, "comp": 1e-6}
FRAC = {  # Plummer spheres with eps = 1/256, N <= 65536
    "plain": {"acc": 0.97, "acc_mag": 0.97, "pot": 0.99, "jerk": 0.95, "jerk_mag": 0.97},
    "comp": {"acc": 0.99, "acc_mag": 0.99, "pot": 0.99, "jerk": 0.97, "jerk_mag": 0.99},
}
# N = 2^20 with eps = 1e-3: more rows have a close neighbour than at N = 65536
FRAC_LARGE = {
    "plain": {"acc": 0.97, "acc_mag": 0.97, "pot": 0.99, "jerk": 0.90, "jerk_mag": 0.95},
    "comp": FRAC["comp"],
}


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_astro_ph_0702058_gb300 import build
    build.build()
    return torch


def rel_vec(got, ref):
    d = np.linalg.norm(got - ref, axis=1)
    r = np.linalg.norm(ref, axis=1)
    return d / np.where(r > 0, r, 1.0)


def rel_mag(got, ref):
    g = np.linalg.norm(got, axis=1)
    r = np.linalg.norm(ref, axis=1)
    return np.abs(g - r) / np.where(r > 0, r, 1.0)


def rel_scalar(got, ref):
    return np.abs(got - ref) / np.where(np.abs(ref) > 0, np.abs(ref), 1.0)


def errors(acc, jerk, pot, ra, rk, rp):
    return {"acc": rel_vec(acc, ra), "acc_mag": rel_mag(acc, ra), "jerk": rel_vec(jerk, rk),
            "jerk_mag": rel_mag(jerk, rk), "pot": rel_scalar(pot, rp)}


def check_threshold_fractions(mode, e, what="", frac=None):
    """Asserts that each key's share of rows within REL[mode] reaches its fraction; returns the shares."""
    need = (frac or FRAC)[mode]
    got = {key: float(np.mean(e[key] <= REL[mode])) for key in need}
    for key, f in got.items():
        assert f >= need[key], f"{what} {mode} {key}: only {f:.3f} of rows within {REL[mode]:.0e} (need {need[key]})"
    return got


def check_force(mode, m, x, v, eps2, rows, got, ref, what="", min_rows=100):
    """Asserts the per-row FP32 bound and the stated thresholds; returns the errors."""
    acc, jerk, pot = got
    ra, rk, rp = ref
    B, _ = bounds(m, x, v, eps2, np.asarray(rows), mode)
    abs_err = np.stack([np.linalg.norm(acc - ra, axis=1), np.linalg.norm(jerk - rk, axis=1),
                        np.abs(pot - rp)], axis=1)
    worst = (abs_err / B).max(axis=0)
    assert np.all(worst <= 1.0), f"{what} {mode}: error over the FP32 bound, max err/bound {worst}"
    e = errors(acc, jerk, pot, ra, rk, rp)
    if len(rows) >= min_rows:
        shares = check_threshold_fractions(mode, e, what)
        print(f"\n{what} {mode}: rows within {REL[mode]:.0e}: " + ", ".join(f"{k} {f:.4f}" for k, f in shares.items()))
    return e


def gpu_force(sim, act):
    na = len(act)
    acc = np.zeros((na, 3))
    jerk = np.zeros((na, 3))
    pot = np.zeros(na)
    sim.force(np.ascontiguousarray(act, dtype=np.int32), acc=acc, jerk=jerk, pot=pot)
    return acc, jerk, pot
