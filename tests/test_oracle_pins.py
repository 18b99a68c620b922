"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test checks one oracle function against what the paper or the
mathematics fixes: exact rational brute force, closed forms (Newtonian
two-body force, Kepler orbits, polynomial trajectories, the Aarseth
criterion on a circular orbit), finite differences, conservation laws and
hand-built block schedules.  A dropped term, a wrong sign, a swapped operand
or an off-by-one level in the oracle fails at least one of them.
"""
import json
import math
import os
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

from synthetic import kepler_pair, plummer_sphere

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# --------------------------------------------------------------------------- force
def _exact_force(m, x, v, eps2, digits=60):
    """Eq. (Force) with the Appendix A softened pair term, exact r^2 and 60-digit r^-1."""
    getcontext().prec = digits
    n = len(m)
    F = lambda z: Fraction(float(z))  # noqa: E731  exact binary value of a double
    X = [[F(c) for c in row] for row in x]
    V = [[F(c) for c in row] for row in v]
    M = [F(c) for c in m]
    e2 = F(eps2)
    acc, jerk, pot = [], [], []
    for i in range(n):
        ai = [Decimal(0)] * 3
        ki = [Decimal(0)] * 3
        pi_ = Decimal(0)
        for j in range(n):
            if j == i:
                continue
            dx = [X[j][c] - X[i][c] for c in range(3)]
            dv = [V[j][c] - V[i][c] for c in range(3)]
            r2 = e2 + sum(d * d for d in dx)
            xv = sum(dx[c] * dv[c] for c in range(3))
            rinv = 1 / Decimal(r2.numerator).__truediv__(Decimal(r2.denominator)).sqrt()
            mj = Decimal(M[j].numerator) / Decimal(M[j].denominator)
            D = lambda f: Decimal(f.numerator) / Decimal(f.denominator)  # noqa: E731
            r3 = rinv ** 3
            r5 = rinv ** 5
            for c in range(3):
                ai[c] += mj * D(dx[c]) * r3
                ki[c] += mj * (D(dv[c]) * r3 - 3 * D(xv) * D(dx[c]) * r5)
            pi_ -= mj * rinv
        acc.append([float(c) for c in ai])
        jerk.append([float(c) for c in ki])
        pot.append(float(pi_))
    return np.array(acc), np.array(jerk), np.array(pot)


@pytest.mark.parametrize("n,eps2", [(2, 0.0), (3, 1.0 / 65536), (5, 0.01), (16, 1.0 / 65536)])
def test_force_matches_exact_brute_force(orc, n, eps2):
    rs = np.random.default_rng(100 + n)
    m = rs.uniform(0.5, 2.0, n) / n
    x = rs.normal(size=(n, 3))
    v = rs.normal(size=(n, 3))
    acc, jerk, pot = orc.force(m, x, v, eps2)
    ea, ek, ep = _exact_force(m, x, v, eps2)
    for got, ref in ((acc, ea), (jerk, ek)):
        err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert err.max() < 1e-13
    assert np.abs((pot - ep) / ep).max() < 1e-14


def test_force_two_body_newton(orc):
    """Two bodies: |a_1| = m_2 d / (d^2 + eps^2)^(3/2) pointing at body 2; phi_1 = -m_2 / sqrt(d^2+eps^2)."""
    d, eps2 = 0.75, 0.04
    u = np.array([2.0, -1.0, 2.0]) / 3.0
    m = np.array([0.3, 0.7])
    x = np.stack([np.zeros(3), d * u])
    v = np.zeros((2, 3))
    acc, jerk, pot = orc.force(m, x, v, eps2)
    s = (d * d + eps2) ** 1.5
    np.testing.assert_allclose(acc[0], m[1] * d / s * u, rtol=1e-15, atol=1e-16)
    np.testing.assert_allclose(acc[1], -m[0] * d / s * u, rtol=1e-15, atol=1e-16)
    np.testing.assert_allclose(pot, [-m[1] / math.sqrt(d * d + eps2), -m[0] / math.sqrt(d * d + eps2)],
                               rtol=1e-15)
    assert np.all(jerk == 0.0)  # no relative motion, no jerk


def test_force_momentum_conservation(orc):
    """Antisymmetry m_i a_ij = -m_j a_ji: sum m a = 0 and sum m k = 0 (unequal masses)."""
    rs = np.random.default_rng(7)
    n = 300
    m = rs.uniform(0.1, 3.0, n)
    x = rs.normal(size=(n, 3))
    v = rs.normal(size=(n, 3))
    acc, jerk, pot = orc.force(m, x, v, 1e-4)
    for f in (acc, jerk):
        tot = np.abs((m[:, None] * f).sum(axis=0)).max()
        scale = (m[:, None] * np.abs(f)).sum(axis=0).max()
        assert tot < 1e-13 * scale
    # phi symmetric: sum_i m_i phi_i counts each unordered pair twice
    iu, ju = np.triu_indices(n, 1)
    w = -(m[iu] * m[ju] / np.sqrt(((x[iu] - x[ju]) ** 2).sum(axis=1) + 1e-4)).sum()
    assert abs((m * pot).sum() - 2 * w) < 1e-12 * abs(w)


def test_jerk_is_time_derivative_of_acceleration(orc):
    """k = da/dt along straight-line motion: central finite difference, O(h^2)."""
    rs = np.random.default_rng(11)
    n = 9
    m = rs.uniform(0.5, 1.5, n) / n
    x = rs.normal(size=(n, 3))
    v = rs.normal(size=(n, 3))
    eps2 = 1e-3
    _, jerk, _ = orc.force(m, x, v, eps2)
    h = 1e-5
    ap, _, _ = orc.force(m, x + h * v, v, eps2)
    am, _, _ = orc.force(m, x - h * v, v, eps2)
    fd = (ap - am) / (2 * h)
    err = np.linalg.norm(fd - jerk, axis=1) / np.linalg.norm(jerk, axis=1)
    assert err.max() < 1e-7


def test_potential_gradient_is_minus_acceleration(orc):
    """d phi_i / d x_i = -a_i (softened potential and force are consistent)."""
    rs = np.random.default_rng(12)
    n = 7
    m = rs.uniform(0.5, 1.5, n) / n
    x = rs.normal(size=(n, 3))
    v = np.zeros((n, 3))
    eps2 = 2e-3
    acc, _, _ = orc.force(m, x, v, eps2)
    h = 1e-6
    for i in range(n):
        g = np.empty(3)
        for c in range(3):
            xp = x.copy(); xp[i, c] += h  # noqa: E702
            xm = x.copy(); xm[i, c] -= h  # noqa: E702
            g[c] = (orc.force(m, xp, v, eps2, [i])[2][0] - orc.force(m, xm, v, eps2, [i])[2][0]) / (2 * h)
        assert np.linalg.norm(g + acc[i]) < 1e-7 * np.linalg.norm(acc[i])


def test_self_term_excluded_with_zero_softening(orc):
    m, x, v = kepler_pair(0.0)
    acc, jerk, pot = orc.force(m, x, v, 0.0)
    assert np.all(np.isfinite(acc)) and np.all(np.isfinite(jerk)) and np.all(np.isfinite(pot))
    acc1, _, pot1 = orc.force(m[:1], x[:1], v[:1], 0.0)   # a lone particle feels nothing
    assert np.all(acc1 == 0) and pot1[0] == 0


# --------------------------------------------------------------------------- energy
def test_energy_closed_forms(orc):
    # Kepler pair m1 = m2 = 1/2, a = 1: E = -m1 m2 / (2a) = -1/8 at any phase.
    for e in (0.0, 0.5, 0.9):
        m, x, v = kepler_pair(e)
        ek, ep = orc.energy(m, x, v, 0.0)
        assert abs(ek + ep + 0.125) < 1e-15
    # Equilateral triangle of side s, masses mu: W = -3 mu^2 / s, at rest.
    s, mu = 0.8, 0.25
    x = np.array([[0, 0, 0], [s, 0, 0], [s / 2, s * math.sqrt(3) / 2, 0]])
    ek, ep = orc.energy(np.full(3, mu), x, np.zeros((3, 3)), 0.0)
    assert ek == 0 and abs(ep + 3 * mu * mu / s) < 1e-15
    # Softening enters as sqrt(r^2 + eps^2).
    ek, ep = orc.energy(np.full(3, mu), x, np.zeros((3, 3)), 0.09)
    assert abs(ep + 3 * mu * mu / math.sqrt(s * s + 0.09)) < 1e-15


def test_energy_plummer_henon_units(orc):
    """Henon units: E = -1/4, virial 2K/|W| = 1 (up to sampling noise and the 0.999 cut)."""
    m, x, v = plummer_sphere(8192, 21)
    ek, ep = orc.energy(m, x, v, 0.0)
    assert abs(ek + ep + 0.25) < 0.02
    assert abs(2 * ek / abs(ep) - 1) < 0.05
    assert abs(ek - 0.25) < 0.02


# --------------------------------------------------------------------------- predictor
def test_predictor_exact_on_cubic_trajectories(orc):
    """x(t) = x + v t + a t^2/2 + k t^3/6 is reproduced exactly, each particle from its own t_i."""
    rs = np.random.default_rng(3)
    n, lmax = 50, 20
    x, v, a, k = (rs.normal(size=(n, 3)) for _ in range(4))
    t = rs.integers(0, 1 << 12, n).astype(np.int64) * 8
    t_new = (1 << 15) + 24
    xp, vp = orc.predict(x, v, a, k, t, t_new, lmax)
    dt = (t_new - t) / float(1 << lmax)
    for i in range(n):
        T = Fraction(int(t_new - t[i]), 1 << lmax)
        for c in range(3):
            X = (Fraction(x[i, c]) + Fraction(v[i, c]) * T + Fraction(a[i, c]) * T ** 2 / 2
                 + Fraction(k[i, c]) * T ** 3 / 6)
            V = Fraction(v[i, c]) + Fraction(a[i, c]) * T + Fraction(k[i, c]) * T ** 2 / 2
            assert abs(xp[i, c] - float(X)) <= 4e-16 * (abs(float(X)) + 1)
            assert abs(vp[i, c] - float(V)) <= 4e-16 * (abs(float(V)) + 1)
    assert np.all(dt > 0)


# --------------------------------------------------------------------------- corrector
def _quintic(c, t):
    """Derivatives 0..3 of x(t) = sum_n c_n t^n / n!, n = 0..5."""
    f = math.factorial
    x = sum(c[n] * t ** n / f(n) for n in range(6))
    v = sum(c[n] * t ** (n - 1) / f(n - 1) for n in range(1, 6))
    a = sum(c[n] * t ** (n - 2) / f(n - 2) for n in range(2, 6))
    k = sum(c[n] * t ** (n - 3) / f(n - 3) for n in range(3, 6))
    return x, v, a, k


def test_corrector_exact_on_quintic_trajectories(orc):
    """Hermite interpolation is exact for cubic a(t): a^(2), a^(3) and the corrected x, v of a
    quintic trajectory are reproduced, and the criterion sees end-of-step derivatives."""
    rs = np.random.default_rng(5)
    n, lmin, lmax, eta = 6, 2, 20, 0.01
    C = rs.normal(size=(6, n, 3))
    st = orc.State(np.ones(n), C[0], C[1], 0.0, eta, lmin=lmin, lmax=lmax)
    st.a[:] = C[2]
    st.k[:] = C[3]
    st.level[:] = 3   # a long step keeps the rounding of Delta a / dt^3 small
    t_new = 1 << (lmax - 3)
    dt = t_new / float(1 << lmax)
    xe, ve, ae, ke = _quintic(C, dt)
    xp, vp = st.predict(t_new)
    act = np.arange(n, dtype=np.int32)
    dtc = st.correct(act, xp, vp, ae, ke, t_new)
    assert _rel(st.x, xe) < 1e-14 and _rel(st.v, ve) < 1e-13
    assert np.array_equal(st.a, ae) and np.array_equal(st.k, ke) and np.all(st.t == t_new)
    for i in range(n):
        ref = orc.dt_aarseth(ae[i], ke[i], C[4, i] + C[5, i] * dt, C[5, i], eta)
        assert abs(dtc[i] - ref) <= 1e-11 * ref


# --------------------------------------------------------------------------- time steps
def test_aarseth_criterion_circular_orbit_closed_form(orc):
    """Uniform circular motion, |a^(n)| = A w^n: Eq. (timestep) gives sqrt(eta)/w, Eq. (initTimestep) eta/w."""
    A, w, th, eta = 2.5, 3.7, 0.4, 0.02
    rot = lambda p: np.array([math.cos(th + p), math.sin(th + p), 0.0])  # noqa: E731
    a = -A * rot(0)
    k = -A * w * rot(math.pi / 2)
    a2 = -A * w * w * rot(math.pi)
    a3 = -A * w ** 3 * rot(3 * math.pi / 2)
    assert abs(orc.dt_aarseth(a, k, a2, a3, eta) - math.sqrt(eta) / w) < 1e-15
    assert abs(orc.dt_initial(a, k, eta) - eta / w) < 1e-16


def test_init_levels_circular_binaries_closed_form(orc):
    """Eq. (initTimestep) through the oracle's start of a run.  For a circular binary of total mass 1 and
    separation d (eps = 0) each body has |a| = 1/(2 d^2) and, since dx.dv = 0, |k| = |dv|/(2 d^3) with
    |dv| = d^(-1/2); so |a|/|k| = d^(3/2) exactly and the first step is the largest power of two not above
    eta_init d^(3/2).  Two binaries 10^6 apart (cross terms ~1e-12 relative) with different d must get the
    levels worked out by hand below; eta is set apart from eta_init, so taking one for the other, an
    off-by-one level or another particle's force changes them."""
    # (d, eta_init, level): eta_init d^1.5 and the bin [2^-L, 2^-(L-1)) it falls in
    cases = [
        (1.0, 0.01, 7),      # 0.01     in [0.0078125, 0.015625)
        (0.25, 0.01, 10),    # 0.00125  in [0.0009765625, 0.001953125)
        (4.0, 0.003, 6),     # 0.024    in [0.015625, 0.03125)
        (0.25, 0.003, 12),   # 0.000375 in [0.000244140625, 0.00048828125)
    ]
    for (d1, eta_init, l1), (d2, eta_init2, l2) in zip(cases[::2], cases[1::2]):
        assert eta_init == eta_init2
        for d, lv in ((d1, l1), (d2, l2)):
            dt = eta_init * d ** 1.5
            assert 2.0 ** -lv <= dt * (1 - 1e-6) and dt * (1 + 1e-6) < 2.0 ** (1 - lv)
        ma, xa, va = kepler_pair(0.0, a=d1)
        mb, xb, vb = kepler_pair(0.0, a=d2)
        m = np.concatenate([ma, mb])
        x = np.concatenate([xa, xb + np.array([1e6, 0.0, 0.0])])
        v = np.concatenate([va, vb])
        st = orc.State(m, x, v, 0.0, 0.05, eta_init=eta_init, lmin=3, lmax=26).init()
        assert list(st.level) == [l1, l1, l2, l2], (d1, d2, eta_init, list(st.level))
        assert np.all(st.t == 0)
        # the forces it stored are the binaries' own, to the 1e-12 of the far pair
        for i, d in enumerate((d1, d1, d2, d2)):
            assert abs(np.linalg.norm(st.a[i]) * 2 * d * d - 1) < 1e-10
            assert abs(np.linalg.norm(st.k[i]) * 2 * d ** 3.5 - 1) < 1e-10


def test_level_quantisation_edges(orc):
    lmin, lmax = 6, 26
    assert orc.level_floor(2.0 ** -7, lmin, lmax) == (7, False)
    assert orc.level_floor(2.0 ** -7 * 1.999, lmin, lmax) == (7, False)
    assert orc.level_floor(2.0 ** -7 * 0.999, lmin, lmax) == (8, False)
    assert orc.level_floor(np.nextafter(2.0 ** -9, 0), lmin, lmax) == (10, False)
    assert orc.level_floor(0.5, lmin, lmax) == (6, False)          # above dt_max: clamp
    assert orc.level_floor(math.inf, lmin, lmax) == (6, False)
    assert orc.level_floor(2.0 ** -26, lmin, lmax) == (26, False)
    assert orc.level_floor(2.0 ** -27, lmin, lmax) == (26, True)   # below dt_min: clamp, flagged
    assert orc.level_floor(0.0, lmin, lmax) == (26, True)
    assert orc.level_floor(math.nan, lmin, lmax)[0] == -1
    # shrink at once; grow one level at most, only on a multiple of twice the old step
    assert orc.next_level(8, 11, 3 << 18, lmin, lmax) == 11
    assert orc.next_level(8, 8, 3 << 18, lmin, lmax) == 8
    assert orc.next_level(8, 6, 4 << 18, lmin, lmax) == 7
    assert orc.next_level(8, 6, 3 << 18, lmin, lmax) == 8
    assert orc.next_level(6, 6, 0, lmin, lmax) == 6


def test_schedule_hand_built(orc):
    lmax = 26
    t = np.array([0, 0, 0], dtype=np.int64)
    lv = np.array([7, 6, 7], dtype=np.int8)
    assert orc.schedule(t, lv, lmax)[0] == 1 << 19
    assert list(orc.schedule(t, lv, lmax)[1]) == [0, 2]
    t = np.array([1 << 19, 0, 1 << 19], dtype=np.int64)
    lv = np.array([8, 6, 7], dtype=np.int8)
    tb, act = orc.schedule(t, lv, lmax)
    assert tb == (1 << 19) + (1 << 18) and list(act) == [0]
    t = np.array([(1 << 19) + (1 << 18), 0, 1 << 19], dtype=np.int64)
    tb, act = orc.schedule(t, lv, lmax)
    assert tb == 1 << 20 and list(act) == [0, 1, 2]
    # the smallest steps: due one tick apart, only the earliest is in the block
    t = np.array([0, 0, 2, 1], dtype=np.int64)
    lv = np.array([25, 26, 26, 26], dtype=np.int8)
    tb, act = orc.schedule(t, lv, lmax)
    assert tb == 1 and list(act) == [1]


def test_block_run_invariants(orc):
    m, x, v = plummer_sphere(256, 9)
    st = orc.State(m, x, v, (1 / 256) ** 2, 0.02, lmin=6, lmax=26).init()
    t_prev = 0
    for _ in range(60):
        t_blk, act, *_ = st.step()
        assert t_blk >= t_prev and np.all(np.diff(act) > 0)
        t_prev = t_blk
        steps = np.left_shift(np.int64(1), (26 - st.level.astype(np.int64)))
        assert np.all(st.t % steps == 0)
        assert np.all(st.t <= t_blk)


# --------------------------------------------------------------------------- integrator
def _kepler_exact(e, t, m1=0.5, m2=0.5):
    mt = m1 + m2
    M = t  # mean motion 1 for a = 1, G(m1 + m2) = 1
    E = M
    for _ in range(60):
        E -= (E - e * math.sin(E) - M) / (1 - e * math.cos(E))
    rel = np.array([math.cos(E) - e, math.sqrt(1 - e * e) * math.sin(E), 0.0])
    return np.stack([-m2 / mt * rel, m1 / mt * rel])


@pytest.mark.parametrize("e", [0.0, 0.5])
def test_hermite_fourth_order_convergence_kepler(orc, e):
    """Shared power-of-two step on a Kepler orbit: halving dt cuts the error by ~2^4."""
    errs, derr = [], []
    t_end = 4.0
    for L in (7, 8):
        m, x, v = kepler_pair(e)
        st = orc.State(m, x, v, 0.0, 0.01, lmin=L, lmax=L).init()
        e0 = sum(st.energy())
        st.evolve(int(t_end * (1 << L)))
        assert np.all(st.t == int(t_end * (1 << L)))
        errs.append(np.abs(st.x - _kepler_exact(e, t_end)).max())
        derr.append(abs(sum(st.energy()) - e0))
    ratio = errs[0] / errs[1]
    assert 10 < ratio < 24, ratio
    assert derr[0] / max(derr[1], 1e-300) > 8


def test_energy_error_band_and_block_statistics(orc):
    """N = 1024, eta = 0.01, dt_max = 1/64, to t = 1/8: the paper's fitted block statistics
    (n_steps ~ 247 N^0.35 per time unit, n_block ~ 0.20 N^0.81) within a factor 2, and an
    FP64 energy error far below the paper's single-precision GPU level."""
    with open(os.path.join(GOLDEN, "paper_block_statistics.json")) as f:
        g = json.load(f)
    N = 1024
    m, x, v = plummer_sphere(N, 1)
    st = orc.State(m, x, v, (1 / 256) ** 2, 0.01, lmin=6, lmax=26).init()
    e0 = sum(st.energy())
    bt, bn, _ = st.evolve(1 << (26 - 3))
    assert np.all(st.t == 1 << 23)
    n_steps_fit = g["n_steps_coeff"] * N ** g["n_steps_exp"] / 8
    n_block_fit = g["n_block_coeff"] * N ** g["n_block_exp"]
    assert 0.5 < len(bt) / n_steps_fit < 2
    assert 0.5 < bn.mean() / n_block_fit < 2
    de = abs((sum(st.energy()) - e0) / e0)
    assert 1e-12 < de < g["gpu_energy_error_mean"]
