"""Pins of the FP64 reverse-mode oracle (oracle/adjoint.py) to things other than itself:
its forward run agrees with the C oracle's shared-step integration, and its gradients
agree with central finite differences of the C oracle's loss."""
import numpy as np
import pytest

import oracle
from oracle import adjoint
from synthetic import plummer_sphere

EPS2 = (1.0 / 128) ** 2
LEVEL = 9  # dt = 1/512, the shared step of the differentiable configuration


def _c_loss(m, x0, v0, steps):
    st = oracle.State(m, x0, v0, EPS2, 0.01, lmin=LEVEL, lmax=LEVEL).init()
    st.evolve(steps)
    ek, ep = oracle.energy(m, st.x, st.v, EPS2)
    return float((st.x ** 2).sum() + ep), st


def test_adjoint_forward_matches_c_oracle():
    m, x, v = plummer_sphere(40, 3)
    a, k = adjoint.force(m, x, v, EPS2)
    ra, rk, _ = oracle.force(m, x, v, EPS2)
    assert np.abs(a - ra).max() <= 1e-13 * np.abs(ra).max()
    assert np.abs(k - rk).max() <= 1e-13 * np.abs(rk).max()
    states = adjoint.rollout(m, x, v, EPS2, 2.0 ** -LEVEL, 24)
    L, st = _c_loss(m, x, v, 24)
    assert np.abs(states[-1][0] - st.x).max() <= 1e-12
    assert abs(adjoint.loss(m, states[-1][0], EPS2) - L) <= 1e-12 * abs(L)


@pytest.mark.parametrize("n,steps", [(8, 16), (16, 32)])
def test_reverse_mode_matches_central_differences(n, steps):
    m, x, v = plummer_sphere(n, 5 + n)
    m = m * np.random.default_rng(n).uniform(0.7, 1.3, n)  # unequal masses exercise dL/dm
    L, gx, gv, gm = adjoint.rollout_grad(m, x, v, EPS2, 2.0 ** -LEVEL, steps)
    assert abs(L - _c_loss(m, x, v, steps)[0]) <= 1e-12 * abs(L)
    h = 1e-6
    for name, arr, g in (("x", x, gx), ("v", v, gv), ("m", m, gm)):
        fd = np.zeros_like(arr)
        flat = arr.reshape(-1)
        for idx in range(flat.size):
            p = flat.copy(); p[idx] += h  # noqa: E702
            q = flat.copy(); q[idx] -= h  # noqa: E702
            args_p = [m, x, v]
            args_q = [m, x, v]
            pos = {"m": 0, "x": 1, "v": 2}[name]
            args_p[pos] = p.reshape(arr.shape)
            args_q[pos] = q.reshape(arr.shape)
            fd.reshape(-1)[idx] = (_c_loss(*args_p, steps)[0] - _c_loss(*args_q, steps)[0]) / (2 * h)
        err = np.abs(fd - g).max() / np.abs(g).max()
        assert err < 1e-6, (name, err)


def test_force_vjp_matches_central_differences_of_the_c_force():
    """One force evaluation: the vector-Jacobian product against central differences of
    S = sum_i (ga_i . a_i + gk_i . k_i) computed with the C oracle's force."""
    n = 6
    m, x, v = plummer_sphere(n, 41)
    rng = np.random.default_rng(41)
    m = m * rng.uniform(0.5, 1.5, n)
    ga, gk = rng.standard_normal((n, 3)), rng.standard_normal((n, 3))

    def S(mm, xx, vv):
        a, k, _ = oracle.force(mm, xx, vv, EPS2)
        return float((ga * a).sum() + (gk * k).sum())

    gx, gv, gm = adjoint.force_vjp(m, x, v, EPS2, ga, gk)
    h = 1e-6
    for name, arr, g in (("x", x, gx), ("v", v, gv), ("m", m, gm)):
        fd = np.zeros(arr.size)
        for idx in range(arr.size):
            p = arr.reshape(-1).copy(); p[idx] += h  # noqa: E702
            q = arr.reshape(-1).copy(); q[idx] -= h  # noqa: E702
            args_p = {"m": m, "x": x, "v": v}
            args_q = dict(args_p)
            args_p[name] = p.reshape(arr.shape)
            args_q[name] = q.reshape(arr.shape)
            fd[idx] = (S(args_p["m"], args_p["x"], args_p["v"]) - S(args_q["m"], args_q["x"], args_q["v"])) / (2 * h)
        err = np.abs(fd - g.reshape(-1)).max() / np.abs(g).max()
        assert err < 1e-7, (name, err)


def test_rollout_vjp_matches_central_differences():
    """The reverse sweep seeded with arbitrary cotangents of the final positions and velocities:
    <g_x0, dx0> + <g_v0, dv0> + <g_m, dm> against central differences of
    S = <g_xT, x_T> + <g_vT, v_T> from the C oracle's forward run, for every input component."""
    n, steps = 8, 16
    m, x, v = plummer_sphere(n, 51)
    rng = np.random.default_rng(51)
    m = m * rng.uniform(0.7, 1.3, n)
    g_xT, g_vT = rng.standard_normal((n, 3)), rng.standard_normal((n, 3))
    xT, vT, gx, gv, gm = adjoint.rollout_vjp(m, x, v, EPS2, 2.0 ** -LEVEL, steps, g_xT, g_vT)
    st = _c_loss(m, x, v, steps)[1]
    assert np.abs(xT - st.x).max() <= 1e-12 and np.abs(vT - st.v).max() <= 1e-11

    def S(mm, xx, vv):
        s = _c_loss(mm, xx, vv, steps)[1]
        return float((g_xT * s.x).sum() + (g_vT * s.v).sum())

    h = 1e-6
    for name, arr, g in (("x", x, gx), ("v", v, gv), ("m", m, gm)):
        fd = np.zeros(arr.size)
        for idx in range(arr.size):
            p = arr.reshape(-1).copy(); p[idx] += h  # noqa: E702
            q = arr.reshape(-1).copy(); q[idx] -= h  # noqa: E702
            args_p = {"m": m, "x": x, "v": v}
            args_q = dict(args_p)
            args_p[name] = p.reshape(arr.shape)
            args_q[name] = q.reshape(arr.shape)
            fd[idx] = (S(args_p["m"], args_p["x"], args_p["v"]) - S(args_q["m"], args_q["x"], args_q["v"])) / (2 * h)
        err = np.abs(fd - g.reshape(-1)).max() / np.abs(g).max()
        assert err < 1e-6, (name, err)
