"""FP64 reverse mode (adjoint) of a shared-step Hermite rollout.  TEST INFRASTRUCTURE ONLY.

The rollout: the force of Eq. (Force) with the Appendix A pair term at t = 0,
then ``steps`` Hermite steps of one shared dt (predictor and corrector of
Sect. 2 of Portegies Zwart, Belleman & Geldof 2007).  The loss is the sum of
squared final positions plus the final softened potential energy,
L = sum_i |x_i|^2 + E_pot, E_pot = -1/2 sum_i sum_{j != i} m_i m_j / sqrt(r_ij^2 + eps^2).

``rollout_grad`` returns L and dL/d(x0, v0, m) by reverse mode: the
corrector and predictor are linear in (x, v, a, k, a_p, k_p), so their
adjoints are their transposes; the force's vector-Jacobian product follows
from the derivatives of the pair term (R = (eps^2 + |d|^2)^(-1/2), d = x_j - x_i,
e = v_j - v_i):
  d a_ij / d d = m_j (R^3 I - 3 R^5 d d^T),  d k_ij / d e = the same matrix,
  d k_ij / d d [delta] = m_j (-3 R^5 (d.delta) e - 3 R^5 (e.delta) d
                              + 15 R^7 (d.e)(d.delta) d - 3 R^5 (d.e) delta).
Plain numpy over all pairs: meant for N <= a few hundred.  Pinned by central
finite differences of the C oracle's forward run (tests/test_oracle_adjoint.py).
"""
from __future__ import annotations

import numpy as np


def _pairs(m, x, v, eps2):
    n = len(m)
    d = x[None, :, :] - x[:, None, :]          # d[i, j] = x_j - x_i
    e = v[None, :, :] - v[:, None, :]
    r2 = eps2 + (d * d).sum(-1)
    off = ~np.eye(n, dtype=bool)
    R = np.zeros((n, n))
    R[off] = 1.0 / np.sqrt(r2[off])
    return d, e, R


def force(m, x, v, eps2):
    """(a, k): acceleration and jerk of every particle (all pairs, j != i)."""
    d, e, R = _pairs(m, x, v, eps2)
    R3, R5 = R ** 3, R ** 5
    de = (d * e).sum(-1)
    a = (m[None, :, None] * R3[..., None] * d).sum(1)
    k = (m[None, :, None] * (R3[..., None] * e - 3.0 * (de * R5)[..., None] * d)).sum(1)
    return a, k


def force_vjp(m, x, v, eps2, ga, gk):
    """(gx, gv, gm) = the force's vector-Jacobian product with upstream (ga, gk)."""
    d, e, R = _pairs(m, x, v, eps2)
    R3, R5, R7 = R ** 3, R ** 5, R ** 7
    de = (d * e).sum(-1)
    dga = (d * ga[:, None, :]).sum(-1)          # d_ij . ga_i
    dgk = (d * gk[:, None, :]).sum(-1)
    egk = (e * gk[:, None, :]).sum(-1)
    mj = m[None, :, None]
    gd = mj * (R3[..., None] * ga[:, None, :] - 3.0 * (R5 * dga)[..., None] * d)
    gd += mj * (-3.0 * (R5 * egk)[..., None] * d - 3.0 * (R5 * dgk)[..., None] * e
                + 15.0 * (R7 * de * dgk)[..., None] * d - 3.0 * (R5 * de)[..., None] * gk[:, None, :])
    ge = mj * (R3[..., None] * gk[:, None, :] - 3.0 * (R5 * dgk)[..., None] * d)
    gx = gd.sum(0) - gd.sum(1)                  # x_j gets +d, x_i gets -d
    gv = ge.sum(0) - ge.sum(1)
    gm = (R3 * dga + R3 * egk - 3.0 * R5 * de * dgk).sum(0)
    return gx, gv, gm


def potential_energy(m, x, eps2):
    d, _, R = _pairs(m, x, np.zeros_like(x), eps2)
    return -0.5 * (m[:, None] * m[None, :] * R).sum()


def loss(m, x, eps2):
    return float((x * x).sum() + potential_energy(m, x, eps2))


def loss_grad(m, x, eps2):
    """(dL/dx, dL/dm) of the loss at the final state."""
    d, _, R = _pairs(m, x, np.zeros_like(x), eps2)
    R3 = R ** 3
    gx = 2.0 * x - m[:, None] * (m[None, :, None] * R3[..., None] * d).sum(1)
    gm = -(m[None, :] * R).sum(1)
    return gx, gm


def rollout(m, x0, v0, eps2, dt, steps):
    """Forward run; returns the list of states (x, v, a, k) at steps 0 .. steps."""
    x, v = np.array(x0, float), np.array(v0, float)
    a, k = force(m, x, v, eps2)
    states = [(x, v, a, k)]
    for _ in range(steps):
        xp = x + v * dt + a * dt ** 2 / 2.0 + k * dt ** 3 / 6.0
        vp = v + a * dt + k * dt ** 2 / 2.0
        ap, kp = force(m, xp, vp, eps2)
        a2 = -6.0 * (a - ap) / dt ** 2 - (4.0 * k + 2.0 * kp) / dt
        a3 = 12.0 * (a - ap) / dt ** 3 + 6.0 * (k + kp) / dt ** 2
        x = xp + a2 / 24.0 * dt ** 4 + a3 / 120.0 * dt ** 5
        v = vp + a2 / 6.0 * dt ** 3 + a3 / 24.0 * dt ** 4
        a, k = ap, kp
        states.append((x, v, a, k))
    return states


def _reverse(m, states, eps2, dt, steps, gx, gv, gm):
    """The reverse sweep from the gradients (gx, gv, gm) of the final x, v and of the masses to
    (dx0, dv0, dm): corrector, force and predictor transposed step by step, then the t = 0 force."""
    ga = np.zeros_like(gx)
    gk = np.zeros_like(gx)
    c1, c2, c3, c4 = dt ** 4 / 24.0, dt ** 5 / 120.0, dt ** 3 / 6.0, dt ** 4 / 24.0
    for s in range(steps - 1, -1, -1):
        x, v, a, k = states[s]
        xp = x + v * dt + a * dt ** 2 / 2.0 + k * dt ** 3 / 6.0
        vp = v + a * dt + k * dt ** 2 / 2.0
        # corrector transposed
        g_a2 = c1 * gx + c3 * gv
        g_a3 = c2 * gx + c4 * gv
        g_xp, g_vp = gx.copy(), gv.copy()
        g_ap = 6.0 / dt ** 2 * g_a2 - 12.0 / dt ** 3 * g_a3 + ga
        g_kp = -2.0 / dt * g_a2 + 6.0 / dt ** 2 * g_a3 + gk
        g_a = -6.0 / dt ** 2 * g_a2 + 12.0 / dt ** 3 * g_a3
        g_k = -4.0 / dt * g_a2 + 6.0 / dt ** 2 * g_a3
        # force at the predicted state
        fx, fv, fm = force_vjp(m, xp, vp, eps2, g_ap, g_kp)
        g_xp += fx
        g_vp += fv
        gm = gm + fm
        # predictor transposed
        gx = g_xp
        gv = g_xp * dt + g_vp
        ga = g_a + g_xp * dt ** 2 / 2.0 + g_vp * dt
        gk = g_k + g_xp * dt ** 3 / 6.0 + g_vp * dt ** 2 / 2.0
    # initial force
    fx, fv, fm = force_vjp(m, states[0][0], states[0][1], eps2, ga, gk)
    return gx + fx, gv + fv, gm + fm


def rollout_grad(m, x0, v0, eps2, dt, steps):
    """(L, dL/dx0, dL/dv0, dL/dm) by reverse mode through the whole rollout."""
    m = np.asarray(m, float)
    states = rollout(m, x0, v0, eps2, dt, steps)
    xf = states[-1][0]
    L = loss(m, xf, eps2)
    gx, gm = loss_grad(m, xf, eps2)
    return (L,) + _reverse(m, states, eps2, dt, steps, gx, np.zeros_like(gx), gm)


def rollout_vjp(m, x0, v0, eps2, dt, steps, g_xT, g_vT):
    """(x_T, v_T, g_x0, g_v0, g_m): the final state of the rollout and the vector-Jacobian product of
    (x0, v0, m) -> (x_T, v_T) with the cotangents (g_xT, g_vT) of the final positions and velocities."""
    m = np.asarray(m, float)
    states = rollout(m, x0, v0, eps2, dt, steps)
    gx = np.array(g_xT, float).reshape(-1, 3)
    gv = np.array(g_vT, float).reshape(-1, 3)
    return (states[-1][0], states[-1][1]) + _reverse(m, states, eps2, dt, steps, gx, gv, np.zeros_like(m))
