"""A-priori per-particle error bounds of the FP32 force kernel against the FP64 oracle.

The force on particle i is a sum of pair terms a_ij, k_ij, phi_ij evaluated in
FP32 (unit roundoff u = 2^-24).  Its error against the exact FP64 sum is bounded
to first order by the sum over j of four contributions, each computed here in
FP64 from the particles' positions and velocities:

  position rounding (plain mode only; compensated mode forms x_j - x_i from
  hi/lo splits, exact to ~u^2): |delta d| <= u (|x_i| + |x_j|), and
      |d a_ij / d d| <= 2 m_j / R^3,
      |d k_ij / d d| <= 24 m_j |dv| / R^4,
      |d phi_ij / d d| <= m_j / R^2,          R^2 = |d|^2 + eps^2;
  velocity rounding (both modes): |delta dv| <= u (|v_i| + |v_j|) and
      |d k_ij / d dv| <= 2 m_j / R^3;
  pair arithmetic: the MUFU reciprocal square root (relative error <= 2^-22.9,
      about 2.1 u, entering r^-3 three times and r^-5 five times) plus the
      roundings of the products and fused multiply-adds: C_ARITH u |term|;
  summation: FP32 partial sums of FOLD = 128 terms, then FP32 additions of the
      partials (plain) or double-single folds (compensated): a statistical
      bound C_SUM u (sqrt(FOLD) + sqrt(n_partials)) sum_j |term| with the
      second root absent in compensated mode.

Nothing here is the method's arithmetic under test: it is an error model
used to set tolerances.
"""
from __future__ import annotations

import math

import numpy as np

U = 2.0 ** -24
FOLD = 128  # pairs per FP32 partial sum in the force kernels
C_ARITH = {"acc": 10.0, "jerk": 24.0, "pot": 6.0}
C_SUM = 2.0


def bounds(m, x, v, eps2, rows, mode):
    """Per-row absolute error bounds (acc, jerk, pot) and the magnitude sums (A, K, P)."""
    m = np.asarray(m, np.float64)
    x = np.asarray(x, np.float64)
    v = np.asarray(v, np.float64)
    n = len(m)
    xn = np.linalg.norm(x, axis=1)
    vn = np.linalg.norm(v, axis=1)
    n_part = math.ceil(n / FOLD)
    s_fac = C_SUM * (math.sqrt(FOLD) + (math.sqrt(n_part) if mode == "plain" else 0.0))
    out = np.zeros((len(rows), 3))
    mags = np.zeros((len(rows), 3))
    for q, i in enumerate(rows):
        d = x - x[i]
        dv = v - v[i]
        R2 = (d * d).sum(1) + eps2
        R2[i] = np.inf
        R = np.sqrt(R2)
        R3 = R2 * R
        dn = np.linalg.norm(d, axis=1)
        dvn = np.linalg.norm(dv, axis=1)
        a_abs = m * dn / R3
        k_abs = m * dvn / R3 + 3 * m * np.abs((d * dv).sum(1)) * dn / (R3 * R2)
        p_abs = m / R
        ddv = U * (vn[i] + vn)
        bk = C_ARITH["jerk"] * U * k_abs + 2 * m * ddv / R3
        ba = C_ARITH["acc"] * U * a_abs
        bp = C_ARITH["pot"] * U * p_abs
        if mode == "plain":
            dd = U * (xn[i] + xn)
            ba = ba + 2 * m * dd / R3
            bk = bk + 24 * m * dvn * dd / (R3 * R)
            bp = bp + m * dd / R2
        A, K, P = a_abs.sum(), k_abs.sum(), p_abs.sum()
        out[q] = (ba.sum() + s_fac * U * A, bk.sum() + s_fac * U * K, bp.sum() + s_fac * U * P)
        mags[q] = (A, K, P)
    return out, mags
