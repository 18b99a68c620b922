"""The a-priori FP32 error bound of tests/fp32_bounds.py against an emulation of the kernel's arithmetic
(CPU only).

The emulation forms every pair term of the packed force kernel in float32 with numpy, in the kernel's
operation order (dx = x_j - x_i from FP32 positions in plain mode, from hi/lo splits in compensated
mode; r2 by fused multiply-adds; xv likewise; rinv, m rinv, m rinv^3, w), with the reciprocal square
root drawn at the worst relative error the MUFU unit may have (the correctly rounded value times
1 +- 2^-22.9, rounded to float32), and sums them as the kernel does: float32 partial sums of 128 terms,
each split into its even-j and odd-j halves, then a float32 running total (plain) or Knuth's TwoSum into
a double-single pair (compensated).  The emulated errors against the FP64 oracle must lie inside the
bound the GPU parity tests apply, with room to spare.  This pins the bound to the arithmetic it claims to
bound; it does not replace the GPU tests.
"""
import numpy as np
import pytest

import oracle
from synthetic import active_subset, plummer_sphere
from tests.fp32_bounds import bounds

F = np.float32
EPS2 = (1.0 / 256) ** 2
MUFU_REL = 2.0 ** -22.9


def _fma(a, b, c):
    """float32 fused multiply-add: the product is exact in float64 (24 + 24 bits), one rounding after."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F)


def _emulate_row(i, m, x, v, mode, rng):
    n = len(m)
    hi = x.astype(F)
    lo = (x - hi.astype(np.float64)).astype(F)
    vf = v.astype(F)
    mf = m.astype(F)
    j = np.arange(n)
    if mode == "comp":
        dx = ((hi[j] - hi[i]).astype(F) + (lo[j] - lo[i]).astype(F)).astype(F)
    else:
        dx = (hi[j] - hi[i]).astype(F)
    dv = (vf[j] - vf[i]).astype(F)
    r2 = _fma(dx[:, 2], dx[:, 2], _fma(dx[:, 1], dx[:, 1], _fma(dx[:, 0], dx[:, 0], np.full(n, F(EPS2)))))
    exact = 1.0 / np.sqrt(r2.astype(np.float64))
    rinv = (exact * (1.0 + MUFU_REL * rng.choice([-1.0, 1.0], n))).astype(F)
    rinv[i] = F(0)  # j = i contributes nothing
    xv = _fma(dx[:, 2], dv[:, 2], _fma(dx[:, 1], dv[:, 1], (dx[:, 0] * dv[:, 0]).astype(F)))
    rinv2 = (rinv * rinv).astype(F)
    mr = (mf * rinv).astype(F)
    mr3 = (mr * rinv2).astype(F)
    wn = ((xv * rinv2).astype(F) * F(-3)).astype(F)
    terms = np.empty((n, 7), F)
    for c in range(3):
        terms[:, c] = (mr3 * dx[:, c]).astype(F)  # the kernel fuses these into its partials: bounded alike
        terms[:, 3 + c] = (mr3 * _fma(wn, dx[:, c], dv[:, c])).astype(F)
    terms[:, 6] = -mr
    # 128-term partials, each as even and odd halves summed in float32, then folded
    out = np.zeros(7)
    tot = np.zeros(7, F)
    low = np.zeros(7, F)
    for b in range(0, n, 128):
        blk = terms[b:b + 128]
        even = np.zeros(7, F)
        odd = np.zeros(7, F)
        for k in range(0, len(blk), 2):
            even = (even + blk[k]).astype(F)
            if k + 1 < len(blk):
                odd = (odd + blk[k + 1]).astype(F)
        part = (even + odd).astype(F)
        if mode == "comp":
            s = (tot + part).astype(F)
            bb = (s - tot).astype(F)
            e = ((tot - (s - bb).astype(F)).astype(F) + (part - bb).astype(F)).astype(F)
            tot, low = s, (low + e).astype(F)
        else:
            tot = (tot + part).astype(F)
    out[:] = tot.astype(np.float64) + (low.astype(np.float64) if mode == "comp" else 0.0)
    return out[:3], out[3:6], out[6]


@pytest.mark.parametrize("mode", ["plain", "comp"])
def test_fp32_bound_holds_for_the_emulated_kernel(mode):
    n = 2048
    m, x, v = plummer_sphere(n, 71)
    rows = active_subset(n, 48, 71)
    rng = np.random.default_rng(71)
    got = [_emulate_row(int(i), m, x, v, mode, rng) for i in rows]
    acc = np.array([g[0] for g in got])
    jerk = np.array([g[1] for g in got])
    pot = np.array([g[2] for g in got])
    ra, rk, rp = oracle.force(m, x, v, EPS2, rows)
    B, _ = bounds(m, x, v, EPS2, rows, mode)
    err = np.stack([np.linalg.norm(acc - ra, axis=1), np.linalg.norm(jerk - rk, axis=1), np.abs(pot - rp)], 1)
    ratio = (err / B).max(axis=0)
    print(f"\n{mode}: largest error / bound over {len(rows)} rows: acc {ratio[0]:.3f} jerk {ratio[1]:.3f} "
          f"pot {ratio[2]:.3f}")
    assert np.all(ratio <= 0.5), ratio  # inside the bound, with at least a factor of two to spare
