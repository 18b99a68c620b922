"""Pins of the summation-check and sorted-summation oracles (orc_rsqrt_rn_f32,
orc_force_fp32_terms, orc_force_sorted_fp32).

The correctly rounded reciprocal square root is checked against 60-digit decimal
arithmetic, and the FP32-term sums against a brute-force reconstruction in exact
rational arithmetic (every FP32 operation rounded from its exact value), so that
a wrong operation order, a dropped term or a wrong rounding shows up."""
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import oracle
from synthetic import plummer_sphere

getcontext().prec = 60


def _fl32(fr: Fraction) -> np.float32:
    """Round an exact rational to the nearest float32 (ties to even)."""
    if fr == 0:
        return np.float32(0.0)
    c = np.float32(float(fr))
    cands = {c, np.nextafter(c, np.float32(np.inf)), np.nextafter(c, np.float32(-np.inf))}
    best = sorted(cands, key=lambda f: (abs(Fraction(float(f)) - fr),
                                        int(np.array(f, dtype=np.float32).view(np.uint32)) & 1))
    return best[0]


def _rsqrt_decimal(r2: np.float32) -> np.float32:
    y = 1 / Decimal(float(r2)).sqrt()
    c = np.float32(float(y))
    cands = [c, np.nextafter(c, np.float32(np.inf)), np.nextafter(c, np.float32(0))]
    return min(cands, key=lambda f: abs(Decimal(float(f)) - y))


def test_rsqrt_rn_matches_60_digit_decimal():
    rng = np.random.default_rng(11)
    r2s = list(np.float32(10.0) ** rng.uniform(-12, 12, 3000).astype(np.float32))
    # hard cases: r2 close to 1/f^2 for floats f (results near a representable value)
    for f in np.float32(2.0) ** rng.uniform(-10, 10, 300).astype(np.float32):
        base = np.float32(1.0) / (np.float32(f) * np.float32(f))
        r2s += [base, np.nextafter(base, np.float32(0)), np.nextafter(base, np.float32(np.inf))]
    r2s += [np.float32(4.0) ** k for k in range(-20, 21)] + [np.float32(2.0), np.float32(3.0)]
    bad = [r for r in r2s if oracle.rsqrt_rn_f32(r) != _rsqrt_decimal(np.float32(r))]
    assert not bad, bad[:5]


def test_rsqrt_rn_exact_powers():
    for k in range(-30, 31):
        assert oracle.rsqrt_rn_f32(np.float32(4.0) ** k) == np.float32(2.0) ** -k


def _terms_exact(m, x, v, eps2, i, comp=True):
    """The 7 lists of FP32 terms over j != i for particle i (as exact rationals), each FP32
    operation rounded from its exact value; comp: dx from the hi/lo split, else from fl32(x)."""
    F = lambda a: Fraction(float(a))
    R = lambda fr: F(_fl32(fr))
    e2 = F(np.float32(eps2))
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    u = v.astype(np.float32)
    mu = m.astype(np.float32)
    terms = [[] for _ in range(7)]
    for j in range(len(m)):
        if j == i:
            continue
        if comp:
            dx = [R(R(F(hi[j, c]) - F(hi[i, c])) + R(F(lo[j, c]) - F(lo[i, c]))) for c in range(3)]
        else:
            dx = [R(F(hi[j, c]) - F(hi[i, c])) for c in range(3)]
        dv = [R(F(u[j, c]) - F(u[i, c])) for c in range(3)]
        r2 = R(dx[2] * dx[2] + R(dx[1] * dx[1] + R(dx[0] * dx[0] + e2)))
        rinv = F(_rsqrt_decimal(np.float32(float(r2))))
        xv = R(dx[2] * dv[2] + R(dx[1] * dv[1] + R(dx[0] * dv[0])))
        rinv2 = R(rinv * rinv)
        mr = R(F(mu[j]) * rinv)
        mr3 = R(mr * rinv2)
        w = R(3 * R(xv * rinv2))
        for c in range(3):
            terms[c].append(R(mr3 * dx[c]))
            terms[3 + c].append(R(mr3 * R(-w * dx[c] + dv[c])))
        terms[6].append(-mr)
    return terms


def test_fp32_terms_match_exact_rational_reconstruction():
    m, x, v = plummer_sphere(7, 19)
    x = x + 1e-9 * np.arange(21).reshape(7, 3)  # nonzero low parts
    eps2 = (1.0 / 64) ** 2
    acc, jerk, pot = oracle.force_fp32_terms(m, x, v, eps2)
    for i in range(7):
        ref = [float(sum(t)) for t in _terms_exact(m, x, v, eps2, i)]
        got = list(acc[i]) + list(jerk[i]) + [pot[i]]
        for c in range(7):
            assert got[c] == pytest.approx(ref[c], rel=1e-15, abs=1e-300), (i, c)


def test_fp32_terms_close_to_fp64_force():
    """The FP32 terms differ from the FP64 pair terms by FP32 rounding only."""
    m, x, v = plummer_sphere(512, 21)
    eps2 = (1.0 / 256) ** 2
    a32, k32, p32 = oracle.force_fp32_terms(m, x, v, eps2)
    a64, k64, p64 = oracle.force(m, x, v, eps2)
    ra = np.linalg.norm(a32 - a64, axis=1) / np.linalg.norm(a64, axis=1)
    rk = np.linalg.norm(k32 - k64, axis=1) / np.linalg.norm(k64, axis=1)
    rp = np.abs(p32 - p64) / np.abs(p64)
    assert np.median(ra) < 1e-6 and np.median(rk) < 1e-5 and np.max(rp) < 1e-6
    assert np.median(ra) > 1e-12  # they are FP32 terms, not FP64 ones


def test_sorted_sums_match_rational_reconstruction_bit_for_bit():
    """Sorted ablation: terms ordered by magnitude (ties by raw bits), added in FP32 from the
    smallest; every addition rounded from its exact value."""
    m, x, v = plummer_sphere(9, 23)
    m = m * (1.0 + 0.1 * np.arange(9))  # unequal masses: no ties in magnitude by symmetry
    eps2 = (1.0 / 64) ** 2
    acc, jerk, pot = oracle.force_sorted_fp32(m, x, v, eps2)
    bits = lambda f: int(np.array(np.float32(float(f)), dtype=np.float32).view(np.uint32))
    for i in range(9):
        got = list(acc[i]) + list(jerk[i]) + [pot[i]]
        for c, ts in enumerate(_terms_exact(m, x, v, eps2, i, comp=False)):
            order = sorted(ts, key=lambda t: (bits(t) & 0x7FFFFFFF, bits(t)))
            s = Fraction(0)
            for t in order:
                s = Fraction(float(_fl32(s + t)))
            assert got[c] == float(s), (i, c)


def test_sorted_order_matters_and_stays_fp32_accurate():
    """The sorted FP32 sum is a different rounding of the same terms as the unsorted one, and
    stays within single-precision accuracy of the FP64 force."""
    m, x, v = plummer_sphere(2048, 24)
    eps2 = (1.0 / 256) ** 2
    act = np.arange(0, 2048, 8, dtype=np.int32)
    a_s, k_s, _ = oracle.force_sorted_fp32(m, x, v, eps2, act)
    a_d, k_d, _ = oracle.force(m, x, v, eps2, act)
    ra = np.linalg.norm(a_s - a_d, axis=1) / np.linalg.norm(a_d, axis=1)
    assert np.median(ra) < 1e-6 and np.max(ra) < 1e-4
