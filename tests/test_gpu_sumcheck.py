"""The compensated summation against the stated 1e-10 bound (read as a bound on the
summation given identical FP32 pair terms).

In the summation-check mode the kernel forms each FP32 pair term of the compensated
pair term with correctly rounded operations in a fixed order, and folds every term
into its double-single sums.  The oracle forms the same FP32 terms on the CPU from
the same FP64 state and adds them exactly; the two must agree to 1e-10 per particle
(denominators floored at 1e-3 of the rms over the compared rows).  The kernel is the
production one (force_kernel_x2): its structure-of-arrays tiles and tile groups, the
packed two-pair loop with its even and odd j halves, the j-ranges, the partial layout
and the FP64 reduction are those the compensated benchmark runs; only the pair term's
rsqrt and the fold length differ."""
import numpy as np
import pytest

import oracle
from synthetic import active_subset, plummer_sphere
from tests.gpu_common import EPS2, gpu_force, need_gpu

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def _rel(got, ref):
    """Per-row relative error of vectors (n x 3) or scalars, denominator floored at 1e-3 rms."""
    got, ref = np.atleast_2d(got.T).T, np.atleast_2d(ref.T).T
    d = np.linalg.norm(got - ref, axis=1)
    r = np.linalg.norm(ref, axis=1)
    floor = 1e-3 * np.sqrt(np.mean(r ** 2))
    return d / np.maximum(r, floor), int(np.sum(r < floor))


def _check(got, ref, what):
    worst = {}
    for name, g, r in zip(("acc", "jerk", "pot"), got, ref):
        e, floored = _rel(g, r)
        worst[name] = float(e.max())
        assert e.max() <= TOL, f"{what} {name}: max rel {e.max():.3e} (floored rows {floored})"
    return worst


@pytest.mark.parametrize("n,n_act,shape", [
    (4099, 4099, (0, 0, 0)),
    (4099, 1111, (64, 1, 3)),
    (4099, 1111, (128, 2, 1)),
    (4099, 300, (256, 4, 5)),
    (65536, 512, (0, 0, 0)),
])
def test_sumcheck_sums_equal_exact_sums_of_fp32_terms(torch, n, n_act, shape):
    from paper_astro_ph_0702058_gb300 import Simulation
    m, x, v = plummer_sphere(n, 31)
    act = active_subset(n, n_act, 5)
    threads, ipt, split = shape
    with Simulation(m, x, v, EPS2, mode="sumcheck", j_tile=threads, i_block=ipt, j_split=split) as sim:
        sim.predict(0.0)
        # the kernel's inputs are the oracle's FP32 split of the same FP64 state
        posm = np.zeros((n, 4), np.float32)
        vel = np.zeros((n, 4), np.float32)
        poslo = np.zeros((n, 4), np.float32)
        sim.get_predicted(posm, vel, poslo)
        hi = x.astype(np.float32)
        assert np.array_equal(posm[:, :3], hi) and np.array_equal(posm[:, 3], m.astype(np.float32))
        assert np.array_equal(poslo[:, :3], (x - hi).astype(np.float32))
        assert np.array_equal(vel[:, :3], v.astype(np.float32))
        got = gpu_force(sim, act)
        st = sim.stats()
    if threads:
        assert (st["last_threads"], st["last_i_per_thread"], st["last_j_split"]) == shape
    ref = oracle.force_fp32_terms(m, x, v, EPS2, act)
    worst = _check(got, ref, f"n={n} n_act={n_act} shape={shape}")
    print(f"\nsumcheck n={n} n_act={n_act} shape={shape}: max rel {worst}")


def test_production_comp_differs_only_by_term_rounding(torch):
    """The production compensated mode (hardware rsqrt, 128-term FP32 partials) sits at FP32
    term-rounding distance from the same exact sums, far above the summation-check mode."""
    from paper_astro_ph_0702058_gb300 import Simulation
    n = 4099
    m, x, v = plummer_sphere(n, 32)
    act = active_subset(n, 700, 6)
    ref = oracle.force_fp32_terms(m, x, v, EPS2, act)
    out = {}
    for mode in ("comp", "sumcheck"):
        with Simulation(m, x, v, EPS2, mode=mode) as sim:
            sim.predict(0.0)
            out[mode] = gpu_force(sim, act)
    e_comp = max(_rel(g, r)[0].max() for g, r in zip(out["comp"], ref))
    e_chk = max(_rel(g, r)[0].max() for g, r in zip(out["sumcheck"], ref))
    print(f"\nvs exact sums of the check terms: comp {e_comp:.2e}, sumcheck {e_chk:.2e}")
    assert e_chk <= TOL < e_comp < 1e-4


def test_sumcheck_integrates(torch):
    """The mode runs through the whole block-step path (schedule, predict, force, correct)."""
    from paper_astro_ph_0702058_gb300 import Simulation
    m, x, v = plummer_sphere(1024, 1)
    with Simulation(m, x, v, EPS2, eta=0.01, mode="sumcheck") as sim:
        e0 = sum(sim.energy())
        nb = sim.step(1.0 / 64)
        e1 = sum(sim.energy())
    assert nb > 0 and abs((e1 - e0) / e0) < 1e-6
