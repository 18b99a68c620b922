"""Degenerate sizes through the C ABI: an empty block, a single particle, every mode."""
import numpy as np
import pytest

import oracle
from synthetic import plummer_sphere
from tests.gpu_common import EPS2, gpu_force, need_gpu

pytestmark = pytest.mark.gpu
MODES = ("plain", "comp", "sumcheck", "sorted", "ds")


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.mark.parametrize("mode", MODES)
def test_empty_block_is_a_no_op(torch, mode):
    from paper_astro_ph_0702058_gb300 import Simulation
    m, x, v = plummer_sphere(300, 3)
    with Simulation(m, x, v, EPS2, mode=mode) as sim:
        sim.predict(0.0)
        before = sim.stats()["force_calls"]
        acc, jerk, pot = gpu_force(sim, np.zeros(0, dtype=np.int32))
        assert acc.shape == (0, 3) and pot.shape == (0,)
        sim.correct(np.zeros(0, dtype=np.int32))
        assert sim.stats()["blocks"] == 0 and sim.stats()["force_calls"] == before + 1


@pytest.mark.parametrize("mode", MODES)
def test_single_particle_moves_ballistically(torch, mode):
    """N = 1: no force, every step at dt_max, and x(t) = x + v t exactly in FP64."""
    from paper_astro_ph_0702058_gb300 import Simulation
    m = np.array([1.0])
    x = np.array([[0.25, -0.5, 0.125]])
    v = np.array([[0.5, 0.25, -1.0]])
    with Simulation(m, x, v, EPS2, lmin=6, lmax=26, mode=mode) as sim:
        sim.predict(0.0)
        acc, jerk, pot = gpu_force(sim, np.array([0], dtype=np.int32))
        assert not acc.any() and not jerk.any() and pot[0] == 0.0
        nb = sim.step(1.0 / 16)
        out = dict(x=np.zeros((1, 3)), v=np.zeros((1, 3)), level=np.zeros(1, dtype=np.int8))
        sim.get_state(**out)
        ek, ep = sim.energy()
    assert nb == 4 and out["level"][0] == 6
    ref = x.copy()
    for _ in range(4):
        ref = ref + (1.0 / 64) * v
    assert np.array_equal(out["x"], ref) and np.array_equal(out["v"], v)
    assert ek == 0.5 * (v ** 2).sum() and ep == 0.0


def test_two_bodies_every_mode_agree_with_oracle(torch):
    from paper_astro_ph_0702058_gb300 import Simulation
    m, x, v = plummer_sphere(2, 4)
    ref = oracle.force(m, x, v, EPS2)
    for mode in MODES:
        with Simulation(m, x, v, EPS2, mode=mode) as sim:
            sim.predict(0.0)
            got = gpu_force(sim, np.array([0, 1], dtype=np.int32))
        for g, r in zip(got, ref):
            assert np.allclose(g, r, rtol=1e-5, atol=0), mode
