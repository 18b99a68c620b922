"""Sorted-summation ablation (Sect. 6 of the paper: add the pair forces by size, smallest
first): the GPU mode against the oracle's sorted FP32 sums, bit for bit."""
import numpy as np
import pytest

import oracle
from synthetic import active_subset, plummer_sphere
from tests.gpu_common import EPS2, gpu_force, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.mark.parametrize("n,n_act", [(1, 1), (2, 2), (3, 3), (257, 257), (1000, 1000), (4099, 700),
                                     (16384, 256), (32768, 64)])
def test_sorted_mode_bit_exact(torch, n, n_act):
    from paper_astro_ph_0702058_gb300 import Simulation
    m, x, v = plummer_sphere(n, 40 + n % 7)
    act = active_subset(n, n_act, 9)
    with Simulation(m, x, v, EPS2, mode="sorted") as sim:
        sim.predict(0.0)
        got = gpu_force(sim, act)
    ref = oracle.force_sorted_fp32(m, x, v, EPS2, act)
    for g, r, name in zip(got, ref, ("acc", "jerk", "pot")):
        bad = np.argwhere(g != r)
        assert bad.size == 0, f"{name}: {len(bad)} mismatches, first row {bad[0]}"


def test_sorted_mode_size_limit(torch):
    from paper_astro_ph_0702058_gb300 import NBodyError, Simulation
    m, x, v = plummer_sphere(32769, 2)
    with pytest.raises(NBodyError):
        Simulation(m, x, v, EPS2, mode="sorted")


def test_sorted_mode_integrates(torch):
    from paper_astro_ph_0702058_gb300 import Simulation
    m, x, v = plummer_sphere(1024, 1)
    with Simulation(m, x, v, EPS2, eta=0.01, mode="sorted") as sim:
        e0 = sum(sim.energy())
        nb = sim.step(1.0 / 64)
        e1 = sum(sim.energy())
    assert nb > 0 and abs((e1 - e0) / e0) < 1e-6
