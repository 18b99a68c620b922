"""Double-single force mode against the FP64 oracle: the stated 1e-10 per-particle bound
applied to the force itself (reading gamma), and a free-running integration that follows
the oracle's block schedule."""
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
    got, ref = np.atleast_2d(got.T).T, np.atleast_2d(ref.T).T
    d = np.linalg.norm(got - ref, axis=1)
    r = np.linalg.norm(ref, axis=1)
    return d / np.maximum(r, 1e-3 * np.sqrt(np.mean(r ** 2)))


@pytest.mark.parametrize("n,n_act,split", [(2, 2, 0), (3, 3, 0), (257, 257, 0), (1000, 1000, 1), (4099, 4099, 0),
                                           (4099, 300, 5), (65536, 256, 0)])
def test_ds_force_within_1e10_of_fp64(torch, n, n_act, split):
    from paper_astro_ph_0702058_gb300 import Simulation
    m, x, v = plummer_sphere(n, 60 + n % 11)
    act = active_subset(n, n_act, 3)
    with Simulation(m, x, v, EPS2, mode="ds", j_split=split) as sim:
        sim.predict(0.0)
        got = gpu_force(sim, act)
    ref = oracle.force(m, x, v, EPS2, act)
    worst = [float(_rel(g, r).max()) for g, r in zip(got, ref)]
    print(f"\nds n={n} n_act={n_act}: max rel acc {worst[0]:.2e} jerk {worst[1]:.2e} pot {worst[2]:.2e}")
    assert max(worst) <= TOL, worst


def test_ds_zero_softening_pair(torch):
    from paper_astro_ph_0702058_gb300 import Simulation
    from synthetic import kepler_pair
    m, x, v = kepler_pair(0.5)
    with Simulation(m, x, v, 0.0, mode="ds") as sim:
        sim.predict(0.0)
        got = gpu_force(sim, np.arange(2))
    ref = oracle.force(m, x, v, 0.0)
    for g, r in zip(got, ref):
        assert np.allclose(g, r, rtol=1e-11, atol=0)


def test_ds_integration_follows_oracle(torch):
    """C1 (N = 1024, eta = 0.01, to t = 1/8): same block count as the FP64 oracle and the same
    energy error to 1%."""
    from paper_astro_ph_0702058_gb300 import Simulation
    m, x, v = plummer_sphere(1024, 1)
    with Simulation(m, x, v, EPS2, eta=0.01, lmin=6, lmax=26, mode="ds") as sim:
        e0 = sum(sim.energy())
        nb = sim.step(0.125)
        e1 = sum(sim.energy())
    st = oracle.State(m, x, v, EPS2, 0.01, lmin=6, lmax=26).init()
    o0 = sum(st.energy())
    bt, _, _ = st.evolve(int(0.125 * 2 ** 26))
    o1 = sum(st.energy())
    de, do = abs((e1 - e0) / e0), abs((o1 - o0) / o0)
    print(f"\nds blocks {nb} oracle {len(bt)}; |dE/E| ds {de:.3e} oracle {do:.3e}")
    assert abs(nb - len(bt)) <= 0.002 * len(bt)
    assert abs(de - do) <= 0.01 * do
