"""nbody_step's small-block CUDA graph: the same bits as separate launches, and it is used."""
import numpy as np
import pytest

from synthetic import plummer_sphere
from tests.gpu_common import EPS2, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def _run(m, x, v, mode, t_end, eta, graphs):
    from paper_astro_ph_0702058_gb300 import Simulation, nbody_debug_step_graphs
    nbody_debug_step_graphs(graphs)
    try:
        with Simulation(m, x, v, EPS2, eta=eta, lmin=6, lmax=26, mode=mode) as sim:
            nb = sim.step(t_end)
            n = len(m)
            out = dict(x=np.zeros((n, 3)), v=np.zeros((n, 3)), a=np.zeros((n, 3)), k=np.zeros((n, 3)),
                       t_tick=np.zeros(n, dtype=np.int64), level=np.zeros(n, dtype=np.int8))
            sim.get_state(**out)
            st = sim.stats()
            e = sum(sim.energy())
    finally:
        nbody_debug_step_graphs(True)
    return nb, out, st, e


@pytest.mark.parametrize("mode", ["plain", "comp"])
@pytest.mark.parametrize("n,t_end,eta", [(1024, 0.125, 0.01), (4099, 1.0 / 64, 0.02), (65536, 1.0 / 64, 0.02)])
def test_graph_blocks_equal_separate_launches(torch, mode, n, t_end, eta):
    m, x, v = plummer_sphere(n, 70 + n % 13)
    nb_g, s_g, st_g, e_g = _run(m, x, v, mode, t_end, eta, True)
    nb_s, s_s, st_s, e_s = _run(m, x, v, mode, t_end, eta, False)
    assert nb_g == nb_s and st_g["pairs"] == st_s["pairs"] and st_g["blocks"] == st_s["blocks"]
    for key in s_g:
        assert np.array_equal(s_g[key], s_s[key]), key
    assert e_g == e_s
    assert st_s["graph_blocks"] == 0
    assert st_g["graph_blocks"] > 0  # small blocks went through the graph
    print(f"\nn={n} {mode}: {nb_g} blocks, {st_g['graph_blocks']} as graph replays")
