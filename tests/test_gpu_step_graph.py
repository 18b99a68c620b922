"""nbody_step's small-block CUDA graph, one block per replay or a device-side loop of blocks per
replay: the same bits as separate launches, and both are used."""
import numpy as np
import pytest

from synthetic import plummer_sphere
from tests.gpu_common import EPS2, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def _run(m, x, v, mode, t_end, eta, graphs, max_steps=0):
    from paper_astro_ph_0702058_gb300 import Simulation, nbody_debug_step_graphs
    nbody_debug_step_graphs(graphs)
    try:
        with Simulation(m, x, v, EPS2, eta=eta, lmin=6, lmax=26, mode=mode) as sim:
            nb = sim.step(t_end, max_steps)
            n = len(m)
            out = dict(x=np.zeros((n, 3)), v=np.zeros((n, 3)), a=np.zeros((n, 3)), k=np.zeros((n, 3)),
                       t_tick=np.zeros(n, dtype=np.int64), level=np.zeros(n, dtype=np.int8))
            sim.get_state(**out)
            st = sim.stats()
            e = sum(sim.energy()) if max_steps == 0 else None  # energy needs synchronised particles
    finally:
        nbody_debug_step_graphs(3)
    return nb, out, st, e


@pytest.mark.parametrize("mode", ["plain", "comp"])
# (1024, 1.0, 0.01) runs ~5000 blocks: replays of the device loop end at its cap (1 + 1024 blocks)
@pytest.mark.parametrize("n,t_end,eta", [(1024, 0.125, 0.01), (1024, 1.0, 0.01), (4099, 1.0 / 64, 0.02),
                                         (65536, 1.0 / 64, 0.02)])
def test_graph_blocks_equal_separate_launches(torch, mode, n, t_end, eta):
    m, x, v = plummer_sphere(n, 70 + n % 13)
    nb_s, s_s, st_s, e_s = _run(m, x, v, mode, t_end, eta, 0)
    assert st_s["graph_blocks"] == 0 and st_s["loop_blocks"] == 0
    for level in (1, 2):
        nb_g, s_g, st_g, e_g = _run(m, x, v, mode, t_end, eta, level)
        assert nb_g == nb_s and st_g["pairs"] == st_s["pairs"] and st_g["blocks"] == st_s["blocks"], level
        for key in s_g:
            assert np.array_equal(s_g[key], s_s[key]), (level, key)
        assert e_g == e_s, level
        assert st_g["graph_blocks"] > 0  # small blocks went through the graph
        if level == 1:
            assert st_g["loop_blocks"] == 0
        else:  # most graph blocks ran without a host round trip
            assert st_g["loop_blocks"] > 0
        print(f"\nn={n} {mode} level {level}: {nb_g} blocks, {st_g['graph_blocks']} in graph replays, "
              f"{st_g['loop_blocks']} added by the device loop")


@pytest.mark.parametrize("max_steps", [1, 7, 300])
def test_device_loop_honours_max_steps(torch, max_steps):
    """The device loop stops after exactly max_steps blocks, as the host loop does."""
    m, x, v = plummer_sphere(1024, 5)
    nb_s, s_s, st_s, _ = _run(m, x, v, "plain", 0.125, 0.01, 0, max_steps)
    nb_g, s_g, st_g, _ = _run(m, x, v, "plain", 0.125, 0.01, 2, max_steps)
    assert nb_s == nb_g == max_steps and st_g["blocks"] == max_steps
    for key in s_g:
        assert np.array_equal(s_g[key], s_s[key]), key


def test_device_loop_stops_at_the_strict_error_block(torch):
    """Strict mode: the device loop stops after the block whose criterion fell below dt_min, and the
    call fails there with the state the host loop leaves."""
    from paper_astro_ph_0702058_gb300 import NBodyError, Simulation, nbody_debug_step_graphs
    m, x, v = plummer_sphere(500, 8)
    n = len(m)
    res = {}
    for level in (0, 2):
        nbody_debug_step_graphs(level)
        try:
            with Simulation(m, x, v, EPS2, lmin=6, lmax=8, strict=True) as sim:  # lmax = 8 is far too coarse
                with pytest.raises(NBodyError) as e:
                    sim.step(1.0 / 64)
                assert e.value.code == -4
                out = dict(x=np.zeros((n, 3)), v=np.zeros((n, 3)), a=np.zeros((n, 3)), k=np.zeros((n, 3)),
                           t_tick=np.zeros(n, dtype=np.int64), level=np.zeros(n, dtype=np.int8))
                sim.get_state(**out)
                res[level] = (sim.stats(), out)
        finally:
            nbody_debug_step_graphs(3)
    (st0, s0), (st2, s2) = res[0], res[2]
    assert st0["blocks"] == st2["blocks"] and st0["below_dt_min"] == st2["below_dt_min"]
    assert st0["graph_blocks"] == 0 and st2["graph_blocks"] == st2["blocks"]
    for key in s0:
        assert np.array_equal(s0[key], s2[key]), key
