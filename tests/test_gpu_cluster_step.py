"""nbody_step's one-cluster block-step kernel (level 3 of nbody_debug_step_graphs, the default for
plain and compensated systems of n_pad <= 4096): schedule, predictor, force and corrector of
Sect. 2 repeated on the device by the CTAs of one thread-block cluster.

Its forces are the packed pair terms of the force kernel summed in another order, so it is
checked against the FP64 oracle as the separate kernels are: block by block, the block list
is the oracle scheduler's on the GPU's own state, the forces the corrector used are within the
per-row FP32 bound of the oracle's at the oracle's prediction, and the corrected state and new
levels are the oracle corrector's given those forces."""
import numpy as np
import pytest

import oracle
from synthetic import plummer_sphere
from tests.gpu_common import EPS2, check_force, need_gpu

pytestmark = pytest.mark.gpu
LMIN, LMAX = 6, 26


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def _sim(m, x, v, mode, eta=0.01, **kw):
    from paper_astro_ph_0702058_gb300 import Simulation
    return Simulation(m, x, v, EPS2, eta=eta, lmin=kw.pop("lmin", LMIN), lmax=kw.pop("lmax", LMAX), mode=mode, **kw)


def _state(sim):
    n = sim.n
    out = dict(x=np.zeros((n, 3)), v=np.zeros((n, 3)), a=np.zeros((n, 3)), k=np.zeros((n, 3)),
               t_tick=np.zeros(n, dtype=np.int64), level=np.zeros(n, dtype=np.int8))
    sim.get_state(**out)
    return out


def _oracle_from(g, m, eta):
    st = oracle.State(m, g["x"], g["v"], EPS2, eta, lmin=LMIN, lmax=LMAX)
    st.a[:], st.k[:], st.t[:], st.level[:] = g["a"], g["k"], g["t_tick"], g["level"]
    return st


@pytest.mark.parametrize("mode", ["plain", "comp"])
@pytest.mark.parametrize("n,blocks", [(1024, 60), (1000, 25), (4096, 12), (1, 3)])
def test_cluster_blocks_against_the_oracle(torch, mode, n, blocks):
    """One block per call (max_steps = 1): list, forces, corrected state and levels per block."""
    eta = 0.01
    m, x, v = plummer_sphere(n, 1 + n % 7)
    with _sim(m, x, v, mode, eta) as sim:
        g = _state(sim)
        for b in range(blocks):
            tick, act = oracle.schedule(g["t_tick"], g["level"], LMAX)
            before = sim.stats()["cluster_blocks"]
            assert sim.step(1.0, 1) == 1
            assert sim.stats()["cluster_blocks"] == before + 1, "the block did not run in the cluster kernel"
            g2 = _state(sim)
            moved = np.nonzero(g2["t_tick"] != g["t_tick"])[0]
            assert np.array_equal(moved, act) and np.all(g2["t_tick"][act] == tick), b
            st = _oracle_from(g, m, eta)
            xp, vp = st.predict(tick)
            ra, rk, rp = oracle.force(m, xp, vp, EPS2, act)
            acc, jerk = g2["a"][act], g2["k"][act]  # the corrector stores the block's forces as a, k
            if n == 1:  # no pair: exactly zero
                assert not acc.any() and not jerk.any() and not ra.any() and not rk.any()
            else:  # the cluster kernel computes no potential: the oracle's stands in for it
                check_force(mode, m, xp, vp, EPS2, act, (acc, jerk, rp), (ra, rk, rp), f"block {b}")
            st.correct(act, xp, vp, acc, jerk, tick)
            assert np.array_equal(g2["level"], st.level) and np.array_equal(g2["t_tick"], st.t), b
            scale = max(np.abs(st.x).max(), 1e-300)
            assert np.abs(g2["x"] - st.x).max() <= 1e-13 * scale, b
            assert np.abs(g2["v"] - st.v).max() <= 1e-13 * max(np.abs(st.v).max(), 1e-300), b
            g = g2


@pytest.mark.parametrize("mode", ["plain", "comp"])
def test_cluster_run_is_independent_of_launch_budget(torch, mode):
    """One launch for the whole run, or launches of at most 7 blocks: the same bits."""
    m, x, v = plummer_sphere(1024, 1)
    with _sim(m, x, v, mode) as a:
        nb_a = a.step(1.0 / 16)
        sa, st_a = _state(a), a.stats()
    with _sim(m, x, v, mode) as b:
        nb_b = 0
        while True:
            k = b.step(1.0 / 16, 7)
            nb_b += k
            if k < 7:
                break
        sb, st_b = _state(b), b.stats()
    assert nb_a == nb_b and st_a["cluster_blocks"] == nb_a and st_b["cluster_blocks"] == nb_b
    assert st_a["pairs"] == st_b["pairs"] and st_a["blocks"] == st_b["blocks"]
    for key in sa:
        assert np.array_equal(sa[key], sb[key]), key


@pytest.mark.parametrize("mode", ["plain", "comp"])
def test_cluster_c1_energy_and_block_count(torch, mode):
    """C1 to t = 1/8: the cluster kernel conserves energy as the separate kernels do and runs a
    block count within a few percent of theirs (level decisions near a boundary may differ)."""
    from paper_astro_ph_0702058_gb300 import nbody_debug_step_graphs
    m, x, v = plummer_sphere(1024, 1)
    res = {}
    for level in (3, 0):
        nbody_debug_step_graphs(level)
        try:
            with _sim(m, x, v, mode) as sim:
                e0 = sum(sim.energy())
                nb = sim.step(0.125)
                e1 = sum(sim.energy())
                res[level] = (nb, abs((e1 - e0) / e0), sim.stats())
        finally:
            nbody_debug_step_graphs(3)
    (nb3, de3, st3), (nb0, de0, st0) = res[3], res[0]
    print(f"\nC1 {mode}: cluster {nb3} blocks |dE/E| {de3:.3e}; separate kernels {nb0} blocks |dE/E| {de0:.3e}")
    assert st3["cluster_blocks"] == nb3 and st0["cluster_blocks"] == 0
    assert abs(nb3 - nb0) <= 0.05 * nb0
    assert de3 < 1e-5 and de3 < 10 * de0 + 1e-9


def test_cluster_stops_at_the_strict_error_block(torch):
    """Strict mode: the cluster loop stops after the block whose criterion fell below dt_min, as the
    separate launches do, and the call fails there."""
    from paper_astro_ph_0702058_gb300 import NBodyError, nbody_debug_step_graphs
    m, x, v = plummer_sphere(500, 8)
    res = {}
    for level in (3, 0):
        nbody_debug_step_graphs(level)
        try:
            with _sim(m, x, v, "plain", 0.01, lmin=6, lmax=8, strict=True) as sim:  # lmax = 8 is far too coarse
                with pytest.raises(NBodyError) as e:
                    sim.step(1.0 / 64)
                assert e.value.code == -4
                res[level] = sim.stats()
        finally:
            nbody_debug_step_graphs(3)
    assert res[3]["blocks"] == res[0]["blocks"] and res[3]["cluster_blocks"] == res[3]["blocks"]
    assert (res[3]["below_dt_min"] > 0) == (res[0]["below_dt_min"] > 0)


@pytest.mark.parametrize("n,mode,kw", [(4097, "comp", {}), (1024, "comp", {"j_split": 1}),
                                       (1024, "plain", {"j_tile": 64}), (2049, "ds", {}),
                                       (1024, "sorted", {}), (1024, "sumcheck", {})])
def test_cluster_kernel_not_taken_outside_its_scope(torch, n, mode, kw):
    """n_pad > 4096 (2048 double-single), a fixed force shape, or the sorted and summation-check modes:
    the tiled kernels."""
    m, x, v = plummer_sphere(n, 2)
    with _sim(m, x, v, mode, 0.02, **kw) as sim:
        nb = sim.step(1.0 / 64)
        st = sim.stats()
    assert nb > 0 and st["cluster_blocks"] == 0


@pytest.mark.parametrize("n,blocks", [(1024, 40), (1000, 15), (2048, 8)])
def test_cluster_ds_blocks_against_the_oracle(torch, n, blocks):
    """Double-single mode in the cluster kernel, one block per call: the list is the oracle scheduler's,
    the forces the corrector used within 1e-10 of the oracle's (reading gamma), the corrected state and
    levels the oracle corrector's given those forces."""
    eta = 0.01
    m, x, v = plummer_sphere(n, 3 + n % 5)
    with _sim(m, x, v, "ds", eta) as sim:
        g = _state(sim)
        for b in range(blocks):
            tick, act = oracle.schedule(g["t_tick"], g["level"], LMAX)
            assert sim.step(1.0, 1) == 1 and sim.stats()["cluster_blocks"] == b + 1
            g2 = _state(sim)
            st = _oracle_from(g, m, eta)
            xp, vp = st.predict(tick)
            ra, rk, _ = oracle.force(m, xp, vp, EPS2, act)
            acc, jerk = g2["a"][act], g2["k"][act]
            for got, ref in ((acc, ra), (jerk, rk)):
                r = np.linalg.norm(ref, axis=1)
                rel = np.linalg.norm(got - ref, axis=1) / np.maximum(r, 1e-3 * np.sqrt(np.mean(r ** 2)))
                assert rel.max() <= 1e-10, (b, rel.max())
            st.correct(act, xp, vp, acc, jerk, tick)
            assert np.array_equal(g2["level"], st.level) and np.array_equal(g2["t_tick"], st.t), b
            assert np.abs(g2["x"] - st.x).max() <= 1e-13 * np.abs(st.x).max(), b
            g = g2


def test_cluster_ds_free_run_follows_the_oracle_100_blocks(torch):
    """C1 (N = 1024, eta = 0.01): the double-single cluster kernel, run free one block per call, and the
    free-running FP64 oracle take the same first 100 block steps: block times, lists and every particle's
    new time and level (the integer time bins)."""
    n, eta = 1024, 0.01
    m, x, v = plummer_sphere(n, 1)
    ref = oracle.State(m, x, v, EPS2, eta, lmin=LMIN, lmax=LMAX).init()
    with _sim(m, x, v, "ds", eta) as sim:
        g = _state(sim)
        assert np.array_equal(g["level"], ref.level)
        for b in range(100):
            t_ref, act_ref, _, _, _, _ = ref.step()
            assert sim.step(1.0, 1) == 1
            g2 = _state(sim)
            moved = np.nonzero(g2["t_tick"] != g["t_tick"])[0]
            assert np.array_equal(moved, act_ref) and np.all(g2["t_tick"][moved] == t_ref), f"block {b}: lists"
            assert np.array_equal(g2["level"], ref.level) and np.array_equal(g2["t_tick"], ref.t), f"block {b}: levels"
            g = g2
        assert sim.stats()["cluster_blocks"] == 100


@pytest.mark.parametrize("mode", ["plain", "comp", "ds"])
def test_cluster_kepler_orbit_unsoftened(torch, mode):
    """Two bodies on an e = 0.5 Kepler ellipse with eps = 0 (the self-term mask and the massless padding),
    one period (t = 402/64 against 2 pi) through the cluster kernel: the same blocks as the FP64 oracle,
    energy conserved to its level, and the final separation within the FP32 force noise of the oracle's."""
    from paper_astro_ph_0702058_gb300 import Simulation
    from synthetic import kepler_pair
    m, x, v = kepler_pair(0.5)
    t_end = 402 / 64
    with Simulation(m, x, v, 0.0, eta=0.01, lmin=LMIN, lmax=LMAX, mode=mode) as sim:
        e0 = sum(sim.energy())
        nb = sim.step(t_end)
        g = _state(sim)
        e1 = sum(sim.energy())
        st = sim.stats()
    ref = oracle.State(m, x, v, 0.0, 0.01, lmin=LMIN, lmax=LMAX).init()
    bt, _, _ = ref.evolve(int(t_end * 2 ** LMAX))
    de, de_ref = abs(e1 / e0 - 1), abs(sum(ref.energy()) / e0 - 1)
    sep, sep_ref = np.linalg.norm(g["x"][1] - g["x"][0]), np.linalg.norm(ref.x[1] - ref.x[0])
    print(f"\n{mode}: blocks {nb} (oracle {len(bt)}), |dE/E| {de:.3e} (oracle {de_ref:.3e}), "
          f"separation {sep:.12f} (oracle {sep_ref:.12f})")
    assert st["cluster_blocks"] == nb and abs(nb - len(bt)) <= 2
    assert abs(e0 + 0.125) < 1e-12 and de < 2 * de_ref + (1e-6 if mode == "plain" else 1e-8)
    assert abs(sep - sep_ref) < (1e-4 if mode == "plain" else 1e-6)
