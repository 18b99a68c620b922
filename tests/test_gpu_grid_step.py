"""nbody_step's whole-GPU block-step kernel (level 3 of nbody_debug_step_graphs, the default for plain
and compensated systems past the one-cluster kernel's sizes): schedule, predictor, force and corrector
of Sect. 2 repeated on the device by one cooperative launch of one CTA per SM, for blocks of up to
4095 rows; larger blocks end the launch and run through the separate kernels.

Its forces are the packed pair terms summed per CTA over the CTA's own particles, then across CTAs, so
it is checked against the FP64 oracle as the separate kernels are: block by block, the list is the
oracle scheduler's on the GPU's own state, the forces the corrector used are within the per-row FP32
bound of the oracle's at the oracle's prediction, and the corrected state and new levels are the
oracle corrector's given those forces."""
import numpy as np
import pytest

import oracle
from synthetic import plummer_sphere
from tests.gpu_common import EPS2, check_force, need_gpu

pytestmark = pytest.mark.gpu
LMIN, LMAX = 6, 26
GRID_ROWS = 4095


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def _sim(m, x, v, mode, eta=0.02, **kw):
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
# 4099: CTAs without particles (27 per CTA rounded up to 28 leaves the last ones empty) and a ragged
# last CTA; 20001: a ragged last CTA; 65536: C2
@pytest.mark.parametrize("n,blocks", [(4099, 30), (20001, 12), (65536, 8)])
def test_grid_blocks_against_the_oracle(torch, mode, n, blocks):
    """One block per call (max_steps = 1): list, forces, corrected state and levels per block; blocks
    of up to 4095 rows run in the grid kernel, larger ones through the separate kernels."""
    eta = 0.02
    m, x, v = plummer_sphere(n, 1 + n % 7)
    ran = 0
    with _sim(m, x, v, mode, eta) as sim:
        g = _state(sim)
        for b in range(blocks):
            tick, act = oracle.schedule(g["t_tick"], g["level"], LMAX)
            before = sim.stats()["grid_blocks"]
            assert sim.step(1.0, 1) == 1
            in_grid = sim.stats()["grid_blocks"] - before
            assert in_grid == (1 if len(act) <= GRID_ROWS else 0), (b, len(act))
            ran += in_grid
            g2 = _state(sim)
            moved = np.nonzero(g2["t_tick"] != g["t_tick"])[0]
            assert np.array_equal(moved, act) and np.all(g2["t_tick"][act] == tick), b
            st = _oracle_from(g, m, eta)
            xp, vp = st.predict(tick)
            ra, rk, rp = oracle.force(m, xp, vp, EPS2, act)
            acc, jerk = g2["a"][act], g2["k"][act]  # the corrector stores the block's forces as a, k
            # the grid kernel computes no potential: the oracle's stands in for it
            check_force(mode, m, xp, vp, EPS2, act, (acc, jerk, rp), (ra, rk, rp), f"n={n} block {b} ({len(act)} rows)")
            st.correct(act, xp, vp, acc, jerk, tick)
            assert np.array_equal(g2["level"], st.level) and np.array_equal(g2["t_tick"], st.t), b
            assert np.abs(g2["x"] - st.x).max() <= 1e-13 * np.abs(st.x).max(), b
            assert np.abs(g2["v"] - st.v).max() <= 1e-13 * np.abs(st.v).max(), b
            g = g2
    assert ran > 0, "no block ran in the grid kernel"


@pytest.mark.parametrize("mode,eps2", [("plain", 0.0), ("comp", 0.0), ("comp", 1e-14)])
def test_grid_blocks_unsoftened_against_the_oracle(torch, mode, eps2):
    """eps = 0 (and eps^2 below 1e-12): the grid kernel masks the pair j = i (with a softening it adds exact
    zeros and is not masked).  One block per call against the FP64 oracle: list, forces within the per-row
    FP32 bound, corrected state and levels."""
    from paper_astro_ph_0702058_gb300 import Simulation
    n, eta = 6000, 0.02
    m, x, v = plummer_sphere(n, 9)
    with Simulation(m, x, v, eps2, eta=eta, lmin=LMIN, lmax=LMAX, mode=mode) as sim:
        g = _state(sim)
        for b in range(6):
            tick, act = oracle.schedule(g["t_tick"], g["level"], LMAX)
            before = sim.stats()["grid_blocks"]
            assert sim.step(1.0, 1) == 1
            assert sim.stats()["grid_blocks"] == before + (1 if len(act) <= GRID_ROWS else 0), b
            g2 = _state(sim)
            st = oracle.State(m, g["x"], g["v"], eps2, eta, lmin=LMIN, lmax=LMAX)
            st.a[:], st.k[:], st.t[:], st.level[:] = g["a"], g["k"], g["t_tick"], g["level"]
            xp, vp = st.predict(tick)
            ra, rk, rp = oracle.force(m, xp, vp, eps2, act)
            acc, jerk = g2["a"][act], g2["k"][act]
            assert np.all(np.isfinite(acc)) and np.all(np.isfinite(jerk)), b
            check_force(mode, m, xp, vp, eps2, act, (acc, jerk, rp), (ra, rk, rp), f"eps2={eps2} block {b}")
            st.correct(act, xp, vp, acc, jerk, tick)
            assert np.array_equal(g2["level"], st.level) and np.array_equal(g2["t_tick"], st.t), b
            g = g2
        assert sim.stats()["grid_blocks"] > 0


@pytest.mark.parametrize("mode", ["plain", "comp"])
def test_grid_run_is_independent_of_launch_budget(torch, mode):
    """One launch per run of small blocks, or launches of at most 5 blocks: the same bits (the
    summation order depends on the block size and the CTA count only)."""
    m, x, v = plummer_sphere(8192, 4)
    with _sim(m, x, v, mode) as a:
        nb_a = a.step(1.0 / 32)
        sa, st_a = _state(a), a.stats()
    with _sim(m, x, v, mode) as b:
        nb_b = 0
        while True:
            k = b.step(1.0 / 32, 5)
            nb_b += k
            if k < 5:
                break
        sb, st_b = _state(b), b.stats()
    assert nb_a == nb_b and st_a["grid_blocks"] == st_b["grid_blocks"] > 0
    assert st_a["pairs"] == st_b["pairs"] and st_a["blocks"] == st_b["blocks"]
    for key in sa:
        assert np.array_equal(sa[key], sb[key]), key


@pytest.mark.parametrize("mode", ["plain", "comp"])
def test_grid_c2_energy_and_block_count(torch, mode):
    """C2 (N = 65536, eta = 0.02) to t = 1/16: the grid kernel conserves energy as the separate kernels
    (level 2) do and runs a block count within a few percent of theirs."""
    from paper_astro_ph_0702058_gb300 import nbody_debug_step_graphs
    m, x, v = plummer_sphere(65536, 2)
    res = {}
    for level in (3, 2):
        nbody_debug_step_graphs(level)
        try:
            from paper_astro_ph_0702058_gb300 import Simulation
            with Simulation(m, x, v, (1.0 / 256) ** 2, eta=0.02, lmin=LMIN, lmax=LMAX, mode=mode) as sim:
                e0 = sum(sim.energy())
                nb = sim.step(1.0 / 16)
                e1 = sum(sim.energy())
                res[level] = (nb, abs((e1 - e0) / e0), sim.stats())
        finally:
            nbody_debug_step_graphs(3)
    (nb3, de3, st3), (nb2, de2, st2) = res[3], res[2]
    print(f"\nC2 {mode} to 1/16: grid {nb3} blocks ({st3['grid_blocks']} in the grid kernel) |dE/E| {de3:.3e}; "
          f"level 2 {nb2} blocks |dE/E| {de2:.3e}")
    assert st3["grid_blocks"] > 0.5 * nb3 and st2["grid_blocks"] == 0
    assert abs(nb3 - nb2) <= 0.05 * nb2
    assert de3 < 10 * de2 + 1e-9


def test_grid_stops_at_the_strict_error_block(torch):
    """Strict mode: the grid loop stops after the block whose criterion fell below dt_min, as the
    separate launches do, and the call fails there."""
    from paper_astro_ph_0702058_gb300 import NBodyError, nbody_debug_step_graphs
    m, x, v = plummer_sphere(5000, 8)
    res = {}
    for level in (3, 0):
        nbody_debug_step_graphs(level)
        try:
            # lmax = 10 is too coarse for the centre; the first block (t = 2^-10) holds 1113 rows
            with _sim(m, x, v, "plain", 0.01, lmin=6, lmax=10, strict=True) as sim:
                with pytest.raises(NBodyError) as e:
                    sim.step(1.0 / 64)
                assert e.value.code == -4
                res[level] = sim.stats()
        finally:
            nbody_debug_step_graphs(3)
    assert res[3]["blocks"] == res[0]["blocks"] and res[3]["grid_blocks"] == res[3]["blocks"]
    assert (res[3]["below_dt_min"] > 0) == (res[0]["below_dt_min"] > 0)


@pytest.mark.parametrize("n,mode,kw", [(5000, "comp", {"j_split": 1}), (5000, "plain", {"j_sub": 1}),
                                       (5000, "ds", {}), (5000, "sorted", {}), (5000, "sumcheck", {}),
                                       (1024, "comp", {}), (600000, "plain", {})])
def test_grid_kernel_not_taken_outside_its_scope(torch, n, mode, kw):
    """A fixed force shape, the double-single, sorted and summation-check modes, systems the cluster
    kernel takes, or more than 3584 particles per SM: not the grid kernel."""
    m, x, v = plummer_sphere(n, 2)
    with _sim(m, x, v, mode, 0.02, **kw) as sim:
        nb = sim.step(1.0 / 64, 3)
        st = sim.stats()
    assert nb > 0 and st["grid_blocks"] == 0


def test_grid_barrier_times_out_and_context_survives(torch):
    """The test hook makes the grid kernel's last CTA leave before its first barrier, so the other CTAs'
    bounded wait gives up after ~1 s: the call reports NBODY_ETIMEOUT without a fault or a hang, no block
    has run, and the next call continues as if the failed one had not happened."""
    import time
    from paper_astro_ph_0702058_gb300 import NBodyError, nbody_debug_skip_tile_copy
    m, x, v = plummer_sphere(8192, 4)
    with _sim(m, x, v, "comp") as ref:
        nb_ref = ref.step(1.0 / 64)
        s_ref = _state(ref)
    with _sim(m, x, v, "comp") as sim:
        nbody_debug_skip_tile_copy(True)
        try:
            t0 = time.perf_counter()
            with pytest.raises(NBodyError) as e:
                sim.step(1.0 / 64)
            waited = time.perf_counter() - t0
        finally:
            nbody_debug_skip_tile_copy(False)
        assert e.value.code == -7, e.value
        assert 0.5 < waited < 30.0
        assert sim.stats()["blocks"] == 0
        nb = sim.step(1.0 / 64)
        s = _state(sim)
        assert nb == nb_ref and sim.stats()["grid_blocks"] > 0
    for key in s:
        assert np.array_equal(s[key], s_ref[key]), key
