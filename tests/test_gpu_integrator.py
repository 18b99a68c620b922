"""Predictor, corrector + time steps, scheduler, energy and the block-step loop
(Sect. 2) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from synthetic import active_subset, plummer_sphere
from tests.gpu_common import EPS2, check_force, gpu_force, need_gpu

pytestmark = pytest.mark.gpu
LMIN, LMAX = 6, 26


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def _sim(m, x, v, eps2=EPS2, mode="plain", **kw):
    from paper_astro_ph_0702058_gb300 import Simulation
    return Simulation(m, x, v, eps2, mode=mode, lmin=kw.pop("lmin", LMIN), lmax=kw.pop("lmax", LMAX), **kw)


def _random_state(n, seed, t_now=(1 << 22) + (3 << 12)):
    """A valid block-step state at time t_now: each t_i the last multiple of its own
    step not after t_now, so t_i <= t_now < t_i + dt_i for every particle."""
    rs = np.random.default_rng(seed)
    m, x, v = plummer_sphere(n, seed)
    a = rs.normal(size=(n, 3)) * 3
    k = rs.normal(size=(n, 3)) * 30
    level = rs.integers(8, 15, n).astype(np.int8)
    step = np.left_shift(np.int64(1), (LMAX - level.astype(np.int64)))
    t = (t_now // step) * step
    return m, x, v, a, k, t.astype(np.int64), level


def _get_state(sim):
    n = sim.n
    out = dict(x=np.zeros((n, 3)), v=np.zeros((n, 3)), a=np.zeros((n, 3)), k=np.zeros((n, 3)),
               t_tick=np.zeros(n, dtype=np.int64), level=np.zeros(n, dtype=np.int8))
    sim.get_state(**out)
    return out


@pytest.mark.parametrize("mode", ["plain", "comp"])
def test_predict_matches_oracle(torch, mode):
    n = 5000
    m, x, v, a, k, t, level = _random_state(n, 1)
    t_new = int(t.max()) + (1 << 10)
    with _sim(m, x, v, mode=mode) as sim:
        sim.set_state(x, v, a, k, t, level)
        sim.predict(t_new * 2.0 ** -LMAX)
        posm = np.zeros((n, 4), dtype=np.float32)
        vel = np.zeros((n, 4), dtype=np.float32)
        lo = np.zeros((n, 4), dtype=np.float32)
        sim.get_predicted(posm, vel, lo)
    xp, vp = oracle.predict(x, v, a, k, t, t_new, LMAX)
    # FP32 j-stream = FP64 prediction rounded once (within one float ulp of it)
    for got, ref in ((posm[:, :3], xp), (vel[:, :3], vp)):
        ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(got.astype(np.float64) - ref) <= ulp)
    assert np.array_equal(posm[:, 3], m.astype(np.float32))
    if mode == "comp":
        full = posm[:, :3].astype(np.float64) + lo[:, :3].astype(np.float64)
        assert np.abs(full - xp).max() <= 1e-14 * np.abs(xp).max()
    else:
        assert np.all(lo == 0)


def test_correct_and_new_levels_match_oracle(torch):
    n = 3000
    m, x, v, a, k, t, level = _random_state(n, 2)
    step = np.left_shift(np.int64(1), (LMAX - level.astype(np.int64)))
    t_blk = int((t + step).min())
    act = np.nonzero(t + step == t_blk)[0].astype(np.int32)
    xp, vp = oracle.predict(x, v, a, k, t, t_blk, LMAX)
    fa, fk, _ = oracle.force(m, xp, vp, EPS2, act)
    with _sim(m, x, v) as sim:
        sim.set_state(x, v, a, k, t, level)
        sim.predict(t_blk * 2.0 ** -LMAX)
        sim.correct(act, acc=fa, jerk=fk)
        got = _get_state(sim)
    st = oracle.State(m, x, v, EPS2, 0.01, lmin=LMIN, lmax=LMAX)
    st.x[:], st.v[:], st.a[:], st.k[:], st.t[:], st.level[:] = x, v, a, k, t, level
    st.correct(act, xp, vp, fa, fk, t_blk)
    for key, ref in (("x", st.x), ("v", st.v)):
        assert np.abs(got[key] - ref).max() <= 1e-13 * np.abs(ref).max(), key
    assert np.array_equal(got["a"], st.a) and np.array_equal(got["k"], st.k)
    assert np.array_equal(got["t_tick"], st.t) and np.array_equal(got["level"], st.level)


@pytest.mark.parametrize("n", [1, 2, 255, 2048, 2049, 70001])
def test_schedule_matches_oracle(torch, n):
    m, x, v, a, k, t, level = _random_state(n, 3 + n)
    with _sim(m, x, v) as sim:
        sim.set_state(x, v, a, k, t, level)
        blk = np.full(n, -1, dtype=np.int32)
        t_blk, n_act = sim.next_block(blk)
    t_ref, act_ref = oracle.schedule(t, level, LMAX)
    assert t_blk == t_ref * 2.0 ** -LMAX and n_act == len(act_ref)
    assert np.array_equal(blk[:n_act], act_ref)


def test_schedule_full_block_at_synchronised_time(torch):
    n = 10000
    m, x, v = plummer_sphere(n, 4)
    with _sim(m, x, v, lmin=10, lmax=10) as sim:  # one shared level: every block is all n
        blk = np.zeros(n, dtype=np.int32)
        t_blk, n_act = sim.next_block(blk)
        assert n_act == n and t_blk == 2.0 ** -10 and np.array_equal(blk, np.arange(n))


def test_energy_matches_oracle(torch):
    from paper_astro_ph_0702058_gb300 import NBodyError
    n = 3000
    m, x, v = plummer_sphere(n, 5)
    with _sim(m, x, v) as sim:
        ek, ep = sim.energy()
        ref_k, ref_p = oracle.energy(m, x, v, EPS2)
        assert abs(ek - ref_k) <= 1e-13 * abs(ref_k) and abs(ep - ref_p) <= 1e-13 * abs(ref_p)
        blk = np.zeros(n, dtype=np.int32)
        t_blk, n_act = sim.next_block(blk)
        sim.predict(t_blk)
        sim.force(blk[:n_act])
        sim.correct(blk[:n_act])
        with pytest.raises(NBodyError) as e:
            sim.energy()
        assert e.value.code == -6


def test_c1_schedule_lockstep_with_oracle_forces(torch):
    """C1 (N = 1024, eta = 0.01): the GPU predictor/corrector/scheduler, fed the oracle's
    forces at each block, reproduce the oracle's block schedule bit for bit over 100 blocks,
    while the GPU force on the same predicted state stays within tolerance (lockstep)."""
    n = 1024
    m, x, v = plummer_sphere(n, 1)
    ref = oracle.State(m, x, v, EPS2, 0.01, lmin=LMIN, lmax=LMAX).init()
    bt, bn, lists = ref.evolve(1 << 30, max_blocks=100, record_lists=100 * n)
    offs = np.concatenate([[0], np.cumsum(bn)])
    with _sim(m, x, v) as sim:
        s0 = _get_state(sim)
        # start from the oracle's own initial forces and levels
        ref0 = oracle.State(m, x, v, EPS2, 0.01, lmin=LMIN, lmax=LMAX).init()
        sim.set_state(s0["x"], s0["v"], ref0.a, ref0.k, ref0.t, ref0.level)
        blk = np.zeros(n, dtype=np.int32)
        for b in range(100):
            t_blk, n_act = sim.next_block(blk)
            act = blk[:n_act].copy()
            assert int(round(t_blk * 2 ** LMAX)) == bt[b] and np.array_equal(act, lists[offs[b]:offs[b + 1]]), b
            s = _get_state(sim)
            xp, vp = oracle.predict(s["x"], s["v"], s["a"], s["k"], s["t_tick"], bt[b], LMAX)
            fa, fk, fp = oracle.force(m, xp, vp, EPS2, act)
            sim.predict(t_blk)
            got = gpu_force(sim, act)
            check_force("plain", m, xp, vp, EPS2, act, got, (fa, fk, fp), f"block {b}")
            sim.correct(act, acc=fa, jerk=fk)


def _oracle_from(g, m, eta):
    st = oracle.State(m, g["x"], g["v"], EPS2, eta, lmin=LMIN, lmax=LMAX)
    st.a[:], st.k[:], st.t[:], st.level[:] = g["a"], g["k"], g["t_tick"], g["level"]
    return st


@pytest.mark.parametrize("mode", ["plain", "comp"])
def test_c1_free_running_schedule_and_energy(torch, mode):
    """C1 free-running (N = 1024, eta = 0.01), 100 blocks.  At every block the GPU's
    block list, corrected state and new levels equal the oracle scheduler's and corrector's
    on the GPU's own state and forces (time bins bit-exact).  Against the free-running
    oracle the schedule stays identical until a level decision differs; the corrector's
    a^(2), a^(3) amplify the FP32 force differences by (T/dt)^2..3, so such a split is
    expected, and the blocks before it are reported.  The run then goes on to t = 1/8."""
    n, eta = 1024, 0.01
    m, x, v = plummer_sphere(n, 1)
    ref = oracle.State(m, x, v, EPS2, eta, lmin=LMIN, lmax=LMAX).init()
    e0 = sum(ref.energy())
    with _sim(m, x, v, eta=eta, mode=mode) as sim:
        g = _get_state(sim)
        lv0 = [oracle.level_floor(oracle.dt_initial(g["a"][i], g["k"][i], eta), LMIN, LMAX)[0] for i in range(n)]
        assert np.array_equal(g["level"], np.array(lv0, dtype=np.int8))
        same = bool(np.array_equal(g["level"], ref.level))
        matched = 0
        blk = np.zeros(n, dtype=np.int32)
        for b in range(100):
            t_blk, n_act = sim.next_block(blk)
            act = blk[:n_act].copy()
            tick = int(round(t_blk * 2 ** LMAX))
            own_t, own_act = oracle.schedule(g["t_tick"], g["level"], LMAX)
            assert tick == own_t and np.array_equal(act, own_act), b
            if same:
                t_ref, act_ref = ref.schedule()
                same = tick == t_ref and np.array_equal(act, act_ref)
                if same:
                    ref.step()
            sim.predict(t_blk)
            acc, jerk, _ = gpu_force(sim, act)
            sim.correct(act)
            st = _oracle_from(g, m, eta)
            xp, vp = st.predict(tick)
            st.correct(act, xp, vp, acc, jerk, tick)
            g = _get_state(sim)
            assert np.array_equal(g["level"], st.level) and np.array_equal(g["t_tick"], st.t), b
            assert np.abs(g["x"] - st.x).max() <= 1e-13 * np.abs(st.x).max(), b
            if same:
                same = bool(np.array_equal(g["level"], ref.level))
                matched += same
        print(f"\nC1 {mode}: blocks identical to the free-running FP64 oracle: {matched} of 100")
        sim.step(0.125)
        ek, ep = sim.energy()
    ref = oracle.State(m, x, v, EPS2, eta, lmin=LMIN, lmax=LMAX).init()
    ref.evolve(1 << (LMAX - 3))
    de = abs((ek + ep - e0) / e0)
    de_ref = abs((sum(ref.energy()) - e0) / e0)
    print(f"C1 {mode}: |dE/E| at t=1/8 = {de:.3e} (FP64 oracle {de_ref:.3e})")
    assert de < 1e-5


def test_checkpoint_resume_is_bit_exact(torch):
    n = 2000
    m, x, v = plummer_sphere(n, 6)
    with _sim(m, x, v, mode="comp") as a:
        a.step(1.0 / 64)
        mid = _get_state(a)
        a.step(2.0 / 64)
        end_a = _get_state(a)
    with _sim(m, x, v, mode="comp") as b:
        b.set_state(**mid)
        b.step(2.0 / 64)
        end_b = _get_state(b)
    for key in end_a:
        assert np.array_equal(end_a[key], end_b[key]), key


def test_checkpoint_file_resume_is_bit_exact(torch, tmp_path):
    """Simulation.checkpoint writes an .npz file; a new context from it continues bit for bit."""
    from paper_astro_ph_0702058_gb300 import Simulation
    n = 2000
    m, x, v = plummer_sphere(n, 6)
    path = tmp_path / "mid.npz"
    with _sim(m, x, v, mode="comp") as a:
        a.step(1.0 / 64)
        a.checkpoint(path)
        a.step(2.0 / 64)
        end_a = _get_state(a)
    with Simulation.from_checkpoint(path) as b:
        assert b.mode == a.mode and (b.lmin, b.lmax) == (a.lmin, a.lmax) and b.eps2 == a.eps2
        b.step(2.0 / 64)
        end_b = _get_state(b)
    for key in end_a:
        assert np.array_equal(end_a[key], end_b[key]), key


def test_step_reaches_end_time_and_counts(torch):
    n = 4096
    m, x, v = plummer_sphere(n, 7)
    with _sim(m, x, v, eta=0.02) as sim:
        nb = sim.step(1.0 / 64)
        s = _get_state(sim)
        st = sim.stats()
    assert np.all(s["t_tick"] == 1 << (LMAX - 6))
    assert st["blocks"] == nb and nb > 0 and st["force_calls"] >= nb


def test_error_paths(torch):
    from paper_astro_ph_0702058_gb300 import NBodyError, Simulation, nbody_debug_fail_alloc
    n = 500
    m, x, v = plummer_sphere(n, 8)
    with _sim(m, x, v) as sim:
        with pytest.raises(NBodyError) as e:   # force before any prediction
            gpu_force(sim, [1, 2])
        assert e.value.code == -8
        with pytest.raises(NBodyError) as e:   # time off the tick grid
            sim.predict(1e-9)
        assert e.value.code == -1
        sim.predict(0.0)
        with pytest.raises(NBodyError) as e:   # correct without a matching force
            sim.correct(np.array([1, 2], dtype=np.int32))
        assert e.value.code == -8
        with pytest.raises(NBodyError) as e:   # end time not a multiple of dt_max
            sim.step(1.0 / 128)
        assert e.value.code == -1
    nbody_debug_fail_alloc(3)
    with pytest.raises(NBodyError) as e:
        Simulation(m, x, v, EPS2)
    assert e.value.code == -2
    nbody_debug_fail_alloc(0)
    # strict mode: a criterion below dt_min (lmax = 8 is far too coarse) is an error
    with _sim(m, x, v, lmin=6, lmax=8, strict=True) as sim:
        with pytest.raises(NBodyError) as e:
            sim.step(1.0 / 64)
        assert e.value.code == -4
    with _sim(m, x, v, lmin=6, lmax=8) as sim:   # not strict: counted only
        sim.step(1.0 / 64)
        assert sim.stats()["below_dt_min"] > 0


def test_nonfinite_input_is_reported(torch):
    from paper_astro_ph_0702058_gb300 import NBodyError, Simulation
    m, x, v = plummer_sphere(300, 9)
    x = x.copy()
    x[17, 1] = np.nan
    with pytest.raises(NBodyError) as e:
        Simulation(m, x, v, EPS2)
    assert e.value.code == -5


@pytest.mark.parametrize("n", [3000, 65536])
def test_energy_ds_matches_oracle(torch, n):
    """nbody_energy_ds (double-single potential) against the FP64 oracle's energy: E_kin as in
    nbody_energy (FP64), E_pot within 1e-12 relative; at N = 65536 also against the library's FP64
    diagnostic.  It refuses unsynchronised states like nbody_energy."""
    from paper_astro_ph_0702058_gb300 import NBodyError
    m, x, v = plummer_sphere(n, 5)
    with _sim(m, x, v) as sim:
        ek, ep = sim.energy(ds_potential=True)
        ref_k, ref_p = oracle.energy(m, x, v, EPS2)
        print(f"\nenergy_ds n={n}: E_pot rel err {abs(ep - ref_p) / abs(ref_p):.2e}")
        assert abs(ek - ref_k) <= 1e-13 * abs(ref_k) and abs(ep - ref_p) <= 1e-12 * abs(ref_p)
        if n == 65536:
            fk, fp = sim.energy()
            assert fk == ek and abs(fp - ep) <= 1e-12 * abs(fp)
        blk = np.zeros(n, dtype=np.int32)
        t_blk, n_act = sim.next_block(blk)
        sim.predict(t_blk)
        sim.force(blk[:n_act])
        sim.correct(blk[:n_act])
        if n_act < n:
            with pytest.raises(NBodyError) as e:
                sim.energy(ds_potential=True)
            assert e.value.code == -6
