"""Batched ensembles of independent clusters (each with its own block schedule)."""
import numpy as np
import pytest

import oracle
from synthetic import plummer_sphere
from tests.fp32_bounds import bounds
from tests.gpu_common import EPS2, need_gpu

pytestmark = pytest.mark.gpu
SIZES = [256, 300, 1000, 513, 2048, 257]
T_END = 1.0 / 64


def _clusters(sizes, seed0=50):
    parts = [plummer_sphere(int(n), seed0 + c) for c, n in enumerate(sizes)]
    m = np.concatenate([p[0] for p in parts])
    x = np.concatenate([p[1] for p in parts])
    v = np.concatenate([p[2] for p in parts])
    return parts, m, x, v


def _state(obj, n):
    out = dict(x=np.zeros((n, 3)), v=np.zeros((n, 3)), a=np.zeros((n, 3)), k=np.zeros((n, 3)),
               t_tick=np.zeros(n, dtype=np.int64), level=np.zeros(n, dtype=np.int8))
    obj.get_state(**out)
    return out


@pytest.mark.parametrize("mode", ["plain", "comp"])
def test_ensemble_equals_single_systems_bit_for_bit(mode):
    """One j-range per cluster: every cluster of the batched, graph-replayed run ends with
    exactly the state (and the block count) of the same cluster run alone."""
    need_gpu()
    from paper_astro_ph_0702058_gb300 import Ensemble, Simulation
    parts, m, x, v = _clusters(SIZES)
    with Ensemble(SIZES, m, x, v, EPS2, eta=0.02, mode=mode, threads=64, i_block=1, tiles_per_range=64) as ens:
        steps = ens.run(T_END)
        got = _state(ens, len(m))
        st = ens.stats()
    assert steps == st["blocks"].max()
    off = np.concatenate([[0], np.cumsum(SIZES)])
    for c, (mc, xc, vc) in enumerate(parts):
        with Simulation(mc, xc, vc, EPS2, eta=0.02, mode=mode, j_split=1) as sim:
            nb = sim.step(T_END)
            ref = _state(sim, len(mc))
        assert nb == st["blocks"][c]
        for key in ref:
            assert np.array_equal(got[key][off[c]:off[c + 1]], ref[key]), (c, key)


def test_one_warp_shape_matches_the_oracle_forces():
    """The 32-thread shape: t = 0 forces within the per-row FP32 bound after a run-free init."""
    need_gpu()
    from paper_astro_ph_0702058_gb300 import Ensemble
    parts, m, x, v = _clusters(SIZES, 130)
    with Ensemble(SIZES, m, x, v, EPS2, mode="comp", threads=32, i_block=1, tiles_per_range=2) as ens:
        s = _state(ens, len(m))
        ens.run(T_END)
        end = _state(ens, len(m))
    off = np.concatenate([[0], np.cumsum(SIZES)])
    for c, (mc, xc, vc) in enumerate(parts):
        ra, rk, _ = oracle.force(mc, xc, vc, EPS2)
        B, _ = bounds(mc, xc, vc, EPS2, np.arange(len(mc)), "comp")
        assert np.all(np.linalg.norm(s["a"][off[c]:off[c + 1]] - ra, axis=1) <= B[:, 0]), c
        assert np.all(np.linalg.norm(s["k"][off[c]:off[c + 1]] - rk, axis=1) <= B[:, 1]), c
    assert np.all(end["t_tick"] == int(T_END * 2 ** 26))


def test_graph_run_equals_stepwise_run():
    need_gpu()
    from paper_astro_ph_0702058_gb300 import Ensemble
    _, m, x, v = _clusters(SIZES, 70)
    with Ensemble(SIZES, m, x, v, EPS2, mode="comp") as a, Ensemble(SIZES, m, x, v, EPS2, mode="comp") as b:
        for e in (a, b):
            e.set_shape(128, 2, 1)  # several j-ranges per cluster
        a.run(T_END, check_every=5)
        while b.step(T_END) > 0:
            pass
        sa, sb = _state(a, len(m)), _state(b, len(m))
        assert np.array_equal(a.stats()["blocks"], b.stats()["blocks"])
    for key in sa:
        assert np.array_equal(sa[key], sb[key]), key


@pytest.mark.parametrize("mode", ["plain", "comp"])
def test_initial_forces_and_energy_match_oracle(mode):
    """The t = 0 force of every cluster (split into j-ranges) against the FP64 oracle within the
    per-row FP32 bound, and the per-cluster energy against the oracle's."""
    need_gpu()
    from paper_astro_ph_0702058_gb300 import Ensemble
    parts, m, x, v = _clusters(SIZES, 90)
    with Ensemble(SIZES, m, x, v, EPS2, mode=mode) as ens:
        s = _state(ens, len(m))
        ek, ep = ens.energy()
    off = np.concatenate([[0], np.cumsum(SIZES)])
    for c, (mc, xc, vc) in enumerate(parts):
        ra, rk, _ = oracle.force(mc, xc, vc, EPS2)
        B, _ = bounds(mc, xc, vc, EPS2, np.arange(len(mc)), mode)
        ga, gk = s["a"][off[c]:off[c + 1]], s["k"][off[c]:off[c + 1]]
        assert np.all(np.linalg.norm(ga - ra, axis=1) <= B[:, 0]), c
        assert np.all(np.linalg.norm(gk - rk, axis=1) <= B[:, 1]), c
        rek, rep = oracle.energy(mc, xc, vc, EPS2)
        assert abs(ek[c] - rek) <= 1e-13 * abs(rek) and abs(ep[c] - rep) <= 1e-13 * abs(rep)


def test_tuner_picks_a_shape_and_keeps_the_state():
    need_gpu()
    from paper_astro_ph_0702058_gb300 import Ensemble
    _, m, x, v = _clusters(SIZES, 110)
    with Ensemble(SIZES, m, x, v, EPS2) as ens:
        before = _state(ens, len(m))
        threads, ipt, tpr, ms = ens.tune(T_END, steps=3)
        after = _state(ens, len(m))
        assert threads in (32, 64, 128) and ipt in (1, 2) and tpr >= 1 and ms > 0
        for key in before:
            assert np.array_equal(before[key], after[key]), key
        assert ens.stats()["blocks"].sum() == 0
        ens.run(T_END)
        end = _state(ens, len(m))
        ek, ep = ens.energy()
    assert np.all(end["t_tick"] == int(T_END * 2 ** 26))
    assert np.all(np.isfinite(ek + ep))


@pytest.mark.parametrize("mode", ["plain", "comp"])
def test_full_size_c4_sampled_clusters(mode):
    """C4 at full size (512 clusters, sizes from seed 4, 1,177,044 particles): the t = 0 forces and
    energies of 8 sampled clusters against the oracle, then a tuned, graph-replayed run to t = 1/64
    in which every cluster arrives and conserves energy to 1e-6."""
    need_gpu()
    from paper_astro_ph_0702058_gb300 import Ensemble
    from synthetic import ensemble_sizes
    sizes = ensemble_sizes(512, 4)
    assert int(sizes.sum()) == 1177044
    parts = [plummer_sphere(int(n), 4_000_000 + c) for c, n in enumerate(sizes)]
    m = np.concatenate([p[0] for p in parts])
    x = np.concatenate([p[1] for p in parts])
    v = np.concatenate([p[2] for p in parts])
    off = np.concatenate([[0], np.cumsum(sizes)])
    sample = np.linspace(0, 511, 8).astype(int)
    with Ensemble(sizes, m, x, v, EPS2, eta=0.02, mode=mode) as ens:
        s = _state(ens, len(m))
        ek0, ep0 = ens.energy()
        for c in sample:
            mc, xc, vc = parts[c]
            ra, rk, _ = oracle.force(mc, xc, vc, EPS2)
            B, _ = bounds(mc, xc, vc, EPS2, np.arange(len(mc)), mode)
            ga, gk = s["a"][off[c]:off[c + 1]], s["k"][off[c]:off[c + 1]]
            assert np.all(np.linalg.norm(ga - ra, axis=1) <= B[:, 0]), c
            assert np.all(np.linalg.norm(gk - rk, axis=1) <= B[:, 1]), c
            rek, rep = oracle.energy(mc, xc, vc, EPS2)
            assert abs(ek0[c] - rek) <= 1e-13 * abs(rek) and abs(ep0[c] - rep) <= 1e-13 * abs(rep)
        ens.tune(T_END, steps=3)
        ens.run(T_END)
        end = _state(ens, len(m))
        ek, ep = ens.energy()
    assert np.all(end["t_tick"] == int(T_END * 2 ** 26))
    de = np.abs((ek + ep - ek0 - ep0) / (ek0 + ep0))
    print(f"\nC4 {mode}: |dE/E| at t = 1/64 median {np.median(de):.2e} max {de.max():.2e}")
    assert de.max() < 1e-6
