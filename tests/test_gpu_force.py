"""Force kernel (Eq. Force, Appendix A pair term) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from synthetic import active_subset, kepler_pair, plummer_sphere
from tests.gpu_common import EPS2, REL, check_force, errors, gpu_force, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def _sim(m, x, v, eps2, mode, **kw):
    from paper_astro_ph_0702058_gb300 import Simulation
    return Simulation(m, x, v, eps2, mode=mode, **kw)


@pytest.mark.parametrize("mode", ["plain", "comp"])
@pytest.mark.parametrize("n", [1, 2, 3, 17, 255, 256, 257, 1000, 4099])
def test_force_small_sizes_all_rows(torch, mode, n):
    """Ragged sizes around the 256-particle tile, every row and several block sizes."""
    m, x, v = plummer_sphere(n, 40 + n)
    for n_act in sorted({1, max(1, n // 3), n}):
        act = active_subset(n, n_act, 7 + n_act)
        with _sim(m, x, v, EPS2, mode) as sim:
            sim.predict(0.0)
            acc, jerk, pot = gpu_force(sim, act)
        ra, rk, rp = oracle.force(m, x, v, EPS2, act)
        if n == 1:
            assert np.all(acc == 0) and np.all(jerk == 0) and np.all(pot == 0)
            continue
        check_force(mode, m, x, v, EPS2, act, (acc, jerk, pot), (ra, rk, rp), f"n={n} n_act={n_act}")


@pytest.mark.parametrize("mode", ["plain", "comp"])
@pytest.mark.parametrize("n_act", [1, 32, 1024, 1594, 32768, 65536])
def test_force_n65536_sweep_sampled(torch, mode, n_act):
    """The n_act sweep at N = 65536 (j-split for small blocks); up to 512 rows checked."""
    n = 65536
    m, x, v = plummer_sphere(n, 2)
    act = active_subset(n, n_act, 11)
    with _sim(m, x, v, EPS2, mode) as sim:
        sim.predict(0.0)
        acc, jerk, pot = gpu_force(sim, act)
        st = sim.stats()
    rows = np.linspace(0, n_act - 1, min(n_act, 512)).astype(int)
    ra, rk, rp = oracle.force(m, x, v, EPS2, act[rows])
    check_force(mode, m, x, v, EPS2, act[rows], (acc[rows], jerk[rows], pot[rows]), (ra, rk, rp), f"n_act={n_act}")
    if n_act <= 1024:
        assert st["last_j_split"] > 1  # small blocks spread j over the GPU


@pytest.mark.parametrize("mode", ["plain", "comp"])
@pytest.mark.parametrize("n,n_act,eps2", [(65536, 512, EPS2), (65536, 777, EPS2), (65536, 4096, EPS2),
                                          (65536, 8191, EPS2), (20001, 3000, EPS2), (16384, 1000, EPS2),
                                          (20001, 600, 0.0)])
def test_force_slice_shape(torch, mode, n, n_act, eps2):
    """Mid-size blocks of streams of 64 tiles or more take the slice shape: one CTA of 512 threads per SM,
    each over its slice of the stream (ragged at 20001, the last slices in the padding), j-split = SMs.
    Up to 1000 rows against the FP64 oracle, potential included (eps = 0: the pair j = i masked)."""
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    m, x, v = plummer_sphere(n, 5)
    act = active_subset(n, n_act, 13)
    with _sim(m, x, v, eps2, mode) as sim:
        sim.predict(0.0)
        acc, jerk, pot = gpu_force(sim, act)
        st = sim.stats()
    assert st["last_threads"] == 512 and st["last_j_split"] == n_sm, st
    rows = np.linspace(0, n_act - 1, min(n_act, 1000)).astype(int)
    ra, rk, rp = oracle.force(m, x, v, eps2, act[rows])
    assert np.all(np.isfinite(acc)) and np.all(np.isfinite(pot))
    check_force(mode, m, x, v, eps2, act[rows], (acc[rows], jerk[rows], pot[rows]), (ra, rk, rp),
                f"slice n={n} n_act={n_act} eps2={eps2}")


def test_force_slice_rejects_bad_index(torch):
    from paper_astro_ph_0702058_gb300 import NBodyError
    n = 20001
    m, x, v = plummer_sphere(n, 6)
    act = active_subset(n, 700, 2).copy()
    act[333] = n
    with _sim(m, x, v, EPS2, "comp") as sim:
        sim.predict(0.0)
        with pytest.raises(NBodyError) as e:
            gpu_force(sim, act)
        assert e.value.code == -1
        good = active_subset(n, 700, 3)
        acc, jerk, pot = gpu_force(sim, good)
        assert sim.stats()["last_threads"] == 512
    rows = np.arange(0, 700, 7)
    ra, rk, rp = oracle.force(m, x, v, EPS2, good[rows])
    check_force("comp", m, x, v, EPS2, good[rows], (acc[rows], jerk[rows], pot[rows]), (ra, rk, rp), "after a bad index")


def test_comp_more_accurate_than_plain(torch):
    """Compensated p99 error strictly below plain's at N = 65536 (acc, jerk, pot)."""
    n = 65536
    m, x, v = plummer_sphere(n, 2)
    act = active_subset(n, 2048, 5)
    ref = oracle.force(m, x, v, EPS2, act)
    p99 = {}
    for mode in ("plain", "comp"):
        with _sim(m, x, v, EPS2, mode) as sim:
            sim.predict(0.0)
            got = gpu_force(sim, act)
        e = errors(*got, *ref)
        p99[mode] = {k: np.percentile(e[k], 99) for k in ("acc", "jerk", "pot")}
    print("\np99 relative errors at N=65536:", p99)
    for k in ("acc", "jerk", "pot"):
        assert p99["comp"][k] < p99["plain"][k], (k, p99)


@pytest.mark.parametrize("mode", ["plain", "comp"])
def test_force_zero_softening(torch, mode):
    """eps = 0: the self pair is masked; two-body and a small cluster match the oracle."""
    m, x, v = kepler_pair(0.5)
    with _sim(m, x, v, 0.0, mode) as sim:
        sim.predict(0.0)
        acc, jerk, pot = gpu_force(sim, [0, 1])
    ra, rk, rp = oracle.force(m, x, v, 0.0)
    assert np.all(np.isfinite(acc)) and np.all(np.isfinite(pot))
    check_force(mode, m, x, v, 0.0, [0, 1], (acc, jerk, pot), (ra, rk, rp), "kepler")
    rs = np.random.default_rng(3)
    m = rs.uniform(0.5, 1.5, 300) / 300
    x = rs.normal(size=(300, 3))
    v = rs.normal(size=(300, 3))
    with _sim(m, x, v, 0.0, mode) as sim:
        sim.predict(0.0)
        got = gpu_force(sim, np.arange(300))
    check_force(mode, m, x, v, 0.0, np.arange(300), got, oracle.force(m, x, v, 0.0), "eps0 cluster")
    # a particle exactly at the origin, with padding entries in the last tile (300 -> 512)
    x = x.copy()
    x[0] = 0.0
    with _sim(m, x, v, 0.0, mode) as sim:
        sim.predict(0.0)
        got = gpu_force(sim, np.arange(300))
    assert np.all(np.isfinite(got[0])) and np.all(np.isfinite(got[2]))
    check_force(mode, m, x, v, 0.0, np.arange(300), got, oracle.force(m, x, v, 0.0), "particle at origin")


@pytest.mark.parametrize("mode", ["plain", "comp"])
def test_force_every_launch_shape(torch, mode):
    n = 3000
    m, x, v = plummer_sphere(n, 8)
    act = active_subset(n, 1111, 2)
    ref = oracle.force(m, x, v, EPS2, act)
    shapes = [(t, i) for t in (64, 128, 256) for i in (1, 2, 4)] + [(512, 1)]
    for threads, ipt in shapes:
        for split in (1, 3):
            with _sim(m, x, v, EPS2, mode, j_tile=threads, i_block=ipt, j_split=split) as sim:
                sim.predict(0.0)
                got = gpu_force(sim, act)
                st = sim.stats()
            assert (st["last_threads"], st["last_i_per_thread"], st["last_j_split"]) == (threads, ipt, split)
            check_force(mode, m, x, v, EPS2, act, got, ref, f"shape {threads}x{ipt} split {split}")
    # the j-subgroup shape (256 threads: 64 rows x 4 tile quarters), with its own split rule and fixed splits
    for split in (0, 1, 3, 12):
        with _sim(m, x, v, EPS2, mode, j_sub=4, j_split=split) as sim:
            sim.predict(0.0)
            got = gpu_force(sim, act)
            st = sim.stats()
        assert (st["last_threads"], st["last_j_sub"]) == (256, 4) and (split == 0 or st["last_j_split"] == split)
        check_force(mode, m, x, v, EPS2, act, got, ref, f"j-subgroups split {split}")


@pytest.mark.parametrize("mode", ["plain", "comp"])
def test_force_deterministic_and_split_consistent(torch, mode):
    n = 4099
    m, x, v = plummer_sphere(n, 9)
    act = active_subset(n, 300, 4)
    outs = []
    for split in (1, 2, 5, 1):
        with _sim(m, x, v, EPS2, mode, j_split=split) as sim:
            sim.predict(0.0)
            outs.append(gpu_force(sim, act))
    for a, b in zip(outs[0], outs[3]):
        assert np.array_equal(a, b)  # same shape twice: bitwise identical
    ref = oracle.force(m, x, v, EPS2, act)
    for o, split in zip(outs[:3], (1, 2, 5)):
        check_force(mode, m, x, v, EPS2, act, o, ref, f"split {split}")


def test_force_device_buffers_and_repeats(torch):
    """Device (torch) list and outputs give the host-path bits; repeated indices repeat rows."""
    n = 2000
    m, x, v = plummer_sphere(n, 12)
    act = np.array([5, 17, 5, 1999, 0, 17], dtype=np.int32)
    with _sim(m, x, v, EPS2, "comp") as sim:
        sim.predict(0.0)
        h = gpu_force(sim, act)
        da = torch.zeros((6, 3), dtype=torch.float64, device="cuda")
        dj = torch.zeros((6, 3), dtype=torch.float64, device="cuda")
        dp = torch.zeros(6, dtype=torch.float64, device="cuda")
        sim.force(torch.from_numpy(act).cuda(), acc=da, jerk=dj, pot=dp)
        sim.sync()
    assert np.array_equal(h[0], da.cpu().numpy()) and np.array_equal(h[1], dj.cpu().numpy())
    assert np.array_equal(h[2], dp.cpu().numpy())
    assert np.array_equal(h[0][0], h[0][2]) and np.array_equal(h[0][1], h[0][5])


def test_force_rejects_bad_index(torch):
    from paper_astro_ph_0702058_gb300 import NBodyError
    m, x, v = plummer_sphere(100, 1)
    with _sim(m, x, v, EPS2, "plain") as sim:
        sim.predict(0.0)
        with pytest.raises(NBodyError) as e:
            gpu_force(sim, [3, 100])
        assert e.value.code == -1
        # the context stays usable
        got = gpu_force(sim, [3, 4])
        check_force("plain", m, x, v, EPS2, [3, 4], got, oracle.force(m, x, v, EPS2, [3, 4]))


@pytest.mark.parametrize("mode", ["plain", "comp"])
def test_force_full_size_bench_launch(torch, mode):
    """N = 2^20, n_act = N in the launch shape the benchmark times: 4096 sampled rows against the
    oracle's full sums (the stated thresholds), every 32nd of them also within the per-row FP32
    bound."""
    n = 1 << 20
    m, x, v = plummer_sphere(n, 3)
    eps2 = 1e-6
    act = np.arange(n, dtype=np.int32)
    with _sim(m, x, v, eps2, mode) as sim:
        sim.predict(0.0)
        acc, jerk, pot = gpu_force(sim, act)
    rows = np.sort(np.random.default_rng(0).choice(n, 4096, replace=False)).astype(np.int32)
    ref = oracle.force(m, x, v, eps2, rows)
    from tests.gpu_common import FRAC_LARGE, check_threshold_fractions
    e_all = errors(acc[rows], jerk[rows], pot[rows], *ref)
    check_threshold_fractions(mode, e_all, "N=2^20", FRAC_LARGE)
    sub = np.arange(0, 4096, 32)
    check_force(mode, m, x, v, eps2, rows[sub], (acc[rows[sub]], jerk[rows[sub]], pot[rows[sub]]),
                tuple(r[sub] for r in ref), "N=2^20", min_rows=1 << 30)  # thresholds checked above
    print(f"\nN=2^20 {mode} (4096 rows): " + ", ".join(f"{k} max {v.max():.2e} p50 {np.median(v):.2e} "
                                          f"within {REL[mode]:.0e}: {np.mean(v <= REL[mode]):.3f}"
                                          for k, v in e_all.items()))
