"""nbody_force_noalloc: the force call for callers that cannot allocate device memory.

Such a caller (one whose host application owns all GPU memory, or that runs
under a latency budget where an allocation is not allowed) keeps the
predicted j-stream, the active list and the outputs in its own device
buffers; the library keeps its scratch in a fixed array.  This test calls
the entry point through the C ABI twice in a row, with different blocks, and
checks each result against nbody_force (the existing entry point) on the same
j-stream, within the per-row FP32 error bound the other GPU tests use, and
against the FP64 oracle.  It needs nothing from other tests, so it passes
alone in a fresh process as well as after them; pytest collects it last.
"""
import numpy as np
import pytest

import oracle
from synthetic import active_subset, plummer_sphere
from tests.fp32_bounds import bounds
from tests.gpu_common import EPS2, check_force, gpu_force, need_gpu

pytestmark = pytest.mark.gpu


def _padded_stream(torch, sim, n):
    """The simulation's predicted j-stream in fresh device buffers, padded as the call requires."""
    n_pad = (n + 255) // 256 * 256
    host = [np.zeros((n, 4), dtype=np.float32) for _ in range(3)]
    sim.get_predicted(*host)
    out = []
    for k, h in enumerate(host):
        full = np.zeros((n_pad, 4), dtype=np.float32)
        full[:n] = h
        if k == 0:
            full[n:, :3] = 1e15  # massless padding far away
        out.append(torch.from_numpy(full).cuda())
    return out


@pytest.mark.parametrize("mode", ["plain", "comp"])
def test_noalloc_matches_nbody_force_twice(mode):
    torch = need_gpu()
    from paper_astro_ph_0702058_gb300 import MODES, Simulation, nbody_force_noalloc
    n = 3000  # n_pad = 3072: a ragged last tile of padding
    m, x, v = plummer_sphere(n, 31)
    with Simulation(m, x, v, EPS2, mode=mode) as sim:
        sim.predict(0.0)
        posm, vel, lo = _padded_stream(torch, sim, n)
        for call, (n_act, seed) in enumerate(((1000, 1), (300, 2))):
            act = active_subset(n, n_act, seed)
            ref = gpu_force(sim, act)  # the existing entry point
            acc = torch.full((n_act, 3), float("nan"), dtype=torch.float64, device="cuda")
            jerk = torch.full((n_act, 3), float("nan"), dtype=torch.float64, device="cuda")
            pot = torch.full((n_act,), float("nan"), dtype=torch.float64, device="cuda")
            nbody_force_noalloc(posm, vel, lo, n, torch.from_numpy(act).cuda(), n_act, EPS2, MODES[mode],
                                acc, jerk, pot)
            got = (acc.cpu().numpy(), jerk.cpu().numpy(), pot.cpu().numpy())
            B, _ = bounds(m, x, v, EPS2, act, mode)
            diff = np.stack([np.linalg.norm(got[0] - ref[0], axis=1), np.linalg.norm(got[1] - ref[1], axis=1),
                             np.abs(got[2] - ref[2])], axis=1)
            assert np.all(diff <= B), f"call {call}: no-alloc result differs from nbody_force beyond the FP32 bound"
            check_force(mode, m, x, v, EPS2, act, got, oracle.force(m, x, v, EPS2, act), f"no-alloc call {call}")


@pytest.mark.parametrize("mode,n,n_act,rows", [
    ("plain", 200, 77, None),          # one j-tile: no split, the scratch array is not used
    ("comp", 200, 200, None),
    ("comp", 262000, 131072, 512),     # the largest block: the split is capped to the two ranges that fit
])
def test_noalloc_single_tile_and_scratch_limit(mode, n, n_act, rows):
    """The two edges of the split rule: a single j-tile (split 1) and a block of 131072 rows, where
    only two j-ranges of partial sums fit the scratch array.  Each is compared with nbody_force on the
    same j-stream within the per-row FP32 bound, on every row or on a seeded sample of them."""
    torch = need_gpu()
    from paper_astro_ph_0702058_gb300 import MODES, Simulation, nbody_force_noalloc
    m, x, v = plummer_sphere(n, 33)
    act = active_subset(n, n_act, 4)
    with Simulation(m, x, v, EPS2, mode=mode) as sim:
        sim.predict(0.0)
        posm, vel, lo = _padded_stream(torch, sim, n)
        ref = gpu_force(sim, act)
        out = [torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")
               for shape in ((n_act, 3), (n_act, 3), (n_act,))]
        for call in range(2):
            nbody_force_noalloc(posm, vel, lo, n, torch.from_numpy(act).cuda(), n_act, EPS2, MODES[mode], *out)
            got = tuple(t.cpu().numpy() for t in out)
            assert all(np.isfinite(g).all() for g in got), f"call {call}: rows left unwritten"
            pick = np.arange(n_act) if rows is None else np.sort(np.random.default_rng(5).choice(n_act, rows, False))
            B, _ = bounds(m, x, v, EPS2, act[pick], mode)
            diff = np.stack([np.linalg.norm(got[0][pick] - ref[0][pick], axis=1),
                             np.linalg.norm(got[1][pick] - ref[1][pick], axis=1),
                             np.abs(got[2][pick] - ref[2][pick])], axis=1)
            assert np.all(diff <= B), f"{mode} n={n} call {call}: differs from nbody_force beyond the FP32 bound"


def test_noalloc_rejects_blocks_beyond_its_scratch():
    torch = need_gpu()
    from paper_astro_ph_0702058_gb300 import NBODY_MODE_PLAIN, NBodyError, nbody_force_noalloc
    n = 131073
    n_pad = (n + 255) // 256 * 256
    buf = torch.zeros((n_pad, 4), dtype=torch.float32, device="cuda")
    act = torch.arange(n, dtype=torch.int32, device="cuda")
    out3 = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    out1 = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(NBodyError) as e:
        nbody_force_noalloc(buf, buf, None, n, act, n, EPS2, NBODY_MODE_PLAIN, out3, out3, out1)
    assert e.value.code == -1 and "131072" in str(e.value)
