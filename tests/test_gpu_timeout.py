"""Failure path of the bounded device-side waits, without a fault or a hang.

The test hook makes the force kernel leave out the copy of its first j-tile,
so the mbarrier wait for it never completes; after ~2 s the kernel records a
timeout and returns.  The call must report NBODY_ETIMEOUT and the context
must stay usable (the next call gives correct forces)."""
import time

import numpy as np
import pytest

import oracle
from synthetic import plummer_sphere
from tests.gpu_common import EPS2, check_force, gpu_force, need_gpu

pytestmark = pytest.mark.gpu


def test_tile_wait_times_out_and_context_survives():
    need_gpu()
    from paper_astro_ph_0702058_gb300 import NBodyError, Simulation, nbody_debug_skip_tile_copy
    n = 200  # one tile, one block: a single bounded wait runs out
    m, x, v = plummer_sphere(n, 1)
    with Simulation(m, x, v, EPS2) as sim:
        sim.predict(0.0)
        nbody_debug_skip_tile_copy(True)
        try:
            t0 = time.perf_counter()
            with pytest.raises(NBodyError) as e:
                gpu_force(sim, [7])
            waited = time.perf_counter() - t0
        finally:
            nbody_debug_skip_tile_copy(False)
        assert e.value.code == -7, e.value
        assert 1.0 < waited < 30.0
        got = gpu_force(sim, [7, 8])
        check_force("plain", m, x, v, EPS2, [7, 8], got, oracle.force(m, x, v, EPS2, [7, 8]))
        assert np.all(np.isfinite(got[0]))
