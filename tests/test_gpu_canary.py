"""Output canaries: the force, state and j-stream calls write exactly their rows.

Device output buffers get extra rows filled with a NaN pattern; after a call the rows it
owns must be finite and the extra rows must still hold the pattern bit for bit (no write
past the end, e.g. from a launch sized for more rows than the block has).  Small sizes,
ragged tails and every launch shape and split kind."""
import numpy as np
import pytest

from synthetic import active_subset, plummer_sphere
from tests.gpu_common import EPS2, need_gpu

pytestmark = pytest.mark.gpu
EXTRA = 37


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def _canary(torch, rows, width):
    shape = (rows + EXTRA, width) if width > 1 else (rows + EXTRA,)
    return torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")


def _intact(torch, buf, rows):
    tail = buf[rows:]
    return bool(torch.isnan(tail).all()) and bool(torch.isfinite(buf[:rows]).all())


@pytest.mark.parametrize("mode", ["plain", "comp", "ds"])
@pytest.mark.parametrize("n,n_act,shape", [(1, 1, (0, 0, 0)), (17, 5, (0, 0, 0)), (257, 257, (64, 1, 2)),
                                           (3000, 1111, (128, 2, 3)), (3000, 99, (256, 4, 0)),
                                           (12000, 8192, (0, 0, 0)), (3000, 1000, (0, -4, 0)),
                                           (20000, 1003, (0, 0, 0))])
def test_force_writes_exactly_its_rows(torch, mode, n, n_act, shape):
    """(i_block -4 stands for the j-subgroup shape, j_sub = 4.)"""
    from paper_astro_ph_0702058_gb300 import Simulation
    m, x, v = plummer_sphere(n, 90 + n % 7)
    if shape[1] < 0:
        kw = {} if mode == "ds" else dict(j_sub=-shape[1], j_split=shape[2])
    else:
        kw = {} if mode == "ds" else dict(j_tile=shape[0], i_block=shape[1], j_split=shape[2])
    act = torch.from_numpy(active_subset(n, n_act, 4)).cuda()
    acc, jerk, pot = _canary(torch, n_act, 3), _canary(torch, n_act, 3), _canary(torch, n_act, 1)
    with Simulation(m, x, v, EPS2, mode=mode, **kw) as sim:
        sim.predict(0.0)
        sim.force(act, n_act, acc=acc, jerk=jerk, pot=pot)
        sim.sync()
    for buf in (acc, jerk, pot):
        assert _intact(torch, buf, n_act)


def test_state_and_jstream_write_exactly_n_rows(torch):
    from paper_astro_ph_0702058_gb300 import Simulation
    n = 1000
    m, x, v = plummer_sphere(n, 95)
    with Simulation(m, x, v, EPS2, mode="comp") as sim:
        sim.step(1.0 / 64)
        bufs = {k: _canary(torch, n, 3) for k in ("x", "v", "a", "k")}
        sim.get_state(**bufs)
        for buf in bufs.values():
            assert _intact(torch, buf, n)
        sim.predict(2.0 / 64)
        f = [torch.full((n + EXTRA, 4), float("nan"), dtype=torch.float32, device="cuda") for _ in range(3)]
        sim.get_predicted(*f)
        for buf in f:
            assert bool(torch.isnan(buf[n:]).all()) and bool(torch.isfinite(buf[:n]).all())
