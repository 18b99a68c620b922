"""The debug build (-DNB_DEBUG): the library's device-side index checks on.

A failed check records an error word and skips the access; the host reports it as
NBODY_ECUDA ("debug build: a device-side index check failed at site ...").  Nothing traps.
This builds the library with the checks into a temporary directory and runs, in a fresh
process loading that build, force evaluations over launch shapes, modes and block sizes,
block runs through the device-side loop, the one-cluster and the whole-GPU block-step kernels
and separate launches, the ensemble and the no-alloc entry point; every call must succeed (no
check may fail)."""
import os
import subprocess
import sys

import pytest

from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np, torch
from paper_astro_ph_0702058_gb300 import (Ensemble, MODES, Simulation, nbody_debug_step_graphs,
                                          nbody_force_noalloc)
from synthetic import active_subset, ensemble_sizes, plummer_sphere
EPS2 = (1 / 256) ** 2
for mode in ("plain", "comp", "sumcheck", "ds", "sorted"):
    for n, n_act, shape in ((1, 1, (0, 0, 0)), (300, 300, (0, 0, 0)), (4099, 1111, (64, 1, 3)),
                            (4099, 777, (128, 2, 0)), (20000, 9000, (256, 4, 0)), (20000, 33, (0, 0, 0))):
        if mode == "sorted" and n > 4099:
            continue
        m, x, v = plummer_sphere(n, 3)
        kw = {} if mode in ("ds", "sorted") else dict(j_tile=shape[0], i_block=shape[1], j_split=shape[2])
        with Simulation(m, x, v, EPS2, mode=mode, **kw) as sim:
            sim.predict(0.0)
            act = active_subset(n, n_act, 1)
            out = (np.zeros((n_act, 3)), np.zeros((n_act, 3)), np.zeros(n_act))
            sim.force(act, acc=out[0], jerk=out[1], pot=out[2])
            assert np.isfinite(out[0]).all()
for level in (3, 2, 0):
    nbody_debug_step_graphs(level)
    for mode in ("plain", "comp", "ds"):
        m, x, v = plummer_sphere(1024, 1)
        with Simulation(m, x, v, EPS2, eta=0.01, mode=mode) as sim:
            sim.step(1.0 / 64)
            sim.energy(); sim.energy(ds_potential=True)
nbody_debug_step_graphs(3)
for n in (4099, 20000):  # the whole-GPU block-step kernel (4099: CTAs without particles)
    m, x, v = plummer_sphere(n, 2)
    for mode in ("plain", "comp"):
        with Simulation(m, x, v, EPS2, eta=0.02, mode=mode) as sim:
            sim.step(1.0 / 64)
            assert sim.stats()["grid_blocks"] > 0
sizes = ensemble_sizes(8, 4)
parts = [plummer_sphere(int(k), 40 + c) for c, k in enumerate(sizes)]
with Ensemble(sizes, *(np.concatenate([p[i] for p in parts]) for i in range(3)), EPS2, eta=0.02) as ens:
    ens.run(1.0 / 64)
n = 3000
m, x, v = plummer_sphere(n, 31)
with Simulation(m, x, v, EPS2, mode="comp") as sim:
    sim.predict(0.0)
    n_pad = (n + 255) // 256 * 256
    host = [np.zeros((n, 4), np.float32) for _ in range(3)]
    sim.get_predicted(*host)
    dev = []
    for k, h in enumerate(host):
        full = np.zeros((n_pad, 4), np.float32)
        full[:n] = h
        if k == 0:
            full[n:, :3] = 1e15
        dev.append(torch.from_numpy(full).cuda())
    act = torch.from_numpy(active_subset(n, 500, 2)).cuda()
    outs = [torch.zeros(s, dtype=torch.float64, device="cuda") for s in ((500, 3), (500, 3), (500,))]
    nbody_force_noalloc(dev[0], dev[1], dev[2], n, act, 500, EPS2, MODES["comp"], *outs)
print("debug build: all calls succeeded")
"""


def test_debug_build_index_checks_stay_silent(tmp_path):
    need_gpu()
    from paper_astro_ph_0702058_gb300 import build
    lib = build.build(extra=["-DNB_DEBUG"], out=str(tmp_path / "libnbody_debug.so"), build_dir=str(tmp_path / "obj"))
    env = dict(os.environ, NBODY_LIB=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "all calls succeeded" in r.stdout
