"""GB300 (sm_103a) direct N-body force evaluation for the 4th-order Hermite
block-time-step integrator of Portegies Zwart, Belleman & Geldof (2007).

The work is done by ``libnbody.so`` (CUDA kernels behind the C ABI of
``include/nbody.h``).  ``_lib`` mirrors the C calls one to one; ``Simulation``
below only owns a context handle and forwards to them.  PyTorch is used only
by callers, for device memory and streams.
"""
from __future__ import annotations

from . import _lib
from ._lib import (NBODY_MODE_COMP, NBODY_MODE_DS, NBODY_MODE_PLAIN, NBODY_MODE_SORTED, NBODY_MODE_SUMCHECK,
                   NBodyError,  # noqa: F401
                   nbody_diff_rollout,
                   nbody_ens_energy, nbody_ens_free, nbody_ens_get_state, nbody_ens_get_stats,
                   nbody_ens_init, nbody_ens_run, nbody_ens_set_shape, nbody_ens_step, nbody_ens_tune,
                   nbody_correct, nbody_debug_fail_alloc, nbody_debug_skip_tile_copy, nbody_debug_step_graphs,
                   nbody_default_params, nbody_energy, nbody_energy_ds,
                   nbody_force, nbody_force_noalloc, nbody_free, nbody_get_predicted, nbody_get_state, nbody_get_stats, nbody_init,
                   nbody_last_error, nbody_next_block, nbody_predict, nbody_set_state, nbody_step,
                   nbody_strerror, nbody_sync)

MODES = {"plain": NBODY_MODE_PLAIN, "comp": NBODY_MODE_COMP, "sumcheck": NBODY_MODE_SUMCHECK,
         "sorted": NBODY_MODE_SORTED, "ds": NBODY_MODE_DS}

_STATE_KEYS = ("x", "v", "a", "k", "t_tick", "level")
_PARAM_KEYS = ("eta", "eta_init", "lmin", "lmax", "mode", "strict", "i_block", "j_tile", "j_split", "j_sub")


def write_checkpoint(path, m, eps2, params, state) -> None:
    """Writes an ``.npz`` checkpoint: the masses ``m`` (n,), eps^2, the integrator parameters (a dict of
    ``Simulation``'s keyword arguments) and the state of ``Simulation.get_state``: x, v, a, k (n, 3)
    float64, t_tick (n,) int64 ticks of 2^-lmax and level (n,) int8 (dt = 2^-level)."""
    import json

    import numpy as np
    m = np.ascontiguousarray(m, dtype=np.float64)
    n = m.shape[0]
    want = {"x": (np.float64, (n, 3)), "v": (np.float64, (n, 3)), "a": (np.float64, (n, 3)),
            "k": (np.float64, (n, 3)), "t_tick": (np.int64, (n,)), "level": (np.int8, (n,))}
    out = {}
    for key, (dt, shape) in want.items():
        a = np.asarray(state[key])
        if a.dtype != dt or a.shape != shape:
            raise ValueError(f"checkpoint field {key}: need {np.dtype(dt).name} {shape}, got {a.dtype} {a.shape}")
        out[key] = a
    unknown = set(params) - set(_PARAM_KEYS)
    if unknown:
        raise ValueError(f"unknown parameters {sorted(unknown)}")
    np.savez(path, m=m, eps2=np.float64(eps2), params=np.array(json.dumps(params, sort_keys=True)), **out)


def read_checkpoint(path):
    """(m, eps2, params, state) from a file of ``write_checkpoint``; no pickled objects are read."""
    import json

    import numpy as np
    with np.load(path, allow_pickle=False) as d:
        m = np.ascontiguousarray(d["m"], dtype=np.float64)
        eps2 = float(d["eps2"])
        params = json.loads(str(d["params"]))
        state = {key: np.ascontiguousarray(d[key]) for key in _STATE_KEYS}
    n = m.shape[0]
    for key in ("x", "v", "a", "k"):
        if state[key].dtype != np.float64 or state[key].shape != (n, 3):
            raise ValueError(f"checkpoint field {key} has {state[key].dtype} {state[key].shape}")
    if state["t_tick"].dtype != np.int64 or state["t_tick"].shape != (n,):
        raise ValueError("checkpoint field t_tick must be int64 (n,)")
    if state["level"].dtype != np.int8 or state["level"].shape != (n,):
        raise ValueError("checkpoint field level must be int8 (n,)")
    return m, eps2, params, state


class Simulation:
    """One library context: masses, FP64 state and j-stream on the current CUDA device.

    ``m`` (n,), ``x`` and ``v`` (n, 3) float64, numpy or torch (host or CUDA).
    ``stream``: a ``torch.cuda.Stream`` (or raw ``cudaStream_t`` int); None
    selects the legacy default stream.
    """

    def __init__(self, m, x, v, eps2, *, eta=0.01, eta_init=None, lmin=6, lmax=26, mode="plain",
                 strict=False, i_block=0, j_tile=0, j_split=0, j_sub=0, stream=None):
        p = nbody_default_params()
        p.eta = float(eta)
        p.eta_init = float(eta_init) if eta_init is not None else 0.0
        p.lmin, p.lmax = int(lmin), int(lmax)
        p.mode = MODES[mode] if isinstance(mode, str) else int(mode)
        p.strict = 1 if strict else 0
        p.i_block, p.j_tile, p.j_split, p.j_sub = int(i_block), int(j_tile), int(j_split), int(j_sub)
        if stream is not None:
            p.stream = int(getattr(stream, "cuda_stream", stream))
        self.n = int(m.shape[0])
        self.lmin, self.lmax = p.lmin, p.lmax
        self.mode = p.mode
        self.stream = stream
        self.eps2 = float(eps2)
        self._m = m.detach().clone() if hasattr(m, "detach") else m.copy()  # fixed masses, for checkpoints
        self._params = {"eta": p.eta, "eta_init": p.eta_init, "lmin": p.lmin, "lmax": p.lmax, "mode": p.mode,
                        "strict": bool(p.strict), "i_block": p.i_block, "j_tile": p.j_tile, "j_split": p.j_split,
                        "j_sub": p.j_sub}
        self._ctx = nbody_init(self.n, m, x, v, eps2, p)

    @property
    def handle(self):
        if self._ctx is None:
            raise RuntimeError("simulation closed")
        return self._ctx

    def next_block(self, active=None):
        """(t_blk, n_act); the block's indices go to ``active`` (int32, room for n) if given."""
        return nbody_next_block(self.handle, active)

    def predict(self, t):
        nbody_predict(self.handle, t)

    def force(self, active, n_act=None, acc=None, jerk=None, pot=None):
        n_act = int(active.shape[0]) if n_act is None else int(n_act)
        nbody_force(self.handle, active, n_act, acc, jerk, pot)

    def correct(self, active, n_act=None, acc=None, jerk=None):
        n_act = int(active.shape[0]) if n_act is None else int(n_act)
        nbody_correct(self.handle, active, n_act, acc, jerk)

    def step(self, t_end, max_steps=0):
        return nbody_step(self.handle, t_end, max_steps)

    def sync(self):
        nbody_sync(self.handle)

    def energy(self, ds_potential=False):
        """(E_kin, E_pot) at a synchronised time; ``ds_potential`` evaluates the potential in
        double-single arithmetic (``nbody_energy_ds``: ~1e-13 relative, fast at large N)."""
        return nbody_energy_ds(self.handle) if ds_potential else nbody_energy(self.handle)

    def get_state(self, x=None, v=None, a=None, k=None, t_tick=None, level=None):
        nbody_get_state(self.handle, self.n, x, v, a, k, t_tick, level)

    def set_state(self, x, v, a, k, t_tick, level):
        nbody_set_state(self.handle, self.n, x, v, a, k, t_tick, level)

    def checkpoint(self, path):
        """Writes masses, eps^2, parameters and the FP64 state to an ``.npz`` file (``write_checkpoint``);
        ``Simulation.from_checkpoint`` resumes from it bit for bit."""
        import numpy as np
        n = self.n
        st = dict(x=np.zeros((n, 3)), v=np.zeros((n, 3)), a=np.zeros((n, 3)), k=np.zeros((n, 3)),
                  t_tick=np.zeros(n, dtype=np.int64), level=np.zeros(n, dtype=np.int8))
        self.get_state(**st)
        m = self._m.detach().cpu().numpy() if hasattr(self._m, "detach") else self._m
        write_checkpoint(path, m, self.eps2, self._params, st)

    @classmethod
    def from_checkpoint(cls, path, stream=None):
        """A new context holding the state of ``path`` (see ``checkpoint``)."""
        m, eps2, params, st = read_checkpoint(path)
        params = dict(params)
        if params.get("eta_init", 0.0) <= 0.0:
            params["eta_init"] = None
        sim = cls(m, st["x"], st["v"], eps2, stream=stream, **params)
        sim.set_state(**st)
        return sim

    def get_predicted(self, posm=None, vel=None, poslo=None):
        nbody_get_predicted(self.handle, self.n, posm, vel, poslo)

    def stats(self):
        s = nbody_get_stats(self.handle)
        return {f: getattr(s, f) for f, _ in s._fields_}

    def close(self):
        if self._ctx is not None:
            nbody_free(self._ctx)
            self._ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ensemble:
    """Independent clusters integrated together (one library ensemble handle).

    ``sizes`` (n_clusters,) particle counts; ``m``, ``x``, ``v`` hold all
    clusters' particles one after the other.  Other arguments as ``Simulation``.
    """

    def __init__(self, sizes, m, x, v, eps2, *, eta=0.02, eta_init=None, lmin=6, lmax=26, mode="plain",
                 strict=False, stream=None, threads=0, i_block=0, tiles_per_range=0):
        import numpy as np
        p = nbody_default_params()
        p.j_tile, p.i_block, p.j_split = int(threads), int(i_block), int(tiles_per_range)
        p.eta = float(eta)
        p.eta_init = float(eta_init) if eta_init is not None else 0.0
        p.lmin, p.lmax = int(lmin), int(lmax)
        p.mode = MODES[mode] if isinstance(mode, str) else int(mode)
        p.strict = 1 if strict else 0
        if stream is not None:
            p.stream = int(getattr(stream, "cuda_stream", stream))
        self.sizes = np.ascontiguousarray(sizes, dtype=np.int64)
        self.n_clusters = int(self.sizes.shape[0])
        self.n = int(self.sizes.sum())
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)])
        self._h = nbody_ens_init(self.n_clusters, self.sizes, m, x, v, eps2, p)

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("ensemble closed")
        return self._h

    def set_shape(self, threads, i_block, tiles_per_range):
        nbody_ens_set_shape(self.handle, threads, i_block, tiles_per_range)

    def tune(self, t_end, steps=4):
        """(threads, i_block, tiles_per_range, ms per batched step) of the fastest shape."""
        return nbody_ens_tune(self.handle, t_end, steps)

    def step(self, t_end):
        return nbody_ens_step(self.handle, t_end)

    def run(self, t_end, check_every=16):
        return nbody_ens_run(self.handle, t_end, check_every)

    def energy(self):
        import numpy as np
        ek = np.zeros(self.n_clusters)
        ep = np.zeros(self.n_clusters)
        nbody_ens_energy(self.handle, self.n_clusters, ek, ep)
        return ek, ep

    def get_state(self, x=None, v=None, a=None, k=None, t_tick=None, level=None):
        nbody_ens_get_state(self.handle, self.n, x, v, a, k, t_tick, level)

    def stats(self):
        import numpy as np
        blocks = np.zeros(self.n_clusters, dtype=np.int64)
        pairs = np.zeros(self.n_clusters, dtype=np.int64)
        launches = nbody_ens_get_stats(self.handle, self.n_clusters, blocks, pairs)
        return {"blocks": blocks, "pairs": pairs, "kernel_launches": launches}

    def close(self):
        if self._h is not None:
            nbody_ens_free(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
