"""ctypes binding of libnbody.so (argument marshalling only).

Every function here has the name and arguments of the C call in
``include/nbody.h`` and does nothing but convert Python objects to pointers
and sizes and turn a negative return code into ``NBodyError``.  All work
runs in the library's CUDA kernels; there is no CPU fallback: if the library
is missing or cannot be loaded, every call raises.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA
memory); they must be C-contiguous with the dtype the C call expects.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from .build import LIB

_lock = threading.Lock()
_lib = None

NBODY_OK = 0
NBODY_EINVAL = -1
NBODY_ENOMEM = -2
NBODY_ECUDA = -3
NBODY_EDTMIN = -4
NBODY_ENONFINITE = -5
NBODY_ENOTSYNC = -6
NBODY_ETIMEOUT = -7
NBODY_ESTATE = -8
NBODY_MODE_PLAIN = 0
NBODY_MODE_COMP = 1
NBODY_MODE_SUMCHECK = 2
NBODY_MODE_SORTED = 3
NBODY_MODE_DS = 4

# Every symbol include/nbody.h declares (checked by the tests against the header).
EXPORTS = ("nbody_default_params", "nbody_init", "nbody_next_block", "nbody_predict", "nbody_force",
           "nbody_correct", "nbody_step", "nbody_sync", "nbody_energy", "nbody_energy_ds", "nbody_get_state",
           "nbody_set_state", "nbody_get_predicted", "nbody_get_stats", "nbody_free", "nbody_strerror", "nbody_last_error",
           "nbody_debug_fail_alloc", "nbody_debug_skip_tile_copy", "nbody_debug_step_graphs", "nbody_force_noalloc",
           "nbody_ens_init", "nbody_ens_set_shape", "nbody_ens_tune", "nbody_ens_step", "nbody_ens_run",
           "nbody_ens_energy", "nbody_ens_get_state", "nbody_ens_get_stats", "nbody_ens_free",
           "nbody_diff_rollout", "nbody_rollout", "nbody_rollout_vjp")


class nbody_params(C.Structure):
    _fields_ = [("eta", C.c_double), ("eta_init", C.c_double), ("lmin", C.c_int), ("lmax", C.c_int),
                ("mode", C.c_int), ("strict", C.c_int), ("i_block", C.c_int), ("j_tile", C.c_int),
                ("j_split", C.c_int), ("j_sub", C.c_int), ("stream", C.c_void_p)]


class nbody_stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_pad", C.c_int64), ("blocks", C.c_int64), ("below_dt_min", C.c_int64),
                ("nonfinite", C.c_int64), ("force_calls", C.c_int64), ("pairs", C.c_int64),
                ("kernel_launches", C.c_int64), ("last_threads", C.c_int), ("last_i_per_thread", C.c_int),
                ("last_j_split", C.c_int), ("mode", C.c_int), ("graph_blocks", C.c_int64),
                ("loop_blocks", C.c_int64), ("last_j_sub", C.c_int),
                ("cluster_blocks", C.c_int64), ("grid_blocks", C.c_int64)]


class NBodyError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        self.code = code
        super().__init__(f"{where}: {detail} (code {code})")


def lib_path() -> str:
    return os.environ.get("NBODY_LIB", LIB)


def lib():
    """Loads libnbody.so (raises if it has not been built: no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libnbody.so not built ({path}); run __graft_entry__.build()")
            L = C.CDLL(path)
            P = C.c_void_p
            L.nbody_default_params.argtypes = [C.POINTER(nbody_params)]
            L.nbody_default_params.restype = None
            L.nbody_init.argtypes = [C.POINTER(C.c_void_p), C.c_int64, P, P, P, C.c_double, C.POINTER(nbody_params)]
            L.nbody_next_block.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_int64), P]
            L.nbody_predict.argtypes = [P, C.c_double]
            L.nbody_force.argtypes = [P, P, C.c_int64, P, P, P]
            L.nbody_correct.argtypes = [P, P, C.c_int64, P, P]
            L.nbody_step.argtypes = [P, C.c_double, C.c_int64, C.POINTER(C.c_int64)]
            L.nbody_sync.argtypes = [P]
            L.nbody_energy.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.nbody_energy_ds.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.nbody_get_state.argtypes = [P, P, P, P, P, P, P]
            L.nbody_set_state.argtypes = [P, P, P, P, P, P, P]
            L.nbody_get_predicted.argtypes = [P, P, P, P]
            L.nbody_get_stats.argtypes = [P, C.POINTER(nbody_stats)]
            L.nbody_free.argtypes = [P]
            L.nbody_free.restype = None
            L.nbody_strerror.argtypes = [C.c_int]
            L.nbody_strerror.restype = C.c_char_p
            L.nbody_last_error.argtypes = []
            L.nbody_last_error.restype = C.c_char_p
            L.nbody_debug_fail_alloc.argtypes = [C.c_int]
            L.nbody_debug_fail_alloc.restype = None
            L.nbody_debug_skip_tile_copy.argtypes = [C.c_int]
            L.nbody_debug_skip_tile_copy.restype = None
            L.nbody_debug_step_graphs.argtypes = [C.c_int]
            L.nbody_debug_step_graphs.restype = None
            L.nbody_force_noalloc.argtypes = [P, P, P, C.c_int64, P, C.c_int64, C.c_double, C.c_int, P, P, P, P]
            L.nbody_force_noalloc.restype = C.c_int
            I = C.POINTER(C.c_int)
            L.nbody_ens_init.argtypes = [C.POINTER(C.c_void_p), C.c_int64, P, P, P, P, C.c_double,
                                         C.POINTER(nbody_params)]
            L.nbody_ens_set_shape.argtypes = [P, C.c_int, C.c_int, C.c_int]
            L.nbody_ens_tune.argtypes = [P, C.c_double, C.c_int, I, I, I, C.POINTER(C.c_double)]
            L.nbody_ens_step.argtypes = [P, C.c_double, C.POINTER(C.c_int64)]
            L.nbody_ens_run.argtypes = [P, C.c_double, C.c_int64, C.POINTER(C.c_int64)]
            L.nbody_ens_energy.argtypes = [P, P, P]
            L.nbody_ens_get_state.argtypes = [P, P, P, P, P, P, P]
            L.nbody_ens_get_stats.argtypes = [P, P, P, C.POINTER(C.c_int64)]
            L.nbody_diff_rollout.argtypes = [C.c_int64, P, P, P, C.c_double, C.c_int, C.c_int64, C.c_int64, C.c_int,
                                             P, P, P, P, P]
            L.nbody_diff_rollout.restype = C.c_int
            L.nbody_rollout.argtypes = [C.c_int64, P, P, P, C.c_double, C.c_int, C.c_int64, C.c_int, P, P, P]
            L.nbody_rollout.restype = C.c_int
            L.nbody_rollout_vjp.argtypes = [C.c_int64, P, P, P, C.c_double, C.c_int, C.c_int64, C.c_int64, C.c_int,
                                            P, P, P, P, P, P]
            L.nbody_rollout_vjp.restype = C.c_int
            L.nbody_ens_free.argtypes = [P]
            L.nbody_ens_free.restype = None
            for name in ("nbody_ens_init", "nbody_ens_set_shape", "nbody_ens_tune", "nbody_ens_step",
                         "nbody_ens_run", "nbody_ens_energy", "nbody_ens_get_state", "nbody_ens_get_stats"):
                getattr(L, name).restype = C.c_int
            for name in ("nbody_init", "nbody_next_block", "nbody_predict", "nbody_force", "nbody_correct",
                         "nbody_step", "nbody_sync", "nbody_energy", "nbody_energy_ds", "nbody_get_state", "nbody_set_state",
                         "nbody_get_predicted", "nbody_get_stats"):
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _check(code: int, where: str) -> None:
    if code != NBODY_OK:
        detail = lib().nbody_last_error().decode() or lib().nbody_strerror(code).decode()
        raise NBodyError(code, where, detail)


_DTYPES = {"f64": ("float64", "torch.float64"), "i32": ("int32", "torch.int32"),
           "i64": ("int64", "torch.int64"), "i8": ("int8", "torch.int8")}


def ptr(a, kind: str, min_len: int = 0):
    """Raw address of a contiguous numpy array / torch tensor of dtype ``kind`` (None passes NULL)."""
    if a is None:
        return None
    np_name, torch_name = _DTYPES[kind]
    if hasattr(a, "data_ptr"):  # torch.Tensor
        if str(a.dtype) != torch_name:
            raise TypeError(f"expected {torch_name}, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if a.numel() < min_len:
            raise ValueError(f"buffer holds {a.numel()} elements, need {min_len}")
        return C.c_void_p(a.data_ptr())
    if hasattr(a, "__array_interface__"):
        if str(a.dtype) != np_name:
            raise TypeError(f"expected {np_name}, got {a.dtype}")
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if a.size < min_len:
            raise ValueError(f"buffer holds {a.size} elements, need {min_len}")
        return C.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported buffer type {type(a)}")


def nbody_default_params() -> nbody_params:
    p = nbody_params()
    lib().nbody_default_params(C.byref(p))
    return p


def nbody_init(n: int, m, x, v, eps2: float, params: nbody_params):
    h = C.c_void_p()
    _check(lib().nbody_init(C.byref(h), int(n), ptr(m, "f64", n), ptr(x, "f64", 3 * n), ptr(v, "f64", 3 * n),
                            float(eps2), C.byref(params)), "nbody_init")
    return h


def nbody_next_block(ctx, active=None):
    t = C.c_double()
    na = C.c_int64()
    _check(lib().nbody_next_block(ctx, C.byref(t), C.byref(na), ptr(active, "i32")), "nbody_next_block")
    return t.value, na.value


def nbody_predict(ctx, t: float) -> None:
    _check(lib().nbody_predict(ctx, float(t)), "nbody_predict")


def nbody_force(ctx, active, n_act: int, acc=None, jerk=None, pot=None) -> None:
    _check(lib().nbody_force(ctx, ptr(active, "i32", n_act), int(n_act), ptr(acc, "f64", 3 * n_act),
                             ptr(jerk, "f64", 3 * n_act), ptr(pot, "f64", n_act)), "nbody_force")


def nbody_correct(ctx, active, n_act: int, acc=None, jerk=None) -> None:
    _check(lib().nbody_correct(ctx, ptr(active, "i32", n_act), int(n_act), ptr(acc, "f64", 3 * n_act),
                               ptr(jerk, "f64", 3 * n_act)), "nbody_correct")


def nbody_step(ctx, t_end: float, max_steps: int = 0) -> int:
    ns = C.c_int64()
    _check(lib().nbody_step(ctx, float(t_end), int(max_steps), C.byref(ns)), "nbody_step")
    return ns.value


def nbody_sync(ctx) -> None:
    _check(lib().nbody_sync(ctx), "nbody_sync")


def nbody_energy(ctx):
    ek, ep = C.c_double(), C.c_double()
    _check(lib().nbody_energy(ctx, C.byref(ek), C.byref(ep)), "nbody_energy")
    return ek.value, ep.value


def nbody_energy_ds(ctx):
    ek, ep = C.c_double(), C.c_double()
    _check(lib().nbody_energy_ds(ctx, C.byref(ek), C.byref(ep)), "nbody_energy_ds")
    return ek.value, ep.value


def nbody_get_state(ctx, n, x=None, v=None, a=None, k=None, t_tick=None, level=None) -> None:
    _check(lib().nbody_get_state(ctx, ptr(x, "f64", 3 * n), ptr(v, "f64", 3 * n), ptr(a, "f64", 3 * n),
                                 ptr(k, "f64", 3 * n), ptr(t_tick, "i64", n), ptr(level, "i8", n)),
           "nbody_get_state")


def nbody_set_state(ctx, n, x, v, a, k, t_tick, level) -> None:
    _check(lib().nbody_set_state(ctx, ptr(x, "f64", 3 * n), ptr(v, "f64", 3 * n), ptr(a, "f64", 3 * n),
                                 ptr(k, "f64", 3 * n), ptr(t_tick, "i64", n), ptr(level, "i8", n)),
           "nbody_set_state")


_F32 = ("float32", "torch.float32")


def _ptr_f32(a, min_len):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if str(a.dtype) != _F32[1] or not a.is_contiguous() or a.numel() < min_len:
            raise ValueError("need a contiguous float32 tensor of n x 4")
        return C.c_void_p(a.data_ptr())
    if str(a.dtype) != _F32[0] or not a.flags["C_CONTIGUOUS"] or a.size < min_len:
        raise ValueError("need a C-contiguous float32 array of n x 4")
    return C.c_void_p(a.ctypes.data)


def nbody_get_predicted(ctx, n, posm=None, vel=None, poslo=None) -> None:
    _check(lib().nbody_get_predicted(ctx, _ptr_f32(posm, 4 * n), _ptr_f32(vel, 4 * n), _ptr_f32(poslo, 4 * n)),
           "nbody_get_predicted")


def nbody_get_stats(ctx) -> nbody_stats:
    s = nbody_stats()
    _check(lib().nbody_get_stats(ctx, C.byref(s)), "nbody_get_stats")
    return s


def nbody_free(ctx) -> None:
    lib().nbody_free(ctx)


def nbody_strerror(code: int) -> str:
    return lib().nbody_strerror(int(code)).decode()


def nbody_last_error() -> str:
    return lib().nbody_last_error().decode()


def nbody_debug_fail_alloc(k: int) -> None:
    lib().nbody_debug_fail_alloc(int(k))


def nbody_debug_skip_tile_copy(on: bool) -> None:
    lib().nbody_debug_skip_tile_copy(1 if on else 0)


def nbody_debug_step_graphs(level: int) -> None:
    """0: separate launches, 1: one graph replay per block, 2: device-side block loop, 3 (default): as 2, and
    the one-cluster block-step kernel for small systems (plain and compensated n_pad <= 4096, double-single
    n_pad <= 2048), the whole-GPU cooperative kernel for the blocks of up to 4095 rows of larger plain and
    compensated systems."""
    lib().nbody_debug_step_graphs(int(level))


def nbody_force_noalloc(posm, vel, poslo, n: int, active, n_act: int, eps2: float, mode: int,
                        acc, jerk, pot, stream=None) -> None:
    """Force on a list from the caller's own device j-stream, with no device allocation."""
    n_pad = (int(n) + 255) // 256 * 256
    st = None if stream is None else C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    _check(lib().nbody_force_noalloc(_ptr_f32(posm, 4 * n_pad), _ptr_f32(vel, 4 * n_pad),
                                     _ptr_f32(poslo, 4 * n_pad), int(n), ptr(active, "i32", n_act),
                                     int(n_act), float(eps2), int(mode), ptr(acc, "f64", 3 * n_act),
                                     ptr(jerk, "f64", 3 * n_act), ptr(pot, "f64", n_act), st),
           "nbody_force_noalloc")


def nbody_ens_init(n_clusters: int, sizes, m, x, v, eps2: float, params: nbody_params):
    h = C.c_void_p()
    n = int(sum(int(s) for s in sizes))
    _check(lib().nbody_ens_init(C.byref(h), int(n_clusters), ptr(sizes, "i64", n_clusters), ptr(m, "f64", n),
                                ptr(x, "f64", 3 * n), ptr(v, "f64", 3 * n), float(eps2), C.byref(params)),
           "nbody_ens_init")
    return h


def nbody_ens_set_shape(ens, threads: int, i_block: int, tiles_per_range: int) -> None:
    _check(lib().nbody_ens_set_shape(ens, int(threads), int(i_block), int(tiles_per_range)), "nbody_ens_set_shape")


def nbody_ens_tune(ens, t_end: float, steps: int = 4):
    t, i, p = C.c_int(), C.c_int(), C.c_int()
    ms = C.c_double()
    _check(lib().nbody_ens_tune(ens, float(t_end), int(steps), C.byref(t), C.byref(i), C.byref(p), C.byref(ms)),
           "nbody_ens_tune")
    return t.value, i.value, p.value, ms.value


def nbody_ens_step(ens, t_end: float) -> int:
    live = C.c_int64()
    _check(lib().nbody_ens_step(ens, float(t_end), C.byref(live)), "nbody_ens_step")
    return live.value


def nbody_ens_run(ens, t_end: float, check_every: int = 16) -> int:
    ns = C.c_int64()
    _check(lib().nbody_ens_run(ens, float(t_end), int(check_every), C.byref(ns)), "nbody_ens_run")
    return ns.value


def nbody_ens_energy(ens, n_clusters: int, ekin, epot) -> None:
    _check(lib().nbody_ens_energy(ens, ptr(ekin, "f64", n_clusters), ptr(epot, "f64", n_clusters)),
           "nbody_ens_energy")


def nbody_ens_get_state(ens, n, x=None, v=None, a=None, k=None, t_tick=None, level=None) -> None:
    _check(lib().nbody_ens_get_state(ens, ptr(x, "f64", 3 * n), ptr(v, "f64", 3 * n), ptr(a, "f64", 3 * n),
                                     ptr(k, "f64", 3 * n), ptr(t_tick, "i64", n), ptr(level, "i8", n)),
           "nbody_ens_get_state")


def nbody_ens_get_stats(ens, n_clusters: int, blocks=None, pairs=None):
    kl = C.c_int64()
    _check(lib().nbody_ens_get_stats(ens, ptr(blocks, "i64", n_clusters), ptr(pairs, "i64", n_clusters),
                                     C.byref(kl)), "nbody_ens_get_stats")
    return kl.value


def nbody_ens_free(ens) -> None:
    lib().nbody_ens_free(ens)


def nbody_diff_rollout(n: int, m, x0, v0, eps2: float, level: int, steps: int, checkpoint_every: int, mode: int,
                       loss, g_x0, g_v0, g_m, stream=None) -> None:
    st = None if stream is None else C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    _check(lib().nbody_diff_rollout(int(n), ptr(m, "f64", n), ptr(x0, "f64", 3 * n), ptr(v0, "f64", 3 * n),
                                    float(eps2), int(level), int(steps), int(checkpoint_every), int(mode),
                                    ptr(loss, "f64", 1), ptr(g_x0, "f64", 3 * n), ptr(g_v0, "f64", 3 * n),
                                    ptr(g_m, "f64", n), st), "nbody_diff_rollout")


def nbody_rollout(n: int, m, x0, v0, eps2: float, level: int, steps: int, mode: int, x_T, v_T, stream=None) -> None:
    st = None if stream is None else C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    _check(lib().nbody_rollout(int(n), ptr(m, "f64", n), ptr(x0, "f64", 3 * n), ptr(v0, "f64", 3 * n), float(eps2),
                               int(level), int(steps), int(mode), ptr(x_T, "f64", 3 * n), ptr(v_T, "f64", 3 * n), st),
           "nbody_rollout")


def nbody_rollout_vjp(n: int, m, x0, v0, eps2: float, level: int, steps: int, checkpoint_every: int, mode: int,
                      g_xT, g_vT, g_x0, g_v0, g_m, stream=None) -> None:
    st = None if stream is None else C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    _check(lib().nbody_rollout_vjp(int(n), ptr(m, "f64", n), ptr(x0, "f64", 3 * n), ptr(v0, "f64", 3 * n),
                                   float(eps2), int(level), int(steps), int(checkpoint_every), int(mode),
                                   ptr(g_xT, "f64", 3 * n), ptr(g_vT, "f64", 3 * n), ptr(g_x0, "f64", 3 * n),
                                   ptr(g_v0, "f64", 3 * n), ptr(g_m, "f64", n), st), "nbody_rollout_vjp")
