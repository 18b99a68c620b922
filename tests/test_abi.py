"""The C ABI: the library builds for sm_103a, loads, and exports every call the
header declares; the binding mirrors them; argument checks that need no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nbody.h")


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(nbody_[a-z_0-9]+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_astro_ph_0702058_gb300 import build
    return build.build()


def test_header_declares_the_calls():
    names = header_functions()
    for required in ("nbody_init", "nbody_predict", "nbody_force", "nbody_correct", "nbody_energy",
                     "nbody_next_block", "nbody_step", "nbody_get_state", "nbody_set_state", "nbody_free",
                     "nbody_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_mirrors_header():
    from paper_astro_ph_0702058_gb300 import _lib
    assert sorted(_lib.EXPORTS) == header_functions()
    for name in _lib.EXPORTS:
        assert callable(getattr(_lib, name)), name


def test_strerror_and_argument_checks_without_gpu(libpath):
    import numpy as np

    from paper_astro_ph_0702058_gb300 import _lib
    L = _lib.lib()
    for code in range(-8, 1):
        assert L.nbody_strerror(code).decode()
    assert L.nbody_strerror(-99).decode() == "unknown error code"
    p = _lib.nbody_default_params()
    assert p.eta == 0.01 and p.lmin == 6 and p.lmax == 26 and p.mode == 0
    m = np.ones(4)
    x = np.zeros((4, 3))
    h = ctypes.c_void_p()
    # rejected before any device call
    assert L.nbody_init(ctypes.byref(h), 0, _lib.ptr(m, "f64"), _lib.ptr(x, "f64"), _lib.ptr(x, "f64"), 0.1,
                        ctypes.byref(p)) == _lib.NBODY_EINVAL
    assert L.nbody_init(ctypes.byref(h), 4, _lib.ptr(m, "f64"), _lib.ptr(x, "f64"), _lib.ptr(x, "f64"), -1.0,
                        ctypes.byref(p)) == _lib.NBODY_EINVAL
    bad = _lib.nbody_default_params()
    bad.lmin, bad.lmax = 10, 5
    assert L.nbody_init(ctypes.byref(h), 4, _lib.ptr(m, "f64"), _lib.ptr(x, "f64"), _lib.ptr(x, "f64"), 0.1,
                        ctypes.byref(bad)) == _lib.NBODY_EINVAL
    assert "lmin" in _lib.nbody_last_error()
    assert L.nbody_predict(None, 0.0) == _lib.NBODY_EINVAL
    L.nbody_free(None)


def test_python_binding_rejects_wrong_dtypes():
    import numpy as np

    from paper_astro_ph_0702058_gb300 import _lib
    with pytest.raises(TypeError):
        _lib.ptr(np.zeros(3, dtype=np.float32), "f64")
    with pytest.raises(ValueError):
        _lib.ptr(np.zeros((3, 3))[:, 0], "f64")


def _c_layout(struct, fields, tmp_path):
    """sizeof and offsetof of a header struct, from a C program compiled against include/nbody.h."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    lines = [f'printf("%zu\\n", sizeof({struct}));'] + [f'printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"nbody.h\"\nint main(void) {\n"
                   + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), [int(v) for v in out[1:]]


@pytest.mark.parametrize("name", ["nbody_params", "nbody_stats"])
def test_binding_structs_match_header_layout(name, tmp_path):
    """The ctypes mirrors have the header's size and field offsets (the library writes whole structs)."""
    import ctypes as C

    from paper_astro_ph_0702058_gb300 import _lib
    cls = getattr(_lib, name)
    fields = [f for f, _ in cls._fields_]
    size, offsets = _c_layout(name, fields, tmp_path)
    assert C.sizeof(cls) == size
    assert [getattr(cls, f).offset for f in fields] == offsets


def test_every_call_rejects_a_null_handle_without_gpu(libpath):
    """Each call that takes a context or ensemble checks its pointers before any device work: with null
    arguments it returns EINVAL (no crash, no CUDA call), on a machine without a GPU."""
    import ctypes as C

    from paper_astro_ph_0702058_gb300 import _lib
    L = _lib.lib()

    def null_args(fn):
        out = []
        for t in fn.argtypes:
            if t in (C.c_int, C.c_int64):
                out.append(1)
            elif t is C.c_double:
                out.append(0.5)
            else:
                out.append(None)
        return out

    names = ["nbody_next_block", "nbody_predict", "nbody_force", "nbody_correct", "nbody_step", "nbody_sync",
             "nbody_energy", "nbody_energy_ds", "nbody_get_state", "nbody_set_state", "nbody_get_predicted", "nbody_get_stats",
             "nbody_ens_init", "nbody_ens_set_shape", "nbody_ens_tune", "nbody_ens_step", "nbody_ens_run",
             "nbody_ens_energy", "nbody_ens_get_state", "nbody_ens_get_stats", "nbody_diff_rollout", "nbody_rollout",
             "nbody_rollout_vjp",
             "nbody_force_noalloc"]
    for name in names:
        fn = getattr(L, name)
        assert fn(*null_args(fn)) == _lib.NBODY_EINVAL, name
        assert _lib.nbody_last_error(), name
    L.nbody_ens_free(None)
    L.nbody_free(None)


def test_noalloc_rejects_misaligned_pointers_without_gpu(libpath):
    """nbody_force_noalloc checks the alignment its kernels need (16 bytes for the j-stream, which
    bulk asynchronous copies read; 8 for the outputs; 4 for the list) before any CUDA call, so a
    misaligned pointer returns EINVAL instead of reaching a kernel.  The addresses below are
    never dereferenced: the call returns before it touches memory."""
    import ctypes as C

    from paper_astro_ph_0702058_gb300 import _lib
    L = _lib.lib()
    good16, good8, good4 = 0x10000, 0x20000, 0x30000
    plain = _lib.NBODY_MODE_PLAIN

    def call(posm=good16, vel=good16, poslo=good16, act=good4, acc=good8, jerk=good8, pot=good8, mode=plain):
        return L.nbody_force_noalloc(C.c_void_p(posm), C.c_void_p(vel), C.c_void_p(poslo), 1000, C.c_void_p(act),
                                     10, C.c_double(1e-4), mode, C.c_void_p(acc), C.c_void_p(jerk),
                                     C.c_void_p(pot), None)

    for kw, what in ((dict(posm=good16 + 8), "16-byte"), (dict(vel=good16 + 4), "16-byte"),
                     (dict(poslo=good16 + 8, mode=_lib.NBODY_MODE_COMP), "16-byte"),
                     (dict(acc=good8 + 4), "8-byte"), (dict(pot=good8 + 2), "8-byte"),
                     (dict(act=good4 + 2), "4-byte")):
        assert call(**kw) == _lib.NBODY_EINVAL, kw
        assert what in _lib.nbody_last_error(), (kw, _lib.nbody_last_error())
