"""The .npz checkpoint format of the Python API (host logic; no GPU)."""
import numpy as np
import pytest

from paper_astro_ph_0702058_gb300 import read_checkpoint, write_checkpoint


def _state(n, seed=0):
    r = np.random.default_rng(seed)
    return dict(x=r.standard_normal((n, 3)), v=r.standard_normal((n, 3)), a=r.standard_normal((n, 3)),
                k=r.standard_normal((n, 3)), t_tick=r.integers(0, 1 << 40, n, dtype=np.int64),
                level=r.integers(6, 27, n, dtype=np.int8))


def test_round_trip_is_exact(tmp_path):
    n = 37
    st = _state(n)
    m = np.random.default_rng(1).random(n)
    params = {"eta": 0.02, "eta_init": 0.0, "lmin": 6, "lmax": 26, "mode": 1, "strict": True, "i_block": 0,
              "j_tile": 0, "j_split": 0}
    path = tmp_path / "ck.npz"
    write_checkpoint(path, m, 1.0 / 65536, params, st)
    m2, eps2, p2, st2 = read_checkpoint(path)
    assert np.array_equal(m2, m) and eps2 == 1.0 / 65536 and p2 == params
    for key in st:
        assert st2[key].dtype == st[key].dtype and np.array_equal(st2[key], st[key]), key
        assert st2[key].flags["C_CONTIGUOUS"]


@pytest.mark.parametrize("key,bad", [("x", np.zeros((5, 3), dtype=np.float32)), ("v", np.zeros((4, 3))),
                                     ("t_tick", np.zeros(5, dtype=np.int32)), ("level", np.zeros(5, dtype=np.int64))])
def test_write_rejects_wrong_fields(tmp_path, key, bad):
    st = _state(5)
    st[key] = bad
    with pytest.raises(ValueError):
        write_checkpoint(tmp_path / "bad.npz", np.ones(5), 0.1, {}, st)


def test_write_rejects_unknown_parameters(tmp_path):
    with pytest.raises(ValueError):
        write_checkpoint(tmp_path / "bad.npz", np.ones(3), 0.1, {"nu": 0.01}, _state(3))


def test_read_rejects_inconsistent_files(tmp_path):
    path = tmp_path / "bad.npz"
    st = _state(4)
    np.savez(path, m=np.ones(4), eps2=np.float64(0.1), params=np.array("{}"),
             **{**st, "level": st["level"].astype(np.int16)})
    with pytest.raises(ValueError):
        read_checkpoint(path)
