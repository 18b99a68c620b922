"""The hand-written adjoint of the shared-step rollout against the FP64 reverse-mode
oracle (itself pinned to finite differences of the C oracle, tests/test_oracle_adjoint.py)."""
import numpy as np
import pytest

from oracle import adjoint
from synthetic import plummer_sphere
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu
EPS2 = (1.0 / 128) ** 2
LEVEL, STEPS = 9, 256


def _gpu_grad(m, x, v, steps=STEPS, ck=16, mode=0):
    from paper_astro_ph_0702058_gb300 import nbody_diff_rollout
    n = len(m)
    loss = np.zeros(1)
    gx, gv, gm = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
    nbody_diff_rollout(n, m, x, v, EPS2, LEVEL, steps, ck, mode, loss, gx, gv, gm)
    return loss[0], gx, gv, gm


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("mode", [0, 1])
def test_gradient_matches_fp64_reverse_mode_n64(mode):
    """N = 64, eps = 1/128, 256 steps of dt = 1/512: loss and dL/d(x0, v0, m)."""
    need_gpu()
    m, x, v = plummer_sphere(64, 12)
    m = m * np.random.default_rng(3).uniform(0.8, 1.2, 64)
    L, gx, gv, gm = _gpu_grad(m, x, v, mode=mode)
    rL, rgx, rgv, rgm = adjoint.rollout_grad(m, x, v, EPS2, 2.0 ** -LEVEL, STEPS)
    print(f"\nmode {mode}: loss rel err {abs(L - rL) / abs(rL):.2e}, grad rel err x {_rel(gx, rgx):.2e} "
          f"v {_rel(gv, rgv):.2e} m {_rel(gm, rgm):.2e}")
    assert abs(L - rL) <= 1e-6 * abs(rL)
    for g, r in ((gx, rgx), (gv, rgv), (gm, rgm)):
        assert _rel(g, r) < 1e-4


def test_checkpoint_spacing_does_not_change_the_gradient():
    need_gpu()
    m, x, v = plummer_sphere(96, 13)
    outs = [_gpu_grad(m, x, v, steps=40, ck=ck) for ck in (1, 7, 16, 40)]
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)


def test_autograd_function():
    torch = need_gpu()
    from paper_astro_ph_0702058_gb300.autodiff import rollout_loss
    m, x, v = plummer_sphere(128, 14)
    xt = torch.tensor(x, device="cuda", requires_grad=True)
    vt = torch.tensor(v, device="cuda", requires_grad=True)
    mt = torch.tensor(m, device="cuda", requires_grad=True)
    loss = rollout_loss(xt, vt, mt, steps=32)
    (3.0 * loss).backward()
    L, gx, gv, gm = _gpu_grad(m, x, v, steps=32)
    assert abs(loss.item() - L) == 0.0
    np.testing.assert_array_equal(xt.grad.cpu().numpy(), 3.0 * gx)
    np.testing.assert_array_equal(vt.grad.cpu().numpy(), 3.0 * gv)
    np.testing.assert_array_equal(mt.grad.cpu().numpy(), 3.0 * gm)


@pytest.mark.parametrize("mode", [0, 1])
def test_full_size_gradient_against_double_single_finite_differences(mode):
    """C5 at full size (N = 4096, eps = 1/128, 256 steps of 1/512, checkpoints every 16): the
    directional derivative g . d of the adjoint gradient against central differences of the loss
    computed with double-single forces (~1e-12 from FP64), along seeded directions in x0, v0 and m."""
    need_gpu()
    from paper_astro_ph_0702058_gb300 import MODES
    n = 4096
    m, x, v = plummer_sphere(n, 5)
    L, gx, gv, gm = _gpu_grad(m, x, v, mode=mode)
    rng = np.random.default_rng(17)
    ds = MODES["ds"]
    for what in ("x", "v", "m"):
        d = rng.standard_normal((n, 3) if what != "m" else n)
        if what == "m":
            d *= m  # relative mass perturbations
        h = 1e-4  # large enough to beat the double-single rounding noise, small against the curvature
        args = {"x": x, "v": v, "m": m}
        lp = _gpu_grad(*(args[k] + h * d if k == what else args[k] for k in ("m", "x", "v")), mode=ds)[0]
        lm = _gpu_grad(*(args[k] - h * d if k == what else args[k] for k in ("m", "x", "v")), mode=ds)[0]
        fd = (lp - lm) / (2 * h)
        g = {"x": gx, "v": gv, "m": gm}[what]
        an = float((g * d).sum())
        print(f"\nmode {mode} d{what}: adjoint {an:.8e} finite difference {fd:.8e} rel {abs(an - fd) / abs(fd):.2e}")
        assert abs(an - fd) <= 1e-3 * abs(fd)


@pytest.mark.parametrize("mode", [0, 1])
def test_rollout_vjp_matches_fp64_reverse_mode_n64(mode):
    """N = 64, eps = 1/128, 256 steps of 1/512: the rollout's final state and its vector-Jacobian
    product for seeded random cotangents of (x_T, v_T), against the FP64 reverse-mode oracle."""
    need_gpu()
    from paper_astro_ph_0702058_gb300._lib import nbody_rollout, nbody_rollout_vjp
    n = 64
    m, x, v = plummer_sphere(n, 22)
    rng = np.random.default_rng(22)
    m = m * rng.uniform(0.8, 1.2, n)
    g_xT, g_vT = rng.standard_normal((n, 3)), rng.standard_normal((n, 3))
    xT, vT = np.zeros((n, 3)), np.zeros((n, 3))
    nbody_rollout(n, m, x, v, EPS2, LEVEL, STEPS, mode, xT, vT)
    gx, gv, gm = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
    nbody_rollout_vjp(n, m, x, v, EPS2, LEVEL, STEPS, 16, mode, g_xT, g_vT, gx, gv, gm)
    rxT, rvT, rgx, rgv, rgm = adjoint.rollout_vjp(m, x, v, EPS2, 2.0 ** -LEVEL, STEPS, g_xT, g_vT)
    print(f"\nmode {mode}: x_T {_rel(xT, rxT):.2e} v_T {_rel(vT, rvT):.2e}; vjp x {_rel(gx, rgx):.2e} "
          f"v {_rel(gv, rgv):.2e} m {_rel(gm, rgm):.2e}")
    assert _rel(xT, rxT) < 1e-6 and _rel(vT, rvT) < 1e-5
    for g, r in ((gx, rgx), (gv, rgv), (gm, rgm)):
        assert _rel(g, r) < 1e-4
    # a missing cotangent is zero
    gx0 = np.zeros((n, 3))
    nbody_rollout_vjp(n, m, x, v, EPS2, LEVEL, STEPS, 16, mode, None, g_vT, gx0, None, None)
    rgx0 = adjoint.rollout_vjp(m, x, v, EPS2, 2.0 ** -LEVEL, STEPS, np.zeros((n, 3)), g_vT)[2]
    assert _rel(gx0, rgx0) < 1e-4


def test_rollout_autograd_inside_a_larger_program():
    """rollout() composes with torch: a loss built from (x_T, v_T) by ordinary torch ops differentiates
    through the library's vector-Jacobian product, which equals the direct C call with those cotangents."""
    torch = need_gpu()
    from paper_astro_ph_0702058_gb300._lib import nbody_rollout_vjp
    from paper_astro_ph_0702058_gb300.autodiff import rollout
    n = 96
    m, x, v = plummer_sphere(n, 23)
    w = torch.tensor(np.random.default_rng(23).standard_normal((n, 3)), device="cuda")
    xt = torch.tensor(x, device="cuda", requires_grad=True)
    vt = torch.tensor(v, device="cuda", requires_grad=True)
    mt = torch.tensor(m, device="cuda", requires_grad=True)
    xT, vT = rollout(xt, vt, mt, steps=24)
    loss = (w * xT).sum() + 0.5 * (vT ** 2).sum() + torch.sin(xT[:, 0]).sum()
    loss.backward()
    g_xT = (w + torch.stack([torch.cos(xT[:, 0]), torch.zeros(n, device="cuda", dtype=torch.float64),
                             torch.zeros(n, device="cuda", dtype=torch.float64)], 1)).detach()
    g_vT = vT.detach()
    gx, gv, gm = (torch.zeros_like(xt), torch.zeros_like(vt), torch.zeros_like(mt))
    nbody_rollout_vjp(n, mt.detach(), xt.detach(), vt.detach(), EPS2, LEVEL, 24, 16, 0, g_xT.contiguous(),
                      g_vT.contiguous(), gx, gv, gm)
    torch.testing.assert_close(xt.grad, gx, rtol=1e-12, atol=0)
    torch.testing.assert_close(vt.grad, gv, rtol=1e-12, atol=0)
    torch.testing.assert_close(mt.grad, gm, rtol=1e-12, atol=0)
