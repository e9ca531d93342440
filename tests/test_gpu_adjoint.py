"""The hand-written adjoint (sph_backward) against the oracle's forward-mode derivative of
the same discrete map (the oracle's dual numbers are themselves pinned to central finite
differences). Bars: FP64 mode <= 1e-8 relative; FP32 pair loops <= 1e-3 relative."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import sim_of

import paper_1909_04504_gb300 as G

pytestmark = pytest.mark.gpu


def _direction(s, dim, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    fluid = s["role"] == W.FLUID
    return [np.where(fluid, rng.normal(size=s["x"].shape), 0.0) for _ in range(dim)]


def _check(wl, K, tol, seed=5, check_alpha=False):
    s = O.state_of(wl)
    d = _direction(s, wl.dim, seed)
    _, dke_u = O.grad(wl, s, wl.dt, K, du=d[0], dv=d[1], dw=d[2] if wl.dim == 3 else None)
    _, dke_nu = O.grad(wl, s, wl.dt, K, dnu=1.0)
    with sim_of(wl) as sim:
        gu, gnu, galpha = sim.backward(G.scheme_of(wl), wl.dt, K)
    got = sum(np.dot(gu[k], d[k]) for k in range(wl.dim))
    assert abs(got - dke_u) <= tol * abs(dke_u), (got, dke_u)
    if wl.nu:
        assert abs(gnu - dke_nu) <= tol * abs(dke_nu), (gnu, dke_nu)
    if check_alpha:
        _, dke_al = O.grad(wl, s, wl.dt, K, dalpha=1.0)
        assert abs(galpha - dke_al) <= tol * abs(dke_al), (galpha, dke_al)
    return gu, gnu, galpha


def _tg2(precision, n=20):
    wl = W.taylor_green_2d(n=n, precision=precision)
    wl.nu = 0.05
    return wl


def test_k0_closed_form():
    wl = _tg2(W.PREC_FP64)
    s = O.state_of(wl)
    with sim_of(wl) as sim:
        gu, gnu, _ = sim.backward(G.scheme_of(wl), wl.dt, 0)
    assert np.allclose(gu[0], s["m"] * s["u"], rtol=0, atol=1e-15)
    assert np.allclose(gu[1], s["m"] * s["v"], rtol=0, atol=1e-15)
    assert gnu == 0.0


def test_taylor_green_2d_fp64():
    _check(_tg2(W.PREC_FP64), K=10, tol=1e-8)


def test_dam_break_2d_fp64_walls_av_xsph():
    wl = W.dam_break_2d(dx=0.08, precision=W.PREC_FP64)
    s = O.state_of(wl)
    rng = np.random.Generator(np.random.PCG64(3))
    fluid = s["role"] == W.FLUID
    wl.arrays[0].u = 0.3 * rng.normal(size=wl.arrays[0].n)
    wl.arrays[0].v = 0.3 * rng.normal(size=wl.arrays[0].n)
    _check(wl, K=6, tol=1e-8, check_alpha=True)


def test_taylor_green_3d_fp32_against_fp64_oracle():
    """The differentiation configuration's 16^3 copy: FP32 forward, FP64 oracle gradient."""
    wl = W.taylor_green_3d(n=16, precision=W.PREC_FP32)
    _check(wl, K=10, tol=1e-3)


def test_taylor_green_3d_fp64():
    wl = W.taylor_green_3d(n=12, precision=W.PREC_FP64)
    _check(wl, K=5, tol=1e-8)


def test_checkpoint_interval_does_not_change_the_gradient_and_final_state():
    wl = W.dam_break_2d(dx=0.05, precision=W.PREC_FP32)
    sch = G.scheme_of(wl)
    K = 9
    outs = []
    for C in (1, 3, 4, 9):  # 4: a remainder segment of one step
        with sim_of(wl) as sim:
            gu, gnu, gal = sim.backward(sch, wl.dt, K, ckpt_every=C)
            outs.append((gu, gal, sim.state()))
    for gu, gal, st in outs[1:]:
        assert np.array_equal(gu, outs[0][0]) and gal == outs[0][1]
        for k in ("x", "y", "u", "v", "rho"):
            assert np.array_equal(st[k], outs[0][2][k])
    with sim_of(wl) as sim:
        sim.eval_rhs(sch)
        sim.step(sch, wl.dt, K)
        st = sim.state()
    for k in ("x", "y", "u", "v", "rho"):
        assert np.array_equal(st[k], outs[0][2][k]), k


def test_backward_rejects_summation_density_and_adaptive_dt():
    wl = _tg2(W.PREC_FP64)
    with sim_of(wl) as sim:
        sch = G.scheme_of(wl, density=G.SUMMATION)
        with pytest.raises(G.SphError):
            sim.backward(sch, wl.dt, 2)
        with pytest.raises(G.SphError):
            sim.backward(G.scheme_of(wl), 0.0, 2)


def test_autograd_function_gives_the_adjoint_gradients():
    import torch
    wl = _tg2(W.PREC_FP64, n=16)
    s = O.state_of(wl)
    K = 6
    with sim_of(wl) as sim:
        u0 = torch.tensor(np.stack([s["u"], s["v"]]), dtype=torch.float64, requires_grad=True)
        nu = torch.tensor(wl.nu, dtype=torch.float64, requires_grad=True)
        ke = G.final_kinetic_energy(sim, G.scheme_of(wl), wl.dt, K, u0, nu)
        ke.backward()
    ke_o, dke_nu = O.grad(wl, s, wl.dt, K, dnu=1.0)
    assert abs(ke.item() - ke_o) <= 1e-12 * ke_o
    assert abs(nu.grad.item() - dke_nu) <= 1e-8 * abs(dke_nu)
    d = _direction(s, 2, 9)
    _, dke_u = O.grad(wl, s, wl.dt, K, du=d[0], dv=d[1])
    got = float((u0.grad.numpy() * np.stack(d)).sum())
    assert abs(got - dke_u) <= 1e-8 * abs(dke_u)


def _dam_break_moving(wl, seed=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    for name in ("u", "v", "w")[:wl.dim]:
        setattr(wl.arrays[0], name, 0.3 * rng.normal(size=wl.arrays[0].n))
    return wl


def test_dam_break_2d_fp32_dalpha():
    """d/d alpha (Monaghan artificial viscosity) with FP32 pair loops, walls and XSPH."""
    _check(_dam_break_moving(W.dam_break_2d(dx=0.08, precision=W.PREC_FP32)), K=6, tol=1e-3,
           check_alpha=True)


@pytest.mark.parametrize("prec,tol", [(W.PREC_FP64, 1e-8), (W.PREC_FP32, 1e-3)])
def test_dam_break_3d_dalpha(prec, tol):
    """d/d alpha and a velocity direction in 3D: walls, artificial viscosity, XSPH, gravity
    along z."""
    wl = _dam_break_moving(W.dam_break_3d(dx=0.1, precision=prec))
    _check(wl, K=4, tol=tol, check_alpha=True)
