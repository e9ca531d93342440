"""The benchmark configurations as configured, against the oracle.

- Dam break 2D (20,000 fluid + 3,618 wall particles, FP32 pair loops, FP64 integrator)
  over its full 2,000 steps: the one-step increments within 1e-4 relative L2, the
  front position (largest fluid x) at the end within 2 dx of the oracle's (a free surface
  is chaotic, so the comparison after many steps is of a global feature), and the
  growth of the FP32-vs-FP64 difference printed.
- Taylor-Green 3D: the adjoint through K = 50 steps with checkpoints on the 16^3 copy
  against the oracle's dual numbers (FP32 pair loops, 1e-3), the adjoint on the full
  64^3 run against central differences of the GPU forward run (relative step 1e-3 in nu
  and along a seeded velocity direction, agreement 1e-2), and the max |u| curve of the
  16^3 copy over 50 steps within 1 % of the oracle's at every step."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import field_error, rel_l2, sim_of

import paper_1909_04504_gb300 as G

pytestmark = pytest.mark.gpu

FIELDS_2D = ("x", "y", "u", "v", "rho")


def _front(x, role):
    return float(np.max(x[role == W.FLUID]))


def test_dam_break_2d_full_run_against_the_oracle():
    wl = W.dam_break_2d()
    assert wl.n_total == 23_618 and wl.steps == 2000
    s = O.state_of(wl)
    sch = G.scheme_of(wl)
    st1, _ = O.run(wl, s, wl.dt, 1)
    st100, _ = O.run(wl, s, wl.dt, 100)
    stK, histK = O.run(wl, s, wl.dt, wl.steps)
    with sim_of(wl) as sim:  # one run; the history holds the records of the last call
        sim.step(sch, wl.dt, 1)
        g1 = sim.state()
        h1 = sim.history()
        sim.step(sch, wl.dt, 99)
        g100 = sim.state()
        h2 = sim.history()
        sim.step(sch, wl.dt, wl.steps - 100)
        gK = sim.state()
        h = np.concatenate([h1, h2, sim.history()])
    for k in FIELDS_2D:  # one step: increments within the FP32 bar
        assert field_error(wl, k, g1[k], st1[k], s[k]) <= 1e-4, k
    growth = {}
    for tag, g, o in (("1", g1, st1), ("100", g100, st100), (str(wl.steps), gK, stK)):
        growth[tag] = {k: field_error(wl, k, g[k], o[k], s[k]) for k in FIELDS_2D}
    dx = 0.01
    fg, fo = _front(gK["x"], s["role"]), _front(stK["x"], s["role"])
    ke_rel = np.abs(h[:, 2] - histK[1:, 2]) / np.maximum(np.abs(histK[1:, 2]), 1e-300)
    print("\ndam break 2D, FP32 vs the FP64 oracle: relative L2 of the change from t = 0")
    for tag, e in growth.items():
        print(f"  step {tag:>5}: " + ", ".join(f"{k} {v:.2e}" for k, v in e.items()))
    print(f"  kinetic energy, relative difference at steps 1/10/100/1000/2000: "
          + ", ".join(f"{ke_rel[i]:.2e}" for i in (0, 9, 99, 999, wl.steps - 1)))
    print(f"  front x at t = {wl.steps * wl.dt:.4f} s: GPU {fg:.6f}, oracle {fo:.6f} m "
          f"(moved {fo - 1.0 + 0.5 * dx:.4f} m)")
    assert h.shape[0] == wl.steps
    assert np.array_equal(h[:, 0], histK[1:, 0]) or np.max(np.abs(h[:, 0] - histK[1:, 0])) < 1e-14
    assert abs(fg - fo) <= 2 * dx
    assert np.all(np.isfinite(ke_rel))


def _direction(s, dim, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    fluid = s["role"] == W.FLUID
    d = [np.where(fluid, rng.normal(size=s["x"].shape), 0.0) for _ in range(dim)]
    nrm = np.sqrt(sum(np.sum(v * v) for v in d))
    return [v / nrm for v in d]


def test_taylor_green_3d_adjoint_k50_fp32_against_dual_numbers():
    """The differentiation configuration's 16^3 copy at its K = 50, checkpoints every
    ceil(sqrt(50)) = 8 steps (the default)."""
    wl = W.taylor_green_3d(n=16, precision=W.PREC_FP32)
    K = 50
    s = O.state_of(wl)
    d = _direction(s, 3, 21)
    _, dke_u = O.grad(wl, s, wl.dt, K, du=d[0], dv=d[1], dw=d[2])
    _, dke_nu = O.grad(wl, s, wl.dt, K, dnu=1.0)
    with sim_of(wl) as sim:
        gu, gnu, _ = sim.backward(G.scheme_of(wl), wl.dt, K)
    got = sum(float(np.dot(gu[k], d[k])) for k in range(3))
    assert abs(got - dke_u) <= 1e-3 * abs(dke_u), (got, dke_u)
    assert abs(gnu - dke_nu) <= 1e-3 * abs(dke_nu), (gnu, dke_nu)


def _final_ke(wl, u0, nu, K):
    with sim_of(wl) as sim:
        for k, name in enumerate(("u", "v", "w")):
            sim.set(name, u0[k])
        sim.step(G.scheme_of(wl, nu=nu), wl.dt, K)
        return float(sim.diagnostics()[2])


def test_taylor_green_3d_full_size_adjoint_against_central_differences():
    """64^3 = 262,144 particles, FP32 pair loops, K = 50: dKE/dnu and dKE/du0 along a
    seeded unit direction against central differences of the GPU's own forward run with a
    relative step of 1e-3 (nu +- 1e-3 nu; u0 +- 1e-3 |u0| d), agreement 1e-2."""
    wl = W.taylor_green_3d()
    K = 50
    s = O.state_of(wl)
    u0 = [s["u"].copy(), s["v"].copy(), s["w"].copy()]
    d = _direction(s, 3, 33)
    with sim_of(wl) as sim:
        gu, gnu, _ = sim.backward(G.scheme_of(wl), wl.dt, K)
    dnu = 1e-3 * wl.nu
    fd_nu = (_final_ke(wl, u0, wl.nu + dnu, K) - _final_ke(wl, u0, wl.nu - dnu, K)) / (2 * dnu)
    eps = 1e-3 * np.sqrt(sum(np.sum(v * v) for v in u0))
    up = [u0[k] + eps * d[k] for k in range(3)]
    um = [u0[k] - eps * d[k] for k in range(3)]
    fd_u = (_final_ke(wl, up, wl.nu, K) - _final_ke(wl, um, wl.nu, K)) / (2 * eps)
    adj_u = sum(float(np.dot(gu[k], d[k])) for k in range(3))
    print(f"\nTG 3D 64^3, K = {K}: dKE/dnu adjoint {gnu:.6e}, central difference {fd_nu:.6e}; "
          f"dKE/du0.d adjoint {adj_u:.6e}, central difference {fd_u:.6e}")
    assert abs(gnu - fd_nu) <= 1e-2 * abs(fd_nu)
    assert abs(adj_u - fd_u) <= 1e-2 * abs(fd_u)


def test_taylor_green_3d_decay_curve_within_one_percent():
    """The 16^3 copy over 50 FP32 steps: max |u| within 1 % of the oracle at every step, and
    the velocity field's change from t = 0 within the FP32 bar at the end."""
    wl = W.taylor_green_3d(n=16, precision=W.PREC_FP32)
    steps = 50
    s = O.state_of(wl)
    st, hist = O.run(wl, s, wl.dt, steps)
    with sim_of(wl) as sim:
        sim.step(G.scheme_of(wl), wl.dt, steps)
        h = sim.history()
        g = sim.state()
    umax_g, umax_o = h[:, 3], hist[1:, 3]
    err = np.max(np.abs(umax_g - umax_o) / umax_o)
    assert err <= 0.01
    # the decay itself: the oracle's max|u| falls over the run
    assert umax_o[-1] < umax_o[0]
    for k in ("u", "v"):
        assert rel_l2(g[k] - s[k], st[k] - s[k]) <= 1e-3, k
