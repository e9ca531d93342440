"""Pins of the oracle's smoothing kernels (Sec. 2, kernel interpolation) against
what mathematics fixes: unit integral, radial derivative, compact support,
smoothness at the spline knots, the first-moment identity of the gradient, and
the lattice sum predicted by the Poisson summation formula."""
import math

import numpy as np
import pytest
import scipy.integrate as integrate
import scipy.special as special

import oracle as O
import workloads as W

KINDS = [(W.QUINTIC, 3.0, [1.0, 2.0]), (W.WENDLAND_C2, 2.0, []), (W.CUBIC_SPLINE, 2.0, [1.0])]
KNOTS = {k: kn for k, _, kn in KINDS}


def _quad(f, kind, h, support):
    knots = [0.0] + [k * h for k in KNOTS[kind]] + [support * h]
    return sum(integrate.quad(f, a, b, limit=200, epsabs=1e-14, epsrel=1e-12)[0]
               for a, b in zip(knots[:-1], knots[1:]))


def _shell(dim, r):
    return 2 * math.pi * r if dim == 2 else 4 * math.pi * r * r


@pytest.mark.parametrize("kind,support,knots", KINDS)
@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("h", [1.0, 0.013, 0.7])
def test_unit_integral(kind, support, knots, dim, h):
    total = _quad(lambda r: O.kernel(kind, dim, h, r)[0] * _shell(dim, r), kind, h, support)
    assert abs(total - 1.0) < 1e-10


@pytest.mark.parametrize("kind,support,knots", KINDS)
@pytest.mark.parametrize("dim", [2, 3])
def test_gradient_first_moment(kind, support, knots, dim):
    """Integration by parts: integral of x . grad W dV = -d * integral W dV = -d."""
    h = 0.9
    total = _quad(lambda r: r * O.kernel(kind, dim, h, r)[1] * _shell(dim, r), kind, h, support)
    assert abs(total + dim) < 1e-10


@pytest.mark.parametrize("kind,support,knots", KINDS)
@pytest.mark.parametrize("dim", [2, 3])
def test_derivative_matches_finite_difference(kind, support, knots, dim):
    h = 1.3
    for r in np.linspace(0.03, support * h - 0.03, 37):
        eps = 1e-6 * h
        fd = (O.kernel(kind, dim, h, r + eps)[0] - O.kernel(kind, dim, h, r - eps)[0]) / (2 * eps)
        d = O.kernel(kind, dim, h, r)[1]
        scale = abs(O.kernel(kind, dim, h, 0.0)[0]) / h
        assert abs(fd - d) < 1e-7 * scale


@pytest.mark.parametrize("kind,support,knots", KINDS)
@pytest.mark.parametrize("dim", [2, 3])
def test_compact_support_and_knots(kind, support, knots, dim):
    h = 1.0
    for r in (support * h, support * h + 1e-9, 5.0 * h):
        W0, dW = O.kernel(kind, dim, h, r)
        assert W0 == 0.0 and dW == 0.0
    W_in, dW_in = O.kernel(kind, dim, h, support * h * (1 - 1e-7))
    # dW vanishes at the support like (support - r)^4 (quintic), ^3 (Wendland C2) or ^2
    # (cubic spline): (2e-7)^2 = 4e-14
    assert abs(W_in) < 1e-20 and abs(dW_in) < (1e-13 if kind == W.CUBIC_SPLINE else 1e-18)
    for q in knots:  # value, slope continuous across the spline knots
        a = O.kernel(kind, dim, h, q * h - 1e-9)
        b = O.kernel(kind, dim, h, q * h + 1e-9)
        assert abs(a[0] - b[0]) < 1e-8 and abs(a[1] - b[1]) < 1e-7
    # radial derivative vanishes at r = 0 and the kernel decreases monotonically
    assert O.kernel(kind, dim, h, 0.0)[1] == 0.0
    rs = np.linspace(0.0, support * h, 200)
    ws = [O.kernel(kind, dim, h, r)[0] for r in rs]
    assert all(a >= b for a, b in zip(ws[:-1], ws[1:]))


def _fourier(kind, dim, h, support, kappa):
    if dim == 2:
        f = lambda r: O.kernel(kind, dim, h, r)[0] * special.j0(kappa * r) * 2 * math.pi * r
    else:
        f = lambda r: (O.kernel(kind, dim, h, r)[0] * np.sinc(kappa * r / math.pi)
                       * 4 * math.pi * r * r)
    return _quad(f, kind, h, support)


def poisson_lattice_sum(kind, dim, hdx, support, K):
    """sum_j dx^d W(x_i - x_j) over an infinite lattice = sum_k W^(2 pi k / dx) (Poisson)."""
    cache = {}
    total = 1.0  # k = 0 term is the unit integral
    for k in np.ndindex(*([2 * K + 1] * dim)):
        n2 = int(sum((c - K) ** 2 for c in k))
        if n2 == 0 or n2 > K * K:
            continue
        if n2 not in cache:
            cache[n2] = _fourier(kind, dim, hdx, support, 2 * math.pi * math.sqrt(n2))
        total += cache[n2]
    return total


@pytest.mark.parametrize("kind,dim,hdx,K,tol", [
    (W.QUINTIC, 2, 1.0, 12, 2e-8),
    (W.WENDLAND_C2, 2, 1.3, 12, 2e-5),
    (W.CUBIC_SPLINE, 2, 1.2, 12, 1e-5),
    (W.QUINTIC, 3, 1.0, 8, 2e-8),
    (W.WENDLAND_C2, 3, 1.3, 8, 2e-5),
    (W.CUBIC_SPLINE, 3, 1.2, 8, 1e-5),
])
def test_summation_density_equals_poisson_lattice_sum(kind, dim, hdx, K, tol):
    """Eq. (2) on a uniform periodic lattice (m = rho0 dx^d) gives rho0 times the lattice
    sum of W, which the Poisson summation formula evaluates in Fourier space."""
    support = 3.0 if kind == W.QUINTIC else 2.0
    expected = poisson_lattice_sum(kind, dim, hdx, support, K)
    n = 16 if dim == 2 else 10
    if dim == 2:
        wl = W.taylor_green_2d(n=n, jitter=0.0, hdx=hdx)
    else:
        wl = W.taylor_green_3d(n=n, jitter=0.0)
        wl.h = hdx / n
    wl.kernel = kind
    wl.density = 1
    s = O.state_of(wl)
    r = O.rhs(wl, s)
    rho = r["rho"] / wl.rho0
    assert np.max(np.abs(rho - expected)) < tol
    # loose statement of the same fact: summation density is close to rho0 on a lattice
    assert np.max(np.abs(rho - 1.0)) < 1.1e-2
