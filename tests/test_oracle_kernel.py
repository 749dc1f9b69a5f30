"""Pins of the oracle's kernel function and Riemann solver against mathematics
that does not come from the oracle itself (quadrature, finite differences,
lattice convergence, the linear acoustic Riemann solution)."""
import math

import numpy as np
import pytest
from scipy import integrate


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("h", [0.013, 1.0, 3.7])
def test_wendland_unit_integral(oracle_mod, dim, h):
    # int W dV = 1: 2 pi int W r dr (2D), 4 pi int W r^2 dr (3D)
    if dim == 2:
        f = lambda r: oracle_mod.W(2, h, r) * 2.0 * math.pi * r
    else:
        f = lambda r: oracle_mod.W(3, h, r) * 4.0 * math.pi * r * r
    val, err = integrate.quad(f, 0.0, 2.0 * h, epsabs=0, epsrel=1e-13, limit=200)
    assert abs(val - 1.0) < 1e-10


@pytest.mark.parametrize("dim", [2, 3])
def test_wendland_derivative_finite_difference(oracle_mod, dim):
    h = 0.7
    for q in np.linspace(0.05, 1.95, 39):
        r = q * h
        eps = 1e-6 * h
        fd = (oracle_mod.W(dim, h, r + eps) - oracle_mod.W(dim, h, r - eps)) / (2 * eps)
        an = oracle_mod.dW(dim, h, r)
        scale = oracle_mod.alpha(dim, h) / h
        assert abs(fd - an) < 1e-7 * scale, (q, fd, an)


@pytest.mark.parametrize("dim", [2, 3])
def test_wendland_support_and_shape(oracle_mod, dim):
    h = 1.0
    assert oracle_mod.W(dim, h, 2.0 * h) == 0.0
    assert oracle_mod.dW(dim, h, 2.0 * h) == 0.0
    assert oracle_mod.W(dim, h, 2.5 * h) == 0.0
    assert oracle_mod.dW(dim, h, 0.0) == 0.0
    rs = np.linspace(0, 2 * h, 101)[:-1]
    w = np.array([oracle_mod.W(dim, h, r) for r in rs])
    assert np.all(w > 0) and np.all(np.diff(w) < 0)
    # W(0) = alpha_d (closed form of the normalisation constant)
    a = 7 / (4 * math.pi) if dim == 2 else 21 / (16 * math.pi)
    assert abs(oracle_mod.W(dim, h, 0.0) - a) < 1e-15


@pytest.mark.parametrize("dim", [2, 3])
def test_lattice_sum_converges_to_one(oracle_mod, dim):
    # sigma0 * dp^d is a Riemann sum of int W dV = 1; it converges as h/dp grows
    errs = [abs(oracle_mod.sigma0(dim, 1.0, hf) - 1.0) for hf in (1.3, 2.0, 3.0, 4.0)]
    assert errs[-1] < 1e-4
    assert errs[0] < 0.02
    # translation of the unit: sigma0 scales as dp^-d
    s1 = oracle_mod.sigma0(dim, 1.0, 1.3)
    s2 = oracle_mod.sigma0(dim, 0.01, 0.013)
    assert abs(s2 * 0.01 ** dim - s1) < 1e-12


def test_riemann_linear_acoustics(oracle_mod):
    """With the limiter saturated (U_L - U_R >= c0/3) the interface state is the
    exact solution of the linear acoustic Riemann problem with impedance
    Z = rho_bar c0 on both sides:  p* = (pL+pR)/2 + Z (UL-UR)/2,
    u* = (UL+UR)/2 + (pL-pR)/(2Z)."""
    rng = np.random.default_rng(7)
    c0 = 12.0
    for _ in range(200):
        pL, pR = rng.normal(size=2) * 50
        rL, rR = 1000 + rng.normal(size=2)
        UR = rng.normal()
        UL = UR + c0 / 3 + abs(rng.normal()) * 3
        Ps, Us = oracle_mod.riemann(pL, pR, rL, rR, UL, UR, c0)
        Z = 0.5 * (rL + rR) * c0
        assert Ps == pytest.approx(0.5 * (pL + pR) + 0.5 * Z * (UL - UR), rel=1e-13, abs=1e-9)
        assert Us == pytest.approx(0.5 * (UL + UR) + (pL - pR) / (2 * Z), rel=1e-13, abs=1e-12)


def test_riemann_special_cases(oracle_mod):
    c0 = 10.0
    # no velocity jump: P* is the mean pressure
    Ps, Us = oracle_mod.riemann(3.0, 5.0, 1.0, 1.2, 0.7, 0.7, c0)
    assert Ps == 4.0
    assert Us == pytest.approx(0.7 + (3.0 - 5.0) / (2 * 1.1 * c0), rel=1e-15)
    # expansion (UL < UR): the limiter switches dissipation off
    Ps, _ = oracle_mod.riemann(3.0, 5.0, 1.0, 1.2, 0.1, 0.9, c0)
    assert Ps == 4.0
    # equal pressures: U* is the mean normal velocity
    _, Us = oracle_mod.riemann(2.0, 2.0, 1.0, 1.0, 0.3, -0.1, c0)
    assert Us == pytest.approx(0.1, rel=1e-15)
    # weak compression: limiter beta = 3 (UL-UR)/c0 < 1
    UL, UR = 0.2, 0.0
    Ps, _ = oracle_mod.riemann(0.0, 0.0, 1.0, 1.0, UL, UR, c0)
    beta = 3 * (UL - UR) / c0
    assert Ps == pytest.approx(0.5 * beta * 1.0 * c0 * (UL - UR), rel=1e-14)


def test_riemann_mirror_symmetry(oracle_mod):
    """Seen from the other side (left and right swapped, normal reversed) the
    interface pressure is the same and the interface velocity flips sign."""
    rng = np.random.default_rng(11)
    for _ in range(500):
        pL, pR = rng.normal(size=2) * 10
        rL, rR = 1 + 0.01 * rng.normal(size=2)
        UL, UR = rng.normal(size=2)
        P1, U1 = oracle_mod.riemann(pL, pR, rL, rR, UL, UR, 5.0)
        P2, U2 = oracle_mod.riemann(pR, pL, rR, rL, -UR, -UL, 5.0)
        assert P1 == pytest.approx(P2, rel=1e-14, abs=1e-14)
        assert U1 == pytest.approx(-U2, rel=1e-14, abs=1e-14)
