"""Pins of the oracle's EPL deflection (Tessore & Metcalf 2015 series) against
closed forms, a library hypergeometric function and the Poisson equation."""
import math

import mpmath
import numpy as np
import pytest

import oracle


def _ellip(e1, e2):
    c = math.hypot(e1, e2)
    return (1 - c) / (1 + c), 0.5 * math.atan2(e2, e1)


@pytest.mark.parametrize("e1,e2,x0,y0", [(0.3, 0.0, 0.0, 0.0), (0.1, -0.25, 0.05, -0.02),
                                          (-0.4, 0.2, -0.1, 0.07)])
def test_sie_closed_form(e1, e2, x0, y0):
    """gamma = 2 is the SIE: kappa = b / (2 sqrt(q^2 x'^2 + y'^2)) has
    alpha'_x = b/k atan(k x'/psi), alpha'_y = b/k atanh(k y'/psi), k = sqrt(1-q^2)
    (Kormann et al. 1994; Keeton 2001), in the lens frame."""
    thetaE = 1.3
    q, phi = _ellip(e1, e2)
    rng = np.random.default_rng(1)
    x = rng.uniform(-3, 3, 50)
    y = rng.uniform(-3, 3, 50)
    ax, ay = oracle.epl_deflection([thetaE, 2.0, e1, e2, x0, y0], x, y)
    b = thetaE * math.sqrt(q)
    k = math.sqrt(1 - q * q)
    cs, sn = math.cos(phi), math.sin(phi)
    dx, dy = x - x0, y - y0
    xp, yp = cs * dx + sn * dy, -sn * dx + cs * dy
    psi = np.sqrt(q * q * xp * xp + yp * yp)
    axp = b / k * np.arctan(k * xp / psi)
    ayp = b / k * np.arctanh(k * yp / psi)
    np.testing.assert_allclose(ax, cs * axp - sn * ayp, rtol=0, atol=1e-13)
    np.testing.assert_allclose(ay, sn * axp + cs * ayp, rtol=0, atol=1e-13)


@pytest.mark.parametrize("gamma", [1.5, 1.8, 2.0, 2.3, 2.7])
def test_circular_power_law(gamma):
    """q = 1: alpha = theta_E (r/theta_E)^(2-gamma) r_hat (mean convergence 1
    inside theta_E)."""
    thetaE, x0, y0 = 1.7, 0.2, -0.1
    rng = np.random.default_rng(2)
    x = rng.uniform(-4, 4, 40)
    y = rng.uniform(-4, 4, 40)
    ax, ay = oracle.epl_deflection([thetaE, gamma, 0.0, 0.0, x0, y0], x, y)
    dx, dy = x - x0, y - y0
    r = np.hypot(dx, dy)
    mag = thetaE * (r / thetaE) ** (2 - gamma)
    np.testing.assert_allclose(ax, mag * dx / r, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(ay, mag * dy / r, rtol=1e-13, atol=1e-14)


def test_einstein_ring_maps_to_source_centre():
    """A circular SIS sends every point of its Einstein ring to beta = 0."""
    thetaE = 1.25
    ang = np.linspace(0, 2 * np.pi, 17)
    x, y = thetaE * np.cos(ang), thetaE * np.sin(ang)
    ax, ay = oracle.epl_deflection([thetaE, 2.0, 0.0, 0.0, 0.0, 0.0], x, y)
    np.testing.assert_allclose(x - ax, 0, atol=1e-14)
    np.testing.assert_allclose(y - ay, 0, atol=1e-14)


@pytest.mark.parametrize("seed", range(6))
def test_hypergeometric_factor_matches_library(seed):
    """Sum Omega_n / e^{i varphi} equals 2F1(1, t/2; 2 - t/2; -f e^{2 i varphi})
    (mpmath.hyp2f1) to FP64 rounding, up to f = 0.75."""
    rng = np.random.default_rng(100 + seed)
    for _ in range(8):
        t = rng.uniform(0.05, 1.95)
        f = rng.uniform(0.0, 0.75)
        ph = rng.uniform(-np.pi, np.pi)
        F = oracle.hyp2f1_series(t, f, ph)
        ref = complex(mpmath.hyp2f1(1, t / 2, 2 - t / 2, -f * mpmath.exp(2j * ph)))
        assert abs(F - ref) < 1e-14 * max(1.0, abs(ref)), (t, f, ph, F, ref)


def test_series_truncation_bound():
    """The number of terms grows with f and the dropped tail stays below the
    stated bound f^N/(1-f) relative to the library value."""
    prev = 0
    for f in [0.0, 0.05, 0.2, 0.4, 0.6, 0.79]:
        n = oracle.series_terms(f)
        assert n >= prev
        prev = n
        assert (n + 2) ** 2 * f ** n / (1 - f) ** 2 < 1e-17
    assert oracle.series_terms(0.0) == 1


def _div_curl(p6, x, y, h=1e-5):
    axp, _ = oracle.epl_deflection(p6, x + h, y)
    axm, _ = oracle.epl_deflection(p6, x - h, y)
    _, ayp = oracle.epl_deflection(p6, x, y + h)
    _, aym = oracle.epl_deflection(p6, x, y - h)
    _, ayxp = oracle.epl_deflection(p6, x + h, y)
    _, ayxm = oracle.epl_deflection(p6, x - h, y)
    axyp, _ = oracle.epl_deflection(p6, x, y + h)
    axym, _ = oracle.epl_deflection(p6, x, y - h)
    div = (axp - axm) / (2 * h) + (ayp - aym) / (2 * h)
    curl = (ayxp - ayxm) / (2 * h) - (axyp - axym) / (2 * h)
    return div, curl


@pytest.mark.parametrize("seed", range(5))
def test_poisson_equation(seed):
    """div alpha = 2 kappa with kappa = (2-t)/2 (b/R)^t, R = sqrt(q^2 x'^2 + y'^2),
    b = theta_E sqrt(q) (the EPL's defining convergence), and curl alpha = 0,
    by FP64 central differences, for general (q, gamma, angle, centre)."""
    rng = np.random.default_rng(200 + seed)
    thetaE = rng.uniform(0.8, 2.5)
    gamma = rng.uniform(1.4, 2.6)
    e1, e2 = rng.uniform(-0.45, 0.45, 2)
    x0, y0 = rng.normal(0, 0.05, 2)
    p6 = [thetaE, gamma, e1, e2, x0, y0]
    x = rng.uniform(-3, 3, 30)
    y = rng.uniform(-3, 3, 30)
    keep = np.hypot(x - x0, y - y0) > 0.2
    x, y = x[keep], y[keep]
    div, curl = _div_curl(p6, x, y)
    q, phi = _ellip(e1, e2)
    cs, sn = math.cos(phi), math.sin(phi)
    xp = cs * (x - x0) + sn * (y - y0)
    yp = -sn * (x - x0) + cs * (y - y0)
    t = gamma - 1
    R = np.sqrt(q * q * xp * xp + yp * yp)
    kappa = (2 - t) / 2 * (thetaE * math.sqrt(q) / R) ** t
    np.testing.assert_allclose(div, 2 * kappa, rtol=2e-7)
    np.testing.assert_allclose(curl, 0, atol=2e-7 * np.max(np.abs(div)))


def test_orientation_convention():
    """e1 > 0 puts the mass's major axis along x; e2 > 0 along x = y
    (convergence, measured as div alpha / 2, is larger along the major axis)."""
    a = 1.0
    for e1, e2, pmaj, pmin in [(0.3, 0.0, (a, 0.0), (0.0, a)),
                               (0.0, 0.3, (a / math.sqrt(2), a / math.sqrt(2)),
                                (a / math.sqrt(2), -a / math.sqrt(2)))]:
        p6 = [1.2, 2.0, e1, e2, 0.0, 0.0]
        dmaj, _ = _div_curl(p6, np.array([pmaj[0]]), np.array([pmaj[1]]))
        dmin, _ = _div_curl(p6, np.array([pmin[0]]), np.array([pmin[1]]))
        assert dmaj[0] > 1.2 * dmin[0]


def test_centre_is_finite():
    """At the centre the clamped radius gives a finite (zero) deflection."""
    ax, ay = oracle.epl_deflection([1.2, 2.2, 0.2, 0.1, 0.3, -0.2], [0.3], [-0.2])
    assert np.isfinite(ax).all() and np.isfinite(ay).all()
    assert abs(ax[0]) < 1e-6 and abs(ay[0]) < 1e-6
