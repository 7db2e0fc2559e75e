"""Pins of the FP64 reference MLP used to check the surrogate's tensor-core
kernels: BF16 rounding against known values, and the backward pass against
central differences in exact arithmetic."""
import mpmath
import numpy as np

import oracle
import oracle.mlp as mlp


def test_bf16_rounding_is_nearest_even():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -2.5, 3.14159])
    np.testing.assert_array_equal(mlp.bf16(v), [1.0, 1.0, 1.0 + 2 ** -6, 1.0, -2.5, 3.140625])


def test_backward_matches_central_differences():
    rng = np.random.default_rng(3)
    p = rng.normal(size=mlp.NPARAM) * 0.3
    X = np.stack([rng.uniform(0.5, 1, 6), rng.uniform(1.7, 2.3, 6), rng.uniform(-3, 1.6, 6),
                  rng.uniform(0, 2 * np.pi, 6)], 1)
    T = rng.normal(size=(6, 2))
    loss, g = mlp.loss_grad(p, X, T, rounding=False)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    for k in idx:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (mlp.loss_grad(pp, X, T, rounding=False)[0] - mlp.loss_grad(pm, X, T, rounding=False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_base_terms_are_the_first_series_terms():
    """1 + c1 z + c2 z^2 agrees with 2F1 to O(f^3) (mpmath)."""
    q, gamma, vp = 0.95, 2.1, 0.7
    X = np.array([[q, gamma, 0.0, vp]])
    f = (1 - q) / (1 + q)
    t = gamma - 1
    F = complex(mpmath.hyp2f1(1, t / 2, 2 - t / 2, -f * mpmath.exp(2j * vp)))
    assert abs(mlp.base_F(X)[0] - F) < 2 * f ** 3
    assert abs(oracle.hyp2f1_series(t, f, vp) - F) < 1e-14


def test_network_output_definition(monkeypatch):
    """surrogate_F = base terms + z^3 y / OUT_SCALE: with y set to OUT_SCALE x
    (2F1 - base terms) / z^3 from mpmath, it returns 2F1 (a wrong power of z or
    scale fails); and that y stays O(1) across the training domain."""
    pts = [(0.5, 1.7, 0.3), (0.5, 2.3, 2.2), (0.62, 2.0, 4.0), (0.9, 1.85, 5.5), (0.99, 2.2, 1.1)]
    X = np.array([[q, g, 0.0, vp] for q, g, vp in pts])
    F = np.empty(len(pts), complex)
    Y = np.empty((len(pts), 2))
    for k, (q, g, vp) in enumerate(pts):
        mpmath.mp.dps = 40
        f = mpmath.mpf(1 - q) / (1 + q)
        t = mpmath.mpf(g) - 1
        z = -f * mpmath.exp(2j * mpmath.mpf(vp))
        c1 = t / (4 - t)
        c2 = c1 * (2 + t) / (6 - t)
        Fm = mpmath.hyp2f1(1, t / 2, 2 - t / 2, z)
        y = mlp.OUT_SCALE * (Fm - (1 + c1 * z + c2 * z * z)) / z ** 3
        F[k] = complex(Fm)
        Y[k] = [float(mpmath.re(y)), float(mpmath.im(y))]
    assert np.all(np.abs(Y) < 2.0) and np.all(np.abs(Y).max(1) > 0.1)
    monkeypatch.setattr(mlp, "forward", lambda params, X, rounding=True: (Y, None))
    np.testing.assert_allclose(mlp.surrogate_F(None, X), F, rtol=0, atol=1e-12)
