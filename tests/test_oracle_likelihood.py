"""Pins of the oracle's likelihood, prior and dual-number gradient."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import synth


def _small(ny=20, nx=20, s=2, seed=11):
    W = synth.ground_60()
    spec = W.prior()
    psf = synth.moffat_psf(5, 0.262, 1.1)
    th0 = W.truth()
    S0 = oracle.System(ny, nx, 0.262, s, np.zeros((ny, nx)), np.ones((ny, nx)), psf, 1, 1, spec)
    m = S0.model_image(th0)[0]
    d, sig = synth.noisy_data(m, synth.noise_draws((ny, nx), seed))
    return oracle.System(ny, nx, 0.262, s, d, sig, psf, 1, 1, spec), th0, spec, m, sig


def test_model_equal_to_data_gives_zero_likelihood():
    S, th0, spec, m, sig = _small()
    S2 = oracle.System(S.ny, S.nx, 0.262, 2, m, sig, S.psf, 1, 1, spec)
    assert abs(S2.log_likelihood(th0)) < 1e-20
    assert S2.logp(th0)[0] == pytest.approx(S2.log_prior(th0), rel=1e-15)


def test_hand_computed_chi2_two_by_two():
    """All intensities zero: m = 0, so log L = -1/2 sum (d/sigma)^2 by hand."""
    spec = synth.config_prior(1, 1)
    d = np.array([[1.0, -2.0], [0.5, 3.0]])
    sig = np.array([[1.0, 2.0], [0.5, 1.5]])
    S = oracle.System(2, 2, 0.262, 2, d, sig, np.ones((3, 3)), 1, 1, spec)
    th = synth.ground_60().truth().copy()
    th[14] = 0.0
    th[21] = 0.0
    assert S.log_likelihood(th) == pytest.approx(-0.5 * (1 + 1 + 1 + 4), rel=1e-15)


def test_log_prior_matches_scipy():
    spec = synth.config_prior(1, 1)
    S = oracle.System(2, 2, 0.262, 1, np.zeros((2, 2)), np.ones((2, 2)), np.ones((1, 1)), 1, 1,
                      spec)
    th = synth.draw(spec, 5, 17)
    for row in th:
        ref = 0.0
        for x, pr in zip(row, spec.params):
            if pr.kind == "uniform":
                ref += stats.uniform(pr.lo, pr.hi - pr.lo).logpdf(x)
            elif pr.kind == "normal":
                ref += stats.norm(pr.a, pr.b).logpdf(x)
            elif pr.kind == "truncnorm":
                ref += stats.truncnorm((pr.lo - pr.a) / pr.b, (pr.hi - pr.a) / pr.b,
                                       loc=pr.a, scale=pr.b).logpdf(x)
            elif pr.kind == "lognormal":
                ref += stats.lognorm(s=pr.b, scale=math.exp(pr.a)).logpdf(x)
        assert S.log_prior(row) == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_support_domain_and_nan():
    S, th0, spec, m, sig = _small(8, 8, 1)
    bad = []
    t = th0.copy(); t[0] = 3.0; bad.append(t)            # theta_E above U(0.8, 2.5)
    t = th0.copy(); t[2], t[3] = 0.4, 0.35; bad.append(t)  # |e_EPL| >= 0.5 disc
    t = th0.copy(); t[10] = 0.2; bad.append(t)            # lens-light e1 outside TN support
    t = th0.copy(); t[21] = -1.0; bad.append(t)           # lognormal intensity <= 0
    lp, g = S.logp_grad(np.array(bad))
    assert np.all(np.isneginf(lp))
    assert np.all(g == 0.0)
    t = th0.copy(); t[5] = np.nan
    lp, g = S.logp_grad(t)
    assert np.isnan(lp[0]) and np.all(np.isnan(g))
    assert np.isnan(S.logp(t)[0])


def test_model_domain_of_the_slope():
    """The EPL exists for 1 < gamma < 3 (t = gamma - 1 in (0, 2)): with a prior
    that does not bound gamma, log p is -inf outside that range and finite
    inside it."""
    S, th0, spec, m, sig = _small(8, 8, 1)
    ps = list(spec.params)
    ps[1] = synth.Prior("normal", 2.0, 1.0)
    wide = synth.PriorSpec(ps, spec.emax)
    S2 = oracle.System(8, 8, 0.262, 1, S.data, S.sigma, S.psf, 1, 1, wide)
    rows = np.repeat(th0[None], 4, 0)
    rows[:, 1] = [0.95, 1.05, 2.95, 3.05]
    lp = S2.logp(rows)
    assert np.isneginf(lp[[0, 3]]).all() and np.isfinite(lp[[1, 2]]).all()


@pytest.mark.parametrize("which", ["truth", "draw0", "draw1"])
def test_dual_gradient_matches_central_differences(which):
    """Forward-mode dual-number gradient against FP64 central differences,
    h = 1e-6 max(|theta|, 1), on every parameter."""
    S, th0, spec, m, sig = _small(16, 16, 2)
    if which == "truth":
        th = th0
    else:
        th = synth.draw(spec, 2, 5)[int(which[-1])]
    lp, g = S.logp_grad(th)
    fd = np.empty_like(th)
    for k in range(th.size):
        h = 1e-6 * max(abs(th[k]), 1.0)
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd[k] = (S.logp(tp)[0] - S.logp(tm)[0]) / (2 * h)
    scale = np.max(np.abs(fd))
    err = np.abs(g - fd)
    assert np.all(err <= 1e-5 * np.maximum(np.abs(fd), 1e-3 * scale)), (g, fd)
    assert lp[0] == pytest.approx(S.logp(th)[0], rel=1e-14)


def test_jacobian_is_consistent_with_gradient_and_differences():
    """d logp/d theta = sum_p (d_p - m_p)/sigma_p^2 dm_p/dtheta + dlog prior, and
    the Jacobian matches central differences of the model image."""
    S, th0, spec, m, sig = _small(12, 12, 2)
    th = synth.draw(spec, 1, 8)[0]
    mm, J = S.model_jacobian(th)
    np.testing.assert_allclose(mm, S.model_image(th)[0], rtol=1e-14)
    lp, g = S.logp_grad(th)
    gp = np.empty_like(th)
    for k in range(th.size):  # prior gradient by differences of the log prior
        h = 1e-6 * max(abs(th[k]), 1.0)
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        gp[k] = (S.log_prior(tp) - S.log_prior(tm)) / (2 * h)
        fd = (S.model_image(tp)[0] - S.model_image(tm)[0]) / (2 * h)
        np.testing.assert_allclose(J[:, :, k], fd, rtol=1e-5, atol=1e-7 * np.abs(fd).max() + 1e-12)
    gl = np.einsum("ij,ijk->k", (S.data - mm) / S.sigma ** 2, J)
    np.testing.assert_allclose(g[0], gl + gp, rtol=1e-6, atol=1e-6 * np.abs(g).max())
