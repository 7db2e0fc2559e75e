"""Pins of the backward-intensity oracle (oracle/backward.py): linearity of
the model in the intensities, exact recovery from noiseless data, vanishing
intensity derivative at the solution, and the envelope-theorem gradient
against finite differences of the profile log p (re-solving every time)."""
import numpy as np
import pytest

import oracle
from oracle import backward as BW
from lenscase import make_case, small_workload


@pytest.fixture(scope="module")
def case():
    return make_case(small_workload(24, 24, 2, 5, 1, 1, seed=313))


def test_model_is_linear_in_the_intensities(case):
    th = case.truth.copy()
    M = BW.component_images(case.oracle, th)
    idx = BW.intensity_indices(1, 1)
    full = case.oracle.model_image(th)[0]
    assert np.allclose(full, np.tensordot(th[idx], M, axes=1), rtol=1e-12, atol=1e-12)


def test_noiseless_data_gives_the_true_intensities(case):
    W = case.W
    m = case.oracle.model_image(case.truth)[0]
    clean = oracle.System(W.ny, W.nx, W.pixel_scale, W.supersample, m, case.sigma, case.psf,
                          1, 1, case.spec)
    I = BW.solve_intensities(clean, case.truth)
    assert np.allclose(I, case.truth[BW.intensity_indices(1, 1)], rtol=1e-9)


def test_intensity_derivative_vanishes_at_the_solution(case):
    prof = BW.profile_system(case.oracle, case.spec)
    th = case.truth + 0.002 * np.random.default_rng(1).normal(size=case.truth.size)
    lp, g, I = BW.logp_grad_backward(case.oracle, prof, th)
    th2 = th.copy()
    th2[BW.intensity_indices(1, 1)] = I[0]
    _, graw = prof.logp_grad(th2)
    idx = BW.intensity_indices(1, 1)
    assert np.all(np.abs(graw[0, idx]) * np.abs(I[0]) < 1e-6 * np.abs(lp[0]) + 1e-6)
    assert np.all(g[0, idx] == 0.0)


def test_envelope_gradient_matches_finite_differences(case):
    prof = BW.profile_system(case.oracle, case.spec)
    th = case.truth + 0.001 * np.random.default_rng(2).normal(size=case.truth.size)
    lp, g, _ = BW.logp_grad_backward(case.oracle, prof, th)
    idx = set(BW.intensity_indices(1, 1))
    h = 1e-6
    for k in range(th.size):
        if k in idx:
            continue
        e = np.zeros(th.size)
        e[k] = h
        fd = (BW.logp_grad_backward(case.oracle, prof, th + e)[0][0]
              - BW.logp_grad_backward(case.oracle, prof, th - e)[0][0]) / (2 * h)
        assert abs(g[0, k] - fd) <= 2e-5 * max(1.0, abs(fd)), (k, g[0, k], fd)
