"""The host-side convergence diagnostics of the inference layer
(paper_2606_30633_b300.infer: FFT autocovariances) against the oracle's
direct-sum implementation, and against the closed forms the oracle is
pinned to."""
import math

import numpy as np
import pytest

from oracle import infer as I


@pytest.fixture(scope="module")
def host():
    from paper_2606_30633_b300 import infer
    return infer


def _ar1(rng, N, M, r, offsets=None):
    x = np.empty((N, M))
    x[0] = rng.normal(size=M)
    e = rng.normal(size=(N, M)) * math.sqrt(1 - r * r)
    for t in range(1, N):
        x[t] = r * x[t - 1] + e[t]
    if offsets is not None:
        x += offsets
    return x


@pytest.mark.parametrize("r", [0.0, 0.3, 0.8])
def test_rhat_and_ess_match_the_oracle(host, r):
    rng = np.random.default_rng(int(r * 10) + 1)
    x = _ar1(rng, 600, 5, r)[:, :, None] * np.array([1.0, 3.0])  # two parameters
    assert np.allclose(host.rhat(x), I.rhat(x), rtol=1e-12)
    assert np.allclose(host.ess(x), I.ess(x), rtol=1e-9)


def test_rhat_flags_separated_chains(host):
    rng = np.random.default_rng(9)
    x = _ar1(rng, 500, 4, 0.2, offsets=np.array([0.0, 0.0, 0.0, 3.0]))
    assert host.rhat(x) > 1.1
    assert abs(host.rhat(rng.normal(size=(2000, 6))) - 1.0) < 0.01


def test_ess_closed_form(host):
    rng = np.random.default_rng(4)
    N, M, r = 4000, 4, 0.6
    x = _ar1(rng, N, M, r)
    want = N * M * (1 - r) / (1 + r)
    assert abs(host.ess(x) - want) < 0.15 * want
