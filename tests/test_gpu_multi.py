"""Uneven multi-system batches (gl_multi_*): one persistent launch per
component-count group reproduces gl_logp_grad of every system bit for bit, in
every shared-memory policy and deflection kind; the autotuner returns the
fastest policy."""
import numpy as np
import pytest

import synth
from lenscase import make_case, small_workload

pytestmark = pytest.mark.gpu

MIX = [  # ny, nx, s, psf, n_light, n_src, rows
    (24, 24, 2, 11, 1, 1, 5),
    (40, 33, 3, 5, 1, 2, 3),
    (17, 20, 1, 11, 1, 3, 4),
    (64, 64, 2, 21, 1, 1, 2),   # two 84x84 buffers: global scratch under "two CTAs"
    (30, 30, 2, 11, 0, 1, 3),
    (20, 25, 4, 3, 2, 2, 2),
]


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2606_30633_b300 import build
    build.build()
    import paper_2606_30633_b300 as gl
    cases, systems, thetas = [], [], []
    for k, (ny, nx, s, K, nl, ns, rows) in enumerate(MIX):
        c = make_case(small_workload(ny, nx, s, K, nl, ns, seed=900 + 7 * k))
        th = c.theta(rows)
        th[0] = c.truth
        cases.append(c)
        systems.append(c.gpu_system())
        thetas.append(torch.tensor(th, dtype=torch.float32, device="cuda"))
    return torch, gl, cases, systems, thetas


@pytest.mark.parametrize("policy", [0, 1, 2])
@pytest.mark.parametrize("defl", ["series", "table"])
def test_multi_matches_per_system(env, policy, defl):
    torch, gl, cases, systems, thetas = env
    d = gl.GL_DEFL_SERIES if defl == "series" else gl.GL_DEFL_TABLE
    plan = gl.Multi(systems, [t.shape[0] for t in thetas], policy)
    lps, gs = plan.logp_grad(thetas, defl=d)
    lps2, gs2 = plan.logp_grad(thetas, lps, gs, defl=d)  # second call reuses the work lists
    torch.cuda.synchronize()
    for s, t, lp, g in zip(systems, thetas, lps2, gs2):
        rl, rg = s.logp_grad(t, defl=d)
        np.testing.assert_array_equal(lp.cpu().numpy(), rl.cpu().numpy())
        np.testing.assert_array_equal(g.cpu().numpy(), rg.cpu().numpy())


def test_multi_against_the_oracle(env):
    torch, gl, cases, systems, thetas = env
    plan = gl.Multi(systems, [t.shape[0] for t in thetas], gl.GL_MULTI_SMEM_TWO_CTAS)
    lps, _ = plan.logp_grad(thetas)
    for c, t, lp in zip(cases, thetas, lps):
        ref = c.oracle.logp(t.double().cpu().numpy())
        assert np.all(np.abs(lp.cpu().numpy() - ref) <= 1e-5 * np.abs(ref) + 2e-3)


def test_autotuner_returns_the_fastest_policy(env):
    torch, gl, cases, systems, thetas = env
    from paper_2606_30633_b300 import autotune
    best, times = autotune.tune_multi(systems, [t.shape[0] for t in thetas], thetas, reps=2)
    assert set(times) == {"global", "two_ctas", "one_cta"}
    assert times[min(times, key=times.get)] == min(times.values())
    assert best.smem_policy == autotune.POLICIES[min(times, key=times.get)]


@pytest.mark.parametrize("defl", ["series", "table"])
def test_systems_without_rows(env, defl):
    """Systems with zero rows are skipped, including a whole component-count
    group without rows; the others still match their own gl_logp_grad bit for
    bit. A plan in which no system has rows launches nothing and succeeds."""
    torch, gl, cases, systems, thetas = env
    d = gl.GL_DEFL_SERIES if defl == "series" else gl.GL_DEFL_TABLE
    th = [t if k % 2 == 0 else t[:0] for k, t in enumerate(thetas)]
    plan = gl.Multi(systems, [t.shape[0] for t in th], gl.GL_MULTI_SMEM_TWO_CTAS)
    lps, gs = plan.logp_grad(th, defl=d)
    torch.cuda.synchronize()
    for s, t, lp, g in zip(systems, th, lps, gs):
        assert lp.shape[0] == t.shape[0] and g.shape == t.shape
        if t.shape[0]:
            rl, rg = s.logp_grad(t, defl=d)
            np.testing.assert_array_equal(lp.cpu().numpy(), rl.cpu().numpy())
            np.testing.assert_array_equal(g.cpu().numpy(), rg.cpu().numpy())
    none = gl.Multi(systems, [0] * len(systems), gl.GL_MULTI_SMEM_GLOBAL)
    lps, gs = none.logp_grad([t[:0] for t in thetas], defl=d)
    torch.cuda.synchronize()
    assert all(lp.numel() == 0 for lp in lps) and all(g.numel() == 0 for g in gs)
