"""HMC leapfrog blocks (gl_leapfrog, one CUDA graph per block) against the same
integrator written with gl_logp_grad and torch, against an FP64 integrator on
the oracle, and against the integrator's own invariants (time reversibility,
energy conservation to O(eps^2)); divergent chains are frozen."""
import numpy as np
import pytest

import synth
from lenscase import make_case, small_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2606_30633_b300 import build
    build.build()
    c = make_case(small_workload(28, 28, 2, 11, 1, 1, seed=71))
    return torch, c, c.gpu_system()


def _start(torch, c, n, seed=1, rel=0.01):
    th = synth.jitter(c.truth, c.W.prior(), n, seed, rel=rel)
    th[0] = c.truth
    spec = c.W.prior()
    widths = np.array([(p.hi - p.lo) / np.sqrt(12) if p.kind == "uniform" else
                       (np.exp(p.a) * p.b if p.kind == "lognormal" else p.b) for p in spec.params])
    inv_mass = (widths ** 2).astype(np.float32)  # M^-1 = prior variance scale
    p0 = np.random.default_rng(seed + 1).standard_normal(th.shape) / np.sqrt(inv_mass)
    dev = "cuda"
    return (torch.tensor(th, dtype=torch.float32, device=dev),
            torch.tensor(p0, dtype=torch.float32, device=dev),
            torch.tensor(inv_mass, device=dev))


def test_graph_block_matches_explicit_loop(env):
    torch, c, s = env
    th, p, im = _start(torch, c, 16)
    eps, L = 2e-3, 10
    lp, g = s.logp_grad(th)
    # explicit integrator through gl_logp_grad
    th2, p2 = th.clone(), p.clone()
    lp2, g2 = lp.clone(), g.clone()
    for _ in range(L):
        p2 = torch.addcmul(p2, g2, torch.full_like(g2, 0.5 * eps))
        th2 = th2 + eps * im * p2
        lp2, g2 = s.logp_grad(th2)
        p2 = p2 + 0.5 * eps * g2
    s.leapfrog(th, p, lp, g, im, eps, L)
    torch.cuda.synchronize()
    torch.testing.assert_close(th, th2, rtol=2e-6, atol=1e-7)
    torch.testing.assert_close(p, p2, rtol=1e-4, atol=1e-3)
    torch.testing.assert_close(lp, lp2, rtol=1e-6, atol=1e-3)


def test_matches_fp64_integrator_on_the_oracle(env):
    torch, c, s = env
    th, p, im = _start(torch, c, 4, seed=3)
    eps, L = 2e-3, 10
    lp, g = s.logp_grad(th)
    th64, p64, im64 = th.double().cpu().numpy(), p.double().cpu().numpy(), im.double().cpu().numpy()
    s.leapfrog(th, p, lp, g, im, eps, L)
    _, gr = c.oracle.logp_grad(th64)
    t0 = th64.copy()
    for _ in range(L):
        p64 = p64 + 0.5 * eps * gr
        th64 = th64 + eps * im64 * p64
        lr, gr = c.oracle.logp_grad(th64)
        p64 = p64 + 0.5 * eps * gr
    moved = th64 - t0
    got = th.double().cpu().numpy() - t0
    err = np.abs(got - moved)
    assert np.all(err <= 2e-3 * np.abs(moved) + 2e-6 * np.abs(t0) + 1e-7), float(err.max())


def test_reversible_and_second_order_in_energy(env):
    """Time reversibility (negate p, integrate back to the start) and the
    leapfrog's O(eps^2) energy error at fixed trajectory time: halving eps
    (doubling the steps) cuts |H1 - H0| by about 4."""
    torch, c, s = env
    dH = []
    for eps, L in ((2e-3, 10), (1e-3, 20)):
        th, p, im = _start(torch, c, 8, seed=5)
        lp, g = s.logp_grad(th)
        th0 = th.clone()
        H0 = -lp.double() + 0.5 * (p.double() ** 2 * im.double()).sum(1)
        s.leapfrog(th, p, lp, g, im, eps, L)
        H1 = -lp.double() + 0.5 * (p.double() ** 2 * im.double()).sum(1)
        dH.append(float(torch.abs(H1 - H0).sum()))
        p.neg_()
        s.leapfrog(th, p, lp, g, im, eps, L)
        torch.cuda.synchronize()
        torch.testing.assert_close(th, th0, rtol=1e-5, atol=2e-6)
    assert dH[0] > 1e-2, dH          # well above the FP32 noise floor of H
    assert 0.12 < dH[1] / dH[0] < 0.4, dH


def test_divergent_chains_are_frozen_and_graph_recaptures(env):
    torch, c, s = env
    th, p, im = _start(torch, c, 6, seed=7)
    th[2, 0] = 3.0  # outside the theta_E prior: -inf at the start
    lp, g = s.logp_grad(th)
    frozen = th[2].clone()
    s.leapfrog(th, p, lp, g, im, 1e-3, 5)
    s.leapfrog(th, p, lp, g, im, 1e-3, 5)   # same arguments: graph replay
    s.leapfrog(th, p, lp, g, im, 5e-4, 3)   # new eps and length: re-capture
    torch.cuda.synchronize()
    assert torch.isneginf(lp[2]) and torch.equal(th[2], frozen)
    assert torch.isfinite(lp[[0, 1, 3, 4, 5]]).all()
    lp_chk, g_chk = s.logp_grad(th)
    torch.testing.assert_close(lp[[0, 1, 3, 4, 5]], lp_chk[[0, 1, 3, 4, 5]])
    torch.testing.assert_close(g[[0, 1, 3, 4, 5]], g_chk[[0, 1, 3, 4, 5]])


def test_space_block_matches_fp64_integrator():
    """One graph block of the space-telescope workload (200 x 200 px at
    0.05"/px, s = 5, 21 x 21 Gaussian-core PSF, two source components: the
    image buffers live in global scratch) against the FP64 integrator on the
    oracle, for 4 chains started near the truth: 10 leapfrogs with the
    benchmark's step scale. Positions agree to the same bound as the small
    case's."""
    import torch
    c = make_case(synth.space_200())
    s = c.gpu_system()
    th, p, im = _start(torch, c, 4, seed=5, rel=0.002)
    eps, L = 1e-4, 10
    lp, g = s.logp_grad(th)
    th64, p64, im64 = th.double().cpu().numpy(), p.double().cpu().numpy(), im.double().cpu().numpy()
    h0 = lp.double().cpu().numpy() - 0.5 * np.sum(im64 * p64 ** 2, 1)
    s.leapfrog(th, p, lp, g, im, eps, L)
    torch.cuda.synchronize()
    _, gr = c.oracle.logp_grad(th64)
    t0 = th64.copy()
    for _ in range(L):
        p64 = p64 + 0.5 * eps * gr
        th64 = th64 + eps * im64 * p64
        lr, gr = c.oracle.logp_grad(th64)
        p64 = p64 + 0.5 * eps * gr
    h1 = lr - 0.5 * np.sum(im64 * p64 ** 2, 1)
    moved = th64 - t0
    got = th.double().cpu().numpy() - t0
    err = np.abs(got - moved)
    lpg = lp.double().cpu().numpy()
    print(f"\nspace block: |dH| (FP64) {np.array2string(np.abs(h1 - h0), precision=3)}; position err / "
          f"bound max {(err / (2e-3 * np.abs(moved) + 2e-6 * np.abs(t0) + 1e-7)).max():.3f}; "
          f"log p rel err {np.abs(lpg - lr).max() / np.abs(lr).max():.2e}")
    assert np.all(np.isfinite(lpg))
    assert np.all(err <= 2e-3 * np.abs(moved) + 2e-6 * np.abs(t0) + 1e-7), float(err.max())
    assert np.all(np.abs(lpg - lr) <= 1e-5 * np.abs(lr))
    s.close()
