"""Edge cases of the inference layer on the GPU: the half-bounded and flat
bijector maps, ragged batch sizes (rows not a multiple of the 8 rows per
block), a chain started at NaN, empty calls, and an SVI step with a ragged
sample count."""
import numpy as np
import pytest

import oracle
import synth
from lenscase import f32, make_case, round_spec, small_workload
from oracle import infer as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def case():
    return make_case(small_workload(32, 32, 2, 7, 1, 1, seed=1601))


def _t(torch, a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


def test_half_bounded_and_flat_maps(torch, case):
    import paper_2606_30633_b300 as gl
    ps = list(case.spec.params)
    ps[6] = synth.Prior("flat", 0.0, 1.0, -0.2, np.inf)      # shear g1: [lo, inf)
    ps[7] = synth.Prior("flat", 0.0, 1.0, -np.inf, 0.3)      # shear g2: (-inf, hi]
    ps[12] = synth.Prior("flat", 0.0, 1.0, -np.inf, np.inf)  # lens-light x: R
    ps[13] = synth.Prior("flat", 0.0, 1.0, -1.0, 1.0)        # lens-light y: [lo, hi]
    spec = round_spec(synth.PriorSpec(ps, case.spec.emax))
    W = case.W
    s = gl.System(W.ny, W.nx, W.pixel_scale, W.supersample, case.data, case.sigma, case.psf, 1, 1,
                  spec)
    bij = I.Bijector.from_spec(spec)
    assert bij.mode[6] == I.LOWER and bij.mode[7] == I.UPPER
    assert bij.mode[12] == I.ID and bij.mode[13] == I.INTERVAL
    u = f32(np.random.default_rng(2).normal(0, 1.2, size=(13, s.P)))
    th, lj = s.bijector_forward(_t(torch, u))
    th_o, lj_o = bij.forward(u)
    assert np.allclose(th.cpu().numpy(), th_o, rtol=2e-7, atol=1e-9)
    assert np.allclose(lj.cpu().numpy(), lj_o, rtol=2e-7, atol=2e-6)
    back = s.bijector_inverse(th).cpu().numpy()
    assert np.allclose(back, bij.inverse(th.cpu().numpy().astype(np.float64)), rtol=1e-5,
                       atol=1e-5)
    s.close()


@pytest.mark.parametrize("B", [1, 9])
def test_ragged_batches_of_the_unconstrained_gradient(torch, case, B):
    s = case.gpu_system()
    bij = I.Bijector.from_spec(case.spec)
    th = f32(synth.jitter(case.truth, case.W.prior(), B, 4, rel=0.003))
    u = f32(bij.inverse(th))
    lp, g = s.logp_grad_unconstrained(_t(torch, u))
    lp_o, g_o = I.logp_grad_unconstrained(case.oracle, bij, u)
    assert np.all(np.abs(lp.cpu().numpy() - lp_o) <= 2e-5 * np.abs(lp_o) + 1e-2)
    assert np.all(np.isfinite(g.cpu().numpy()))


def test_empty_and_zero_step_calls(torch, case):
    s = case.gpu_system()
    z = torch.zeros(0, s.P, device="cuda")
    th, lj = s.bijector_forward(z)
    assert th.shape == (0, s.P) and lj.shape == (0,)
    u = torch.zeros(4, s.P, device="cuda")
    m, v = torch.zeros_like(u), torch.zeros_like(u)
    before = u.clone()
    s.map_adam(u, m, v, 0)
    assert torch.equal(u, before)


def test_hmc_with_ragged_chains_and_a_nan_start(torch, case):
    import paper_2606_30633_b300 as gl
    B, L, eps, seed = 5, 2, 1e-3, 9
    bij = I.Bijector.from_spec(case.spec)
    u0 = f32(bij.inverse(f32(synth.jitter(case.truth, case.W.prior(), B, 12, rel=0.003))))
    u0[2, :] = np.nan
    h = gl.Hmc(case.gpu_system(), _t(torch, u0), L, eps, seed=seed)
    h.run(2)
    u, lp, _, _ = h.state()
    h.close()
    u, lp = u.cpu().numpy(), lp.cpu().numpy()
    assert np.isnan(lp[2]) and np.all(np.isnan(u[2]))
    good = [0, 1, 3, 4]
    assert np.all(np.isfinite(lp[good])) and np.all(np.isfinite(u[good]))
    # the finite chains follow the oracle's transitions on the same draws
    lg = lambda x: I.logp_grad_unconstrained(case.oracle, bij, x)
    uo = u0[good].copy()
    lpo, go = lg(uo)
    for step in range(2):
        z, a = I.hmc_draws(seed, step, B, u0.shape[1])
        uo, lpo, go, _, _ = I.hmc_transition(uo, lpo, go, np.ones(u0.shape[1]), eps, L,
                                             z[good], a[good], lg)
    assert np.allclose(u[good], uo, atol=5e-5)


def test_svi_step_with_a_ragged_sample_count(torch, case):
    from paper_2606_30633_b300 import infer
    s = case.gpu_system()
    bij = I.Bijector.from_spec(case.spec)
    P = s.P
    n, seed = 37, 5
    mu0 = f32(bij.inverse(case.truth[None]))[0]
    phi, opt = infer.svi_init(s, _t(torch, mu0), scale=0.01)
    phi0 = phi.cpu().numpy().astype(np.float64)
    elbo = s.svi_adabelief(phi, opt, n, 1, seed=seed).cpu().numpy()
    Lr = phi0[P:].reshape(P, P)
    L = np.tril(Lr, -1) + np.diag(np.exp(np.diag(Lr)))
    z = I.svi_draws(seed, 0, n, P)
    w, _ = I.svi_terms(phi0[:P], L, z, lambda x: I.logp_unconstrained(case.oracle, bij, x))
    assert abs(elbo[0] - w.mean()) <= 1e-4 * abs(w.mean()) + 0.05
