"""GPU parity of the inference layer (bijector, log p~ and its gradient,
multi-start MAP with Adam, HMC transitions, SVI steps) against the FP64
oracle (oracle/infer.py) on the same inputs and the same counter-based
random numbers."""
import math

import numpy as np
import pytest

import synth
from lenscase import f32, grad_bound, make_case, small_workload
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
    return make_case(small_workload(40, 40, 2, 11, 1, 1, seed=1201))


@pytest.fixture(scope="module")
def bij(case):
    return I.Bijector.from_spec(case.spec)


@pytest.fixture(scope="module")
def sysg(torch, case):
    return case.gpu_system()


def _u_near_mode(case, bij, n, seed):
    th = f32(synth.jitter(case.truth, case.W.prior(), n, seed, rel=0.003))
    th[0] = case.truth
    return f32(bij.inverse(th))


def _u_prior(case, bij, n, seed):
    return f32(bij.inverse(case.theta(n, seed=seed)))


def _lg(case, bij):
    return lambda u: I.logp_grad_unconstrained(case.oracle, bij, u)


def test_bijector_matches_oracle(torch, sysg, bij):
    rng = np.random.default_rng(3)
    u = f32(rng.normal(0, 1.5, size=(64, sysg.P)))
    u[0, 2:4] = 0.0      # EPL ellipticity at the disc centre
    u[1, 2:4] = [2e-4, -1e-4]
    ug = torch.tensor(u, dtype=torch.float32, device="cuda")
    th, lj = sysg.bijector_forward(ug)
    th_o, lj_o = bij.forward(u)
    th = th.cpu().numpy()
    assert np.all(np.abs(th - th_o) <= 2e-7 * np.abs(th_o) + 1e-9), np.abs(th - th_o).max()
    assert np.allclose(lj.cpu().numpy(), lj_o, rtol=2e-7, atol=2e-6)
    ui = sysg.bijector_inverse(torch.tensor(th, dtype=torch.float32, device="cuda")).cpu().numpy()
    uo = bij.inverse(th.astype(np.float64))
    assert np.all(np.abs(ui - uo) <= 1e-5 * np.abs(uo) + 1e-5), np.abs(ui - uo).max()


@pytest.mark.parametrize("where", ["mode", "prior"])
def test_unconstrained_logp_and_gradient_match_oracle(torch, case, sysg, bij, where):
    u = _u_near_mode(case, bij, 8, 5) if where == "mode" else _u_prior(case, bij, 8, 6)
    lp, g = sysg.logp_grad_unconstrained(torch.tensor(u, dtype=torch.float32, device="cuda"))
    lp, g = lp.cpu().numpy(), g.cpu().numpy()
    lp_o, g_o = I.logp_grad_unconstrained(case.oracle, bij, u)
    assert np.all(np.abs(lp - lp_o) <= 2e-5 * np.abs(lp_o) + 1e-2), np.abs(lp - lp_o).max()
    th_o, _ = bij.forward(u)
    J = np.abs(bij.jacobian(u))
    bound = np.einsum("bij,bi->bj", J, grad_bound(case, th_o)) + 1e-5 * np.abs(g_o) + 1e-6
    err = np.abs(g - g_o)
    assert np.all(err <= bound), float((err / bound).max())


def test_map_adam_first_step_and_trajectory(torch, case, sysg, bij):
    u0 = _u_near_mode(case, bij, 12, 7)
    lr = 1e-3
    u = torch.tensor(u0, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(u)
    v = torch.zeros_like(u)
    lp = sysg.map_adam(u, m, v, 1, lr=lr).cpu().numpy()
    lp_o, g_o = I.logp_grad_unconstrained(case.oracle, bij, u0)
    assert np.all(np.abs(lp - lp_o) <= 2e-5 * np.abs(lp_o) + 1e-2)
    # Adam's first step moves every coordinate by lr g/(|g| + eps): lr sign(g)
    th_o, _ = bij.forward(u0)
    gb = np.einsum("bij,bi->bj", np.abs(bij.jacobian(u0)), grad_bound(case, th_o))
    step = u.cpu().numpy() - u0
    sure = np.abs(g_o) > 2 * gb
    assert sure.mean() > 0.5
    assert np.all(np.abs(step[sure] - lr * np.sign(g_o[sure])) <= 1e-3 * lr + 1e-6)
    assert np.all(np.abs(step) <= lr * (1 + 1e-5) + 1e-6)
    # 40 more steps on the GPU against the FP64 Adam from the same start
    lp40 = sysg.map_adam(u, m, v, 40, t0=1, lr=lr).cpu().numpy()
    _, hist = I.adam(u0, _lg(case, bij), 41, lr=lr)
    assert np.all(lp40 > lp)  # ascending
    assert np.all(np.abs(lp40 - hist[-1]) <= 1e-4 * np.abs(hist[-1]) + 0.5), \
        np.abs(lp40 - hist[-1]).max()


def test_hmc_transition_matches_oracle(torch, case, sysg, bij):
    import paper_2606_30633_b300 as gl
    B, L, eps, seed = 48, 3, 1.5e-3, 123
    u0 = _u_near_mode(case, bij, B, 9)
    h = gl.Hmc(sysg, torch.tensor(u0, dtype=torch.float32, device="cuda"), L, eps, seed=seed)
    draws = torch.empty(1, B, sysg.P, device="cuda")
    acc = torch.empty(1, device="cuda")
    h.run(1, 0, draws, acc)
    ug, lpg, im, eps_out = h.state()
    h.close()
    ug, lpg = ug.cpu().numpy(), lpg.cpu().numpy()
    assert eps_out == pytest.approx(eps) and np.all(im.cpu().numpy() == 1.0)
    z, a = I.hmc_draws(seed, 0, B, sysg.P)
    lp0, g0 = I.logp_grad_unconstrained(case.oracle, bij, u0)
    uo, lpo, _, prob, acc_o = I.hmc_transition(u0, lp0, g0, np.ones(sysg.P), eps, L, z, a,
                                               _lg(case, bij))
    log_acc = np.log(np.maximum(prob, 1e-300))
    robust = np.abs(np.log(a) - log_acc) > 0.05
    moved = np.any(ug != u0, axis=1)
    assert robust.sum() >= B // 2
    assert np.all(moved[robust] == acc_o[robust])
    both = robust & acc_o
    assert both.sum() >= 5
    assert np.allclose(ug[both], uo[both], atol=2e-5, rtol=0)
    assert np.allclose(lpg[both], lpo[both], rtol=2e-5, atol=1e-2)
    # recorded draws are theta(u) of the new state
    assert np.allclose(draws[0].cpu().numpy(), bij.forward(ug)[0], rtol=1e-6, atol=1e-7)
    assert abs(float(acc[0]) - prob.mean()) < 0.02


def test_hmc_sampling_with_adaptation(torch, case, sysg, bij):
    from paper_2606_30633_b300 import infer
    B = 96
    u0 = torch.tensor(_u_near_mode(case, bij, B, 11), dtype=torch.float32, device="cuda")
    res = infer.hmc_sample(sysg, u0, n_burnin=80, n_samples=40, n_leapfrog=5, step_size=1e-3,
                           target_accept=0.75, seed=5)
    d = res.draws.cpu().numpy()
    assert np.all(np.isfinite(d))
    assert res.step_size > 0 and np.all(res.inv_mass > 0) and np.all(np.isfinite(res.inv_mass))
    assert 0.3 < res.accept.mean() < 0.99
    # draws stay inside the prior's support
    lo = np.array([p.lo for p in case.spec.params])
    hi = np.array([p.hi for p in case.spec.params])
    assert np.all((d >= lo - 1e-6) & (d <= hi + 1e-6))
    assert np.all(np.hypot(d[..., 2], d[..., 3]) < case.spec.emax[0])
    assert res.rhat.shape == (sysg.P,) and res.ess.shape == (sysg.P,)
    assert np.all(np.isfinite(res.rhat)) and np.all(res.ess > 0)


def test_svi_step_matches_oracle(torch, case, sysg, bij):
    from paper_2606_30633_b300 import infer
    P = sysg.P
    n, seed, lr = 256, 77, 1e-3
    mu0 = _u_near_mode(case, bij, 1, 13)[0]
    phi, opt = infer.svi_init(sysg, torch.tensor(mu0, dtype=torch.float32, device="cuda"), scale=0.01)
    phi0 = phi.cpu().numpy().astype(np.float64)
    elbo = sysg.svi_adabelief(phi, opt, n, 1, lr=lr, seed=seed).cpu().numpy()
    phi1 = phi.cpu().numpy().astype(np.float64)
    mu = phi0[:P]
    Lr = phi0[P:].reshape(P, P)
    L = np.tril(Lr, -1) + np.diag(np.exp(np.diag(Lr)))
    z = I.svi_draws(seed, 0, n, P)
    lpu = lambda u: I.logp_unconstrained(case.oracle, bij, u)
    w, u = I.svi_terms(mu, L, z, lpu)
    assert abs(elbo[0] - w.mean()) <= 1e-4 * abs(w.mean()) + 0.05, (elbo[0], w.mean())
    _, g_mu, g_L = I.svi_grad(mu, L, z, lpu)
    g = np.concatenate([g_mu, (np.tril(g_L, -1) + np.diag(np.diag(g_L) * np.diag(L))).ravel()])
    # FP32 log p~ errors move each w_i by ~1e-5 |log p~|: bound the estimate's error
    a = np.linalg.solve(L.T, z.T).T
    dw = 2e-5 * np.abs(lpu(u)) + 1e-2
    err_mu = (dw[:, None] * np.abs(a)).mean(0)
    err_L = np.einsum("i,ij,ik->jk", dw, np.abs(a), np.abs(z)) / n
    err_L = np.tril(err_L, -1) + np.diag(np.diag(err_L) * np.diag(L) + dw.mean())
    err = np.concatenate([err_mu, err_L.ravel()])
    lower = np.concatenate([np.ones(P, bool), np.tril(np.ones((P, P), bool)).ravel()])
    step = phi1 - phi0
    sure = lower & (np.abs(g) > 3 * err)
    assert sure.sum() > 0.5 * lower.sum()
    # AdaBelief's first step is -lr g / (b1 |g|) (+ O(eps))
    assert np.allclose(step[sure], -lr * np.sign(g[sure]) / 0.95, rtol=1e-3, atol=1e-8)
    assert np.all(step[~lower] == 0.0)


def test_svi_pathwise_step_matches_oracle(torch, case, sysg, bij):
    """One SVI step with the reparameterisation gradient against the oracle's
    svi_grad_pathwise on the same draws (the shared counter-based generator)."""
    import paper_2606_30633_b300 as gl
    from paper_2606_30633_b300 import infer
    P = sysg.P
    n, seed, lr = 256, 78, 1e-3
    mu0 = _u_near_mode(case, bij, 1, 14)[0]
    phi, opt = infer.svi_init(sysg, torch.tensor(mu0, dtype=torch.float32, device="cuda"),
                              scale=0.01)
    phi0 = phi.cpu().numpy().astype(np.float64)
    elbo = sysg.svi_adabelief(phi, opt, n, 1, lr=lr, seed=seed,
                              estimator=gl.GL_SVI_PATHWISE).cpu().numpy()
    phi1 = phi.cpu().numpy().astype(np.float64)
    mu = phi0[:P]
    Lr = phi0[P:].reshape(P, P)
    L = np.tril(Lr, -1) + np.diag(np.exp(np.diag(Lr)))
    z = I.svi_draws(seed, 0, n, P)
    lg = lambda u: I.logp_grad_unconstrained(case.oracle, bij, u)
    w, g_mu, g_L = I.svi_grad_pathwise(mu, L, z, lg)
    assert abs(elbo[0] - w) <= 1e-4 * abs(w) + 0.05, (elbo[0], w)
    g = np.concatenate([g_mu, (np.tril(g_L, -1) + np.diag(np.diag(g_L) * np.diag(L))).ravel()])
    # FP32 gradients: per draw and parameter 2e-3 |g_ik| + 1e-3 max_k |g_ik| bounds the error
    _, gi = lg(mu[None, :] + z @ L.T)
    e = 2e-3 * np.abs(gi) + 1e-3 * np.abs(gi).max(1, keepdims=True)
    err_mu = e.mean(0)
    err_L = np.einsum("ij,ik->jk", e, np.abs(z)) / n
    err_L = np.tril(err_L, -1) + np.diag(np.diag(err_L) * np.diag(L))
    err = np.concatenate([err_mu, err_L.ravel()])
    lower = np.concatenate([np.ones(P, bool), np.tril(np.ones((P, P), bool)).ravel()])
    step = phi1 - phi0
    sure = lower & (np.abs(g) > 3 * err)
    assert sure.sum() > 0.5 * lower.sum()
    assert np.allclose(step[sure], -lr * np.sign(g[sure]) / 0.95, rtol=1e-3, atol=1e-8)
    assert np.all(step[~lower] == 0.0)


def test_whole_fit_recovers_the_posterior(torch, case, sysg, bij):
    """infer.fit runs the stages of Sec. 3 in order (at reduced sizes): the best
    of the multi-start MAP reaches at least the truth's log p~ (the mode is at
    least as probable); SVI with the paper's AdaBelief settings (and the
    reparameterisation gradient) stays near it: at lr 1e-4 and 300 steps q can
    barely move, so only boundedness is asserted; HMC started from
    SVI's draws puts the truth inside the posterior and mixes in most
    directions (median R-hat < 1.2). The slope gamma, degenerate with theta_E
    in this small image, mixes slowly under a diagonal mass matrix (R-hat near
    1.9 here even with 1000 burn-in and 1000 sampling transitions), so no bound
    is put on the largest R-hat."""
    from paper_2606_30633_b300 import infer
    starts = np.concatenate([f32(synth.jitter(case.truth, case.W.prior(), 16, 3, rel=0.01)),
                             case.theta(112, seed=5)])
    r = infer.fit(sysg, torch.tensor(starts, dtype=torch.float32, device="cuda"),
                  map_steps=400, n_vi=256, svi_steps=300, n_chains=32,
                  n_burnin=200, n_samples=300, seed=4)
    u_true = torch.tensor(f32(bij.inverse(case.truth[None])), dtype=torch.float32, device="cuda")
    lp_true = float(sysg.logp_grad_unconstrained(u_true)[0][0])
    assert r.map_logp >= lp_true - 0.5, (r.map_logp, lp_true)
    e = r.svi_elbo
    assert e.shape == (300,) and np.isfinite(e).all()
    assert e[-30:].mean() < e[:30].mean() + 0.1 * abs(e[:30].mean()), (e[:30].mean(),
                                                                        e[-30:].mean())
    d = r.hmc.draws.double().cpu().numpy()
    assert np.isfinite(d).all()
    assert np.all(np.isfinite(r.hmc.rhat)) and np.median(r.hmc.rhat) < 1.2, r.hmc.rhat
    assert 0.3 < r.hmc.accept.mean() < 0.99
    flat = d.reshape(-1, sysg.P)
    z = np.abs(flat.mean(0) - case.truth) / flat.std(0)
    assert np.max(z) < 6.0, z
    assert set(r.seconds) == {"map", "svi", "hmc"} and min(r.seconds.values()) > 0
