"""Pins of the inference-layer oracle (oracle/infer.py) against what the
mathematics and the published algorithms fix: finite differences, closed
forms, published generator outputs, hand-computed diagnostics and the
stationary distribution of HMC on a Gaussian."""
import math

import numpy as np
import pytest

import synth
from oracle import infer as I

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _mixed_bijector():
    kinds = ["uniform", "normal", "normal", "normal", "lognormal", "truncnorm", "flat", "flat",
             "flat"]
    lo = [0.8, -np.inf, -np.inf, -np.inf, 0.0, -0.5, 1.0, -np.inf, -np.inf]
    hi = [2.5, np.inf, np.inf, np.inf, np.inf, 0.5, np.inf, 3.0, np.inf]
    # indices 2, 3 are the EPL ellipticity: normal priors + a disc of radius 0.5
    return I.Bijector(kinds, lo, hi, [0.5])


def _fd_jacobian(bij, u, h=1e-6):
    P = u.size
    J = np.empty((P, P))
    for k in range(P):
        e = np.zeros(P)
        e[k] = h
        J[:, k] = (bij.forward(u + e)[0][0] - bij.forward(u - e)[0][0]) / (2 * h)
    return J


def test_bijector_modes_and_ranges():
    bij = _mixed_bijector()
    assert list(bij.mode) == [I.INTERVAL, I.ID, I.DISC, I.DISC, I.EXP, I.INTERVAL, I.LOWER,
                              I.UPPER, I.ID]
    rng = np.random.default_rng(0)
    u = rng.normal(0, 3, size=(500, 9))
    th, _ = bij.forward(u)
    assert np.all((th[:, 0] > 0.8) & (th[:, 0] < 2.5))
    assert np.all(np.hypot(th[:, 2], th[:, 3]) < 0.5)
    assert np.all(th[:, 4] > 0) and np.all(th[:, 6] > 1.0) and np.all(th[:, 7] < 3.0)
    assert np.all(np.abs(th[:, 5]) < 0.5)


def test_bijector_round_trip():
    bij = _mixed_bijector()
    rng = np.random.default_rng(1)
    u = rng.normal(0, 1.5, size=(200, 9))
    u[0, 2:4] = 0.0  # the disc centre
    u[1, 2:4] = [1e-5, -2e-5]
    th, _ = bij.forward(u)
    assert np.allclose(bij.inverse(th), u, atol=1e-9, rtol=1e-9)


@pytest.mark.parametrize("seed", [2, 3, 4])
def test_bijector_jacobian_and_logdet_match_finite_differences(seed):
    bij = _mixed_bijector()
    rng = np.random.default_rng(seed)
    u = rng.normal(0, 1.2, size=9)
    if seed == 4:
        u[2:4] = [3e-4, -2e-4]  # near the disc centre
    Jfd = _fd_jacobian(bij, u)
    assert np.allclose(bij.jacobian(u)[0], Jfd, atol=1e-8, rtol=1e-6)
    _, logj = bij.forward(u)
    assert abs(logj[0] - math.log(abs(np.linalg.det(Jfd)))) < 1e-7
    h = 1e-6
    g = np.array([(bij.forward(u + h * e)[1][0] - bij.forward(u - h * e)[1][0]) / (2 * h)
                  for e in np.eye(9)])
    assert np.allclose(bij.grad_logj(u)[0], g, atol=1e-7)


def test_bijector_from_the_benchmark_prior():
    bij = I.Bijector.from_spec(synth.config_prior(1, 1))
    # EPL: theta_E, gamma uniform; e disc; centre, shear normal
    assert list(bij.mode[:8]) == [I.INTERVAL, I.INTERVAL, I.DISC, I.DISC, I.ID, I.ID, I.ID, I.ID]
    # lens light: R, n uniform, e truncated normal, centre normal, I log-normal
    assert list(bij.mode[8:15]) == [I.INTERVAL] * 4 + [I.ID, I.ID, I.EXP]


def test_unconstrained_gradient_matches_finite_differences():
    from lenscase import make_case, small_workload
    c = make_case(small_workload(24, 24, 2, 5, 1, 1, seed=77))
    sysm = c.oracle
    bij = I.Bijector.from_spec(c.spec)
    u = bij.inverse(c.truth[None, :].astype(np.float64))[0]
    u = u + np.random.default_rng(5).normal(0, 0.02, size=u.size)
    lp, g = I.logp_grad_unconstrained(sysm, bij, u)
    h = 1e-6
    for k in range(u.size):
        e = np.zeros(u.size)
        e[k] = h
        fd = (I.logp_unconstrained(sysm, bij, u + e)[0]
              - I.logp_unconstrained(sysm, bij, u - e)[0]) / (2 * h)
        assert abs(g[0, k] - fd) <= 1e-5 * max(1.0, abs(fd)), (k, g[0, k], fd)


def test_splitmix64_published_outputs():
    # the first outputs of SplitMix64 seeded with 1234567 (Vigna's reference code)
    gamma = 0x9E3779B97F4A7C15
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    got = [I.splitmix64((1234567 + k * gamma) & ((1 << 64) - 1)) for k in range(5)]
    assert got == want


def test_draws_are_on_the_grid_and_normal():
    vals = np.array([I.uniform(99, k) for k in range(20000)])
    assert np.all((vals > 0) & (vals < 1))
    assert np.allclose((vals * 16777216.0 - 0.5) % 1.0, 0.0)
    assert abs(vals.mean() - 0.5) < 0.01 and abs(vals.var() - 1 / 12) < 0.003
    z, a = I.hmc_draws(7, 3, 400, 10)
    assert abs(z.mean()) < 0.03 and abs(z.var() - 1.0) < 0.05
    assert abs(np.mean(z[:, 0] * z[:, 1])) < 0.08
    # different steps and rows give different numbers
    z2, _ = I.hmc_draws(7, 4, 400, 10)
    assert not np.allclose(z, z2)


def test_leapfrog_on_the_harmonic_oscillator_is_the_known_linear_map():
    # H = u^2/2 + p^2/2: one leapfrog step is
    # [u, p] -> [(1 - e^2/2) u + e p, -e (1 - e^2/4) u + (1 - e^2/2) p]
    eps = 0.3
    u0, p0 = np.array([[0.7]]), np.array([[-0.4]])
    lg = lambda u: (-0.5 * (u * u).sum(1), -u)
    lp, g = lg(u0)
    u1, p1, _, _ = I.leapfrog(u0, p0, lp, g, np.ones(1), eps, 1, lg)
    A = np.array([[1 - eps ** 2 / 2, eps], [-eps * (1 - eps ** 2 / 4), 1 - eps ** 2 / 2]])
    want = A @ np.array([0.7, -0.4])
    assert np.allclose([u1[0, 0], p1[0, 0]], want, atol=1e-14)
    # five steps = A^5
    u5, p5, _, _ = I.leapfrog(u0, p0, lp, g, np.ones(1), eps, 5, lg)
    assert np.allclose([u5[0, 0], p5[0, 0]], np.linalg.matrix_power(A, 5) @ [0.7, -0.4])
    # inverse mass c (H = u^2/2 + c p^2/2): the half kicks are unchanged and the
    # drift moves u by e c p, so one step is
    # [u, p] -> [(1 - c e^2/2) u + c e p, -e (1 - c e^2/4) u + (1 - c e^2/2) p]
    c = 2.5
    uc, pc, _, _ = I.leapfrog(u0, p0, lp, g, np.full(1, c), eps, 1, lg)
    Ac = np.array([[1 - c * eps ** 2 / 2, c * eps],
                   [-eps * (1 - c * eps ** 2 / 4), 1 - c * eps ** 2 / 2]])
    assert np.allclose([uc[0, 0], pc[0, 0]], Ac @ [0.7, -0.4], atol=1e-14)
    assert abs(np.linalg.det(Ac) - 1) < 1e-14  # leapfrog is volume preserving


@pytest.mark.parametrize("inv_mass", [(1.0, 1.0), (0.3, 5.0)])
def test_hmc_leaves_a_gaussian_invariant(inv_mass):
    # target N(0, diag(1, 4)); 4000 chains started from the target; the
    # Metropolis-Hastings correction keeps it invariant even at a step with
    # large energy errors, for any (here deliberately mismatched) mass matrix,
    # provided the momenta are drawn from N(0, M)
    inv_mass = np.array(inv_mass)
    sd = np.array([1.0, 2.0])
    lg = lambda u: (-0.5 * ((u / sd) ** 2).sum(1), -u / sd ** 2)
    rng = np.random.default_rng(11)
    B = 4000
    u = rng.normal(size=(B, 2)) * sd
    lp, g = lg(u)
    rates = []
    for step in range(60):
        z, a = I.hmc_draws(5, step, B, 2)
        u, lp, g, acc_p, acc = I.hmc_transition(u, lp, g, inv_mass, 1.6, 3, z, a, lg)
        rates.append(acc.mean())
    assert 0.2 < np.mean(rates) < 0.95
    assert np.allclose(u.mean(0), 0.0, atol=0.1)
    assert np.allclose(u.std(0), sd, rtol=0.05)
    assert np.allclose(np.mean(u[:, 0] * u[:, 1]), 0.0, atol=0.1)


def test_dual_averaging_reaches_the_target_rate():
    # a monotone acceptance curve a(eps) = exp(-eps^2): the averaged step must
    # converge to eps* = sqrt(-ln 0.75)
    da = I.DualAveraging(2.0, target=0.75)
    eps = 2.0
    for _ in range(2000):
        eps = da.update(math.exp(-eps * eps))
    assert abs(da.final - math.sqrt(-math.log(0.75))) < 0.02


def test_mass_from_burnin_uses_the_last_90_percent():
    s = np.zeros((10, 3, 2))
    s[0] = 100.0  # the first 10 % is dropped
    s[1:, :, 0] = np.arange(27).reshape(9, 3)
    m = I.mass_from_burnin(s)
    assert np.isclose(m[0], np.var(np.arange(27.0))) and m[1] == 0.0


def test_adam_first_step_and_convergence():
    # f = -log p = sum (u - c)^2 / 2; Adam's first step is -lr sign(grad f)
    c = np.array([[1.0, -2.0, 0.5]])
    gf = lambda u: (-0.5 * ((u - c) ** 2).sum(1), -(u - c))
    u0 = np.zeros((1, 3))
    u1, _ = I.adam(u0, gf, 1, lr=0.1)
    assert np.allclose(u1, 0.1 * np.sign(c), atol=1e-8)
    uN, hist = I.adam(u0, gf, 2000, lr=0.05)
    assert np.allclose(uN, c, atol=1e-3) and hist[-1] > hist[0]


def test_adabelief_first_step_and_convergence():
    g = np.array([0.3, -2.0])
    x1, m, s = I.adabelief_step(np.zeros(2), g, np.zeros(2), np.zeros(2), 1, lr=0.01)
    # m1 = (1-b1) g, s1 = (1-b2) (b1 g)^2 (+eps): step = lr g / (b1 |g|)
    assert np.allclose(x1, -0.01 * np.sign(g) / 0.95, rtol=1e-6)
    c = np.array([1.5, -0.5])
    x, m, s = np.zeros(2), np.zeros(2), np.zeros(2)
    for t in range(1, 4001):
        x, m, s = I.adabelief_step(x, x - c, m, s, t, lr=0.01)
    assert np.allclose(x, c, atol=1e-3)


def test_svi_score_gradient_is_unbiased_for_a_gaussian_target():
    # target N(m, S): the ELBO is KL(q || p) up to a constant, with closed-form gradients
    m = np.array([0.5, -1.0])
    S = np.array([[1.0, 0.3], [0.3, 0.5]])
    Si = np.linalg.inv(S)
    logp = lambda u: -0.5 * np.einsum("bi,ij,bj->b", u - m, Si, u - m)
    mu = np.array([0.2, -0.6])
    L = np.array([[0.8, 0.0], [0.1, 0.6]])
    z = np.random.default_rng(3).normal(size=(400000, 2))
    _, g_mu, g_L = I.svi_grad(mu, L, z, logp)
    # d KL/d mu = S^-1 (mu - m); d KL/d L = S^-1 L - L^-T (lower triangle)
    want_mu = Si @ (mu - m)
    want_L = np.tril(Si @ L - np.linalg.inv(L).T)
    assert np.allclose(g_mu, want_mu, atol=0.03)
    assert np.allclose(g_L, want_L, atol=0.05)


def test_svi_pathwise_gradient_is_unbiased_for_a_gaussian_target():
    # the same closed form as above, from the reparameterisation estimator; it
    # needs the target's gradient and has far less variance (fewer draws)
    m = np.array([0.5, -1.0])
    S = np.array([[1.0, 0.3], [0.3, 0.5]])
    Si = np.linalg.inv(S)
    logp = lambda u: -0.5 * np.einsum("bi,ij,bj->b", u - m, Si, u - m)
    logp_grad = lambda u: (logp(u), -(u - m) @ Si)
    mu = np.array([0.2, -0.6])
    L = np.array([[0.8, 0.0], [0.1, 0.6]])
    z = np.random.default_rng(4).normal(size=(40000, 2))
    e_p, g_mu, g_L = I.svi_grad_pathwise(mu, L, z, logp_grad)
    want_mu = Si @ (mu - m)
    want_L = np.tril(Si @ L - np.linalg.inv(L).T)
    assert np.allclose(g_mu, want_mu, atol=0.02)
    assert np.allclose(g_L, want_L, atol=0.02)
    # the ELBO estimate is the same quantity the score-function path reports
    e_s, _, _ = I.svi_grad(mu, L, z, logp)
    assert e_p == pytest.approx(e_s, rel=1e-12)
    # and with z = 0 the mu-gradient is exactly -grad log p~(mu)
    _, g0, _ = I.svi_grad_pathwise(mu, L, np.zeros((1, 2)), logp_grad)
    assert np.allclose(g0, Si @ (mu - m), atol=1e-15)


def test_rhat_by_hand():
    # chains [0, 2] and [4, 6]: means 1, 5; B = 2/1 (4 + 4) = 16; s^2 = 2, 2 so W = 2;
    # var+ = (1/2) 2 + 16/2 = 9; R = sqrt(9/2)
    x = np.array([[0.0, 4.0], [2.0, 6.0]])
    assert np.isclose(I.rhat(x), math.sqrt(4.5))
    rng = np.random.default_rng(2)
    assert abs(I.rhat(rng.normal(size=(2000, 8))) - 1.0) < 0.01


def test_ess_of_ar1_chains_matches_the_closed_form():
    # AR(1) with coefficient r: integrated autocorrelation time (1 + r)/(1 - r)
    rng = np.random.default_rng(4)
    N, M, r = 4000, 4, 0.5
    x = np.empty((N, M))
    x[0] = rng.normal(size=M)
    e = rng.normal(size=(N, M)) * math.sqrt(1 - r * r)
    for t in range(1, N):
        x[t] = r * x[t - 1] + e[t]
    want = N * M * (1 - r) / (1 + r)
    assert abs(I.ess(x) - want) < 0.15 * want
    iid = rng.normal(size=(2000, 4))
    assert abs(I.ess(iid) - 8000) < 0.15 * 8000
