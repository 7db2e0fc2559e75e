"""Host drivers of the inference layer (Sec. 3): multi-start MAP, SVI and HMC
with adaptation, over the library's device-resident steps, plus the
convergence diagnostics of Sec. 3.4 (R-hat and the cross-chain effective
sample size), which run on the host over the draws.

Every step of the computation runs in libgl (gl_map_adam, gl_svi_adabelief,
gl_hmc_*); this module chooses the phases and moves the draws to the host.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import (GL_DEFL_SERIES, GL_HMC_ADAPT_STEP, GL_HMC_COLLECT_MOMENTS, GL_SVI_PATHWISE, Hmc,
               System, _torch)


# ----------------------------------------------------------- diagnostics --
def rhat(draws) -> np.ndarray:
    """Potential scale reduction factor (Gelman et al. 2014, without chain
    splitting) of draws [N, M, ...]: sqrt(((N-1)/N W + B/N) / W), with W the
    mean within-chain variance and B/N the variance of the chain means."""
    x = np.asarray(draws, dtype=np.float64)
    N, M = x.shape[:2]
    means = x.mean(axis=0)
    within = x.var(axis=0, ddof=1).mean(axis=0)
    between_over_n = means.var(axis=0, ddof=1)
    with np.errstate(divide="ignore", invalid="ignore"):  # chains that never moved: inf / nan
        return np.sqrt(((N - 1) / N * within + between_over_n) / within)


def _autocov(c: np.ndarray) -> np.ndarray:
    """Biased autocovariances (divided by N) of centred series c [N, M] along
    axis 0, by FFT with zero padding."""
    N = c.shape[0]
    n2 = 1 << (2 * N - 1).bit_length()
    f = np.fft.rfft(c, n=n2, axis=0)
    return np.fft.irfft(f * np.conj(f), n=n2, axis=0)[:N] / N


def ess(draws) -> np.ndarray:
    """Effective sample size with the cross-chain variance of Vehtari et al.
    (2021): rho_t = 1 - (W - mean_m s_m^2 rho_{t,m}) / var+, summed over
    Geyer's initial monotone sequence of pair sums; ESS = N M / tau."""
    x = np.asarray(draws, dtype=np.float64)
    N, M = x.shape[:2]
    tail = x.shape[2:]
    x = x.reshape(N, M, -1)
    out = np.empty(x.shape[2])
    for k in range(x.shape[2]):
        xs = x[:, :, k]
        c = xs - xs.mean(axis=0)
        ac = _autocov(c)
        s2 = ac[0] * N / (N - 1)
        W = s2.mean()
        var_plus = (N - 1) / N * W + (xs.mean(axis=0).var(ddof=1) if M > 1 else 0.0)
        # s2_m rho_{t,m} = s2_m ac_{t,m} / ac_{0,m} = ac_{t,m} N / (N - 1), also for a
        # chain that never moved (ac = 0); all chains constant gives var+ = 0: nan
        with np.errstate(divide="ignore", invalid="ignore"):
            rho = 1.0 - (W - (ac * (N / (N - 1))).mean(axis=1)) / var_plus
        pairs = rho[0:N - 1:2] + rho[1:N:2]
        pos = np.flatnonzero(pairs <= 0)
        pairs = pairs[:pos[0]] if pos.size else pairs
        pairs = np.minimum.accumulate(pairs)
        tau = -1.0 + 2.0 * pairs.sum()
        with np.errstate(divide="ignore", invalid="ignore"):
            out[k] = N * M / tau
    return out.reshape(tail)


# -------------------------------------------------------------- drivers --
def map_fit(system: System, u0, n_steps: int, lr: float = 1e-2, defl: int = GL_DEFL_SERIES,
            chunk: int = 100):
    """Multi-start MAP (Sec. 3.1): Adam on every row of u0 for n_steps, in
    graph-captured chunks. Returns (u, log p~ at the last evaluated point)."""
    torch = _torch()
    u = u0.clone().contiguous()
    m = torch.zeros_like(u)
    v = torch.zeros_like(u)
    lp = None
    done = 0
    while done < n_steps:
        k = min(chunk, n_steps - done)
        lp = system.map_adam(u, m, v, k, t0=done, lr=lr, defl=defl)
        done += k
    return u, lp


def svi_init(system: System, mu, scale: float = 1e-2):
    """phi = (mu, L = scale I with log diagonal) and a zero AdaBelief state."""
    torch = _torch()
    P = system.P
    L = torch.zeros(P, P, device=mu.device)
    L.fill_diagonal_(math.log(scale))
    phi = torch.cat([mu.reshape(P).float(), L.reshape(-1)]).contiguous()
    opt = torch.zeros(2 * phi.numel(), device=mu.device)
    return phi, opt


def svi_unpack(system: System, phi):
    """(mu [P], L [P, P] lower triangular) from phi."""
    torch = _torch()
    P = system.P
    mu = phi[:P]
    L = torch.tril(phi[P:].reshape(P, P), -1) + torch.diag(torch.exp(phi[P:].reshape(P, P).diag()))
    return mu, L


def svi_fit(system: System, mu0, n_samples: int, n_steps: int, lr: float = 1e-4,
            scale: float = 1e-3, seed: int = 0, defl: int = GL_DEFL_SERIES, chunk: int = 100,
            estimator: int = GL_SVI_PATHWISE):
    """SVI (Sec. 3.2) from q = N(mu0, scale^2 I): n_steps AdaBelief steps with
    the paper's defaults (lr 1e-4, b1 0.95, b2 0.99), n_samples draws each, in
    graph-captured chunks, with the reparameterisation gradient by default
    (the gradient automatic differentiation of the sampled ELBO gives).
    Returns (mu [P], L [P, P], per-step ELBO estimates)."""
    torch = _torch()
    phi, opt = svi_init(system, mu0, scale)
    elbo = []
    done = 0
    while done < n_steps:
        k = min(chunk, n_steps - done)
        elbo.append(system.svi_adabelief(phi, opt, n_samples, k, t0=done, lr=lr, seed=seed,
                                         defl=defl, estimator=estimator))
        done += k
    mu, L = svi_unpack(system, phi)
    e = torch.cat(elbo).cpu().numpy() if elbo else np.zeros(0)
    return mu.clone(), L, e


@dataclass
class HmcResult:
    draws: "object"          # device tensor [n_samples, B, P] (theta)
    accept: np.ndarray       # mean acceptance probability per sampling transition
    step_size: float
    inv_mass: np.ndarray
    rhat: np.ndarray
    ess: np.ndarray


def hmc_sample(system: System, u0, n_burnin: int, n_samples: int, n_leapfrog: int = 10,
               step_size: float = 1e-2, target_accept: float = 0.75, seed: int = 0,
               defl: int = GL_DEFL_SERIES, adapt_mass: bool = True, inv_mass=None,
               n_retune: Optional[int] = None) -> HmcResult:
    """The sampling stage: burn-in with dual-averaging step size, and over its
    last 90 % the moments of u for the diagonal mass matrix (Sec. 3.3); then
    n_samples transitions at the adapted step and mass, with R-hat and ESS of
    the draws (Sec. 3.4).

    inv_mass (device [P]) is the starting M^-1, e.g. the SVI surrogate's
    variances (Sec. 3.3: SVI sets the scale); ones by default. n_retune
    transitions after the mass update retune the step size to it (the second
    burn-in the paper suggests; n_burnin // 2 by default, 0 for none)."""
    torch = _torch()
    h = Hmc(system, u0, n_leapfrog, step_size, target_accept, seed, defl)
    try:
        if inv_mass is not None:
            h.set_inv_mass(inv_mass)
        first = n_burnin - int(math.ceil(0.9 * n_burnin))
        if first:
            h.run(first, GL_HMC_ADAPT_STEP)
        if n_burnin - first:
            h.run(n_burnin - first, GL_HMC_ADAPT_STEP | GL_HMC_COLLECT_MOMENTS)
        mass = adapt_mass and n_burnin > first
        h.end_adaptation(set_inv_mass=mass)
        retune = (n_burnin // 2 if n_retune is None else n_retune) if mass else 0
        if retune:
            h.run(retune, GL_HMC_ADAPT_STEP)
            h.end_adaptation(set_inv_mass=False)
        B, P = h.B, h.P
        draws = torch.empty(n_samples, B, P, device=u0.device)
        acc = torch.empty(n_samples, device=u0.device)
        h.run(n_samples, 0, draws, acc)
        _, _, im, eps = h.state()
    finally:
        h.close()
    d = draws.double().cpu().numpy()
    return HmcResult(draws, acc.cpu().numpy(), eps, im.cpu().numpy(), rhat(d), ess(d))


@dataclass
class FitResult:
    map_u: "object"                  # best MAP point, device [P] (unconstrained)
    map_logp: float                  # its log p~
    svi_mu: "object"                 # device [P]
    svi_L: "object"                  # device [P, P], lower triangular
    svi_elbo: np.ndarray             # per-step estimates of E_q[log q - log p~]
    hmc: HmcResult
    seconds: dict = field(default_factory=dict)   # wall-clock per stage


def fit(system: System, theta_starts, map_steps: int = 1000, map_lr: float = 1e-2,
        n_vi: int = 1000, svi_steps: int = 5000, svi_lr: float = 1e-4, svi_scale: float = 1e-3,
        n_chains: int = 64, n_burnin: int = 500, n_samples: int = 1500, n_leapfrog: int = 10,
        step_size: float = 0.1, seed: int = 0, defl: int = GL_DEFL_SERIES,
        svi_estimator: int = GL_SVI_PATHWISE) -> FitResult:
    """The pipeline of Sec. 3, stage after stage. The defaults are the
    hyperparameter table of the hundred simulated systems (Sec. 4.2; n_MAP is
    the number of rows of theta_starts, 2000 there):
      1. multi-start MAP: Adam from every row of theta_starts (device [n_MAP, P],
         e.g. prior draws) for map_steps; the row with the highest log p~ wins;
      2. SVI: AdaBelief on a full-covariance Gaussian q started at the MAP point,
         n_vi draws per step for svi_steps (reparameterisation gradient by
         default; GL_SVI_SCORE gives the printed score-function form, which is
         mostly noise on narrow lensing posteriors);
      3. HMC: n_chains chains started from draws of q, with q's marginal
         variances as the first inverse mass, burn-in with step-size and mass
         adaptation (hmc_sample), then n_samples transitions, R-hat and ESS.
    Every step runs in libgl; this function only orders them. The chains'
    start draws u0 = mu + L z use torch's generator (seeded)."""
    torch = _torch()
    sec = {}

    def now():
        torch.cuda.synchronize()
        return time.perf_counter()

    t0 = now()
    u_map, lp_map = map_fit(system, system.bijector_inverse(theta_starts), map_steps, map_lr,
                            defl)
    lp = lp_map.cpu().numpy().astype(np.float64)
    lp[~np.isfinite(lp)] = -np.inf
    best = int(np.argmax(lp))
    t1 = now()
    sec["map"] = t1 - t0
    mu, L, elbo = svi_fit(system, u_map[best].contiguous(), n_vi, svi_steps, svi_lr, svi_scale,
                          seed, defl, estimator=svi_estimator)
    t2 = now()
    sec["svi"] = t2 - t1
    g = torch.Generator(device=mu.device)
    g.manual_seed(seed)
    z = torch.randn(n_chains, system.P, device=mu.device, generator=g)
    u0 = (mu[None, :] + z @ L.T).contiguous()
    inv_mass = (L * L).sum(1).contiguous()
    res = hmc_sample(system, u0, n_burnin, n_samples, n_leapfrog, step_size, seed=seed + 1,
                     defl=defl, inv_mass=inv_mass)
    sec["hmc"] = now() - t2
    return FitResult(u_map[best].clone(), float(lp[best]), mu, L, elbo, res, sec)
