"""FP64 oracle of the inference layer around the log-posterior (test
infrastructure; only the tests may import it). Plain numpy, written from the
paper's description of its MAP -> SVI -> HMC pipeline (Sec. 3) and from the
published algorithms it names; it shares no code with the CUDA library.

  * Bijector: the map from an unconstrained vector u to the parameters theta
    (Sec. 3.1: SVI and HMC work on parameters "mapped into an unconstrained
    space via a bijective transformation"), with log|det d theta/d u|.
    The paper defers the transformation to its earlier release; the reading
    taken here is one map per prior support:
        unbounded (normal, flat on R)    theta = u
        interval [lo, hi]                theta = lo + (hi - lo) sigmoid(u)
        (0, inf) (log-normal)            theta = exp(u)
        [lo, inf) / (-inf, hi]           theta = lo + exp(u) / hi - exp(u)
    (uniform, truncated-normal and flat priors take the form their finite
    bounds give) and, for a component whose ellipticity is restricted to the disc
    |e| < emax while both e priors are unbounded, the radial map
        e = v emax tanh(|v|)/|v|.
  * Counter-based random numbers: SplitMix64 (Steele, Lea & Flood 2014), used
    as a counter-based generator, uniforms on a 2^-24 grid, Box-Muller
    normals.
  * Leapfrog / HMC transition with Metropolis-Hastings acceptance (Sec. 3,
    sampling stage), diagonal mass matrix.
  * Dual-averaging step-size adaptation (Hoffman & Gelman 2014, Sec. 3.2).
  * Mass-matrix adaptation (Sec. 3.3): a Gaussian fitted to the last 90 % of
    the burn-in samples; its variances become the inverse mass.
  * Adam (Kingma & Ba 2015) for multi-start MAP (Sec. 3.1), AdaBelief
    (Zhuang et al. 2020) for SVI (Sec. 3.2).
  * The ELBO and its score-function gradient estimate (Eqs. elbo,
    elbo-grad) for a full-covariance Gaussian surrogate.
  * R-hat (Gelman et al. 2014) and the cross-chain effective sample size
    (Vehtari et al. 2021), Sec. 3.4.
"""
from __future__ import annotations

import math
from typing import Callable, Optional, Sequence, Tuple

import numpy as np

# ----------------------------------------------------------------- bijector --
ID, INTERVAL, EXP, LOWER, UPPER, DISC = 0, 1, 2, 3, 4, 5


def _ellip_index(c: int) -> int:
    """Index of e1 of component c (0 = EPL, then the light components)."""
    return 2 if c == 0 else 8 + 7 * (c - 1) + 2


class Bijector:
    """theta(u) for the system's priors (see the module docstring)."""

    def __init__(self, kinds: Sequence[str], lo: Sequence[float], hi: Sequence[float],
                 emax: Sequence[float]):
        P = len(kinds)
        self.P = P
        self.mode = np.zeros(P, dtype=int)
        self.lo = np.asarray(lo, dtype=np.float64).copy()
        self.hi = np.asarray(hi, dtype=np.float64).copy()
        self.rmax = np.zeros(P)  # disc radius, on the e1 index of a disc pair
        for k, kind in enumerate(kinds):
            lo_k, hi_k = self.lo[k], self.hi[k]
            bounded = kind in ("uniform", "truncnorm", "flat")
            if kind == "lognormal":
                self.mode[k] = EXP
            elif bounded and math.isfinite(lo_k) and math.isfinite(hi_k):
                self.mode[k] = INTERVAL
            elif bounded and math.isfinite(lo_k):
                self.mode[k] = LOWER
            elif bounded and math.isfinite(hi_k):
                self.mode[k] = UPPER
            else:
                self.mode[k] = ID
        for c, em in enumerate(emax):
            i = _ellip_index(c)
            if em > 0 and self.mode[i] == ID and self.mode[i + 1] == ID:
                self.mode[i] = DISC
                self.mode[i + 1] = DISC
                self.rmax[i] = em

    @staticmethod
    def from_spec(spec) -> "Bijector":
        """From a synth.PriorSpec."""
        return Bijector([p.kind for p in spec.params], [p.lo for p in spec.params],
                        [p.hi for p in spec.params], spec.emax)

    def _disc_pairs(self):
        return [k for k in range(self.P) if self.mode[k] == DISC and self.rmax[k] > 0]

    def forward(self, u) -> Tuple[np.ndarray, np.ndarray]:
        """theta [B, P] and log|det d theta / d u| [B] for u [B, P]."""
        u = np.atleast_2d(np.asarray(u, dtype=np.float64))
        th = u.copy()
        logj = np.zeros(u.shape[0])
        for k in range(self.P):
            m, x = self.mode[k], u[:, k]
            if m == INTERVAL:
                w = self.hi[k] - self.lo[k]
                s = 1.0 / (1.0 + np.exp(-x))
                th[:, k] = self.lo[k] + w * s
                # log sigmoid(x) + log sigmoid(-x), written without overflow
                logj += math.log(w) - np.abs(x) - 2.0 * np.log1p(np.exp(-np.abs(x)))
            elif m == EXP:
                th[:, k] = np.exp(x)
                logj += x
            elif m == LOWER:
                th[:, k] = self.lo[k] + np.exp(x)
                logj += x
            elif m == UPPER:
                th[:, k] = self.hi[k] - np.exp(x)
                logj += x
        for i in self._disc_pairs():
            v1, v2 = u[:, i], u[:, i + 1]
            rho = np.hypot(v1, v2)
            R = self.rmax[i]
            g = R * _tanh_over(rho)
            th[:, i], th[:, i + 1] = g * v1, g * v2
            # |J| = r'(rho) r(rho)/rho with r = R tanh(rho)
            logj += 2.0 * math.log(R) - 2.0 * np.log(np.cosh(rho)) + np.log(_tanh_over(rho))
        return th, logj

    def inverse(self, theta) -> np.ndarray:
        th = np.atleast_2d(np.asarray(theta, dtype=np.float64))
        u = th.copy()
        for k in range(self.P):
            m, x = self.mode[k], th[:, k]
            if m == INTERVAL:
                s = (x - self.lo[k]) / (self.hi[k] - self.lo[k])
                u[:, k] = np.log(s) - np.log1p(-s)
            elif m == EXP:
                u[:, k] = np.log(x)
            elif m == LOWER:
                u[:, k] = np.log(x - self.lo[k])
            elif m == UPPER:
                u[:, k] = np.log(self.hi[k] - x)
        for i in self._disc_pairs():
            e1, e2 = th[:, i], th[:, i + 1]
            r = np.hypot(e1, e2)
            R = self.rmax[i]
            rho = np.arctanh(r / R)
            f = np.where(r > 0, rho / np.where(r > 0, r, 1.0), 1.0 / R)
            u[:, i], u[:, i + 1] = f * e1, f * e2
        return u

    def jacobian(self, u) -> np.ndarray:
        """d theta / d u, [B, P, P] (block diagonal)."""
        u = np.atleast_2d(np.asarray(u, dtype=np.float64))
        B = u.shape[0]
        J = np.zeros((B, self.P, self.P))
        for k in range(self.P):
            m, x = self.mode[k], u[:, k]
            if m == ID:
                J[:, k, k] = 1.0
            elif m == INTERVAL:
                s = 1.0 / (1.0 + np.exp(-x))
                J[:, k, k] = (self.hi[k] - self.lo[k]) * s * (1.0 - s)
            elif m in (EXP, LOWER):
                J[:, k, k] = np.exp(x)
            elif m == UPPER:
                J[:, k, k] = -np.exp(x)
        for i in self._disc_pairs():
            v = u[:, i:i + 2]
            rho = np.hypot(v[:, 0], v[:, 1])
            R = self.rmax[i]
            g = R * _tanh_over(rho)
            gp_over = R * _dtanh_over_over(rho)  # g'(rho)/rho
            for a in range(2):
                for b in range(2):
                    J[:, i + a, i + b] = (g if a == b else 0.0) + gp_over * v[:, a] * v[:, b]
        return J

    def grad_logj(self, u) -> np.ndarray:
        """d log|J| / d u, [B, P]."""
        u = np.atleast_2d(np.asarray(u, dtype=np.float64))
        G = np.zeros_like(u)
        for k in range(self.P):
            m, x = self.mode[k], u[:, k]
            if m == INTERVAL:
                G[:, k] = 1.0 - 2.0 / (1.0 + np.exp(-x))
            elif m in (EXP, LOWER, UPPER):
                G[:, k] = 1.0
        for i in self._disc_pairs():
            v1, v2 = u[:, i], u[:, i + 1]
            rho = np.hypot(v1, v2)
            k_over = _dlogj_disc_over(rho)  # (d log|J| / d rho) / rho
            G[:, i], G[:, i + 1] = k_over * v1, k_over * v2
        return G


def _tanh_over(rho):
    """tanh(rho)/rho, with its limit 1 at 0."""
    rho = np.asarray(rho, dtype=np.float64)
    small = rho < 1e-4
    r = np.where(small, 1.0, rho)
    return np.where(small, 1.0 - rho * rho / 3.0, np.tanh(r) / r)


def _dtanh_over_over(rho):
    """(d/drho [tanh(rho)/rho... times rho]) i.e. g'(rho)/rho for g = tanh(rho)/rho,
    = (rho sech^2 rho - tanh rho)/rho^3, with its limit -2/3 at 0."""
    rho = np.asarray(rho, dtype=np.float64)
    small = rho < 1e-3
    r = np.where(small, 1.0, rho)
    big = (r / np.cosh(r) ** 2 - np.tanh(r)) / r ** 3
    return np.where(small, -2.0 / 3.0 + 8.0 * rho * rho / 15.0, big)


def _dlogj_disc_over(rho):
    """(d/drho log|J|)/rho for log|J| = const - 2 log cosh rho + log(tanh rho / rho):
    (-2 tanh rho + 2/sinh(2 rho) - 1/rho)/rho, with its limit -8/3 at 0."""
    rho = np.asarray(rho, dtype=np.float64)
    small = rho < 1e-3
    r = np.where(small, 1.0, rho)
    big = (-2.0 * np.tanh(r) + 2.0 / np.sinh(2.0 * r) - 1.0 / r) / r
    return np.where(small, -8.0 / 3.0 + 0.0 * rho, big)


def logp_unconstrained(system, bij: Bijector, u):
    """log p~(u) = log p(theta(u)) + log|J|(u), FP64 (system: oracle.System)."""
    th, logj = bij.forward(u)
    return system.logp(th) + logj


def logp_grad_unconstrained(system, bij: Bijector, u):
    """log p~(u) and its gradient: J^T grad_theta log p + grad log|J|."""
    u = np.atleast_2d(np.asarray(u, dtype=np.float64))
    th, logj = bij.forward(u)
    lp, g = system.logp_grad(th)
    J = bij.jacobian(u)
    gu = np.einsum("bij,bi->bj", J, g) + bij.grad_logj(u)
    return lp + logj, gu


# -------------------------------------------------------- random numbers --
_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """The SplitMix64 output function of state x + gamma (Steele et al. 2014)."""
    z = (x + _GAMMA) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def uniform(seed: int, counter: int) -> float:
    """Uniform in (0, 1) on the grid (k + 1/2) 2^-24 from the top 24 bits of
    SplitMix64 at state seed + counter * gamma."""
    z = splitmix64((seed + counter * _GAMMA) & _M64)
    return ((z >> 40) + 0.5) * (1.0 / 16777216.0)


def hmc_draws(seed: int, step: int, B: int, P: int):
    """Standard normal momenta [B, P] and acceptance uniforms [B] of one HMC
    transition: row b, draw index j uses counter ((step B + b)(2P + 2) + j);
    normal k is Box-Muller on uniforms 2k, 2k+1 (radius from the first), the
    acceptance uniform is index 2P."""
    z = np.empty((B, P))
    a = np.empty(B)
    for b in range(B):
        base = (step * B + b) * (2 * P + 2)
        for k in range(P):
            u1 = uniform(seed, base + 2 * k)
            u2 = uniform(seed, base + 2 * k + 1)
            z[b, k] = math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)
        a[b] = uniform(seed, base + 2 * P)
    return z, a


def svi_draws(seed: int, step: int, n: int, P: int):
    """Standard normals [n, P] of one SVI step (counter (step n + i) 2P + j)."""
    z = np.empty((n, P))
    for i in range(n):
        base = (step * n + i) * (2 * P)
        for k in range(P):
            u1 = uniform(seed, base + 2 * k)
            u2 = uniform(seed, base + 2 * k + 1)
            z[i, k] = math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)
    return z


# ------------------------------------------------------------------ HMC --
def leapfrog(u, p, lp, g, inv_mass, eps: float, n_steps: int,
             logp_grad: Callable):
    """n_steps leapfrog steps (half kick, drift, new gradient, half kick)."""
    u, p, g = u.copy(), p.copy(), g.copy()
    for _ in range(n_steps):
        p = p + 0.5 * eps * g
        u = u + eps * inv_mass * p
        lp, g = logp_grad(u)
        p = p + 0.5 * eps * g
    return u, p, lp, g


def hmc_transition(u, lp, g, inv_mass, eps: float, n_steps: int, z, a,
                   logp_grad: Callable):
    """One HMC transition per row: momenta p = z / sqrt(inv_mass), a leapfrog
    trajectory, Metropolis-Hastings acceptance with log a < min(0, H0 - H1)
    (H = -log p + p^T M^-1 p / 2; a non-finite H1 rejects). Returns the new
    (u, lp, g), the acceptance probability and the accept flags."""
    p0 = z / np.sqrt(inv_mass)
    H0 = -lp + 0.5 * np.sum(inv_mass * p0 * p0, axis=1)
    u1, p1, lp1, g1 = leapfrog(u, p0, lp, g, inv_mass, eps, n_steps, logp_grad)
    H1 = -lp1 + 0.5 * np.sum(inv_mass * p1 * p1, axis=1)
    dH = H0 - H1
    ok = np.isfinite(dH)
    log_acc = np.where(ok, np.minimum(0.0, np.where(ok, dH, 0.0)), -np.inf)
    acc = np.log(a) < log_acc
    un = np.where(acc[:, None], u1, u)
    lpn = np.where(acc, lp1, lp)
    gn = np.where(acc[:, None], g1, g)
    return un, lpn, gn, np.exp(log_acc), acc


class DualAveraging:
    """Step-size adaptation by dual averaging (Hoffman & Gelman 2014, Sec. 3.2),
    driven by the mean acceptance probability over chains."""

    def __init__(self, eps0: float, target: float = 0.75, gamma: float = 0.05,
                 t0: float = 10.0, kappa: float = 0.75):
        self.mu = math.log(10.0 * eps0)
        self.target, self.gamma, self.t0, self.kappa = target, gamma, t0, kappa
        self.m = 0
        self.hbar = 0.0
        self.log_eps = math.log(eps0)
        self.log_eps_bar = 0.0

    def update(self, accept_prob: float) -> float:
        self.m += 1
        m = self.m
        w = 1.0 / (m + self.t0)
        self.hbar = (1.0 - w) * self.hbar + w * (self.target - accept_prob)
        self.log_eps = self.mu - math.sqrt(m) / self.gamma * self.hbar
        eta = m ** (-self.kappa)
        self.log_eps_bar = eta * self.log_eps + (1.0 - eta) * self.log_eps_bar
        return math.exp(self.log_eps)

    @property
    def final(self) -> float:
        return math.exp(self.log_eps_bar)


def mass_from_burnin(samples: np.ndarray) -> np.ndarray:
    """Inverse (diagonal) mass: variances of a Gaussian fitted to the last 90 %
    of burn-in samples [steps, chains, P] (Sec. 3.3)."""
    n = samples.shape[0]
    tail = samples[n - int(math.ceil(0.9 * n)):]
    flat = tail.reshape(-1, samples.shape[-1])
    return flat.var(axis=0)


# ----------------------------------------------------------- optimizers --
def adam(u, grad_fn: Callable, n_steps: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """n_steps of Adam ascending log p~ per row (descending -log p~); returns u
    and the log p~ of every step (before its update)."""
    u = np.array(u, dtype=np.float64)
    m = np.zeros_like(u)
    v = np.zeros_like(u)
    hist = []
    for t in range(1, n_steps + 1):
        lp, g = grad_fn(u)
        hist.append(lp)
        gd = -g
        m = b1 * m + (1 - b1) * gd
        v = b2 * v + (1 - b2) * gd * gd
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        u = u - lr * mh / (np.sqrt(vh) + eps)
    return u, np.array(hist)


def adabelief_step(x, g, m, s, t: int, lr: float, b1=0.95, b2=0.99, eps=1e-16):
    """One AdaBelief step (Zhuang et al. 2020) minimising with gradient g."""
    m = b1 * m + (1 - b1) * g
    d = g - m
    s = b2 * s + (1 - b2) * d * d + eps
    mh = m / (1 - b1 ** t)
    sh = s / (1 - b2 ** t)
    x = x - lr * mh / (np.sqrt(sh) + eps)
    return x, m, s


# ------------------------------------------------------------------- SVI --
def svi_terms(mu, L, z, logp_u: Callable):
    """Per-sample ELBO terms for the Gaussian q(u; mu, L L^T) at u_i = mu + L z_i:
    log q(u_i) - log p~(u_i) (Eq. elbo)."""
    u = mu[None, :] + z @ L.T
    P = mu.size
    logq = (-0.5 * np.sum(z * z, axis=1) - np.sum(np.log(np.abs(np.diag(L))))
            - 0.5 * P * math.log(2.0 * math.pi))
    return logq - logp_u(u), u


def svi_grad(mu, L, z, logp_u: Callable):
    """ELBO estimate and its score-function gradient (Eq. elbo-grad) with
    respect to mu and the lower triangle of L, from the samples z:
      grad = mean_i (log q - log p~)(u_i) grad log q(u_i),
      grad_mu log q = L^-T z,  grad_L log q = tril(L^-T z z^T) - diag(1/L_ii)."""
    w, _ = svi_terms(mu, L, z, logp_u)
    a = np.linalg.solve(L.T, z.T).T  # L^-T z_i
    n = z.shape[0]
    g_mu = (w[:, None] * a).sum(0) / n
    g_L = np.einsum("i,ij,ik->jk", w, a, z) / n
    g_L = np.tril(g_L) - np.diag(w.mean() / np.diag(L))
    return w.mean(), g_mu, g_L


def svi_grad_pathwise(mu, L, z, logp_grad_u: Callable):
    """ELBO estimate and its reparameterisation (pathwise) gradient, the
    gradient that automatic differentiation of the sampled ELBO gives
    (Sec. 3.2 states the gradient is taken that way). With u_i = mu + L z_i,
    log q(u_i) = -|z_i|^2/2 - sum log L_jj - const does not depend on mu, so
      grad_mu ELBO = -mean_i g_i,   grad_L ELBO = -tril(mean_i g_i z_i^T) - diag(1/L_jj),
    g_i = grad_u log p~(u_i). Both estimators have the same expectation."""
    u = mu[None, :] + z @ L.T
    P = mu.size
    lp, g = logp_grad_u(u)
    logq = (-0.5 * np.sum(z * z, axis=1) - np.sum(np.log(np.abs(np.diag(L))))
            - 0.5 * P * math.log(2.0 * math.pi))
    w = logq - lp
    n = z.shape[0]
    g_mu = -g.sum(0) / n
    g_L = -np.tril(g.T @ z / n) - np.diag(1.0 / np.diag(L))
    return w.mean(), g_mu, g_L


# ----------------------------------------------------------- diagnostics --
def rhat(samples: np.ndarray) -> np.ndarray:
    """Potential scale reduction factor (Gelman et al. 2014, BDA3 Sec. 11.4,
    without splitting) for samples [draws N, chains M, ...]:
      B = N/(M-1) sum_m (mean_m - mean)^2,  W = mean_m s_m^2,
      var+ = (N-1)/N W + B/N,  R = sqrt(var+/W)."""
    x = np.asarray(samples, dtype=np.float64)
    N, M = x.shape[0], x.shape[1]
    cm = x.mean(axis=0)
    B = N / (M - 1) * ((cm - cm.mean(axis=0)) ** 2).sum(axis=0)
    W = x.var(axis=0, ddof=1).mean(axis=0)
    var_plus = (N - 1) / N * W + B / N
    return np.sqrt(var_plus / W)


def ess(samples: np.ndarray) -> np.ndarray:
    """Effective sample size with cross-chain variance (Vehtari et al. 2021,
    Sec. 3.2): rho_t = 1 - (W - mean_m s_m^2 rho_{t,m}) / var+, summed by
    Geyer's initial monotone sequence; ESS = N M / tau."""
    x = np.asarray(samples, dtype=np.float64)
    N, M = x.shape[0], x.shape[1]
    rest = x.shape[2:]
    x = x.reshape(N, M, -1)
    out = np.empty(x.shape[2])
    for k in range(x.shape[2]):
        c = x[:, :, k] - x[:, :, k].mean(axis=0)
        s2 = c.var(axis=0, ddof=1)
        # autocovariances per chain (biased, divided by N), by direct sums
        acov = np.empty((N, M))
        for t in range(N):
            acov[t] = (c[:N - t] * c[t:]).sum(axis=0) / N
        W = s2.mean()
        cm = x[:, :, k].mean(axis=0)
        B = N / (M - 1) * ((cm - cm.mean()) ** 2).sum() if M > 1 else 0.0
        var_plus = (N - 1) / N * W + B / N
        rho_m = acov / acov[0]
        rho = 1.0 - (W - (s2 * rho_m).mean(axis=1)) / var_plus
        # Geyer: pairs P_t = rho_2t + rho_2t+1 while positive, made monotone
        tau_sum = 0.0
        prev = np.inf
        t = 0
        while 2 * t + 1 < N:
            Pt = rho[2 * t] + rho[2 * t + 1]
            if Pt <= 0:
                break
            Pt = min(Pt, prev)
            tau_sum += Pt
            prev = Pt
            t += 1
        tau = -1.0 + 2.0 * tau_sum
        out[k] = N * M / tau
    return out.reshape(rest)
