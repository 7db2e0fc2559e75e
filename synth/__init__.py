"""Seeded synthetic inputs for the strong-lens log-posterior.

This module draws parameter vectors from the priors, builds PSF kernels and
turns a noiseless model image into a noise map and noisy data. It holds none
of the lens model's arithmetic (no deflection, no light profile, no binning,
no convolution, no likelihood): the image that the noise is added to is
rendered by whichever side uses these inputs. Both the FP64 oracle and the
CUDA path draw their inputs from here, so that the two see identical numbers.

Parameter order (the 22-parameter model of Eq. sim-dist, Sec. 4.2, extended
to any number of light components):

    [thetaE, gamma, e1, e2, x, y]_EPL, [gamma1, gamma2]_ext,
    then per lens-light Sersic component [R, n, e1, e2, x, y, I],
    then per source Sersic component     [R, n, e1, e2, x, y, I].

Prior kinds are named by strings here ("uniform", "normal", "truncnorm",
"lognormal", "flat"); each consumer maps them to its own codes.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

EPL_NAMES = ["thetaE", "gamma", "e1", "e2", "x", "y"]
SHEAR_NAMES = ["gamma1", "gamma2"]
SERSIC_NAMES = ["R", "n", "e1", "e2", "x", "y", "I"]


def num_params(n_lens_light: int, n_source: int) -> int:
    return 8 + 7 * (n_lens_light + n_source)


def param_names(n_lens_light: int, n_source: int) -> List[str]:
    names = [f"epl.{k}" for k in EPL_NAMES] + [f"shear.{k}" for k in SHEAR_NAMES]
    for c in range(n_lens_light):
        names += [f"light{c}.{k}" for k in SERSIC_NAMES]
    for c in range(n_source):
        names += [f"source{c}.{k}" for k in SERSIC_NAMES]
    return names


@dataclasses.dataclass(frozen=True)
class Prior:
    """One parameter's prior. uniform: [lo, hi]; normal: mean a, sd b;
    truncnorm: mean a, sd b on [lo, hi]; lognormal: log x ~ N(a, b); flat: no
    density (support [lo, hi] if finite)."""
    kind: str
    a: float = 0.0
    b: float = 1.0
    lo: float = -math.inf
    hi: float = math.inf


def U(lo, hi):
    return Prior("uniform", 0.0, 1.0, lo, hi)


def N(mu, sd):
    return Prior("normal", mu, sd)


def TN(mu, sd, lo, hi):
    return Prior("truncnorm", mu, sd, lo, hi)


def LogN(mu_log, sd_log):
    return Prior("lognormal", mu_log, sd_log, 0.0, math.inf)


@dataclasses.dataclass
class PriorSpec:
    params: List[Prior]
    # one entry per component (EPL, lens lights..., sources...): |e| < emax, 0 = none
    emax: List[float]


def config_prior(n_lens_light: int = 1, n_source: int = 1) -> PriorSpec:
    """Priors of the benchmark workloads: the ranges stated for the lens and
    source (theta_E, gamma, e_EPL, shear, lens-light n and R, source n, R and
    centre); every parameter they leave out takes the simulation column of
    Eq. sim-dist (Sec. 4.2)."""
    p: List[Prior] = [U(0.8, 2.5), U(1.7, 2.3), N(0.0, 0.15), N(0.0, 0.15),
                      N(0.0, 0.03), N(0.0, 0.03), N(0.0, 0.05), N(0.0, 0.05)]
    for _ in range(n_lens_light):
        p += [U(0.5, 2.0), U(2.0, 6.0), TN(0.0, 0.05, -0.15, 0.15),
              TN(0.0, 0.05, -0.15, 0.15), N(0.0, 0.01), N(0.0, 0.01),
              LogN(math.log(300.0), 0.3)]
    for _ in range(n_source):
        p += [U(0.05, 0.5), U(0.5, 4.0), TN(0.0, 0.15, -0.5, 0.5),
              TN(0.0, 0.15, -0.5, 0.5), N(0.0, 0.3), N(0.0, 0.3),
              LogN(math.log(150.0), 0.5)]
    emax = [0.5] + [0.0] * (n_lens_light + n_source)
    return PriorSpec(p, emax)


def paper_prior(column: str = "prior", n_lens_light: int = 1, n_source: int = 1) -> PriorSpec:
    """Eq. sim-dist (Sec. 4.2): the simulation distribution (column
    "simulation") that generated the paper's 100 test systems, or the wider
    modelling prior (column "prior") used to fit them. Extra light components
    repeat the first one's distributions."""
    sim = column == "simulation"
    if column not in ("simulation", "prior"):
        raise ValueError(column)
    pick = (lambda a, b: a) if sim else (lambda a, b: b)
    p: List[Prior] = [LogN(math.log(1.25), pick(0.25, 0.4)), TN(2.0, pick(0.25, 0.5), 1.0, 3.0),
                      N(0.0, pick(0.1, 0.2)), N(0.0, pick(0.1, 0.2)),
                      N(0.0, pick(0.03, 0.06)), N(0.0, pick(0.03, 0.06)),
                      N(0.0, pick(0.05, 0.1)), N(0.0, pick(0.05, 0.1))]
    for _ in range(n_lens_light):
        p += [LogN(math.log(1.6), pick(0.15, 0.25)), U(pick(2.0, 0.5), pick(6.0, 8.0)),
              TN(0.0, pick(0.05, 0.1), -0.15, 0.15), TN(0.0, pick(0.05, 0.1), -0.15, 0.15),
              N(0.0, pick(0.01, 0.02)), N(0.0, pick(0.01, 0.02)),
              LogN(math.log(300.0), pick(0.3, 0.5))]
    for _ in range(n_source):
        p += [LogN(math.log(0.25), pick(0.15, 0.25)), U(0.5, pick(4.0, 8.0)),
              TN(0.0, pick(0.15, 0.3), -0.5, 0.5), TN(0.0, pick(0.15, 0.3), -0.5, 0.5),
              N(0.0, pick(0.25, 0.5)), N(0.0, pick(0.25, 0.5)),
              LogN(math.log(150.0), pick(0.5, 0.9))]
    return PriorSpec(p, [0.0] * (1 + n_lens_light + n_source))


def _draw_one(pr: Prior, rng: np.random.Generator) -> float:
    if pr.kind == "uniform":
        return float(rng.uniform(pr.lo, pr.hi))
    if pr.kind == "normal":
        return float(rng.normal(pr.a, pr.b))
    if pr.kind == "truncnorm":
        while True:
            v = float(rng.normal(pr.a, pr.b))
            if pr.lo <= v <= pr.hi:
                return v
    if pr.kind == "lognormal":
        return float(math.exp(rng.normal(pr.a, pr.b)))
    raise ValueError(f"cannot draw from prior kind {pr.kind!r}")


def component_slices(n_lens_light: int, n_source: int) -> List[Tuple[int, int]]:
    """(e1 index, e2 index) of every component, in emax order."""
    out = [(2, 3)]
    for c in range(n_lens_light + n_source):
        base = 8 + 7 * c
        out.append((base + 2, base + 3))
    return out


def draw(spec: PriorSpec, n: int, seed: int, n_lens_light: int = 1,
         n_source: int = 1) -> np.ndarray:
    """n parameter vectors [n, P] (float64) from the priors, with the |e| < emax
    pairs enforced by redrawing the pair."""
    rng = np.random.default_rng(seed)
    P = len(spec.params)
    assert P == num_params(n_lens_light, n_source)
    pairs = component_slices(n_lens_light, n_source)
    out = np.empty((n, P), dtype=np.float64)
    for r in range(n):
        for k in range(P):
            out[r, k] = _draw_one(spec.params[k], rng)
        for (i1, i2), em in zip(pairs, spec.emax):
            if em > 0:
                while math.hypot(out[r, i1], out[r, i2]) >= em:
                    out[r, i1] = _draw_one(spec.params[i1], rng)
                    out[r, i2] = _draw_one(spec.params[i2], rng)
    return out


def jitter(theta0: np.ndarray, spec: PriorSpec, n: int, seed: int,
           rel: float = 0.01) -> np.ndarray:
    """n vectors near theta0: theta0 + N(0, rel * prior width) per parameter,
    kept inside each prior's support. Used for HMC chain starts."""
    rng = np.random.default_rng(seed)
    widths = []
    for pr in spec.params:
        if pr.kind in ("uniform", "flat") and math.isfinite(pr.hi - pr.lo):
            widths.append((pr.hi - pr.lo) / math.sqrt(12.0))
        elif pr.kind == "lognormal":
            widths.append(math.exp(pr.a) * pr.b)
        else:
            widths.append(pr.b)
    w = np.asarray(widths)
    out = theta0[None, :] + rel * w[None, :] * rng.standard_normal((n, theta0.size))
    for k, pr in enumerate(spec.params):
        lo = pr.lo if math.isfinite(pr.lo) else -np.inf
        hi = pr.hi if math.isfinite(pr.hi) else np.inf
        if pr.kind == "lognormal":
            lo = max(lo, 1e-6)
        span = 1e-9 * max(1.0, abs(theta0[k]))
        out[:, k] = np.clip(out[:, k], lo + span, hi - span)
    return out


# ----------------------------------------------------------------- PSFs ----

def moffat_psf(size: int, pixel_scale: float, fwhm: float,
               beta: float = 4.765) -> np.ndarray:
    """Moffat (1969) profile (1 + r^2/alpha^2)^-beta sampled at pixel centres,
    alpha = FWHM / (2 sqrt(2^(1/beta) - 1)); beta = 4.765 (Trujillo et al.
    2001). Normalised to unit sum."""
    assert size % 2 == 1
    alpha = fwhm / (2.0 * math.sqrt(2.0 ** (1.0 / beta) - 1.0))
    c = (size - 1) / 2.0
    yy, xx = np.mgrid[0:size, 0:size].astype(np.float64)
    r2 = ((xx - c) ** 2 + (yy - c) ** 2) * pixel_scale ** 2
    k = (1.0 + r2 / alpha ** 2) ** (-beta)
    return k / k.sum()


def gaussian_core_psf(size: int, pixel_scale: float, fwhm_core: float = 0.08,
                      fwhm_wing: float = 0.25, core_frac: float = 0.9) -> np.ndarray:
    """Space-telescope-like PSF: core_frac * G(fwhm_core) + (1 - core_frac) *
    G(fwhm_wing), unit-integral 2-D Gaussians sampled at pixel centres, then
    normalised to unit sum."""
    assert size % 2 == 1
    c = (size - 1) / 2.0
    yy, xx = np.mgrid[0:size, 0:size].astype(np.float64)
    r2 = ((xx - c) ** 2 + (yy - c) ** 2) * pixel_scale ** 2
    k = np.zeros_like(r2)
    for frac, fw in ((core_frac, fwhm_core), (1.0 - core_frac, fwhm_wing)):
        s = fw / (2.0 * math.sqrt(2.0 * math.log(2.0)))
        k += frac * np.exp(-r2 / (2.0 * s * s)) / (2.0 * math.pi * s * s)
    return k / k.sum()


# ---------------------------------------------------------------- noise ----

def noise_draws(shape: Sequence[int], seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(tuple(shape))


def noisy_data(m_true: np.ndarray, eps: np.ndarray,
               sky: float = 0.01, gain: float = 10.0) -> Tuple[np.ndarray, np.ndarray]:
    """Noise map sigma = sqrt(sky^2 + m_true / gain) from the noiseless truth
    and data d = m_true + sigma * eps (eps ~ N(0, 1), drawn by noise_draws)."""
    sigma = np.sqrt(sky * sky + np.maximum(m_true, 0.0) / gain)
    return m_true + sigma * eps, sigma


# -------------------------------------------------------------- systems ----

@dataclasses.dataclass
class Workload:
    """Shape of one synthetic lens system and its sample batch."""
    name: str
    ny: int
    nx: int
    pixel_scale: float
    supersample: int
    psf: np.ndarray
    n_lens_light: int
    n_source: int
    batch: int
    seed_truth: int
    seed_noise: int
    seed_samples: int

    @property
    def P(self) -> int:
        return num_params(self.n_lens_light, self.n_source)

    def prior(self) -> PriorSpec:
        return config_prior(self.n_lens_light, self.n_source)

    def truth(self) -> np.ndarray:
        return draw(self.prior(), 1, self.seed_truth, self.n_lens_light, self.n_source)[0]

    def samples(self, n: int | None = None) -> np.ndarray:
        return draw(self.prior(), self.batch if n is None else n, self.seed_samples,
                    self.n_lens_light, self.n_source)

    def noise(self) -> np.ndarray:
        return noise_draws((self.ny, self.nx), self.seed_noise)


def ground_60() -> Workload:
    """60x60 px at 0.262"/px, s = 2, 11x11 Moffat FWHM 1.1", 64 samples."""
    return Workload("ground-60x60-s2", 60, 60, 0.262, 2, moffat_psf(11, 0.262, 1.1),
                    1, 1, 64, 101, 102, 103)


def ground_100() -> Workload:
    """100x100 px at 0.262"/px, s = 3, 11x11 Moffat FWHM 1.1", 4096 samples."""
    return Workload("ground-100x100-s3", 100, 100, 0.262, 3, moffat_psf(11, 0.262, 1.1),
                    1, 1, 4096, 201, 202, 203)


def space_200() -> Workload:
    """200x200 px at 0.05"/px, s = 5, 21x21 Gaussian-core PSF, two source
    components, 16384 chains."""
    return Workload("space-200x200-s5", 200, 200, 0.05, 5, gaussian_core_psf(21, 0.05),
                    1, 2, 16384, 301, 302, 303)


def uneven_systems(n_systems: int = 100, samples_each: int = 256,
                   seed: int = 501) -> List[Workload]:
    """Systems of uneven size: sides from {40, 64, 100, 150, 200} px, s from
    {2, 3, 4, 5}, 1-3 source components; ground-based pixel scale and PSF."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_systems):
        side = int(rng.choice([40, 64, 100, 150, 200]))
        s = int(rng.choice([2, 3, 4, 5]))
        ns = int(rng.integers(1, 4))
        out.append(Workload(f"uneven-{k}-{side}px-s{s}-src{ns}", side, side, 0.262, s,
                            moffat_psf(11, 0.262, 1.1), 1, ns, samples_each,
                            seed * 1000 + 3 * k, seed * 1000 + 3 * k + 1,
                            seed * 1000 + 3 * k + 2))
    return out
