"""FP64 oracle of "backward" intensity modelling (test infrastructure; only
the tests may import it).

Sec. 3 (methodology) offers two ways to set the lens and source light
intensities: sample them as parameters ("forward" modelling, the rest of this
oracle) or solve for them by linear inversion ("backward" modelling). The
model image is linear in the Sersic intensities, m = sum_k I_k M_k with M_k
the binned, PSF-convolved image of component k at unit intensity, so the
intensities that maximise the Gaussian likelihood solve the weighted normal
equations
    (M^T W M) I = M^T W d,   W = diag(sigma^-2).
Reading taken here (the paper gives no formula): the backward log-posterior is
the profile log-likelihood at the solved intensities plus the log prior of
the other parameters (intensities carry no prior and may come out negative),
and its gradient with respect to the other parameters is the ordinary
gradient at the solved intensities (the intensity derivative of the
likelihood vanishes there, so the solve contributes nothing to first order).
"""
from __future__ import annotations

import numpy as np

import synth

from . import System


def intensity_indices(n_lens_light: int, n_source: int):
    """Indices of the Sersic intensities in theta (the 7th entry of each
    light component, Eq. sim-dist order)."""
    return [8 + 7 * c + 6 for c in range(n_lens_light + n_source)]


def profile_system(system: System, spec: synth.PriorSpec) -> System:
    """The same system with the intensities' priors replaced by flat ones on R
    (the backward model's prior)."""
    idx = set(intensity_indices(system.n_lens_light, system.n_source))
    ps = [synth.Prior("flat", 0.0, 1.0, -np.inf, np.inf) if k in idx else p
          for k, p in enumerate(spec.params)]
    return System(system.ny, system.nx, system.pixel_scale, system.supersample, system.data,
                  system.sigma, system.psf, system.n_lens_light, system.n_source,
                  synth.PriorSpec(ps, spec.emax))


def component_images(system: System, theta) -> np.ndarray:
    """M_k [K, ny, nx] for one row: the model image with intensity k set to 1
    and every other intensity to 0."""
    th = np.asarray(theta, dtype=np.float64)
    idx = intensity_indices(system.n_lens_light, system.n_source)
    rows = np.repeat(th[None, :], len(idx), axis=0)
    rows[:, idx] = 0.0
    for c, k in enumerate(idx):
        rows[c, k] = 1.0
    return system.model_image(rows)


def solve_intensities(system: System, theta) -> np.ndarray:
    """I* [K] of one row from the weighted normal equations."""
    M = component_images(system, theta).reshape(len(intensity_indices(
        system.n_lens_light, system.n_source)), -1)
    w = (1.0 / system.sigma ** 2).ravel()
    A = (M * w) @ M.T
    b = (M * w) @ system.data.ravel()
    return np.linalg.solve(A, b)


def logp_grad_backward(system: System, profile: System, theta):
    """Backward log p, its gradient (zero in the intensity entries) and the
    solved intensities, per row of theta [B, P]."""
    th = np.atleast_2d(np.asarray(theta, dtype=np.float64)).copy()
    idx = intensity_indices(system.n_lens_light, system.n_source)
    I = np.stack([solve_intensities(system, row) for row in th])
    th[:, idx] = I
    lp, g = profile.logp_grad(th)
    g[:, idx] = 0.0
    return lp, g, I
