"""Shared set-up of parity cases: one seeded synthetic lens system handed to
both the FP64 oracle and the CUDA library with identical (float32-rounded)
inputs: parameters, priors, data, noise map, PSF and pixel scale. The
noiseless truth is rendered by the oracle only."""
from __future__ import annotations

import concurrent.futures
import dataclasses
import os

import numpy as np

import oracle
import synth


def f32(a):
    return np.asarray(np.asarray(a, dtype=np.float32), dtype=np.float64)


def round_spec(spec: synth.PriorSpec) -> synth.PriorSpec:
    ps = [synth.Prior(p.kind, float(np.float32(p.a)), float(np.float32(p.b)),
                      float(np.float32(p.lo)), float(np.float32(p.hi))) for p in spec.params]
    return synth.PriorSpec(ps, [float(np.float32(e)) for e in spec.emax])


@dataclasses.dataclass
class Case:
    W: synth.Workload
    spec: synth.PriorSpec
    data: np.ndarray
    sigma: np.ndarray
    psf: np.ndarray
    truth: np.ndarray
    oracle: oracle.System

    def theta(self, n, seed=None):
        spec = self.W.prior()
        th = synth.draw(spec, n, self.W.seed_samples if seed is None else seed,
                        self.W.n_lens_light, self.W.n_source)
        return f32(th)

    def gpu_system(self):
        import paper_2606_30633_b300 as gl
        return gl.System(self.W.ny, self.W.nx, self.W.pixel_scale, self.W.supersample,
                         self.data, self.sigma, self.psf, self.W.n_lens_light,
                         self.W.n_source, self.spec)


def make_case(W: synth.Workload, nthreads: int = 0) -> Case:
    # the library takes the pixel scale as a float: both sides get that value
    W = dataclasses.replace(W, pixel_scale=float(np.float32(W.pixel_scale)))
    spec = round_spec(W.prior())
    psf = f32(W.psf)
    truth = f32(W.truth())
    blank = oracle.System(W.ny, W.nx, W.pixel_scale, W.supersample, np.zeros((W.ny, W.nx)),
                          np.ones((W.ny, W.nx)), psf, W.n_lens_light, W.n_source, spec)
    m = blank.model_image(truth, nthreads=nthreads)[0]
    d, s = synth.noisy_data(m, W.noise())
    d, s = f32(d), f32(s)
    osys = oracle.System(W.ny, W.nx, W.pixel_scale, W.supersample, d, s, psf,
                         W.n_lens_light, W.n_source, spec)
    return Case(W, spec, d, s, psf, truth, osys)


def small_workload(ny, nx, s, psf_size, n_light=1, n_src=1, pixel_scale=0.262, batch=8,
                   seed=11, fwhm=1.1):
    return synth.Workload(f"case-{ny}x{nx}-s{s}-k{psf_size}-{n_light}{n_src}", ny, nx,
                          pixel_scale, s, synth.moffat_psf(psf_size, pixel_scale, fwhm),
                          n_light, n_src, batch, seed, seed + 1, seed + 2)


def image_close(got, ref, rel=1e-5, peak=1e-4):
    """Per-pixel tolerance: a pixel fails only if it misses both the relative
    bound rel |m| and the absolute bound peak max|m| (unit-peak images)."""
    err = np.abs(got - ref)
    bad = (err > rel * np.abs(ref)) & (err > peak * np.max(np.abs(ref)))
    return not bad.any(), float(np.max(err / np.maximum(np.abs(ref), 1e-30)))


def grad_close(got, ref, rel=1e-3, floor=1e-2):
    """|g - g_ref| <= rel max(|g_ref|, floor ||g_ref||_inf), per row."""
    scale = np.maximum(np.abs(ref), floor * np.max(np.abs(ref), axis=-1, keepdims=True))
    return np.all(np.abs(got - ref) <= rel * scale), float(np.max(np.abs(got - ref) / scale))


EPS_MODEL = 5e-6  # per-pixel relative FP32 model error the gradient bound allows for
MODEL_REL = 1e-5  # the stated per-pixel relative model tolerance


def logp_bound(case: "Case", th: np.ndarray, eps=MODEL_REL) -> np.ndarray:
    """Per-row log p tolerance: the stated relative 1e-6, or the first-order
    log p change that a per-pixel relative model error eps (the stated
    per-pixel tolerance) causes, eps sum_p |d_p - m_p| |m_p| / sigma_p^2,
    whichever is larger."""
    th = np.atleast_2d(th)
    ref = case.oracle.logp(th)
    m = case.oracle.model_image(th)
    r = np.abs(case.data[None] - m) * np.abs(m) / case.sigma[None] ** 2
    return np.maximum(1e-6 * np.abs(ref), eps * r.reshape(len(th), -1).sum(1))


def logp_close(case: "Case", th: np.ndarray, got) -> tuple:
    """(ok, worst error / bound) of GPU log p values against logp_bound."""
    th = np.atleast_2d(th)
    err = np.abs(np.asarray(got, np.float64) - case.oracle.logp(th))
    tol = logp_bound(case, th)
    return bool(np.all(err <= tol)), float(np.max(err / tol))


POS_DELTA = 2e-6  # arcsec: FP32 position precision of grid and deflection


def centre_indices(n_comp: int):
    xs = [4] + [8 + 7 * k + 4 for k in range(n_comp)]
    return xs, [i + 1 for i in xs]


def grad_bound(case: "Case", th: np.ndarray, rel=1e-3, eps=EPS_MODEL,
               pos_delta=POS_DELTA) -> np.ndarray:
    """Per-row, per-parameter gradient tolerance, the sum of
      rel |g_ref|;
      the first-order gradient change that a per-pixel relative model error
      eps (in m and in dm/dtheta) causes,
        eps sum_p (|m_p| + |d_p - m_p|) |dm_p/dtheta_k| / sigma_p^2,
      from the oracle's FP64 Jacobian (near the mode the gradient is a small
      difference of large sums, so this term sets the bound there);
      the gradient change under a coherent shift of every component centre by
      pos_delta in x and in y (FP32 grid and deflection positions are good to
      ~1e-6 arcsec; far from the mode, where a steep deflection or Sersic cusp
      meets the grid, the gradient moves by up to ~5e-3 per 1e-6 arcsec)."""
    th = np.atleast_2d(th)
    out = np.empty_like(th)
    w = 1.0 / case.sigma ** 2
    _, gref = case.oracle.logp_grad(th)
    xs, ys = centre_indices(case.W.n_lens_light + case.W.n_source)
    tx, ty = th.copy(), th.copy()
    tx[:, xs] += pos_delta
    ty[:, ys] += pos_delta
    _, gx = case.oracle.logp_grad(tx)
    _, gy = case.oracle.logp_grad(ty)
    def model_term(b):
        m, J = case.oracle.model_jacobian(th[b])
        wt = w * (np.abs(m) + np.abs(case.data - m))
        return eps * np.einsum("ij,ijk->k", wt, np.abs(J))

    # the oracle's Jacobian is serial per row; ctypes releases the GIL, so rows run in parallel
    with concurrent.futures.ThreadPoolExecutor(max(1, min(th.shape[0], os.cpu_count() or 1))) as ex:
        terms = list(ex.map(model_term, range(th.shape[0])))
    for b in range(th.shape[0]):
        out[b] = (rel * np.abs(gref[b]) + terms[b]
                  + np.abs(gx[b] - gref[b]) + np.abs(gy[b] - gref[b]))
    return out


def central_differences(case: "Case", th: np.ndarray) -> np.ndarray:
    """FP64 central differences of the oracle's log p, h = 1e-6 max(|theta_k|, 1),
    for every row and parameter (all 2 P shifted rows of a row in one call)."""
    th = np.atleast_2d(np.asarray(th, np.float64))
    B, P = th.shape
    h = 1e-6 * np.maximum(np.abs(th), 1.0)
    shifted = np.repeat(th, 2 * P, axis=0).reshape(B, 2 * P, P)
    for k in range(P):
        shifted[:, 2 * k, k] += h[:, k]
        shifted[:, 2 * k + 1, k] -= h[:, k]
    lp = case.oracle.logp(shifted.reshape(-1, P)).reshape(B, P, 2)
    return (lp[:, :, 0] - lp[:, :, 1]) / (2 * h)


def grad_close_bound(got, ref, bound):
    """(ok, worst ratio err/bound and where: (row, parameter index, got, ref))."""
    err = np.abs(np.asarray(got, np.float64) - ref)
    # an exact zero bound (an entry that is exactly 0 on both sides) counts as ratio 0
    # unless the error is non-zero
    r = np.atleast_2d(np.divide(err, bound, out=np.where(err > 0, np.inf, 0.0), where=bound > 0))
    b, k = np.unravel_index(int(np.argmax(r)), r.shape)
    g2, r2 = np.atleast_2d(got), np.atleast_2d(ref)
    return bool(np.all(err <= bound)), (float(r[b, k]), int(b), int(k), float(g2[b, k]),
                                       float(r2[b, k]))


FP32_POS = 1.2e-7  # arcsec: half an FP32 ulp of a 2" coordinate (the Einstein radius)


def position_floor(case: "Case", th: np.ndarray, delta=FP32_POS) -> np.ndarray:
    """Per-row, per-parameter conditioning floor of the gradient at the FP32
    precision of positions: the largest change of the oracle's FP64 gradient
    when a single component centre (lens, lens light or source) moves by
    delta in x or in y. An FP32 evaluation's lens-frame and source-plane
    positions carry rounding of that size, so no FP32 evaluation can be held
    below this floor on an entry whose floor exceeds the stated bound."""
    th = np.atleast_2d(np.asarray(th, np.float64))
    B, P = th.shape
    xs, ys = centre_indices(case.W.n_lens_light + case.W.n_source)
    idx = list(xs) + list(ys)
    shifted = np.repeat(th, len(idx), axis=0).reshape(B, len(idx), P)
    for m, k in enumerate(idx):
        shifted[:, m, k] += delta
    _, g0 = case.oracle.logp_grad(th)
    _, g = case.oracle.logp_grad(shifted.reshape(-1, P))
    return np.abs(g.reshape(B, len(idx), P) - g0[:, None, :]).max(1)
