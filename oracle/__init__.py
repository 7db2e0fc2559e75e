"""FP64 CPU oracle of the strong-lens log-posterior (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It wraps ``gl_oracle.cpp`` (compiled by
``oracle/build.py`` into ``liboracle.so``) with ctypes and numpy. It shares no
code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB: Optional[ctypes.CDLL] = None

_KIND = {"flat": 0, "uniform": 1, "normal": 2, "truncnorm": 3, "lognormal": 4}

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class _System(ctypes.Structure):
    _fields_ = [
        ("ny", ctypes.c_int), ("nx", ctypes.c_int), ("pixel_scale", ctypes.c_double),
        ("supersample", ctypes.c_int),
        ("data", _dp), ("sigma", _dp), ("psf", _dp),
        ("psf_ny", ctypes.c_int), ("psf_nx", ctypes.c_int),
        ("n_lens_light", ctypes.c_int), ("n_source", ctypes.c_int),
        ("prior_kind", _ip), ("prior_a", _dp), ("prior_b", _dp),
        ("prior_lo", _dp), ("prior_hi", _dp), ("emax", _dp),
    ]


def lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        sp = ctypes.POINTER(_System)
        L.or_num_params.argtypes = [ctypes.c_int, ctypes.c_int]
        L.or_series_terms.argtypes = [ctypes.c_double]
        L.or_hyp2f1_series.argtypes = [ctypes.c_double] * 3 + [_dp, _dp]
        L.or_epl_deflection.argtypes = [_dp, ctypes.c_int, _dp, _dp, _dp, _dp]
        L.or_sersic.argtypes = [_dp, ctypes.c_int, _dp, _dp, _dp]
        L.or_surface_brightness.argtypes = [sp, _dp, ctypes.c_int, _dp, _dp, _dp]
        L.or_convolve_same.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int,
                                       ctypes.c_int, _dp]
        L.or_binned_image.argtypes = [sp, _dp, _dp]
        L.or_model_image.argtypes = [sp, _dp, ctypes.c_int, _dp, ctypes.c_int]
        L.or_in_support.argtypes = [sp, _dp]
        L.or_log_prior.argtypes = [sp, _dp]
        L.or_log_prior.restype = ctypes.c_double
        L.or_log_likelihood.argtypes = [sp, _dp]
        L.or_log_likelihood.restype = ctypes.c_double
        L.or_logp.argtypes = [sp, _dp, ctypes.c_int, _dp, ctypes.c_int]
        L.or_logp_grad.argtypes = [sp, _dp, ctypes.c_int, _dp, _dp, ctypes.c_int]
        L.or_model_jacobian.argtypes = [sp, _dp, _dp, _dp]
        _LIB = L
    return _LIB


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def max_threads() -> int:
    return int(lib().or_max_threads())


def num_params(n_lens_light: int, n_source: int) -> int:
    return int(lib().or_num_params(n_lens_light, n_source))


def series_terms(f: float) -> int:
    return int(lib().or_series_terms(float(f)))


def hyp2f1_series(t: float, f: float, varphi: float) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().or_hyp2f1_series(t, f, varphi, ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def epl_deflection(p6: Sequence[float], x, y):
    p = _f64(p6)
    x, y = _f64(x).ravel(), _f64(y).ravel()
    ax, ay = np.empty_like(x), np.empty_like(x)
    lib().or_epl_deflection(_d(p), x.size, _d(x), _d(y), _d(ax), _d(ay))
    return ax, ay


def sersic(p7: Sequence[float], x, y):
    p = _f64(p7)
    x, y = _f64(x), _f64(y)
    shape = x.shape
    x, y = x.ravel(), y.ravel()
    out = np.empty_like(x)
    lib().or_sersic(_d(p), x.size, _d(x), _d(y), _d(out))
    return out.reshape(shape)


def convolve_same(img, psf):
    img, psf = _f64(img), _f64(psf)
    out = np.empty_like(img)
    lib().or_convolve_same(_d(img), img.shape[0], img.shape[1], _d(psf), psf.shape[0],
                           psf.shape[1], _d(out))
    return out


class System:
    """One lens system: image geometry, data, noise map, PSF, model spec and
    priors (a synth.PriorSpec). All arrays are held as float64 copies."""

    def __init__(self, ny, nx, pixel_scale, supersample, data, sigma, psf,
                 n_lens_light, n_source, prior_spec):
        self.ny, self.nx = int(ny), int(nx)
        self.pixel_scale, self.supersample = float(pixel_scale), int(supersample)
        self.n_lens_light, self.n_source = int(n_lens_light), int(n_source)
        self.P = num_params(self.n_lens_light, self.n_source)
        self.data = _f64(data).reshape(self.ny, self.nx)
        self.sigma = _f64(sigma).reshape(self.ny, self.nx)
        self.psf = _f64(psf)
        pr = prior_spec.params
        assert len(pr) == self.P
        self.kind = np.ascontiguousarray([_KIND[p.kind] for p in pr], dtype=np.int32)
        self.pa = _f64([p.a for p in pr])
        self.pb = _f64([p.b for p in pr])
        self.plo = _f64([p.lo for p in pr])
        self.phi = _f64([p.hi for p in pr])
        self.emax = _f64(prior_spec.emax)
        assert self.emax.size == 1 + self.n_lens_light + self.n_source
        self._s = _System(self.ny, self.nx, self.pixel_scale, self.supersample,
                          _d(self.data), _d(self.sigma), _d(self.psf),
                          self.psf.shape[0], self.psf.shape[1],
                          self.n_lens_light, self.n_source,
                          self.kind.ctypes.data_as(_ip), _d(self.pa), _d(self.pb),
                          _d(self.plo), _d(self.phi), _d(self.emax))

    @property
    def ref(self):
        return ctypes.byref(self._s)

    def _theta(self, theta) -> np.ndarray:
        th = _f64(theta)
        if th.ndim == 1:
            th = th[None, :]
        assert th.shape[1] == self.P
        return np.ascontiguousarray(th)

    def surface_brightness(self, theta, x, y):
        th = _f64(theta)
        x, y = _f64(x), _f64(y)
        shape = x.shape
        x, y = x.ravel(), y.ravel()
        out = np.empty_like(x)
        lib().or_surface_brightness(self.ref, _d(th), x.size, _d(x), _d(y), _d(out))
        return out.reshape(shape)

    def binned_image(self, theta):
        th = _f64(theta)
        out = np.empty((self.ny, self.nx))
        lib().or_binned_image(self.ref, _d(th), _d(out))
        return out

    def model_image(self, theta, nthreads: int = 0):
        th = self._theta(theta)
        out = np.empty((th.shape[0], self.ny, self.nx))
        lib().or_model_image(self.ref, _d(th), th.shape[0], _d(out), nthreads)
        return out

    def model_jacobian(self, theta):
        """Model image [ny, nx] and d m / d theta [ny, nx, P] (dual numbers)."""
        th = _f64(theta)
        m = np.empty((self.ny, self.nx))
        J = np.empty((self.ny, self.nx, self.P))
        lib().or_model_jacobian(self.ref, _d(th), _d(m), _d(J))
        return m, J

    def in_support(self, theta) -> bool:
        return bool(lib().or_in_support(self.ref, _d(_f64(theta))))

    def log_prior(self, theta) -> float:
        return float(lib().or_log_prior(self.ref, _d(_f64(theta))))

    def log_likelihood(self, theta) -> float:
        return float(lib().or_log_likelihood(self.ref, _d(_f64(theta))))

    def logp(self, theta, nthreads: int = 0):
        th = self._theta(theta)
        out = np.empty(th.shape[0])
        lib().or_logp(self.ref, _d(th), th.shape[0], _d(out), nthreads)
        return out

    def logp_grad(self, theta, nthreads: int = 0):
        """log p and its gradient by forward-mode dual numbers. Undefined (NaN)
        where a component's ellipticity is exactly e = 0: |e| = sqrt(e1^2 + e2^2)
        has no derivative there although log p is smooth in (e1, e2); the tests
        use central differences of logp() at such points."""
        th = self._theta(theta)
        lp = np.empty(th.shape[0])
        g = np.empty_like(th)
        lib().or_logp_grad(self.ref, _d(th), th.shape[0], _d(lp), _d(g), nthreads)
        return lp, g
