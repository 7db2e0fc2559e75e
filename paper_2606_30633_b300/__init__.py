"""Python binding of libgl, the B300 strong-lens log-posterior library.

Argument marshalling only: every step of the computation runs in libgl's CUDA
kernels behind the C ABI declared in include/gl.h. Torch tensors provide the
device memory and the stream. If libgl.so is missing, or no CUDA device is
present, the calls raise: there is no CPU fallback.

    sys = System(ny, nx, pixel_scale, supersample, data, sigma, psf,
                 n_lens_light, n_source, prior_spec)
    logp = sys.logp(theta)                # theta: cuda float32 [B, P]
    logp, grad = sys.logp_grad(theta)
    img = sys.model_image(theta)
    logp = LogPosterior.apply(theta, sys)   # autograd through the adjoint
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgl.so")

GL_OK, GL_EINVAL, GL_ENOMEM, GL_ECUDA, GL_ENOSURROGATE, GL_ETIMEOUT = range(6)
GL_DEFL_SERIES, GL_DEFL_SURROGATE, GL_DEFL_TABLE, GL_DEFL_TABLE32 = 0, 1, 2, 3
GL_DEFL_SURROGATE_FUSED = 4
PRIOR_KIND = {"flat": 0, "uniform": 1, "normal": 2, "truncnorm": 3, "lognormal": 4}

_STATUS_NAMES = {0: "GL_OK", 1: "GL_EINVAL", 2: "GL_ENOMEM", 3: "GL_ECUDA",
                 4: "GL_ENOSURROGATE", 5: "GL_ETIMEOUT"}


class GLError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class gl_prior(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("a", ctypes.c_float), ("b", ctypes.c_float),
                ("lo", ctypes.c_float), ("hi", ctypes.c_float)]


_fp = ctypes.POINTER(ctypes.c_float)


class gl_system_desc(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int), ("nx", ctypes.c_int), ("pixel_scale", ctypes.c_float),
                ("supersample", ctypes.c_int), ("data", _fp), ("sigma", _fp), ("psf", _fp),
                ("psf_ny", ctypes.c_int), ("psf_nx", ctypes.c_int),
                ("n_lens_light", ctypes.c_int), ("n_source", ctypes.c_int),
                ("prior", ctypes.POINTER(gl_prior)), ("emax", _fp),
                ("inputs_on_device", ctypes.c_int)]


# (name, restype, argtypes) of every entry point in include/gl.h
_VP = ctypes.c_void_p
SIGNATURES = {
    "gl_system_create": (ctypes.c_int, [ctypes.POINTER(gl_system_desc), ctypes.POINTER(_VP)]),
    "gl_system_destroy": (ctypes.c_int, [_VP]),
    "gl_system_num_params": (ctypes.c_int, [_VP]),
    "gl_logp": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, ctypes.c_int, _VP]),
    "gl_logp_grad": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP, ctypes.c_int, _VP]),
    "gl_logp_grad_host": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP, ctypes.c_int, _VP]),
    "gl_model_image": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, ctypes.c_int, _VP]),
    "gl_leapfrog": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_float, ctypes.c_int,
                                   ctypes.c_int, _VP]),
    "gl_logp_grad_noalloc": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP, _VP]),
    "gl_last_error": (ctypes.c_char_p, []),
    "gl_surrogate_num_params": (ctypes.c_int, []),
    "gl_surrogate_train": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(ctypes.c_float)]),
    "gl_surrogate_create": (ctypes.c_int, [_VP, ctypes.POINTER(_VP)]),
    "gl_surrogate_params": (ctypes.c_int, [_VP, _VP]),
    "gl_surrogate_infer": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP]),
    "gl_series_F": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP]),
    "gl_unit_rates": (ctypes.c_int, [_VP, _VP, _VP]),
    "gl_surrogate_loss_grad": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP, _VP]),
    "gl_debug_force_wait_timeout": (ctypes.c_int, [ctypes.c_int]),
    "gl_surrogate_save": (ctypes.c_int, [_VP, ctypes.c_char_p]),
    "gl_surrogate_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(_VP)]),
    "gl_surrogate_destroy": (None, [_VP]),
    "gl_system_set_surrogate": (ctypes.c_int, [_VP, _VP]),
    "gl_multi_create": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int, ctypes.POINTER(_VP)]),
    "gl_multi_create_ex": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP,
                                          ctypes.POINTER(_VP)]),
    "gl_multi_logp_grad": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int, _VP]),
    "gl_multi_destroy": (ctypes.c_int, [_VP]),
    "gl_bijector_forward": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP, _VP]),
    "gl_bijector_inverse": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP]),
    "gl_logp_grad_unconstrained": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP, ctypes.c_int,
                                                  _VP]),
    "gl_map_adam": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                   _VP, ctypes.c_int, _VP]),
    "gl_hmc_create": (ctypes.c_int, [_VP, _VP, _VP, ctypes.POINTER(_VP), _VP]),
    "gl_hmc_set_inv_mass": (ctypes.c_int, [_VP, _VP, _VP]),
    "gl_hmc_run": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP]),
    "gl_hmc_end_adaptation": (ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    "gl_hmc_state": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.POINTER(ctypes.c_float), _VP]),
    "gl_hmc_destroy": (ctypes.c_int, [_VP]),
    "gl_logp_grad_backward": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _VP, _VP, ctypes.c_int,
                                             _VP]),
    "gl_svi_adabelief": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                        ctypes.c_float, ctypes.c_ulonglong, _VP, ctypes.c_int,
                                        _VP]),
    "gl_svi_adabelief_ex": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                           ctypes.c_float, ctypes.c_float, ctypes.c_ulonglong,
                                           _VP, ctypes.c_int, ctypes.c_int, _VP]),
}

GL_HMC_ADAPT_STEP, GL_HMC_COLLECT_MOMENTS = 1, 2
GL_SVI_SCORE, GL_SVI_PATHWISE = 0, 1


class gl_hmc_desc(ctypes.Structure):
    _fields_ = [("chains", ctypes.c_int), ("n_leapfrog", ctypes.c_int),
                ("step_size", ctypes.c_float), ("target_accept", ctypes.c_float),
                ("seed", ctypes.c_ulonglong), ("deflection", ctypes.c_int)]

GL_MULTI_SMEM_GLOBAL, GL_MULTI_SMEM_TWO_CTAS, GL_MULTI_SMEM_ONE_CTA = 0, 1, 2


class gl_surrogate_train_desc(ctypes.Structure):
    _fields_ = [("n_samples", ctypes.c_longlong), ("epochs", ctypes.c_int),
                ("batch", ctypes.c_int), ("lr", ctypes.c_float), ("lr_min", ctypes.c_float),
                ("seed_data", ctypes.c_ulonglong), ("seed_init", ctypes.c_ulonglong),
                ("q_lo", ctypes.c_float), ("q_hi", ctypes.c_float),
                ("gamma_lo", ctypes.c_float), ("gamma_hi", ctypes.c_float),
                ("r_lo", ctypes.c_float), ("r_hi", ctypes.c_float)]

_LIB: Optional[ctypes.CDLL] = None


def load() -> ctypes.CDLL:
    """Loads libgl.so (built by paper_2606_30633_b300/build.py)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_2606_30633_b300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def last_error() -> str:
    return load().gl_last_error().decode()


def _check(status: int):
    if status != GL_OK:
        raise GLError(status, last_error())


def _torch():
    import torch
    return torch


def _stream_ptr(stream) -> int:
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _ptr(t) -> Optional[int]:
    return None if t is None else int(t.data_ptr())


def _need(t, shape, name: str):
    """t must be a contiguous CUDA float32 tensor of exactly this shape: the
    library reads or writes through its raw pointer, so a short buffer would
    be accessed out of bounds."""
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA float32 tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, not {tuple(t.shape)}")
    return t


def prior_array(prior_spec) -> ctypes.Array:
    arr = (gl_prior * len(prior_spec.params))()
    for k, p in enumerate(prior_spec.params):
        arr[k] = gl_prior(PRIOR_KIND[p.kind], p.a, p.b, p.lo, p.hi)
    return arr


class System:
    """One lens system resident on the current CUDA device."""

    def __init__(self, ny: int, nx: int, pixel_scale: float, supersample: int, data, sigma, psf,
                 n_lens_light: int, n_source: int, prior_spec):
        lib = load()
        self._lib = lib
        data = np.ascontiguousarray(np.asarray(data, dtype=np.float32).reshape(ny, nx))
        sigma = np.ascontiguousarray(np.asarray(sigma, dtype=np.float32).reshape(ny, nx))
        psf = np.ascontiguousarray(np.asarray(psf, dtype=np.float32))
        self._prior = prior_array(prior_spec)
        emax = np.ascontiguousarray(np.asarray(prior_spec.emax, dtype=np.float32))
        desc = gl_system_desc(ny, nx, pixel_scale, supersample,
                              data.ctypes.data_as(_fp), sigma.ctypes.data_as(_fp),
                              psf.ctypes.data_as(_fp), psf.shape[0], psf.shape[1],
                              n_lens_light, n_source, self._prior, emax.ctypes.data_as(_fp), 0)
        h = _VP()
        _check(lib.gl_system_create(ctypes.byref(desc), ctypes.byref(h)))
        self._h = h
        self.ny, self.nx, self.P = ny, nx, int(lib.gl_system_num_params(h))
        self.s, self.psf_size = int(supersample), int(psf.shape[0])
        self.n_lens_light, self.n_source = n_lens_light, n_source

    @property
    def handle(self):
        return self._h

    def set_surrogate(self, sur: Optional["Surrogate"]):
        """Attach a surrogate (kept alive by this object) or detach with None."""
        self._sur = sur
        _check(self._lib.gl_system_set_surrogate(self._h, None if sur is None else sur._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gl_system_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _theta(self, theta):
        torch = _torch()
        if not (isinstance(theta, torch.Tensor) and theta.is_cuda and theta.dtype == torch.float32):
            raise TypeError("theta must be a CUDA float32 tensor")
        theta = theta.contiguous()
        if theta.dim() != 2 or theta.shape[1] != self.P:
            raise ValueError(f"theta must be [B, {self.P}]")
        return theta

    def logp(self, theta, defl: int = GL_DEFL_SERIES, out=None, stream=None):
        torch = _torch()
        theta = self._theta(theta)
        B = theta.shape[0]
        out = (torch.empty(B, device=theta.device, dtype=torch.float32) if out is None
               else _need(out, (B,), "out"))
        _check(self._lib.gl_logp(self._h, _ptr(theta), B, _ptr(out), defl, _stream_ptr(stream)))
        return out

    def logp_grad(self, theta, defl: int = GL_DEFL_SERIES, out=None, grad=None, stream=None):
        torch = _torch()
        theta = self._theta(theta)
        B = theta.shape[0]
        out = (torch.empty(B, device=theta.device, dtype=torch.float32) if out is None
               else _need(out, (B,), "out"))
        grad = torch.empty_like(theta) if grad is None else _need(grad, (B, self.P), "grad")
        _check(self._lib.gl_logp_grad(self._h, _ptr(theta), B, _ptr(out), _ptr(grad), defl,
                                      _stream_ptr(stream)))
        return out, grad

    def leapfrog(self, theta, p, logp, grad, inv_mass, eps: float, n_steps: int, stream=None):
        """n_steps leapfrog steps in place (one CUDA graph launch; see gl.h).
        theta, p, grad: CUDA float32 [B, P]; logp [B]; inv_mass [P]."""
        torch = _torch()
        for t in (theta, p, logp, grad, inv_mass):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
                    and t.is_contiguous()):
                raise TypeError("leapfrog buffers must be contiguous CUDA float32 tensors")
        B = theta.shape[0]
        if theta.shape != (B, self.P) or p.shape != theta.shape or grad.shape != theta.shape \
                or logp.shape != (B,) or inv_mass.shape != (self.P,):
            raise ValueError("leapfrog buffer shapes do not match [B, P]")
        _check(self._lib.gl_leapfrog(self._h, _ptr(theta), _ptr(p), _ptr(logp), _ptr(grad),
                                     _ptr(inv_mass), float(eps), int(n_steps), B,
                                     _stream_ptr(stream)))

    # ---- inference layer (unconstrained parameters u; see include/gl.h) ----
    def _rows(self, x, name="u"):
        torch = _torch()
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float32):
            raise TypeError(f"{name} must be a CUDA float32 tensor")
        x = x.contiguous()
        if x.dim() != 2 or x.shape[1] != self.P:
            raise ValueError(f"{name} must be [B, {self.P}]")
        return x

    def bijector_forward(self, u, stream=None):
        """theta(u) and log|det d theta/d u| per row."""
        torch = _torch()
        u = self._rows(u)
        B = u.shape[0]
        th = torch.empty_like(u)
        lj = torch.empty(B, device=u.device, dtype=torch.float32)
        _check(self._lib.gl_bijector_forward(self._h, _ptr(u), B, _ptr(th), _ptr(lj),
                                             _stream_ptr(stream)))
        return th, lj

    def bijector_inverse(self, theta, stream=None):
        torch = _torch()
        theta = self._rows(theta, "theta")
        u = torch.empty_like(theta)
        _check(self._lib.gl_bijector_inverse(self._h, _ptr(theta), theta.shape[0], _ptr(u),
                                             _stream_ptr(stream)))
        return u

    def logp_grad_unconstrained(self, u, defl: int = GL_DEFL_SERIES, stream=None):
        """log p~(u) = log p(theta(u)) + log|J| and its gradient w.r.t. u."""
        torch = _torch()
        u = self._rows(u)
        B = u.shape[0]
        lp = torch.empty(B, device=u.device, dtype=torch.float32)
        g = torch.empty_like(u)
        _check(self._lib.gl_logp_grad_unconstrained(self._h, _ptr(u), B, _ptr(lp), _ptr(g), defl,
                                                    _stream_ptr(stream)))
        return lp, g

    def map_adam(self, u, m, v, n_steps: int, t0: int = 0, lr: float = 1e-2, beta1: float = 0.9,
                 beta2: float = 0.999, eps: float = 1e-8, defl: int = GL_DEFL_SERIES,
                 logp=None, stream=None):
        """n_steps of Adam on every row of u in place (multi-start MAP); m, v
        are the Adam moments (zeros for a fresh start). Returns log p~ at the
        last point evaluated."""
        torch = _torch()
        B = u.shape[0] if isinstance(u, torch.Tensor) and u.dim() == 2 else -1
        for t, name in ((u, "u"), (m, "m"), (v, "v")):
            _need(t, (B, self.P), name)
        logp = (torch.empty(B, device=u.device, dtype=torch.float32) if logp is None
                else _need(logp, (B,), "logp"))
        _check(self._lib.gl_map_adam(self._h, _ptr(u), _ptr(m), _ptr(v), B, int(n_steps),
                                     int(t0), float(lr), float(beta1), float(beta2), float(eps),
                                     _ptr(logp), defl, _stream_ptr(stream)))
        return logp

    def svi_adabelief(self, phi, opt, n_samples: int, n_steps: int, t0: int = 0,
                      lr: float = 1e-4, beta1: float = 0.95, beta2: float = 0.99,
                      eps: float = 1e-16, seed: int = 0, defl: int = GL_DEFL_SERIES,
                      stream=None, estimator: int = GL_SVI_SCORE):
        """n_steps of SVI (AdaBelief on phi = (mu, L with log diagonal)) in
        place; opt is AdaBelief's state [2 (P + P^2)]. estimator:
        GL_SVI_SCORE (the printed score-function gradient) or GL_SVI_PATHWISE
        (the reparameterisation gradient; see gl_svi_adabelief_ex). Returns the
        per-step ELBO estimates [n_steps]."""
        torch = _torch()
        P = self.P
        if phi.shape != (P + P * P,) or opt.shape != (2 * (P + P * P),):
            raise ValueError("phi must be [P + P^2] and opt [2 (P + P^2)]")
        for t in (phi, opt):
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise TypeError("phi and opt must be contiguous CUDA float32 tensors")
        elbo = torch.empty(max(int(n_steps), 1), device=phi.device, dtype=torch.float32)
        _check(self._lib.gl_svi_adabelief_ex(self._h, _ptr(phi), _ptr(opt), int(n_samples),
                                             int(n_steps), int(t0), float(lr), float(beta1),
                                             float(beta2), float(eps), int(seed), _ptr(elbo),
                                             defl, int(estimator), _stream_ptr(stream)))
        return elbo[:int(n_steps)]

    def logp_grad_backward(self, theta, defl: int = GL_DEFL_SERIES, stream=None):
        """Backward intensity modelling: (log p, gradient, solved intensities
        [B, n_lens_light + n_source]); theta's intensity entries are ignored."""
        torch = _torch()
        theta = self._theta(theta)
        B = theta.shape[0]
        lp = torch.empty(B, device=theta.device, dtype=torch.float32)
        g = torch.empty_like(theta)
        inten = torch.empty(B, self.n_lens_light + self.n_source, device=theta.device,
                            dtype=torch.float32)
        _check(self._lib.gl_logp_grad_backward(self._h, _ptr(theta), B, _ptr(lp), _ptr(g),
                                               _ptr(inten), defl, _stream_ptr(stream)))
        return lp, g, inten

    def logp_grad_noalloc(self, theta, out=None, grad=None, stream=None):
        """gl_logp_grad_noalloc: the same result without any device allocation
        inside the call (fixed library scratch; see include/gl.h)."""
        torch = _torch()
        theta = self._theta(theta)
        B = theta.shape[0]
        out = (torch.empty(B, device=theta.device, dtype=torch.float32) if out is None
               else _need(out, (B,), "out"))
        grad = torch.empty_like(theta) if grad is None else _need(grad, (B, self.P), "grad")
        _check(self._lib.gl_logp_grad_noalloc(self._h, _ptr(theta), B, _ptr(out), _ptr(grad),
                                              _stream_ptr(stream)))
        return out, grad

    def logp_grad_host(self, theta: np.ndarray, defl: int = GL_DEFL_SERIES, want_grad=True,
                       stream=None, out=None):
        """Host arrays in and out (the copies happen inside the call). out:
        optional (logp [B], grad [B, P] or None) float32 arrays to fill. Arrays
        from pinned_array() are copied to and from the device directly."""
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float32))
        if th.ndim != 2 or th.shape[1] != self.P:
            raise ValueError(f"theta must be [B, {self.P}]")
        B = th.shape[0]
        if out is None:
            lp = np.empty(B, dtype=np.float32)
            g = np.empty_like(th) if want_grad else None
        else:
            lp, g = out
            for a, shape, name in ((lp, (B,), "logp"), (g, (B, self.P), "grad")):
                if a is None and name == "grad":
                    continue
                if (not isinstance(a, np.ndarray) or a.dtype != np.float32 or a.shape != shape
                        or not a.flags.c_contiguous or not a.flags.writeable):
                    raise ValueError(f"out {name} must be a writable contiguous float32 "
                                     f"array of shape {shape}")
        _check(self._lib.gl_logp_grad_host(self._h, th.ctypes.data, B, lp.ctypes.data,
                                           None if g is None else g.ctypes.data, defl,
                                           _stream_ptr(stream)))
        return lp, g

    def model_image(self, theta, defl: int = GL_DEFL_SERIES, out=None, stream=None):
        torch = _torch()
        theta = self._theta(theta)
        B = theta.shape[0]
        out = (torch.empty((B, self.ny, self.nx), device=theta.device, dtype=torch.float32)
               if out is None else _need(out, (B, self.ny, self.nx), "out"))
        _check(self._lib.gl_model_image(self._h, _ptr(theta), B, _ptr(out), defl,
                                        _stream_ptr(stream)))
        return out


class Hmc:
    """HMC sampler on log p~(u) (gl_hmc_*; see include/gl.h): B chains, each
    transition a leapfrog trajectory with a Metropolis-Hastings correction,
    all on the device."""

    def __init__(self, system: System, u0, n_leapfrog: int, step_size: float,
                 target_accept: float = 0.75, seed: int = 0, defl: int = GL_DEFL_SERIES,
                 stream=None):
        self._lib = system._lib
        self.system = system
        u0 = system._rows(u0)
        self.B, self.P = u0.shape[0], system.P
        desc = gl_hmc_desc(self.B, int(n_leapfrog), float(step_size), float(target_accept),
                           int(seed), int(defl))
        h = _VP()
        _check(self._lib.gl_hmc_create(system._h, ctypes.byref(desc), _ptr(u0), ctypes.byref(h),
                                       _stream_ptr(stream)))
        self._h = h

    def set_inv_mass(self, inv_mass, stream=None):
        _need(inv_mass.contiguous(), (self.P,), "inv_mass")
        _check(self._lib.gl_hmc_set_inv_mass(self._h, _ptr(inv_mass.contiguous()),
                                             _stream_ptr(stream)))

    def run(self, n: int, flags: int = 0, draws=None, accept=None, stream=None):
        """n transitions; draws [n, B, P] (theta) and accept [n] are optional
        CUDA float32 outputs."""
        torch = _torch()
        for t, shape in ((draws, (n, self.B, self.P)), (accept, (n,))):
            if t is not None and (tuple(t.shape) != shape or t.dtype != torch.float32
                                  or not t.is_cuda or not t.is_contiguous()):
                raise ValueError(f"output must be a contiguous CUDA float32 tensor {shape}")
        _check(self._lib.gl_hmc_run(self._h, int(n), int(flags), _ptr(draws), _ptr(accept),
                                    _stream_ptr(stream)))

    def end_adaptation(self, set_inv_mass: bool = True, stream=None):
        _check(self._lib.gl_hmc_end_adaptation(self._h, int(bool(set_inv_mass)),
                                               _stream_ptr(stream)))

    def state(self, stream=None):
        """(u [B, P], log p~ [B], inv_mass [P], step size) — waits for the stream."""
        torch = _torch()
        dev = torch.device("cuda", torch.cuda.current_device())
        u = torch.empty(self.B, self.P, device=dev)
        lp = torch.empty(self.B, device=dev)
        im = torch.empty(self.P, device=dev)
        eps = ctypes.c_float()
        _check(self._lib.gl_hmc_state(self._h, _ptr(u), _ptr(lp), _ptr(im), ctypes.byref(eps),
                                      _stream_ptr(stream)))
        return u, lp, im, eps.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gl_hmc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Multi:
    """An uneven multi-system batch plan (gl_multi_create_ex /
    gl_multi_logp_grad). threads / pairs: per-system launch shapes (threads per
    CTA in {128, 256}, phase-1 pixel pairs in {2, 3}); None gives 256 / 2."""

    def __init__(self, systems, rows, smem_policy: int = GL_MULTI_SMEM_TWO_CTAS,
                 threads: Optional[Sequence[int]] = None, pairs: Optional[Sequence[int]] = None):
        self._lib = load()
        self.systems = list(systems)
        self.rows = [int(r) for r in rows]
        n = len(self.systems)
        if len(self.rows) != n:
            raise ValueError("one row count per system")
        self.threads = [256] * n if threads is None else [int(t) for t in threads]
        self.pairs = [2] * n if pairs is None else [int(p) for p in pairs]
        if len(self.threads) != n or len(self.pairs) != n:
            raise ValueError("one launch shape per system")
        hs = (_VP * n)(*[s.handle for s in self.systems])
        rs = (ctypes.c_int * n)(*self.rows)
        ts = (ctypes.c_int * n)(*self.threads)
        ps = (ctypes.c_int * n)(*self.pairs)
        h = _VP()
        _check(self._lib.gl_multi_create_ex(hs, n, rs, int(smem_policy), ts, ps, ctypes.byref(h)))
        self._h = h
        self.smem_policy = smem_policy

    def shapes(self):
        """(threads per CTA, pixel pairs) of each system."""
        return list(zip(self.threads, self.pairs))

    def logp_grad(self, thetas, logps=None, grads=None, defl: int = GL_DEFL_SERIES, stream=None):
        """thetas: list of CUDA float32 [rows_k, P_k]; returns lists of logp, grad."""
        torch = _torch()
        n = len(self.systems)
        if len(thetas) != n:
            raise ValueError(f"need one theta per system ({n})")
        thetas = [_need(t.contiguous(), (r, s.P), f"thetas[{k}]")
                  for k, (t, r, s) in enumerate(zip(thetas, self.rows, self.systems))]
        if logps is None:
            logps = [torch.empty(t.shape[0], device=t.device, dtype=torch.float32) for t in thetas]
        if grads is None:
            grads = [torch.empty_like(t) for t in thetas]
        if len(logps) != n or len(grads) != n:
            raise ValueError(f"need one logp and one grad buffer per system ({n})")
        for k, (t, lp_k, g_k) in enumerate(zip(thetas, logps, grads)):
            _need(lp_k, (t.shape[0],), f"logps[{k}]")
            _need(g_k, tuple(t.shape), f"grads[{k}]")
        tp = (_VP * n)(*[_ptr(t) for t in thetas])
        lp = (_VP * n)(*[_ptr(t) for t in logps])
        gp = (_VP * n)(*[_ptr(t) for t in grads])
        _check(self._lib.gl_multi_logp_grad(self._h, tp, lp, gp, int(defl), _stream_ptr(stream)))
        return logps, grads

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gl_multi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Surrogate:
    """The learned EPL deflection surrogate (include/gl.h)."""

    def __init__(self, handle):
        self._lib = load()
        self._h = handle
        self.final_loss = float("nan")

    @staticmethod
    def num_params() -> int:
        return int(load().gl_surrogate_num_params())

    @classmethod
    def train(cls, n_samples=10_000_000, epochs=120, batch=16384, lr=2e-3, lr_min=1e-5,
              seed_data=401, seed_init=402, q=(0.5, 1.0), gamma=(1.7, 2.3), r=(0.05, 5.0)):
        lib = load()
        d = gl_surrogate_train_desc(n_samples, epochs, batch, lr, lr_min, seed_data, seed_init,
                                    q[0], q[1], gamma[0], gamma[1], r[0], r[1])
        h = _VP()
        loss = ctypes.c_float()
        _check(lib.gl_surrogate_train(ctypes.byref(d), ctypes.byref(h), ctypes.byref(loss)))
        s = cls(h)
        s.final_loss = loss.value
        return s

    @classmethod
    def from_params(cls, params):
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        if p.size != cls.num_params():
            raise ValueError(f"the surrogate has {cls.num_params()} parameters, not {p.size}")
        h = _VP()
        _check(load().gl_surrogate_create(p.ctypes.data, ctypes.byref(h)))
        return cls(h)

    @classmethod
    def load_file(cls, path: str):
        h = _VP()
        _check(load().gl_surrogate_load(path.encode(), ctypes.byref(h)))
        return cls(h)

    def save(self, path: str):
        _check(self._lib.gl_surrogate_save(self._h, path.encode()))

    def params(self) -> np.ndarray:
        out = np.empty(self.num_params(), dtype=np.float32)
        _check(self._lib.gl_surrogate_params(self._h, out.ctypes.data))
        return out

    def infer(self, x, stream=None):
        """x: CUDA float32 [N, 4] raw (q, gamma, log R/theta_E, vphi) -> F [N, 2]."""
        torch = _torch()
        x = _need(x.contiguous(), (x.shape[0], 4) if x.dim() == 2 else (-1, 4), "x")
        y = torch.empty((x.shape[0], 2), device=x.device, dtype=torch.float32)
        _check(self._lib.gl_surrogate_infer(self._h, _ptr(x), x.shape[0], _ptr(y),
                                            _stream_ptr(stream)))
        return y

    def loss_grad(self, x, target):
        """Mean squared loss and its parameter gradient (x [N, 4], target [N, 2]
        CUDA float32; N a multiple of 128)."""
        N = x.shape[0] if x.dim() == 2 else -1
        x = _need(x.contiguous(), (N, 4), "x")
        target = _need(target.contiguous(), (N, 2), "target")
        loss = np.empty(1, dtype=np.float32)
        grad = np.empty(self.num_params(), dtype=np.float32)
        _check(self._lib.gl_surrogate_loss_grad(self._h, _ptr(x), _ptr(target), x.shape[0],
                                                loss.ctypes.data, grad.ctypes.data))
        return float(loss[0]), grad

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gl_surrogate_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pinned_array(shape, dtype=np.float32) -> np.ndarray:
    """An uninitialised numpy array in page-locked host memory (a view of a
    pinned torch tensor, which the array keeps alive)."""
    torch = _torch()
    tdt = {np.dtype(np.float32): torch.float32, np.dtype(np.float64): torch.float64}[
        np.dtype(dtype)]
    return torch.empty(shape, dtype=tdt, pin_memory=True).numpy()


def debug_force_wait_timeout(on: bool) -> None:
    """Test hook: the tensor-core surrogate kernels take their wait-timeout path
    at their first wait (see gl_debug_force_wait_timeout in include/gl.h)."""
    _check(load().gl_debug_force_wait_timeout(1 if on else 0))


def series_F(x, stream=None):
    """The exact F of the EPL series in FP64 on the device (gl_series_F):
    x CUDA float32 [N, 4] raw (q, gamma, ., vphi) -> F [N, 2] (Re, Im)."""
    torch = _torch()
    x = _need(x.contiguous(), (x.shape[0], 4) if x.dim() == 2 else (-1, 4), "x")
    F = torch.empty((x.shape[0], 2), device=x.device, dtype=torch.float32)
    _check(load().gl_series_F(_ptr(x), x.shape[0], _ptr(F), _stream_ptr(stream)))
    return F


def unit_rates() -> dict:
    """Measured pipe throughput of the current device in operations per SM per
    SM clock (gl_unit_rates): {"fp32", "fp32x2", "mufu"}."""
    v = [ctypes.c_double() for _ in range(3)]
    _check(load().gl_unit_rates(*[ctypes.addressof(x) for x in v]))
    return {"fp32": v[0].value, "fp32x2": v[1].value, "mufu": v[2].value}


def system_from_workload(W, data, sigma) -> System:
    """System for a synth.Workload with the given data and noise map."""
    return System(W.ny, W.nx, W.pixel_scale, W.supersample, data, sigma, W.psf,
                  W.n_lens_light, W.n_source, W.prior())


def _autograd_function():
    torch = _torch()

    class LogPosterior(torch.autograd.Function):
        """log p(theta) per row with its gradient from the fused adjoint kernel."""

        @staticmethod
        def forward(ctx, theta, system: System, defl: int = GL_DEFL_SERIES):
            lp, g = system.logp_grad(theta.detach().float(), defl)
            ctx.save_for_backward(g)
            return lp

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return grad_out[:, None] * g, None, None

    return LogPosterior


def __getattr__(name):
    if name == "LogPosterior":
        fn = _autograd_function()
        globals()["LogPosterior"] = fn
        return fn
    raise AttributeError(name)
