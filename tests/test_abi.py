"""The C-ABI library loads and exports every entry point include/gl.h declares,
and rejects invalid system descriptions on the host (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2606_30633_b300 as gl
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(gl_[a-z_0-9]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2606_30633_b300 import build
    build.build()
    return gl.load()


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert "gl_logp_grad" in declared and "gl_system_create" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert declared <= set(gl.SIGNATURES), declared - set(gl.SIGNATURES)


def _desc(**kw):
    W = synth.ground_60()
    spec = W.prior()
    args = dict(ny=W.ny, nx=W.nx, ps=W.pixel_scale, s=W.supersample, psf=W.psf, nl=1, ns=1)
    args.update(kw)
    data = np.zeros((args["ny"], args["nx"]), np.float32)
    sig = np.ones_like(data)
    psf = np.asarray(args["psf"], np.float32)
    prior = gl.prior_array(spec)
    keep = (data, sig, psf, prior)
    fp = ctypes.POINTER(ctypes.c_float)
    d = gl.gl_system_desc(args["ny"], args["nx"], args["ps"], args["s"],
                          data.ctypes.data_as(fp), sig.ctypes.data_as(fp), psf.ctypes.data_as(fp),
                          psf.shape[0], psf.shape[1], args["nl"], args["ns"], prior, None, 0)
    return d, keep


@pytest.mark.parametrize("kw,msg", [
    (dict(psf=np.ones((4, 4))), "PSF"),
    (dict(psf=np.ones((23, 23))), "PSF"),
    (dict(s=0), "supersample"),
    (dict(s=9), "supersample"),
    (dict(ns=0), "n_source"),
    (dict(nl=3), "n_lens_light"),
    (dict(ny=0), "image size"),
    (dict(ps=-1.0), "pixel_scale"),
])
def test_invalid_descriptions_are_rejected(lib, kw, msg):
    d, keep = _desc(**kw)
    h = ctypes.c_void_p()
    st = lib.gl_system_create(ctypes.byref(d), ctypes.byref(h))
    assert st == gl.GL_EINVAL
    assert h.value is None
    assert msg in gl.last_error()


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.gl_system_create(None, ctypes.byref(h)) == gl.GL_EINVAL
    assert lib.gl_system_num_params(None) == -1
    assert lib.gl_system_destroy(None) == gl.GL_OK
    assert lib.gl_logp(None, None, 0, None, 0, None) == gl.GL_EINVAL


def test_invalid_sigma_and_prior(lib):
    d, keep = _desc()
    keep[1][0, 0] = 0.0  # sigma must be > 0
    h = ctypes.c_void_p()
    assert lib.gl_system_create(ctypes.byref(d), ctypes.byref(h)) == gl.GL_EINVAL
    assert "sigma" in gl.last_error()
    d, keep = _desc()
    keep[3][0].kind = 1
    keep[3][0].lo, keep[3][0].hi = 2.0, 1.0
    assert lib.gl_system_create(ctypes.byref(d), ctypes.byref(h)) == gl.GL_EINVAL
    assert "prior" in gl.last_error()


def test_inference_entry_points_reject_bad_arguments(lib):
    """Host-side validation of the inference layer (no GPU work is issued)."""
    P = ctypes.c_void_p
    assert lib.gl_bijector_forward(None, None, 0, None, None, None) == gl.GL_EINVAL
    assert lib.gl_bijector_inverse(None, None, 0, None, None) == gl.GL_EINVAL
    assert lib.gl_logp_grad_unconstrained(None, None, 0, None, None, 0, None) == gl.GL_EINVAL
    assert lib.gl_logp_grad_backward(None, None, 0, None, None, None, 0, None) == gl.GL_EINVAL
    assert lib.gl_map_adam(None, None, None, None, 0, 0, 0, 1e-2, 0.9, 0.999, 1e-8, None, 0,
                           None) == gl.GL_EINVAL
    assert lib.gl_svi_adabelief(None, None, None, 1, 1, 0, 1e-4, 0.95, 0.99, 1e-16, 0, None, 0,
                                None) == gl.GL_EINVAL
    assert lib.gl_svi_adabelief_ex(None, None, None, 1, 1, 0, 1e-4, 0.95, 0.99, 1e-16, 0, None,
                                   0, gl.GL_SVI_PATHWISE, None) == gl.GL_EINVAL
    h = P()
    assert lib.gl_hmc_create(None, None, None, ctypes.byref(h), None) == gl.GL_EINVAL
    assert h.value is None
    assert lib.gl_hmc_create(None, None, None, None, None) == gl.GL_EINVAL
    assert lib.gl_hmc_run(None, 1, 0, None, None, None) == gl.GL_EINVAL
    assert lib.gl_hmc_end_adaptation(None, 1, None) == gl.GL_EINVAL
    assert lib.gl_hmc_set_inv_mass(None, None, None) == gl.GL_EINVAL
    assert lib.gl_hmc_state(None, None, None, None, None, None) == gl.GL_EINVAL
    assert lib.gl_hmc_destroy(None) == gl.GL_OK
    assert "NULL" in gl.last_error() or "sampler" in gl.last_error()


def _ground_system_args():
    W = synth.ground_60()
    return (W.ny, W.nx, W.pixel_scale, W.supersample, np.zeros((W.ny, W.nx)),
            np.ones((W.ny, W.nx)), W.psf, 1, 1, W.prior())


def test_missing_library_raises(monkeypatch, tmp_path):
    """No libgl.so: the binding raises ImportError instead of computing anything."""
    monkeypatch.setattr(gl, "_LIB", None)
    monkeypatch.setattr(gl, "LIB_PATH", str(tmp_path / "libgl.so"))
    with pytest.raises(ImportError, match="missing"):
        gl.load()
    with pytest.raises(ImportError):
        gl.System(*_ground_system_args())


def test_no_cpu_fallback_without_a_device(lib):
    """Without a CUDA device, creating a system fails with GL_ECUDA (there is no
    host code path to fall back to)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(gl.GLError) as e:
        gl.System(*_ground_system_args())
    assert e.value.status == gl.GL_ECUDA


def test_deflection_kinds_match_the_header():
    """The binding's deflection constants are the header's enum values."""
    text = open(os.path.join(ROOT, "include", "gl.h")).read()
    body = re.search(r"typedef enum \{([^}]*)\} gl_deflection;", text).group(1)
    values = dict((k, int(v)) for k, v in re.findall(r"(GL_DEFL_[A-Z0-9_]+)\s*=\s*(\d+)", body))
    assert values == {"GL_DEFL_SERIES": gl.GL_DEFL_SERIES, "GL_DEFL_SURROGATE": gl.GL_DEFL_SURROGATE,
                      "GL_DEFL_TABLE": gl.GL_DEFL_TABLE, "GL_DEFL_TABLE32": gl.GL_DEFL_TABLE32,
                      "GL_DEFL_SURROGATE_FUSED": gl.GL_DEFL_SURROGATE_FUSED}


def test_multi_plan_rejects_bad_arguments(lib):
    """Host-side validation of gl_multi_create_ex and gl_multi_logp_grad: the
    launch shapes are checked before any system is touched (the fake system
    pointer below is never dereferenced)."""
    h = ctypes.c_void_p()
    one = (ctypes.c_int * 1)(8)
    fake = (ctypes.c_void_p * 1)(ctypes.c_void_p(16))
    assert lib.gl_multi_create_ex(None, 1, one, 1, None, None, ctypes.byref(h)) == gl.GL_EINVAL
    assert lib.gl_multi_create_ex(fake, 0, one, 1, None, None, ctypes.byref(h)) == gl.GL_EINVAL
    assert lib.gl_multi_create_ex(fake, 1, one, 3, None, None, ctypes.byref(h)) == gl.GL_EINVAL
    assert "smem_policy" in gl.last_error()
    bad_threads = (ctypes.c_int * 1)(192)
    assert lib.gl_multi_create_ex(fake, 1, one, 1, bad_threads, None, ctypes.byref(h)) == gl.GL_EINVAL
    assert "threads_per_cta" in gl.last_error()
    bad_pairs = (ctypes.c_int * 1)(4)
    assert lib.gl_multi_create_ex(fake, 1, one, 1, None, bad_pairs, ctypes.byref(h)) == gl.GL_EINVAL
    assert "pixel_pairs" in gl.last_error()
    assert lib.gl_multi_create_ex(fake, 1, one, 1, None, None, None) == gl.GL_EINVAL
    assert h.value is None
    assert lib.gl_multi_logp_grad(None, None, None, None, 0, None) == gl.GL_EINVAL
    assert lib.gl_multi_destroy(None) == gl.GL_OK


def test_autotuner_image_classes():
    """The tuner groups systems by image size, supersampling and PSF size."""
    from types import SimpleNamespace as NS
    from paper_2606_30633_b300 import autotune
    a = NS(ny=100, nx=100, s=3, psf_size=11)
    b = NS(ny=100, nx=100, s=3, psf_size=11)
    c = NS(ny=100, nx=100, s=4, psf_size=11)
    assert autotune.image_class(a) == autotune.image_class(b) != autotune.image_class(c)
    assert set(autotune.SHAPES) == {(256, 2), (256, 3), (128, 2), (128, 3)}
