"""The tensor-core surrogate kernels' wait-timeout path, taken through the
library's test hook (gl_debug_force_wait_timeout): the kernels act as if their
first completion wait had run out, without waiting, so no wait really runs
out and every issued MMA is still drained before the tensor memory is freed.

Checked: the table build (the stand-alone one, and the one inside the fused
gradient kernel) gives NaN log p and gradient on the rows it served, the next GL_DEFL_SURROGATE call on that surrogate returns
GL_ETIMEOUT, the
synchronous training entry points return GL_ETIMEOUT at once, and with the
hook off the same calls succeed again with the results they had before (the
context stays usable)."""
import numpy as np
import pytest

from lenscase import make_case, small_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2606_30633_b300 import build
    build.build()
    import paper_2606_30633_b300 as gl
    sur = gl.Surrogate.train(n_samples=1 << 15, epochs=2, batch=4096)
    c = make_case(small_workload(24, 24, 2, 5, 1, 1, seed=71))
    s = c.gpu_system()
    s.set_surrogate(sur)
    th = c.theta(16, seed=3)
    th[:, 2:4] = np.clip(th[:, 2:4], -0.2, 0.2)  # inside the surrogate's q domain
    th[np.abs(th[:, 2]) < 0.02, 2] = 0.05        # |e| >= 0.01: the table path
    t = torch.tensor(th, dtype=torch.float32, device="cuda")
    yield torch, gl, sur, s, t
    gl.debug_force_wait_timeout(False)
    s.close()
    sur.close()


def test_table_build_timeout_is_reported(env):
    torch, gl, sur, s, t = env
    lp0, g0 = s.logp_grad(t, defl=gl.GL_DEFL_SURROGATE)
    torch.cuda.synchronize()
    assert np.isfinite(lp0.cpu().numpy()).all()
    gl.debug_force_wait_timeout(True)
    try:
        lp1, g1 = s.logp_grad(t, defl=gl.GL_DEFL_SURROGATE)  # asynchronous: returns GL_OK
        torch.cuda.synchronize()
        assert np.isnan(lp1.cpu().numpy()).all() and np.isnan(g1.cpu().numpy()).all()
        with pytest.raises(gl.GLError) as err:
            s.logp_grad(t, defl=gl.GL_DEFL_SURROGATE)
        assert err.value.status == gl.GL_ETIMEOUT
        # the network inside the gradient kernel's CTA as well
        lpf, gf = s.logp_grad(t, defl=gl.GL_DEFL_SURROGATE_FUSED)
        torch.cuda.synchronize()
        assert np.isnan(lpf.cpu().numpy()).all() and np.isnan(gf.cpu().numpy()).all()
        with pytest.raises(gl.GLError) as err:
            s.logp_grad(t, defl=gl.GL_DEFL_SURROGATE_FUSED)
        assert err.value.status == gl.GL_ETIMEOUT
        # the exact series does not use the tensor cores and is unaffected
        lps, _ = s.logp_grad(t, defl=gl.GL_DEFL_SERIES)
        assert np.isfinite(lps.cpu().numpy()).all()
    finally:
        gl.debug_force_wait_timeout(False)
    lp2, g2 = s.logp_grad(t, defl=gl.GL_DEFL_SURROGATE)
    lp3, g3 = s.logp_grad(t, defl=gl.GL_DEFL_SURROGATE_FUSED)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(lp2.cpu().numpy(), lp0.cpu().numpy())
    np.testing.assert_array_equal(g2.cpu().numpy(), g0.cpu().numpy())
    np.testing.assert_array_equal(lp3.cpu().numpy(), lp0.cpu().numpy())
    np.testing.assert_array_equal(g3.cpu().numpy(), g0.cpu().numpy())


def test_training_timeout_is_reported(env):
    torch, gl, sur, _, _ = env
    g = torch.Generator(device="cpu").manual_seed(5)
    x = torch.rand((256, 4), generator=g).cuda()
    y = torch.rand((256, 2), generator=g).cuda()
    loss0, grad0 = sur.loss_grad(x, y)
    gl.debug_force_wait_timeout(True)
    try:
        with pytest.raises(gl.GLError) as err:
            sur.loss_grad(x, y)
        assert err.value.status == gl.GL_ETIMEOUT
        with pytest.raises(gl.GLError) as err:
            gl.Surrogate.train(n_samples=1 << 13, epochs=1, batch=4096)
        assert err.value.status == gl.GL_ETIMEOUT
    finally:
        gl.debug_force_wait_timeout(False)
    loss1, grad1 = sur.loss_grad(x, y)
    assert loss1 == loss0
    np.testing.assert_array_equal(grad1, grad0)
