"""The binding rejects buffers that the library would access out of bounds:
a wrong shape, dtype or device raises before anything is launched, and valid
caller-provided buffers give the same results as the allocating calls."""
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
    c = make_case(small_workload(16, 16, 2, 5, 1, 1, seed=31))
    S = c.gpu_system()
    th = torch.tensor(c.theta(4), dtype=torch.float32, device="cuda")
    return torch, gl, S, th


def test_wrong_buffers_are_rejected(env):
    torch, gl, S, th = env
    B, P = th.shape
    dev = "cuda"
    short = torch.empty(B - 1, device=dev)
    with pytest.raises(ValueError):
        S.logp(th, out=short)
    with pytest.raises(ValueError):
        S.logp_grad(th, out=short)
    with pytest.raises(ValueError):
        S.logp_grad(th, grad=torch.empty(B, P - 1, device=dev))
    with pytest.raises(ValueError):
        S.logp_grad_noalloc(th, grad=torch.empty(B - 1, P, device=dev))
    with pytest.raises(ValueError):
        S.model_image(th, out=torch.empty(B, 16, 15, device=dev))
    with pytest.raises(TypeError):
        S.logp(th, out=torch.empty(B, device=dev, dtype=torch.float64))
    with pytest.raises(TypeError):
        S.logp(th, out=torch.empty(B))  # host memory
    with pytest.raises(ValueError):
        S.logp_grad_host(np.zeros((B, P + 1), np.float32))
    u = S.bijector_inverse(th)
    with pytest.raises(ValueError):
        S.map_adam(u, torch.zeros(B - 1, P, device=dev), torch.zeros_like(u), 1)
    hmc = gl.Hmc(S, u, 2, 1e-3)
    with pytest.raises(ValueError):
        hmc.set_inv_mass(torch.ones(P - 1, device=dev))
    hmc.close()
    out, grad = torch.empty(B, device=dev), torch.empty_like(th)
    S.logp_grad(th, out=out, grad=grad)
    lp, g = S.logp_grad(th)
    assert torch.equal(out, lp) and torch.equal(grad, g)


def test_multi_rejects_mismatched_buffers(env):
    torch, gl, S, th = env
    with pytest.raises(ValueError):
        gl.Multi([S, S], [4])
    plan = gl.Multi([S, S], [4, 2])
    with pytest.raises(ValueError):
        plan.logp_grad([th])
    with pytest.raises(ValueError):
        plan.logp_grad([th, th[:1]])
    with pytest.raises(ValueError):
        plan.logp_grad([th, th[:2]], logps=[torch.empty(3, device="cuda"),
                                            torch.empty(2, device="cuda")])
    lps, gs = plan.logp_grad([th, th[:2]])
    lp, g = S.logp_grad(th)
    assert torch.equal(lps[0], lp) and torch.equal(gs[0], g)
    assert torch.equal(lps[1], lp[:2]) and torch.equal(gs[1], g[:2])


def test_network_calls_reject_wrong_shapes(env):
    torch, gl, S, th = env
    x = torch.rand(256, 3, device="cuda")
    with pytest.raises(ValueError):
        gl.series_F(x)
    with pytest.raises(ValueError):
        gl.Surrogate.from_params(np.zeros(7, np.float32))
    sur = gl.Surrogate.from_params(np.zeros(gl.Surrogate.num_params(), np.float32))
    with pytest.raises(ValueError):
        sur.infer(x)
    with pytest.raises(ValueError):
        sur.loss_grad(torch.rand(256, 4, device="cuda"), torch.rand(255, 2, device="cuda"))
    y = sur.infer(torch.rand(256, 4, device="cuda") + 0.5)
    assert y.shape == (256, 2) and bool(torch.isfinite(y).all())
    sur.close()


def test_unknown_svi_estimator_is_rejected(env):
    torch, gl, S, th = env
    from paper_2606_30633_b300 import infer
    phi, opt = infer.svi_init(S, S.bijector_inverse(th)[0])
    before = phi.clone()
    with pytest.raises(gl.GLError) as e:
        S.svi_adabelief(phi, opt, 8, 1, estimator=7)
    assert e.value.status == gl.GL_EINVAL
    assert torch.equal(phi, before)
