"""GPU parity of backward intensity modelling (gl_logp_grad_backward)
against the FP64 oracle (oracle/backward.py): solved intensities, profile
log p and the envelope-theorem gradient, near the mode and at prior draws, for
no lens light, one or two sources, and the most components (2 + 3)."""
import numpy as np
import pytest

import synth
from lenscase import f32, grad_bound, make_case, small_workload
from oracle import backward as BW

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module", params=[(1, 1), (1, 2), (0, 1), (2, 3)])
def case(request):
    nl, ns = request.param
    return make_case(small_workload(40, 40, 2, 11, nl, ns, seed=1401 + ns))


def test_backward_matches_oracle(torch, case):
    W = case.W
    s = case.gpu_system()
    near = f32(synth.jitter(case.truth, W.prior(), 6, 3, rel=0.003))
    near[0] = case.truth
    th = np.concatenate([near, case.theta(4, seed=9)])
    idx = BW.intensity_indices(W.n_lens_light, W.n_source)
    th_in = th.copy()
    th_in[:, idx] = 7.0  # ignored on input
    lp, g, I = s.logp_grad_backward(torch.tensor(th_in, dtype=torch.float32, device="cuda"))
    lp, g, I = lp.cpu().numpy(), g.cpu().numpy(), I.cpu().numpy()
    prof = BW.profile_system(case.oracle, case.spec)
    lp_o, g_o, I_o = BW.logp_grad_backward(case.oracle, prof, th)
    assert np.all(np.abs(I - I_o) <= 1e-4 * np.abs(I_o) + 1e-6), np.abs((I - I_o) / I_o).max()
    assert np.all(np.abs(lp - lp_o) <= 2e-5 * np.abs(lp_o) + 1e-2), np.abs(lp - lp_o).max()
    assert np.all(g[:, idx] == 0.0)
    # bound: the forward-model gradient bound at theta*, plus the gradient's
    # change under the GPU's intensity error
    ts = th.copy()
    ts[:, idx] = I_o
    tg = th.copy()
    tg[:, idx] = I
    _, g_at_gpu_I = prof.logp_grad(tg)
    g_at_gpu_I[:, idx] = 0.0
    bound = grad_bound(case, ts) + np.abs(g_at_gpu_I - g_o)
    bound[:, idx] = 0.0
    err = np.abs(g - g_o)
    assert np.all(err <= bound), float(np.max(err / np.where(bound > 0, bound, 1)))


def test_backward_with_tables_follows_the_series(torch, case):
    """The same solve with the exact series tabulated per row (GL_DEFL_TABLE):
    the component images of source rows read the tables, lens-light rows need
    no deflection; intensities and log p follow the series path to the tables'
    interpolation error."""
    import paper_2606_30633_b300 as gl
    W = case.W
    s = case.gpu_system()
    th = f32(synth.jitter(case.truth, W.prior(), 6, 5, rel=0.003))
    th[0] = case.truth
    t = torch.tensor(th, dtype=torch.float32, device="cuda")
    lps, _, Is = s.logp_grad_backward(t)
    lpt, _, It = s.logp_grad_backward(t, defl=gl.GL_DEFL_TABLE)
    lps, Is, lpt, It = lps.cpu().numpy(), Is.cpu().numpy(), lpt.cpu().numpy(), It.cpu().numpy()
    assert np.all(np.abs(It - Is) <= 1e-4 * np.abs(Is) + 1e-6), np.abs((It - Is) / Is).max()
    assert np.all(np.abs(lpt - lps) <= 2e-6 * np.abs(lps) + 2e-3), np.abs(lpt - lps).max()
