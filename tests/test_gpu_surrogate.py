"""The learned EPL deflection surrogate: its tensor-core training and
inference kernels against the FP64 reference MLP (with the same BF16
rounding points), a trained network against the exact series, and the
lens path with tabulated deflections (exact-series tables against the
per-sub-pixel series; the trained surrogate against the exact model)."""
import numpy as np
import pytest

import oracle
import oracle.mlp as mlp
import synth
from lenscase import make_case, small_workload

pytestmark = pytest.mark.gpu


def _tuples(n, seed):
    r = np.random.default_rng(seed)
    return np.stack([r.uniform(0.5, 1, n), r.uniform(1.7, 2.3, n),
                     r.uniform(np.log(0.05), np.log(5), n), r.uniform(0, 2 * np.pi, n)],
                    1).astype(np.float32)


@pytest.fixture(scope="module")
def gl():
    import torch
    from paper_2606_30633_b300 import build
    build.build()
    import paper_2606_30633_b300 as g
    return torch, g


@pytest.fixture(scope="module")
def trained(gl):
    torch, g = gl
    # the benchmark's training run: 1e7 exact-series tuples, 120 epochs
    return g.Surrogate.train(n_samples=10_000_000, epochs=120, batch=16384, lr=2e-3, lr_min=1e-5,
                             seed_data=401, seed_init=402)


def test_loss_and_gradient_match_fp64_reference(gl):
    torch, g = gl
    rng = np.random.default_rng(5)
    p = (rng.normal(size=mlp.NPARAM) * 0.2).astype(np.float32)
    sur = g.Surrogate.from_params(p)
    X = _tuples(256, 1)
    T = rng.normal(size=(256, 2)).astype(np.float32)
    loss, grad = sur.loss_grad(torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"))
    lref, gref = mlp.loss_grad(p.astype(np.float64), X, T.astype(np.float64))
    assert abs(loss - lref) <= 1e-5 * lref
    err = np.abs(grad - gref)
    assert np.all(err <= 1e-3 * np.abs(gref) + 1e-3 * np.abs(gref).max()), err.max()


def test_inference_matches_fp64_reference_and_save_load(gl, tmp_path):
    torch, g = gl
    rng = np.random.default_rng(6)
    p = (rng.normal(size=mlp.NPARAM) * 0.2).astype(np.float32)
    sur = g.Surrogate.from_params(p)
    X = _tuples(1000, 2)
    F = sur.infer(torch.tensor(X, device="cuda")).cpu().numpy()
    Fref = mlp.surrogate_F(p.astype(np.float64), X)
    assert np.max(np.abs(F[:, 0] + 1j * F[:, 1] - Fref)) < 2e-5
    path = str(tmp_path / "sur.bin")
    sur.save(path)
    sur2 = g.Surrogate.load_file(path)
    np.testing.assert_array_equal(sur2.params(), p)
    F2 = sur2.infer(torch.tensor(X, device="cuda")).cpu().numpy()
    np.testing.assert_array_equal(F2, F)


def test_trained_network_against_the_exact_series(gl, trained):
    """F error and deflection error (arcsec, at theta_E = 1.25") on held-out tuples."""
    torch, g = gl
    X = _tuples(20000, 99)
    Fs = trained.infer(torch.tensor(X, device="cuda")).cpu().numpy()
    Fs = Fs[:, 0] + 1j * Fs[:, 1]
    Xd = X.astype(np.float64)
    Fe = np.array([oracle.hyp2f1_series(x[1] - 1, (1 - x[0]) / (1 + x[0]), x[3]) for x in Xd])
    d = np.abs(Fs - Fe)
    thE = 1.25
    q, t, R = Xd[:, 0], Xd[:, 1] - 1, np.exp(Xd[:, 2]) * thE
    b = thE * np.sqrt(q)
    dal = 2 * b / (1 + q) * (b / R) ** (t - 1) * d
    base = np.abs(mlp.base_F(Xd) - Fe)
    assert np.sqrt(np.mean(d ** 2)) < 3e-5, np.sqrt(np.mean(d ** 2))
    assert np.sqrt(np.mean(dal ** 2)) < 6e-5 and dal.max() < 3e-3, (np.sqrt(np.mean(dal ** 2)),
                                                                    dal.max())
    assert np.sqrt(np.mean(d ** 2)) < 0.01 * np.sqrt(np.mean(base ** 2))  # the network's gain
    assert trained.final_loss < 1e-4
    # the library's own exact series (the reference the surrogate is measured against)
    Fx = g.series_F(torch.tensor(X, device="cuda")).cpu().numpy()
    np.testing.assert_allclose(Fx[:, 0] + 1j * Fx[:, 1], Fe, rtol=0, atol=3e-7)


def test_series_F_edges(gl):
    """gl_series_F: q = 1 gives F = 1 exactly; tuples outside the series'
    domain give NaN; an empty call is a no-op."""
    torch, g = gl
    X = np.array([[1.0, 2.1, 0.0, 0.4], [0.005, 2.0, 0.0, 0.1], [0.7, 3.0, 0.0, 0.2],
                  [0.7, 2.0, 0.0, np.nan], [0.01, 2.99, 0.0, 1.3]], dtype=np.float32)
    F = g.series_F(torch.tensor(X, device="cuda")).cpu().numpy()
    np.testing.assert_array_equal(F[0], [1.0, 0.0])
    assert np.all(np.isnan(F[1:4]))
    Fe = oracle.hyp2f1_series(X[4, 1] - 1.0, (1 - X[4, 0]) / (1 + X[4, 0]), X[4, 3])
    assert abs(F[4, 0] + 1j * F[4, 1] - Fe) <= 1e-6 * abs(Fe)
    assert g.series_F(torch.zeros((0, 4), device="cuda")).shape == (0, 2)


@pytest.fixture(scope="module")
def lens(gl):
    return make_case(small_workload(60, 60, 2, 11, 1, 1, seed=1121))


def test_exact_tables_reproduce_the_series_path(gl, lens):
    """GL_DEFL_TABLE (exact series tabulated per row, Hermite-interpolated)
    against the per-sub-pixel series: log p and gradients agree to the
    interpolation error; rows with |e| > 0.5 take the series exactly."""
    torch, g = gl
    c = lens
    s = c.gpu_system()
    th = np.concatenate([synth.jitter(c.truth, c.W.prior(), 6, 1, rel=0.01), c.theta(10)])
    th = th.astype(np.float32)
    th[0] = c.truth
    tt = torch.tensor(th, device="cuda")
    lps, gs = s.logp_grad(tt)
    lpt, gt = s.logp_grad(tt, defl=g.GL_DEFL_TABLE)
    lps, lpt = lps.cpu().numpy(), lpt.cpu().numpy()
    assert np.all(np.abs(lpt - lps) <= 2e-6 * np.abs(lps) + 2e-3), np.abs(lpt - lps).max()
    gs, gt = gs.cpu().numpy(), gt.cpu().numpy()
    scale = np.maximum(np.abs(gs), 1e-2 * np.abs(gs).max(1, keepdims=True))
    assert np.all(np.abs(gt - gs) <= 2e-3 * scale), (np.abs(gt - gs) / scale).max()
    img_s = s.model_image(tt).cpu().numpy()
    img_t = s.model_image(tt, defl=g.GL_DEFL_TABLE).cpu().numpy()
    assert np.all(np.abs(img_t - img_s) <= 1e-5 * np.abs(img_s) + 1e-5 * img_s.max())


def test_surrogate_lens_path(gl, trained, lens):
    """With the trained surrogate: |d log p| <= 0.1 against the exact model near
    the mode; gradients follow the exact model's; rows outside the training
    domain (q < 0.5) use the series exactly."""
    torch, g = gl
    c = lens
    s = c.gpu_system()
    s.set_surrogate(trained)
    th = synth.jitter(c.truth, c.W.prior(), 8, 1, rel=0.01).astype(np.float32)
    th[0] = c.truth
    out = c.theta(400, seed=7).astype(np.float32)
    q = (1 - np.hypot(out[:, 2], out[:, 3])) / (1 + np.hypot(out[:, 2], out[:, 3]))
    out = out[q < 0.5][:2]
    assert len(out) == 2
    th = np.concatenate([th, out])
    tt = torch.tensor(th, device="cuda")
    lpu, gu = s.logp_grad(tt, defl=g.GL_DEFL_SURROGATE)
    lps, gs = s.logp_grad(tt)
    ref = c.oracle.logp(th.astype(np.float64))
    lpu = lpu.cpu().numpy()
    assert np.all(np.abs(lpu[:8] - ref[:8]) <= 0.1), lpu[:8] - ref[:8]
    np.testing.assert_array_equal(lpu[8:], lps.cpu().numpy()[8:])
    np.testing.assert_array_equal(gu.cpu().numpy()[8:], gs.cpu().numpy()[8:])
    gu, gs = gu.cpu().numpy()[:8], gs.cpu().numpy()[:8]
    scale = np.maximum(np.abs(gs), 1e-2 * np.abs(gs).max(1, keepdims=True))
    assert np.all(np.abs(gu - gs) <= 0.25 * scale), (np.abs(gu - gs) / scale).max()
    lpf = s.logp(tt, defl=g.GL_DEFL_SURROGATE).cpu().numpy()
    np.testing.assert_array_equal(lpf, lpu)


def test_surrogate_requires_attachment(gl, lens):
    torch, g = gl
    s = lens.gpu_system()
    with pytest.raises(g.GLError) as e:
        s.logp(torch.tensor(lens.theta(2), dtype=torch.float32, device="cuda"),
               defl=g.GL_DEFL_SURROGATE)
    assert e.value.status == g.GL_ENOSURROGATE
