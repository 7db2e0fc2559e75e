"""gl_logp_grad_noalloc: the gradient entry point for callers that may not
allocate device memory (code under a framework that owns a fixed device
memory budget, or a real-time loop that cannot take cudaMalloc's implicit
synchronisation). It takes its scratch from a fixed array inside the library
instead of cudaMalloc.

The image here is too large for shared memory, so the kernel's padded image
buffers live in that scratch. Two calls in a row, through the C ABI, must give
the same log p and gradient as gl_logp_grad (the same kernel: compared bit for
bit), and a batch whose scratch would exceed the fixed array is refused with
GL_EINVAL. Collected last so that a run stopping at the first failure has run
every other test first; it also passes alone in a fresh process."""
import numpy as np
import pytest

from lenscase import make_case, small_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_2606_30633_b300 import build
    build.build()
    import paper_2606_30633_b300 as gl
    # 160x160 px, s = 2, 21x21 PSF: two padded 180x180 FP32 buffers per row
    # (253 KB) do not fit in shared memory, so every row uses a scratch slot
    c = make_case(small_workload(160, 160, 2, 21, 1, 1, pixel_scale=0.05, fwhm=0.3, seed=61))
    return torch, gl, c, c.gpu_system()


def test_matches_gl_logp_grad_on_two_calls(setup):
    """A fresh system (it has never run gl_logp_grad, so it owns no scratch of
    its own): after one warm-up call per batch shape (the first call looks up
    the array's address), further calls leave the device's free memory
    unchanged; then gl_logp_grad gives the same results bit for bit."""
    torch, gl, c, _ = setup
    sysg = c.gpu_system()
    th1 = torch.tensor(c.theta(32, seed=1), dtype=torch.float32, device="cuda")
    th2 = torch.tensor(c.theta(24, seed=2), dtype=torch.float32, device="cuda")
    th1[0] = torch.tensor(c.truth, dtype=torch.float32)
    outs = [(torch.empty(t.shape[0], device="cuda"), torch.empty_like(t)) for t in (th1, th2, th1)]
    sysg.logp_grad_noalloc(th1, *outs[0])
    sysg.logp_grad_noalloc(th2, *outs[1])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    got1 = sysg.logp_grad_noalloc(th1, *outs[0])
    got2 = sysg.logp_grad_noalloc(th2, *outs[1])
    again1 = sysg.logp_grad_noalloc(th1, *outs[2])  # the shared scratch keeps no state that matters
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ref1 = sysg.logp_grad(th1)
    ref2 = sysg.logp_grad(th2)
    torch.cuda.synchronize()
    for got, ref in ((got1, ref1), (got2, ref2), (again1, ref1)):
        np.testing.assert_array_equal(got[0].cpu().numpy(), ref[0].cpu().numpy())
        np.testing.assert_array_equal(got[1].cpu().numpy(), ref[1].cpu().numpy())
    assert np.isfinite(got1[0].cpu().numpy()).all()
    sysg.close()


def test_small_image_without_scratch(setup):
    torch, gl, _, _ = setup
    c = make_case(small_workload(40, 40, 2, 11, 1, 1, seed=62))
    s = c.gpu_system()
    th = torch.tensor(c.theta(16, seed=3), dtype=torch.float32, device="cuda")
    ref = s.logp_grad(th)
    for _ in range(2):
        got = s.logp_grad_noalloc(th)
        np.testing.assert_array_equal(got[0].cpu().numpy(), ref[0].cpu().numpy())
        np.testing.assert_array_equal(got[1].cpu().numpy(), ref[1].cpu().numpy())


def test_batch_beyond_the_fixed_scratch_is_refused(setup):
    torch, gl, c, sysg = setup
    slot = 2 * 180 * 180  # floats per row
    max_rows = (16 * 1024 * 1024) // slot
    th = torch.tensor(c.theta(max_rows + 1, seed=4), dtype=torch.float32, device="cuda")
    with pytest.raises(gl.GLError) as err:
        sysg.logp_grad_noalloc(th)
    assert err.value.status == gl.GL_EINVAL
    assert f"at most {max_rows} rows" in str(err.value)
    ok = sysg.logp_grad_noalloc(th[:max_rows])  # the largest batch that fits runs
    ref = sysg.logp_grad(th[:max_rows])
    np.testing.assert_array_equal(ok[1].cpu().numpy(), ref[1].cpu().numpy())
