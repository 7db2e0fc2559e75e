"""Pins of the oracle's grid, binning, PSF convolution, shear and lens equation."""
import math

import numpy as np
import pytest
from scipy import signal

import oracle
import synth


def _system(ny, nx, D, s, psf, n_src=1, data=None, sigma=None):
    spec = synth.config_prior(1, n_src)
    data = np.zeros((ny, nx)) if data is None else data
    sigma = np.ones((ny, nx)) if sigma is None else sigma
    return oracle.System(ny, nx, D, s, data, sigma, psf, 1, n_src, spec)


def _brute_conv(img, psf):
    ny, nx = img.shape
    ky, kx = psf.shape
    cy, cx = (ky - 1) // 2, (kx - 1) // 2
    out = np.zeros_like(img)
    for i in range(ny):
        for j in range(nx):
            acc = 0.0
            for u in range(ky):
                for v in range(kx):
                    ii, jj = i + cy - u, j + cx - v
                    if 0 <= ii < ny and 0 <= jj < nx:
                        acc += psf[u, v] * img[ii, jj]
            out[i, j] = acc
    return out


@pytest.mark.parametrize("shape,kshape", [((7, 9), (3, 5)), ((5, 5), (3, 3)), ((9, 6), (5, 1)),
                                          ((4, 3), (7, 7))])
def test_convolution_brute_force(shape, kshape):
    """"same" convolution with zero padding against direct loops and
    scipy.signal.convolve2d, with an asymmetric kernel (catches a flipped or
    transposed kernel)."""
    rng = np.random.default_rng(7)
    img = rng.normal(size=shape)
    psf = rng.uniform(0.1, 1.0, size=kshape)
    psf /= psf.sum()
    out = oracle.convolve_same(img, psf)
    np.testing.assert_allclose(out, _brute_conv(img, psf), rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(out, signal.convolve2d(img, psf, mode="same"), rtol=1e-12,
                               atol=1e-14)


def test_convolution_normalises_and_delta_is_identity():
    rng = np.random.default_rng(8)
    img = rng.normal(size=(6, 8))
    delta = np.zeros((5, 5))
    delta[2, 2] = 3.0  # any positive sum: renormalised to 1
    np.testing.assert_allclose(oracle.convolve_same(img, delta), img, rtol=1e-15)
    shift = np.zeros((3, 3))
    shift[1, 2] = 1.0  # true convolution moves content one pixel to +x
    out = oracle.convolve_same(img, shift)
    np.testing.assert_allclose(out[:, 1:], img[:, :-1], rtol=1e-15)
    np.testing.assert_allclose(out[:, 0], 0.0)


def test_grid_orientation():
    """x grows with the column index and y with the row index, origin at the
    image centre: a source light at (+0.5", -0.25") peaks right of and above
    (lower row than) the centre."""
    ny, nx, D = 21, 21, 0.05
    S = _system(ny, nx, D, 1, np.ones((1, 1)))
    th = np.zeros(S.P)
    th[:8] = [1e-8, 2.0, 0, 0, 0, 0, 0, 0]  # negligible deflection
    th[8:15] = [0.2, 1.0, 0, 0, 0, 0, 0.0]  # lens light switched off
    th[15:22] = [0.05, 1.0, 0, 0, 0.5, -0.25, 1.0]
    img = S.binned_image(th)
    i, j = np.unravel_index(np.argmax(img), img.shape)
    assert (i, j) == (10 - 5, 10 + 10)


def test_binning_s1_is_point_sampling_and_supersampling_is_the_mean():
    """s = 1 samples the surface brightness at pixel centres (times D^2); s = 3
    averages the nine sub-pixel centres at offsets (-1/3, 0, 1/3) D."""
    ny, nx, D = 8, 10, 0.2
    W = synth.ground_60()
    th = W.truth()
    S1 = _system(ny, nx, D, 1, np.ones((1, 1)))
    S3 = _system(ny, nx, D, 3, np.ones((1, 1)))
    xs = (np.arange(nx) - (nx - 1) / 2) * D
    ys = (np.arange(ny) - (ny - 1) / 2) * D
    X, Y = np.meshgrid(xs, ys)
    sb = S1.surface_brightness(th, X, Y)
    np.testing.assert_allclose(S1.binned_image(th), sb * D * D, rtol=1e-14)
    acc = np.zeros_like(X)
    for oy in (-1 / 3, 0.0, 1 / 3):
        for ox in (-1 / 3, 0.0, 1 / 3):
            acc += S3.surface_brightness(th, X + ox * D, Y + oy * D)
    np.testing.assert_allclose(S3.binned_image(th), acc / 9 * D * D, rtol=1e-13)


def test_flux_is_conserved_by_binning_and_psf():
    """Total counts approach the analytic Sersic flux of the lens light as s
    grows, and a normalised PSF keeps the total for light well inside the image."""
    ny = nx = 81
    D = 0.1
    psf = synth.moffat_psf(11, D, 0.5)
    th = np.zeros(22)
    th[:8] = [1e-8, 2.0, 0, 0, 0, 0, 0, 0]
    Re, n_s, I_e = 0.6, 1.0, 2.0
    th[8:15] = [Re, n_s, 0.1, 0.05, 0.0, 0.0, I_e]
    th[15:22] = [0.1, 1.0, 0, 0, 0, 0, 0.0]
    bn = 1.9992 * n_s - 0.3271
    from scipy import special
    Rmax = (nx // 2 - 8) * D  # enclosed flux inside an aperture that fits
    S = _system(ny, nx, D, 4, psf)
    b = S.binned_image(th)
    m = S.model_image(th)[0]
    inner_total = (2 * math.pi * n_s * I_e * Re ** 2 * math.exp(bn) * bn ** (-2 * n_s)
                   * special.gamma(2 * n_s))
    assert abs(b.sum() / inner_total - 1) < 2e-3
    assert abs(m.sum() / b.sum() - 1) < 1e-4
    assert Rmax > 3 * Re


def test_shear_and_lens_equation():
    """With a negligible EPL the source is seen at beta = theta - alpha_shear,
    alpha_shear = (g1 x + g2 y, g2 x - g1 y) = grad of psi = g1 (x^2-y^2)/2 + g2 x y
    (checked by differencing the potential)."""
    g1, g2 = 0.07, -0.04
    S = _system(4, 4, 0.1, 1, np.ones((1, 1)))
    th = np.zeros(22)
    th[:8] = [1e-12, 2.0, 0, 0, 0, 0, g1, g2]
    th[8:15] = [0.2, 1.0, 0, 0, 0, 0, 0.0]
    src = [0.3, 1.0, 0.1, -0.2, 0.05, 0.02, 1.0]
    th[15:22] = src
    rng = np.random.default_rng(3)
    x, y = rng.uniform(-1, 1, 20), rng.uniform(-1, 1, 20)
    psi = lambda a, b: 0.5 * g1 * (a * a - b * b) + g2 * a * b
    h = 1e-6
    ax = (psi(x + h, y) - psi(x - h, y)) / (2 * h)
    ay = (psi(x, y + h) - psi(x, y - h)) / (2 * h)
    sb = S.surface_brightness(th, x, y)
    ref = oracle.sersic(src, x - ax, y - ay)
    np.testing.assert_allclose(sb, ref, rtol=1e-8)


def test_sis_images_of_an_offset_source():
    """Singular isothermal sphere (gamma = 2, e = 0) with Einstein radius
    theta_E and a round source at (beta0, 0), beta0 < theta_E: the lens equation
    beta = theta - theta_E theta/|theta| has the two images theta = beta0 +
    theta_E and beta0 - theta_E on the x axis (Schneider, Ehlers & Falco 1992,
    Sec. 8.1). There the lensed surface brightness equals the source's central
    brightness, and it falls off on both sides along the axis."""
    thetaE, beta0 = 1.2, 0.3
    S = _system(4, 4, 0.1, 1, np.ones((1, 1)))
    th = np.zeros(22)
    th[:8] = [thetaE, 2.0, 0, 0, 0, 0, 0, 0]
    th[8:15] = [0.2, 1.0, 0, 0, 0, 0, 0.0]     # no lens light
    src = [0.15, 0.5, 0.0, 0.0, beta0, 0.0, 1.0]
    th[15:22] = src
    peak = oracle.sersic(src, np.array([beta0]), np.array([0.0]))[0]
    for x_img in (beta0 + thetaE, beta0 - thetaE):
        sb = S.surface_brightness(th, np.array([x_img]), np.array([0.0]))[0]
        assert abs(sb / peak - 1) < 1e-9, (x_img, sb, peak)
        side = S.surface_brightness(th, np.array([x_img - 0.02, x_img + 0.02]), np.zeros(2))
        assert np.all(side < 0.99 * peak)
    # the unlensed position of the source is not an image: the brightness there is tiny
    assert S.surface_brightness(th, np.array([beta0]), np.array([0.0]))[0] < 1e-3 * peak
