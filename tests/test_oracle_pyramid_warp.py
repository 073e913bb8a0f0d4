"""Pins of the oracle's coarse-to-fine pieces (Sec. 4 names a standard pyramid with warping and
gives no details; the readings are pinned by exactness properties) and end-to-end recovery of
a known motion (the optical-flow constraint of Sec. 1)."""
import numpy as np
import pytest

from paper_2011_10979_gb300 import synth


def test_level_sizes(orc):
    s = orc.level_sizes(480, 640, 0.5, 5)
    assert s == [(480, 640), (240, 320), (120, 160), (60, 80), (30, 40)]
    assert sum(h * w for h, w in s) == 409200
    s = orc.level_sizes(436, 1024, 0.5, 6)
    assert s[-1] == (14, 32) and sum(h * w for h, w in s) == 595264
    assert orc.level_sizes(48, 64, 0.5, 3) == [(48, 64), (24, 32), (12, 16)]
    assert orc.level_sizes(1, 3, 0.5, 4) == [(1, 3), (1, 2), (1, 1), (1, 1)]


@pytest.mark.parametrize("H,W", [(1, 1), (3, 2), (17, 23), (40, 30)])
def test_smoothing_and_downsampling_keep_constants(orc, H, W):
    img = np.full((H, W), 0.37)
    np.testing.assert_allclose(orc.gauss_smooth(img, 0.5), 0.37, atol=1e-15)
    Hc, Wc = orc.level_size(H, 0.5), orc.level_size(W, 0.5)
    np.testing.assert_allclose(orc.downsample(img, Hc, Wc, 0.5), 0.37, atol=1e-15)


def test_smoothing_keeps_linear_ramps_in_the_interior(orc):
    H, W = 30, 40
    i, j = np.mgrid[0:H, 0:W].astype(float)
    ramp = 0.3 * j - 0.7 * i + 2.0
    sm = orc.gauss_smooth(ramp, 0.5)
    R = 4   # ceil(3 * 0.6 * sqrt(3))
    np.testing.assert_allclose(sm[R:-R, R:-R], ramp[R:-R, R:-R], atol=1e-12)
    assert np.max(np.abs(sm - ramp)) > 1e-3          # the symmetric extension bends the border


def test_downsampling_samples_pixel_centres(orc):
    """At eta = 0.5 the coarse pixel centre sits at fine x = 2 x_c + 0.5: a ramp stays a ramp."""
    H, W = 32, 48
    i, j = np.mgrid[0:H, 0:W].astype(float)
    ramp = 0.3 * j - 0.7 * i
    out = orc.downsample(ramp, 16, 24, 0.5)
    ic, jc = np.mgrid[0:16, 0:24].astype(float)
    exp = 0.3 * (2 * jc + 0.5) - 0.7 * (2 * ic + 0.5)
    np.testing.assert_allclose(out[3:-3, 3:-3], exp[3:-3, 3:-3], atol=1e-12)


def test_upsampling_constant_and_ramp(orc):
    c = np.full((15, 20), 1.25)
    np.testing.assert_allclose(orc.upsample(c, 30, 40, 2.0), 2.5, atol=1e-15)
    ic, jc = np.mgrid[0:15, 0:20].astype(float)
    out = orc.upsample(0.5 * jc + 0.25 * ic, 30, 40, 1.0)
    i, j = np.mgrid[0:30, 0:40].astype(float)
    exp = 0.5 * ((j + 0.5) / 2 - 0.5) + 0.25 * ((i + 0.5) / 2 - 0.5)
    np.testing.assert_allclose(out[1:-1, 1:-1], exp[1:-1, 1:-1], atol=1e-14)


def test_derivatives_of_a_plane(orc):
    i, j = np.mgrid[0:9, 0:11].astype(float)
    Ix, Iy = orc.derivatives(0.4 * j - 0.2 * i + 1.0)
    np.testing.assert_allclose(Ix[:, 1:-1], 0.4, atol=1e-15)
    np.testing.assert_allclose(Iy[1:-1, :], -0.2, atol=1e-15)
    np.testing.assert_allclose(Ix[:, 0], 0.2, atol=1e-15)        # clamped one-sided half difference


def test_warp_identities(orc):
    rng = np.random.default_rng(0)
    H, W = 20, 24
    I0, I1 = rng.random((H, W)), rng.random((H, W))
    I1x, I1y = orc.derivatives(I1)
    z = np.zeros((H, W))
    Ix, Iy, It, ms = orc.warp_linearise(I0, I1, I1x, I1y, z, z, 0.05)
    np.testing.assert_array_equal(Ix, I1x)
    np.testing.assert_array_equal(Iy, I1y)
    np.testing.assert_allclose(It, I1 - I0, atol=1e-15)
    assert ms == pytest.approx(np.max(0.05 ** 2 + I1x ** 2 + I1y ** 2), rel=1e-15)
    # integer motion: exact shift in the interior; rho(d0) = I1w - I0 at the linearisation point
    u0, v0 = np.full((H, W), 3.0), np.full((H, W), -2.0)
    Ix, Iy, It, _ = orc.warp_linearise(I0, I1, I1x, I1y, u0, v0, 0.05)
    np.testing.assert_array_equal(Ix[2:, :W - 3], I1x[:-2, 3:])
    rho = Ix * u0 + Iy * v0 + It
    np.testing.assert_allclose(rho[2:, :W - 3], I1[:-2, 3:] - I0[2:, :W - 3], atol=1e-14)
    # a plane is sampled exactly at fractional positions
    i, j = np.mgrid[0:H, 0:W].astype(float)
    plane = 0.02 * j + 0.03 * i
    px, py = orc.derivatives(plane)
    u0, v0 = np.full((H, W), 1.3), np.full((H, W), 0.6)
    Ix, Iy, It, _ = orc.warp_linearise(plane, plane, px, py, u0, v0, 0.0)
    inner = (slice(1, H - 2), slice(1, W - 3))
    np.testing.assert_allclose(Ix[inner], 0.02, atol=1e-15)
    np.testing.assert_allclose(It[inner], 0.0, atol=1e-14)


@pytest.mark.parametrize("method", [0, 1, 2, 3])
def test_known_flow_recovery(orc, method):
    """64 x 48 sinusoid pair with a piecewise-constant motion: with a data weight that lets the
    data term speak (lambda = 5 on [0, 1] intensities) every solver recovers the motion.
    The 0.1 px threshold was calibrated once on this oracle (EPE 0.05-0.07 px) and frozen."""
    pr = synth.sinusoid_pair()
    P = orc.Params(method=method, lam=5.0, levels=3, warps=5, iters=50,
                   r=1.0 if method == 0 else 1.0, rho=1.9)
    u, v, w, st = orc.solve(pr.I0, pr.I1, P)
    epe = np.hypot(u - pr.u_true, v - pr.v_true)
    assert epe.mean() < 0.1, epe.mean()
    assert st["iters_run"] == 3 * 5 * 50


@pytest.mark.parametrize("method", [0, 1, 2, 3])
def test_known_flow_recovery_on_the_bilinearly_warped_pair(orc, method):
    """The same pair in its literal form (frame 1 = frame 0 resampled bilinearly, so frame 1 is
    smoother than frame 0 and shares its noise): every solver still recovers the motion.  The
    0.2 px threshold was calibrated once on this oracle (EPE 0.08-0.14 px) and frozen."""
    pr = synth.sinusoid_pair(render="bilinear")
    u, v, w, st = orc.solve(pr.I0, pr.I1, orc.Params(method=method, lam=5.0, levels=3, warps=5, iters=50))
    assert np.hypot(u - pr.u_true, v - pr.v_true).mean() < 0.2


def test_stopping_test_and_out_level(orc):
    pr = synth.sinusoid_pair()
    u, v, w, st = orc.solve(pr.I0, pr.I1, orc.Params(lam=5.0, tol=1e-2, iters=200))
    assert st["iters_run"] < 3 * 5 * 200 and st["iters_run"] % 10 == 0
    assert st["residual"] < 1e-2
    u1, v1, _, _ = orc.solve(pr.I0, pr.I1, orc.Params(lam=5.0, out_level=1))
    assert u1.shape == (24, 32)
