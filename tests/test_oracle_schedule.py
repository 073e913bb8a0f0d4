"""Pins of the oracle's coarse-to-fine pieces against library routines and hand computation.

Sec. 4 of the paper names a standard coarse-to-fine pyramid with warping and gives no details;
the oracle takes one reading of it (pyramid sizes, Gaussian pre-smoothing of width
sigma_g = 0.6 sqrt(eta^-2 - 1) and radius ceil(3 sigma_g) with a half-sample symmetric border,
bilinear sampling at pixel centres, u and v scaled by the size ratio when a level is handed to
the next finer one, the duals restarting at zero there, and all state carried from one warp to
the next).  These tests fix that reading independently of the oracle's own code:

  * smoothing  = scipy.ndimage.gaussian_filter1d along rows, then columns (mode 'reflect' is the
    half-sample symmetric extension; truncate = R / sigma_g gives the radius R);
  * resampling = scipy.ndimage.map_coordinates (order 1, mode 'nearest' = clamped coordinates) at
    the pixel-centre coordinates, after that smoothing for the pyramid step;
  * warping    = map_coordinates of I1, I1x, I1y at (x + u0, y + v0);
  * schedule   = a 1 x 1 pair solved by hand (gradient and divergence vanish, so every method
    collapses to a scalar recursion written out from its component equations), and a two-level
    pair composed step by step from the separately pinned pieces, with plants of the plausible
    mistakes (no u/v scaling, no dual restart, no Xbar = X) shown to change the result.
"""
import math

import numpy as np
import pytest

ndi = pytest.importorskip("scipy.ndimage")


def _sigma_r(eta):
    sg = 0.6 * math.sqrt(1.0 / (eta * eta) - 1.0)
    return sg, math.ceil(3.0 * sg)


def _scipy_smooth(img, eta):
    sg, R = _sigma_r(eta)
    t = ndi.gaussian_filter1d(img, sg, axis=1, mode="reflect", truncate=R / sg)
    return ndi.gaussian_filter1d(t, sg, axis=0, mode="reflect", truncate=R / sg)


SIZES = [(1, 1), (1, 6), (5, 1), (3, 2), (2, 5), (9, 13), (40, 31), (48, 64)]


# ------------------------------------------------------------------------------ smoothing
@pytest.mark.parametrize("eta", [0.5, 0.6, 0.75, 0.8])
@pytest.mark.parametrize("H,W", SIZES)
def test_gauss_smooth_is_separable_gaussian_with_half_sample_reflection(orc, eta, H, W):
    rng = np.random.default_rng(H * 131 + W)
    img = rng.random((H, W))
    np.testing.assert_allclose(orc.gauss_smooth(img, eta), _scipy_smooth(img, eta), rtol=0, atol=1e-14)


@pytest.mark.parametrize("pos", ["corner", "top", "left", "bottom_right", "interior", "near_border"])
def test_gauss_smooth_impulse_response(orc, pos):
    """Impulses at the border and inside: the response is the separable Gaussian folded back by
    the half-sample reflection (a whole-sample reflection, a wrong width or radius all fail)."""
    H, W = 17, 23
    i, j = dict(corner=(0, 0), top=(0, 11), left=(8, 0), bottom_right=(H - 1, W - 1), interior=(8, 11),
                near_border=(1, 2))[pos]
    img = np.zeros((H, W))
    img[i, j] = 1.0
    for eta in (0.5, 0.7):
        np.testing.assert_allclose(orc.gauss_smooth(img, eta), _scipy_smooth(img, eta), rtol=0, atol=1e-14)
    # interior impulse at eta = 0.5: the 9-tap kernel exp(-k^2 / (2 sigma_g^2)), normalised
    if pos == "interior":
        sg, R = _sigma_r(0.5)
        k = np.arange(-R, R + 1)
        g = np.exp(-k * k / (2 * sg * sg))
        g /= g.sum()
        out = orc.gauss_smooth(img, 0.5)
        np.testing.assert_allclose(out[i - R:i + R + 1, j - R:j + R + 1], np.outer(g, g), rtol=0, atol=1e-15)
        assert np.count_nonzero(out) == (2 * R + 1) ** 2


# ------------------------------------------------------------------------------ resampling
@pytest.mark.parametrize("eta", [0.5, 0.6])
@pytest.mark.parametrize("H,W", SIZES)
def test_downsample_is_smoothing_then_bilinear_at_pixel_centres(orc, eta, H, W):
    rng = np.random.default_rng(H * 7 + W)
    img = rng.random((H, W))
    Hc, Wc = orc.level_size(H, eta), orc.level_size(W, eta)
    ic, jc = np.mgrid[0:Hc, 0:Wc].astype(float)
    coords = [(ic + 0.5) * H / Hc - 0.5, (jc + 0.5) * W / Wc - 0.5]
    ref = ndi.map_coordinates(_scipy_smooth(img, eta), coords, order=1, mode="nearest")
    np.testing.assert_allclose(orc.downsample(img, Hc, Wc, eta), ref, rtol=0, atol=1e-14)


@pytest.mark.parametrize("Hc,Wc,Hf,Wf", [(1, 1, 2, 2), (1, 3, 2, 5), (5, 7, 9, 13), (20, 16, 40, 31), (29, 38, 48, 64)])
def test_upsample_is_bilinear_at_pixel_centres_times_scale(orc, Hc, Wc, Hf, Wf):
    rng = np.random.default_rng(Hc * 3 + Wf)
    f = rng.normal(size=(Hc, Wc))
    i, j = np.mgrid[0:Hf, 0:Wf].astype(float)
    coords = [(i + 0.5) * Hc / Hf - 0.5, (j + 0.5) * Wc / Wf - 0.5]
    for scale in (1.0, Wf / Wc, Hf / Hc):
        ref = scale * ndi.map_coordinates(f, coords, order=1, mode="nearest")
        np.testing.assert_allclose(orc.upsample(f, Hf, Wf, scale), ref, rtol=0, atol=1e-13)


# ------------------------------------------------------------------------------ warping
@pytest.mark.parametrize("H,W", [(1, 1), (1, 9), (7, 1), (20, 24), (45, 61)])
def test_warp_samples_bilinearly_at_the_displaced_position(orc, H, W):
    rng = np.random.default_rng(H + 100 * W)
    I0, I1 = rng.random((H, W)), rng.random((H, W))
    I1x, I1y = orc.derivatives(I1)
    u0 = rng.uniform(-6, 6, (H, W))          # reaches well outside the image: clamped sampling
    v0 = rng.uniform(-6, 6, (H, W))
    beta = 0.05
    Ix, Iy, It, ms = orc.warp_linearise(I0, I1, I1x, I1y, u0, v0, beta)
    i, j = np.mgrid[0:H, 0:W].astype(float)
    coords = [i + v0, j + u0]
    s1 = ndi.map_coordinates(I1, coords, order=1, mode="nearest")
    sx = ndi.map_coordinates(I1x, coords, order=1, mode="nearest")
    sy = ndi.map_coordinates(I1y, coords, order=1, mode="nearest")
    np.testing.assert_allclose(Ix, sx, rtol=0, atol=1e-14)
    np.testing.assert_allclose(Iy, sy, rtol=0, atol=1e-14)
    np.testing.assert_allclose(It, s1 - I0 - sx * u0 - sy * v0, rtol=0, atol=1e-13)
    assert ms == pytest.approx(float(np.max(beta ** 2 + sx ** 2 + sy ** 2)), rel=1e-14)


def test_derivatives_are_central_differences_with_clamped_indices(orc):
    rng = np.random.default_rng(11)
    I = rng.random((13, 17))
    Ix, Iy = orc.derivatives(I)
    gy, gx = np.gradient(I)                  # central differences inside, one-sided at the border
    np.testing.assert_allclose(Ix[:, 1:-1], gx[:, 1:-1], rtol=0, atol=1e-15)
    np.testing.assert_allclose(Iy[1:-1, :], gy[1:-1, :], rtol=0, atol=1e-15)
    # at the border the clamped index halves the one-sided difference
    np.testing.assert_allclose(Ix[:, 0], 0.5 * gx[:, 0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(Iy[-1, :], 0.5 * gy[-1, :], rtol=0, atol=1e-15)


# ------------------------------------------------------------------------------ schedule, 1 x 1
def _prox_w(zw, It, beta, lam, sg):
    """Resolvent of sigma * lambda |beta w + It| in w (Ix = Iy = 0): the three cases of eq.
    (resolvent) along e = (beta, 0, 0)."""
    e2 = beta * beta
    rho = It + beta * zw
    if e2 <= 0.0:
        return zw
    if rho < -sg * lam * e2:
        t = sg * lam
    elif rho > sg * lam * e2:
        t = -sg * lam
    else:
        t = -rho / e2
    return zw + t * beta


def _scalar_schedule(a, b, m, levels, warps, iters, beta, lam, c, r, rho, a_tilde, sigma, cp_sigma):
    """The whole schedule on a 1 x 1 pair I0 = a, I1 = b, by hand.  On one pixel the forward
    differences and the divergence vanish and the clamped central differences give Ix = Iy = 0,
    so u = v = 0 throughout, p, q stay at 0, the warped residual is It = b - a at every warp,
    M_s = beta^2, and each method reduces to a recursion in w (and s) read off its component
    equations in Sec. 3.1.1 (rpADMMI, rpADMMII), Sec. 3.1.2 (pDR) and Sec. 4 (ALG1).  Every
    level is 1 x 1 too; a level change keeps w and restarts the duals (s = 0; pDR and ALG1:
    Xbar = X)."""
    It = b - a
    at = a_tilde if a_tilde > 0 else max(beta * beta, 1e-12)
    w = s = wb = 0.0
    res2 = 0.0
    for lev in range(levels):
        s = 0.0
        wb = w
        for _ in range(warps):
            for _ in range(iters):
                if m == 0:       # rpADMMI: s with the old w, then w -= r c (beta s' - div p')
                    s_new = (1 - beta * beta / at) * s + (It + beta * w) / (at * c)
                    s_new = min(max(s_new, -lam), lam)
                    w -= r * c * beta * s_new
                    res2 = (beta * s_new) ** 2
                    s = s_new
                elif m == 1:     # rpADMMII
                    s_new = (1 - rho * beta * beta / at) * s + (It + beta * w) / (at * c)
                    s_new = min(max(s_new, -lam), lam)
                    w -= c * (beta * s_new - (1 - rho) * beta * s)
                    res2 = (beta * s_new) ** 2
                    s = s_new
                elif m == 2:     # pDR: b = Xbar, the Gauss-Seidel solve is X' = b on one pixel
                    x_new = wb
                    wb = wb + _prox_w(2 * x_new - wb, It, beta, lam, sigma) - x_new
                    res2 = (x_new - w) ** 2
                    w = x_new
                else:            # ALG1: X' = prox(X + sigma div y) with div y = 0, Xbar = 2X' - X
                    x_new = _prox_w(w, It, beta, lam, cp_sigma)
                    res2 = (x_new - w) ** 2
                    wb = 2 * x_new - w
                    w = x_new
    rows = 3.0 if beta != 0 else 2.0
    energy = lam * abs(It + beta * w)
    return w, s, math.sqrt(res2 / rows), energy, It * s


CASES_1x1 = [
    # (a, b, method, r, rho, a_tilde, lam)
    (0.3, 0.8, 0, 1.0, 1.9, 0.0, 5.0),        # pADMM, s clamped at lambda
    (0.5, 0.5001, 0, 1.0, 1.9, 0.0, 5.0),     # pADMM, s inside the box
    (0.3, 0.8, 0, 1.618, 1.9, 0.0, 0.5),      # rpADMMI
    (0.3, 0.8, 0, 1.0, 1.9, 0.01, 5.0),       # pADMM with a fixed a~ > M_s: s^k enters the update
    (0.62, 0.6, 1, 1.0, 1.9, 0.0, 5.0),       # rpADMMII: (1 - rho) s^k in both updates
    (0.62, 0.6, 1, 1.0, 1.3, 0.0, 0.02),      # rpADMMII, clamped
    (0.3, 0.8, 2, 1.0, 1.9, 0.0, 5.0),        # pDR
    (0.5, 0.5003, 2, 1.0, 1.9, 0.0, 5.0),     # pDR, prox in its middle case
    (0.62, 0.5, 2, 1.0, 1.9, 0.0, 0.05),      # pDR, clamped prox steps: the Xbar = X restart shows
    (0.3, 0.8, 3, 1.0, 1.9, 0.0, 5.0),        # ALG1
    (0.5, 0.5003, 3, 1.0, 1.9, 0.0, 5.0),     # ALG1, prox in its middle case
]


@pytest.mark.parametrize("case", CASES_1x1)
@pytest.mark.parametrize("levels,warps,iters", [(1, 1, 7), (1, 3, 9), (3, 2, 13)])
def test_schedule_on_a_single_pixel_by_hand(orc, case, levels, warps, iters):
    a, b, m, r, rho, a_tilde, lam = case
    beta, c, sigma, cp_sigma = 0.05, 0.05, 2.0, 1.25
    P = orc.Params(method=m, lam=lam, beta=beta, c=c, r=r, rho=rho, a_tilde=a_tilde, sigma=sigma, tau=0.4,
                   cp_tau=0.1, cp_sigma=cp_sigma, levels=levels, warps=warps, iters=iters)
    u, v, w, st = orc.solve(np.full((1, 1), a), np.full((1, 1), b), P)
    ew, es, eres, eE, edual = _scalar_schedule(a, b, m, levels, warps, iters, beta, lam, c, r, rho, a_tilde,
                                               sigma, cp_sigma)
    assert u[0, 0] == 0.0 and v[0, 0] == 0.0
    assert w[0, 0] == pytest.approx(ew, rel=1e-12, abs=1e-13)
    assert st["iters_run"] == levels * warps * iters
    assert st["residual"] == pytest.approx(eres, rel=1e-9, abs=1e-14)
    assert st["energy"] == pytest.approx(eE, rel=1e-9, abs=1e-14)
    if m <= 1:
        assert st["dual_value"] == pytest.approx(edual, rel=1e-9, abs=1e-14)


def test_single_pixel_hand_schedule_sees_the_dual_restart():
    """The 1 x 1 cases above can tell a restart of the duals at a level change from none: the
    hand recursion without the restart gives another w (so a schedule that kept s, or kept the
    old Xbar, would fail them)."""
    def no_restart(m, lam):
        It, beta, c, at, rho = 0.5 - 0.62, 0.05, 0.05, 0.0025, 1.9
        w = s = 0.0
        wb = 0.0
        for _ in range(3 * 2 * 13):
            if m == 1:
                s_new = min(max((1 - rho * beta * beta / at) * s + (It + beta * w) / (at * c), -lam), lam)
                w -= c * (beta * s_new - (1 - rho) * beta * s)
                s = s_new
            else:
                x_new = wb
                wb = wb + _prox_w(2 * x_new - wb, It, beta, lam, 2.0) - x_new
                w = x_new
        return w
    for m, lam in ((1, 5.0), (2, 0.05)):
        with_restart = _scalar_schedule(0.62, 0.5, m, 3, 2, 13, 0.05, lam, 0.05, 1.0, 1.9, 0.0, 2.0, 1.25)[0]
        assert abs(no_restart(m, lam) - with_restart) > 1e-6


# ------------------------------------------------------------------------------ schedule, two levels
def _run_level(orc, st, I0, I1, P):
    I1x, I1y = orc.derivatives(I1)
    for _ in range(P.warps):
        Ix, Iy, It, ms = orc.warp_linearise(I0, I1, I1x, I1y, st["u"].copy(), st["v"].copy(), P.beta)
        at = P.a_tilde if P.a_tilde > 0 else max(ms, 1e-12)
        orc.inner(st, Ix, Iy, It, at, P, P.iters)


def _compose_two_levels(orc, I0, I1, P, scale_uv=True, reset_duals=True, xbar_is_x=True, warm=True):
    """The two-level schedule built from the separately pinned pieces: pyramid step, derivatives,
    warping and the inner iterations; the keyword switches plant the plausible mistakes."""
    H, W = I0.shape
    Hc, Wc = orc.level_size(H, P.eta), orc.level_size(W, P.eta)
    c0, c1 = orc.downsample(I0, Hc, Wc, P.eta), orc.downsample(I1, Hc, Wc, P.eta)
    st = orc.State.zeros(Hc, Wc)
    _run_level(orc, st, c0, c1, P)
    fine = orc.State.zeros(H, W)
    if not reset_duals:
        for k in ("p1", "p2", "q11", "q12", "q21", "q22", "s"):
            fine[k] = orc.upsample(st[k], H, W, 1.0)
    if warm:
        fine["w"] = orc.upsample(st["w"], H, W, 1.0)
        fine["u"] = orc.upsample(st["u"], H, W, W / Wc if scale_uv else 1.0)
        fine["v"] = orc.upsample(st["v"], H, W, H / Hc if scale_uv else 1.0)
    if P.beta == 0.0:
        fine["w"] = np.zeros((H, W))
    if P.method in (2, 3) and xbar_is_x:
        for a, b in (("wb", "w"), ("ub", "u"), ("vb", "v")):
            fine[a] = fine[b].copy()
    _run_level(orc, fine, I0, I1, P)
    return fine["u"], fine["v"], fine["w"]


def _two_level_pair(H=12, W=16):
    i, j = np.mgrid[0:H, 0:W].astype(float)
    f = lambda y, x: 0.5 + 0.25 * np.sin(0.7 * x + 0.3 * y) + 0.2 * np.cos(0.45 * y - 0.5 * x + 1.0)
    return f(i, j), f(i + 0.4, j - 0.9)      # I1(x + d) = I0(x) for d = (0.9, -0.4)


SCHED_METHODS = {"padmm": dict(method=0), "rpadmm2": dict(method=1, rho=1.9), "zach": dict(method=0, beta=0.0),
                 "pdr": dict(method=2), "alg1": dict(method=3)}


@pytest.mark.parametrize("name", list(SCHED_METHODS))
def test_two_level_schedule_is_the_composition_of_its_pinned_steps(orc, name):
    I0, I1 = _two_level_pair()
    P = orc.Params(lam=5.0, levels=2, warps=2, iters=9, **SCHED_METHODS[name])
    u, v, w, _ = orc.solve(I0, I1, P)
    cu, cv, cw = _compose_two_levels(orc, I0, I1, P)
    np.testing.assert_allclose(u, cu, rtol=0, atol=1e-12)
    np.testing.assert_allclose(v, cv, rtol=0, atol=1e-12)
    np.testing.assert_allclose(w, cw, rtol=0, atol=1e-12)
    # each planted mistake moves the result well past that agreement
    plants = [dict(scale_uv=False), dict(warm=False)]
    if name in ("pdr", "alg1"):
        plants.append(dict(xbar_is_x=False))
    plants.append(dict(reset_duals=False))
    for plant in plants:
        pu, pv, _ = _compose_two_levels(orc, I0, I1, P, **plant)
        assert max(np.abs(pu - u).max(), np.abs(pv - v).max()) > 1e-6, plant


@pytest.mark.parametrize("name", ["padmm", "pdr", "alg1"])
def test_coarse_level_of_a_pyramid_is_a_one_level_solve_of_the_downsampled_pair(orc, name):
    """The coarsest level starts from zero and out_level returns right after it."""
    I0, I1 = _two_level_pair(24, 32)
    P2 = orc.Params(lam=5.0, levels=2, warps=3, iters=11, out_level=1, **SCHED_METHODS[name])
    P1 = orc.Params(lam=5.0, levels=1, warps=3, iters=11, **SCHED_METHODS[name])
    Hc, Wc = orc.level_size(24, 0.5), orc.level_size(32, 0.5)
    u2, v2, w2, s2 = orc.solve(I0, I1, P2)
    u1, v1, w1, s1 = orc.solve(orc.downsample(I0, Hc, Wc, 0.5), orc.downsample(I1, Hc, Wc, 0.5), P1)
    assert np.array_equal(u2, u1) and np.array_equal(v2, v1) and np.array_equal(w2, w1)
    assert s2["iters_run"] == s1["iters_run"] == 3 * 11
