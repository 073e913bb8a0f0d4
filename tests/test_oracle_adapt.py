"""Pins of the oracle's residual balancing of the ADMM step c (an extension: the paper fixes c;
eq. (stepsize:constraint) of Sec. 3.1.1 bounds only a and a~, so any c > 0 keeps Prop. 3.1's
metrics positive semidefinite), and of pDR's sigma and tau (Sec. 3.1.2 leaves them free; the
balancing keeps sigma tau and so the preconditioned system).

* the balancing rule's two thresholds and its ties;
* the residuals against the optimality conditions of the two subproblems of eq. (aug:pre1:vector),
  written with sparse operators built entry by entry from the definitions (tests/_mats.py): after
  a pADMM step, B^*Lambda + d_y lies in the normal cone of the unit balls at y^{k+1} and
  I_t + A^*Lambda + d_s in the normal cone of [-lambda, lambda] at s^{k+1};
* the window schedule (first warp of each level, every 10th iteration, c carried to the next
  level, frozen after the window) as the composition of those pinned pieces, with planted
  mistakes;
* convergence with the frozen step (Prop. 3.1): residual -> 0 and primal energy = dual value at
  the fixed-c minimum, from starting steps far too small and far too large."""
from dataclasses import replace

import numpy as np
import pytest

from tests._mats import grad_matrix


def test_balancing_rule_thresholds(orc):
    c = 0.05
    assert orc.adapt_rule(c, 10.0001, 1.0) == 2 * c
    assert orc.adapt_rule(c, 10.0, 1.0) == c          # ties keep c
    assert orc.adapt_rule(c, 1.0, 10.0001) == 0.5 * c
    assert orc.adapt_rule(c, 1.0, 10.0) == c
    assert orc.adapt_rule(c, 3.0, 2.0) == c
    assert orc.adapt_rule(c, 0.0, 0.0) == c
    assert orc.adapt_rule(c, 1e-3, 0.0) == 2 * c
    assert orc.adapt_rule(c, 0.0, 1e-3) == 0.5 * c


def _ball(x, radius=1.0):
    n = np.sqrt(np.sum(x * x, axis=0))
    return x / np.maximum(1.0, n / radius)


def _state(orc, rng, H, W, lam, beta):
    """A random ADMM state that keeps the vanishing boundary of the iterates (x-components zero in
    the last column, y-components in the last row), some duals on their ball's surface."""
    st = orc.State.zeros(H, W)
    p = _ball(1.6 * rng.normal(size=(2, H * W)))
    q = _ball(1.6 * rng.normal(size=(4, H * W)))
    for name, arr in (("p1", p[0]), ("p2", p[1]), ("q11", q[0]), ("q12", q[1]), ("q21", q[2]), ("q22", q[3])):
        a = arr.reshape(H, W).copy()
        if name in ("p1", "q11", "q21"):
            a[:, -1] = 0.0
        else:
            a[-1, :] = 0.0
        if beta == 0.0 and name in ("p1", "p2"):
            a[:] = 0.0
        st[name] = a
    st["s"] = np.clip(1.5 * lam * rng.uniform(-1, 1, (H, W)), -lam, lam)
    for k in ("u", "v"):
        st[k] = rng.normal(size=(H, W))
    st["w"] = rng.normal(size=(H, W)) if beta != 0.0 else np.zeros((H, W))
    return st


COMPS = (("w", ("p1", "p2")), ("u", ("q11", "q12")), ("v", ("q21", "q22")))


@pytest.mark.parametrize("beta", [0.05, 0.0])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("c", [0.05, 3.0])
def test_residuals_are_the_subproblem_optimality_gaps(orc, beta, mode, c):
    H, W = 6, 7
    N = H * W
    rng = np.random.default_rng(int(100 * c) + 7 * mode + int(100 * beta))
    lam, a = 0.3, 8.0
    Ix, Iy = rng.normal(size=(H, W)) * 0.5, rng.normal(size=(H, W)) * 0.5
    It = rng.normal(size=(H, W)) * 0.3 * c     # so that the s-step lands inside and on the box
    P = orc.Params(method=0, r=1.0, lam=lam, beta=beta, c=c, a=a, a_tilde_mode=mode)
    ms = beta ** 2 + Ix ** 2 + Iy ** 2
    at = float(ms.max())
    prev = _state(orc, rng, H, W, lam, beta)
    for k in ("w", "u", "v"):
        prev[k] = prev[k] * c
    cur = prev.copy()
    orc.admm_step(cur, Ix, Iy, It, at, P)
    rn, dn = orc.adapt_residuals(prev, cur, Ix, Iy, at, c, P)

    Dx, Dy = grad_matrix(H, W)
    G = np.vstack([Dx.toarray(), Dy.toarray()])      # 2N x N, forward differences
    coef = {"w": np.full(N, beta), "u": Ix.ravel(), "v": Iy.ravel()}
    s1, ds = cur["s"].ravel(), (cur["s"] - prev["s"]).ravel()
    r2, d2 = 0.0, 0.0
    interior = boundary = 0
    for lam_name, (y1, y2) in COMPS:
        if lam_name == "w" and beta == 0.0:
            continue
        y = np.concatenate([cur[y1].ravel(), cur[y2].ravel()])
        dy = y - np.concatenate([prev[y1].ravel(), prev[y2].ravel()])
        A = coef[lam_name]
        r = A * s1 + G.T @ y                              # A s + B y, with B = G^T (B y = -div y)
        dyres = c * (G @ (A * ds) - a * dy + G @ (G.T @ dy))   # c (B^*A ds - (aI - B^*B) dy)
        r2 += r @ r
        d2 += dyres @ dyres
        if lam_name == "w":
            # y-subproblem optimality for p: B^*Lambda^{k+1} + d_y in the normal cone of the unit
            # ball of R^2 at p^{k+1} (per pixel)
            g = (G @ cur["w"].ravel() + dyres).reshape(2, N)
            yy = y.reshape(2, N)
            on = np.sqrt(np.sum(yy * yy, axis=0)) > 1 - 1e-12
            assert np.abs(g[:, ~on]).max(initial=0) < 1e-10
            mu = np.sum(g[:, on] * yy[:, on], axis=0)
            assert np.all(mu > -1e-10)
            assert np.abs(g[:, on] - mu * yy[:, on]).max(initial=0) < 1e-10
            interior += int((~on).sum())
            boundary += int(on.sum())
    # q1, q2 share one ball in R^4: check the joint normal cone
    gq, yq = [], []
    for lam_name, (y1, y2) in COMPS[1:]:
        dy = np.concatenate([(cur[y1] - prev[y1]).ravel(), (cur[y2] - prev[y2]).ravel()])
        A = coef[lam_name]
        dyres = c * (G @ (A * ds) - a * dy + G @ (G.T @ dy))
        gq.append((G @ cur[lam_name].ravel() + dyres).reshape(2, N))
        yq.append(np.vstack([cur[y1].ravel(), cur[y2].ravel()]))
    gq, yq = np.vstack(gq), np.vstack(yq)
    on = np.sqrt(np.sum(yq * yq, axis=0)) > 1 - 1e-12
    assert np.abs(gq[:, ~on]).max(initial=0) < 1e-10
    mu = np.sum(gq[:, on] * yq[:, on], axis=0)
    assert np.all(mu > -1e-10)
    assert np.abs(gq[:, on] - mu * yq[:, on]).max(initial=0) < 1e-10
    interior += int((~on).sum())
    boundary += int(on.sum())
    # s-subproblem: I_t + A^*Lambda^{k+1} + d_s in the normal cone of [-lambda, lambda] at s^{k+1}
    M = beta ** 2 + Ix.ravel() ** 2 + Iy.ravel() ** 2          # A^*A, diagonal
    at_k = np.maximum(M, 1e-12) if mode == 1 else np.full(N, at)
    dsres = c * (M - at_k) * ds
    d2 += dsres @ dsres
    gs = It.ravel() + beta * cur["w"].ravel() + Ix.ravel() * cur["u"].ravel() + Iy.ravel() * cur["v"].ravel() + dsres
    top, bot = s1 > lam - 1e-12, s1 < -lam + 1e-12
    mid = ~(top | bot)
    assert np.abs(gs[mid]).max(initial=0) < 1e-10
    assert np.all(gs[top] > -1e-10) and np.all(gs[bot] < 1e-10)
    assert interior > 0 and boundary > 0 and mid.any() and (top | bot).any()
    assert rn == pytest.approx(np.sqrt(r2), rel=1e-12)
    assert dn == pytest.approx(np.sqrt(d2), rel=1e-12)
    assert dn > 0


def test_residuals_vanish_without_motion_and_scale_with_c(orc):
    """No change of y and s: d = 0.  d is linear in c for the same pair of states."""
    H, W = 5, 4
    rng = np.random.default_rng(3)
    Ix, Iy = rng.normal(size=(H, W)), rng.normal(size=(H, W))
    st = _state(orc, rng, H, W, 0.3, 0.05)
    P = orc.Params(method=0, lam=0.3, beta=0.05)
    rn, dn = orc.adapt_residuals(st, st.copy(), Ix, Iy, 2.0, 0.05, P)
    assert dn == 0.0 and rn > 0
    nxt = st.copy()
    orc.admm_step(nxt, Ix, Iy, rng.normal(size=(H, W)), 2.0, P)
    _, d1 = orc.adapt_residuals(st, nxt, Ix, Iy, 2.0, 0.05, P)
    _, d2 = orc.adapt_residuals(st, nxt, Ix, Iy, 2.0, 0.4, P)
    assert d2 == pytest.approx(8.0 * d1, rel=1e-12)


# ------------------------------------------------------------------ the window schedule
def _adaptive_level(orc, st, I0, I1, P, c, every_warp=False, period=10):
    I1x, I1y = orc.derivatives(I1)
    for wp in range(P.warps):
        Ix, Iy, It, ms = orc.warp_linearise(I0, I1, I1x, I1y, st["u"].copy(), st["v"].copy(), P.beta)
        at = P.a_tilde if P.a_tilde > 0 else max(ms, 1e-12)
        K = P.c_adapt_iters if (wp == 0 or every_warp) else 0
        for k in range(P.iters):
            test = k < K and (k + 1) % period == 0
            prev = st.copy() if test else None
            orc.admm_step(st, Ix, Iy, It, at, replace(P, c=c))
            if test:
                rn, dn = orc.adapt_residuals(prev, st, Ix, Iy, at, c, P)
                c = orc.adapt_rule(c, rn, dn)
    return c


def _adaptive_two_levels(orc, I0, I1, P, carry=True, every_warp=False, period=10):
    H, W = I0.shape
    Hc, Wc = orc.level_size(H, P.eta), orc.level_size(W, P.eta)
    st = orc.State.zeros(Hc, Wc)
    c = _adaptive_level(orc, st, orc.downsample(I0, Hc, Wc, P.eta), orc.downsample(I1, Hc, Wc, P.eta), P, P.c,
                        every_warp, period)
    fine = orc.State.zeros(H, W)
    fine["w"] = orc.upsample(st["w"], H, W, 1.0)
    fine["u"] = orc.upsample(st["u"], H, W, W / Wc)
    fine["v"] = orc.upsample(st["v"], H, W, H / Hc)
    if P.beta == 0.0:
        fine["w"] = np.zeros((H, W))
    c = _adaptive_level(orc, fine, I0, I1, P, c if carry else P.c, every_warp, period)
    return fine["u"], fine["v"], c


def _pair(H=12, W=16):
    i, j = np.mgrid[0:H, 0:W].astype(float)
    f = lambda y, x: 0.5 + 0.25 * np.sin(0.7 * x + 0.3 * y) + 0.2 * np.cos(0.45 * y - 0.5 * x + 1.0)
    return f(i, j), f(i + 0.4, j - 0.9)


@pytest.mark.parametrize("kw", [dict(method=0, c=500.0), dict(method=1, rho=1.9, c=5e-5), dict(method=0, beta=0.0, c=400.0)])
def test_window_schedule_is_the_composition_of_its_pinned_steps(orc, kw):
    I0, I1 = _pair()
    P = orc.Params(lam=5.0, levels=2, warps=2, iters=35, c_adapt_iters=20, **kw)
    u, v, _, st = orc.solve(I0, I1, P)
    cu_, cv_, c = _adaptive_two_levels(orc, I0, I1, P)
    np.testing.assert_allclose(u, cu_, rtol=0, atol=1e-12)
    np.testing.assert_allclose(v, cv_, rtol=0, atol=1e-12)
    assert st["c_final"] == c and c != P.c
    assert np.isfinite(st["adapt_margin"]) and st["adapt_margin"] > 0
    assert st["iters_run"] == 2 * 2 * 35
    # planted mistakes: the step reset at the finer level, the window in every warp, a test
    # every 5 iterations; each changes the final step or the flow.  (While no projection is
    # active the iteration is invariant under c -> 2^k c with the duals scaled by 2^-k, so a
    # plant can leave the flow bitwise unchanged and show only in c.)
    for plant in (dict(carry=False), dict(every_warp=True), dict(period=5)):
        pu, pv, pc = _adaptive_two_levels(orc, I0, I1, P, **plant)
        assert pc != c or max(np.abs(pu - u).max(), np.abs(pv - v).max()) > 1e-6, plant
    # no window: the fixed-step schedule
    u0, v0, _, s0 = orc.solve(I0, I1, replace(P, c_adapt_iters=0))
    assert s0["c_final"] == P.c and not np.array_equal(u0, u)


def test_stopping_test_starts_after_the_window(orc):
    """With tol > 0 the first warp's window runs in full; the test then runs every 10 iterations
    counted from the warp's start, so the run count stays a multiple of 10 (or the budget).  With a
    step 1000 times too large the constraint residual passes the test while the flow is still far
    from the minimum; the balanced step runs longer and stops at a much lower energy."""
    I0, I1 = _pair(24, 32)
    P = orc.Params(lam=5.0, levels=1, warps=1, iters=400, c_adapt_iters=30, c=50.0, tol=1e-3)
    _, _, _, st = orc.solve(I0, I1, P)
    assert 30 <= st["iters_run"] < 400 and st["iters_run"] % 10 == 0
    _, _, _, s0 = orc.solve(I0, I1, replace(P, c_adapt_iters=0))
    assert s0["iters_run"] < 30 and s0["iters_run"] % 10 == 0
    assert st["iters_run"] > s0["iters_run"] and st["energy"] < 0.7 * s0["energy"]


def test_bad_parameters_are_rejected(orc):
    I0, I1 = _pair()
    for kw in (dict(c_adapt_iters=15), dict(c_adapt_iters=-10), dict(c_adapt_iters=20, method=3)):
        with pytest.raises(ValueError):
            orc.solve(I0, I1, orc.Params(levels=1, warps=1, iters=5, **kw))


# ------------------------------------------------------------------ convergence with the frozen step
@pytest.mark.slow
def test_frozen_step_reaches_the_certified_minimum(orc):
    """After the window the iteration is Prop. 3.1's fixed-metric pADMM / rpADMMII, so it converges
    to the saddle point: residual -> 0 and primal energy = dual value <I_t, s> = the fixed-step
    minimum, from a step 100 times too small and 1000 times too large."""
    H, W = 8, 8
    rng = np.random.default_rng(21)
    y_, x_ = np.mgrid[0:H, 0:W].astype(float)
    img = np.sin(0.9 * x_ + 0.3) + np.cos(0.7 * y_ - 0.2 * x_)
    d = dict(Ix=0.3 * np.cos(0.9 * x_ + 0.3), Iy=-0.2 * np.sin(0.7 * y_ - 0.2 * x_),
             It=0.15 * img + 0.05 * rng.normal(size=(H, W)))
    beta, lam = 0.05, 0.8
    at = float((beta ** 2 + d["Ix"] ** 2 + d["Iy"] ** 2).max())
    st = orc.State.zeros(H, W)
    orc.inner(st, d["Ix"], d["Iy"], d["It"], at, orc.Params(method=0, lam=lam, beta=beta), 150000)
    ref = orc.energy(st["w"], st["u"], st["v"], d["Ix"], d["Iy"], d["It"], beta, lam)
    for kw in (dict(method=0, c=0.0005), dict(method=0, c=50.0), dict(method=1, rho=1.9, c=50.0)):
        P = orc.Params(lam=lam, beta=beta, **kw)
        st = orc.State.zeros(H, W)
        n, res, c, margin = orc.inner_adapt(st, d["Ix"], d["Iy"], d["It"], at, P, 250000, 100, P.c)
        E = orc.energy(st["w"], st["u"], st["v"], d["Ix"], d["Iy"], d["It"], beta, lam)
        assert n == 250000 and c != P.c and 0.05 <= c <= 5.0, (kw, c)
        assert res < 1e-7, (kw, res)
        assert abs(E - orc.dual_value(d["It"], st["s"])) < 1e-6 * E, kw
        assert abs(E - ref) < 1e-6 * ref, (kw, E, ref)


def test_balancing_rescues_a_bad_step(orc):
    """With tol = 1e-6 and a step 100 times too small, the fixed-step pADMM does not reach the
    tolerance in 20,000 iterations; with a 100-iteration window it does, well inside."""
    H, W = 8, 8
    y_, x_ = np.mgrid[0:H, 0:W].astype(float)
    rng = np.random.default_rng(21)
    img = np.sin(0.9 * x_ + 0.3) + np.cos(0.7 * y_ - 0.2 * x_)
    Ix, Iy = 0.3 * np.cos(0.9 * x_ + 0.3), -0.2 * np.sin(0.7 * y_ - 0.2 * x_)
    It = 0.15 * img + 0.05 * rng.normal(size=(H, W))
    at = float((0.05 ** 2 + Ix ** 2 + Iy ** 2).max())
    P = orc.Params(method=0, lam=0.8, beta=0.05, c=0.0005, tol=1e-6)
    n0, r0 = orc.inner(orc.State.zeros(H, W), Ix, Iy, It, at, P, 20000)
    n1, r1, c1, _ = orc.inner_adapt(orc.State.zeros(H, W), Ix, Iy, It, at, P, 20000, 100, P.c)
    assert n0 == 20000 and r0 > 1e-5
    assert n1 < 20000 and r1 < 1e-6 and c1 > 0.05


# ------------------------------------------------------------------ pDR: sigma and tau with sigma tau fixed
def test_pdr_balancing_keeps_the_preconditioned_system(orc):
    """Scaling sigma by theta and tau by 1 / theta (theta a power of two) keeps sigma tau, hence
    T = I - sigma tau Laplace and its SRBGS preconditioner: with ybar = 0 and Xbar = X the right-hand
    side is X for every theta, so the X-update is bitwise the same; a step that scaled sigma alone
    would differ."""
    H, W = 7, 9
    rng = np.random.default_rng(8)
    Ix, Iy, It = (rng.normal(size=(H, W)) * s for s in (0.4, 0.4, 0.2))
    base = orc.State.zeros(H, W)
    for k in ("w", "u", "v"):
        base[k] = rng.normal(size=(H, W))
    for a, b in (("wb", "w"), ("ub", "u"), ("vb", "v")):
        base[a] = base[b].copy()
    out = {}
    for th in (1.0, 4.0, 0.125):
        st = base.copy()
        orc.pdr_step(st, Ix, Iy, It, orc.Params(method=2, lam=0.3, sigma=2.0 * th, tau=0.4 / th))
        out[th] = st
    for th in (4.0, 0.125):
        for k in ("w", "u", "v"):
            assert np.array_equal(out[th][k], out[1.0][k]), (th, k)
    st = base.copy()
    orc.pdr_step(st, Ix, Iy, It, orc.Params(method=2, lam=0.3, sigma=8.0, tau=0.4))
    assert not np.array_equal(st["u"], out[1.0]["u"])


def test_pdr_residuals_are_the_per_step_changes(orc):
    H, W = 5, 6
    rng = np.random.default_rng(9)
    a, b = orc.State.zeros(H, W), orc.State.zeros(H, W)
    for st in (a, b):
        for k in orc.STATE_FIELDS:
            st[k] = rng.normal(size=(H, W))
    for beta in (0.05, 0.0):
        P = orc.Params(method=2, beta=beta)
        rx, ry = orc.pdr_adapt_residuals(a, b, 2.0, 0.4, P)
        xs = ("w", "u", "v") if beta else ("u", "v")
        ys = ("p1", "p2", "q11", "q12", "q21", "q22") if beta else ("q11", "q12", "q21", "q22")
        assert rx == pytest.approx(np.sqrt(sum(((b[k] - a[k]) ** 2).sum() for k in xs)) / 2.0, rel=1e-14)
        assert ry == pytest.approx(np.sqrt(sum(((b[k] - a[k]) ** 2).sum() for k in ys)) / 0.4, rel=1e-14)


def _pdr_adaptive_level(orc, st, I0, I1, P, theta, every_warp=False, period=10):
    I1x, I1y = orc.derivatives(I1)
    for wp in range(P.warps):
        Ix, Iy, It, _ = orc.warp_linearise(I0, I1, I1x, I1y, st["u"].copy(), st["v"].copy(), P.beta)
        K = P.c_adapt_iters if (wp == 0 or every_warp) else 0
        for k in range(P.iters):
            test = k < K and (k + 1) % period == 0
            prev = st.copy() if test else None
            Q = replace(P, sigma=P.sigma * theta, tau=P.tau / theta)
            orc.pdr_step(st, Ix, Iy, It, Q)
            if test:
                rx, ry = orc.pdr_adapt_residuals(prev, st, Q.sigma, Q.tau, P)
                theta = orc.adapt_rule(theta, rx, ry)
    return theta


def _pdr_adaptive_two_levels(orc, I0, I1, P, carry=True, every_warp=False, period=10):
    H, W = I0.shape
    Hc, Wc = orc.level_size(H, P.eta), orc.level_size(W, P.eta)
    st = orc.State.zeros(Hc, Wc)
    th = _pdr_adaptive_level(orc, st, orc.downsample(I0, Hc, Wc, P.eta), orc.downsample(I1, Hc, Wc, P.eta), P, 1.0,
                             every_warp, period)
    fine = orc.State.zeros(H, W)
    fine["w"] = orc.upsample(st["w"], H, W, 1.0)
    fine["u"] = orc.upsample(st["u"], H, W, W / Wc)
    fine["v"] = orc.upsample(st["v"], H, W, H / Hc)
    for a, b in (("wb", "w"), ("ub", "u"), ("vb", "v")):
        fine[a] = fine[b].copy()
    th = _pdr_adaptive_level(orc, fine, I0, I1, P, th if carry else 1.0, every_warp, period)
    return fine["u"], fine["v"], th


@pytest.mark.parametrize("kw,plants", [(dict(sigma=32.0, tau=0.025), True), (dict(sigma=64.0, tau=0.0125), True),
                                       (dict(sigma=0.125, tau=6.4), False)])
def test_pdr_window_schedule_is_the_composition_of_its_pinned_steps(orc, kw, plants):
    """The ratio far too large (the planted mistakes each change the result) and far too small
    (balanced within the first warp, so the window-in-every-warp plant would not show)."""
    I0, I1 = _pair()
    P = orc.Params(method=2, lam=5.0, levels=2, warps=2, iters=35, c_adapt_iters=20, **kw)
    u, v, _, st = orc.solve(I0, I1, P)
    cu_, cv_, th = _pdr_adaptive_two_levels(orc, I0, I1, P)
    np.testing.assert_allclose(u, cu_, rtol=0, atol=1e-12)
    np.testing.assert_allclose(v, cv_, rtol=0, atol=1e-12)
    assert st["c_final"] == P.sigma * th and th != 1.0
    for plant in ((dict(carry=False), dict(every_warp=True), dict(period=5)) if plants else ()):
        pu, pv, pth = _pdr_adaptive_two_levels(orc, I0, I1, P, **plant)
        assert pth != th or max(np.abs(pu - u).max(), np.abs(pv - v).max()) > 1e-6, plant


@pytest.mark.slow
def test_pdr_frozen_steps_reach_the_certified_minimum(orc):
    """With theta frozen after the window the iteration is Prop. 3.2's pDR with fixed steps: from a
    sigma / tau ratio 256 times too large or too small it reaches the pADMM-certified minimum."""
    H, W = 8, 8
    rng = np.random.default_rng(21)
    y_, x_ = np.mgrid[0:H, 0:W].astype(float)
    img = np.sin(0.9 * x_ + 0.3) + np.cos(0.7 * y_ - 0.2 * x_)
    d = dict(Ix=0.3 * np.cos(0.9 * x_ + 0.3), Iy=-0.2 * np.sin(0.7 * y_ - 0.2 * x_),
             It=0.15 * img + 0.05 * rng.normal(size=(H, W)))
    beta, lam = 0.05, 0.8
    at = float((beta ** 2 + d["Ix"] ** 2 + d["Iy"] ** 2).max())
    st = orc.State.zeros(H, W)
    orc.inner(st, d["Ix"], d["Iy"], d["It"], at, orc.Params(method=0, lam=lam, beta=beta), 150000)
    ref = orc.energy(st["w"], st["u"], st["v"], d["Ix"], d["Iy"], d["It"], beta, lam)
    for th0 in (1 / 16.0, 16.0):
        P = orc.Params(method=2, lam=lam, beta=beta, sigma=2.0 * th0, tau=0.4 / th0)
        st = orc.State.zeros(H, W)
        n, res, th, _ = orc.inner_adapt_pdr(st, d["Ix"], d["Iy"], d["It"], P, 100000, 100)
        E = orc.energy(st["w"], st["u"], st["v"], d["Ix"], d["Iy"], d["It"], beta, lam)
        assert th != 1.0 and 0.25 <= th0 * th <= 1.0, (th0, th)   # the ratio ends balanced
        assert abs(E - ref) < 1e-5 * ref, (th0, E, ref)
        assert res < 1e-8
