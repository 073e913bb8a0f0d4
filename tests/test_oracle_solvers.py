"""Pins of the oracle's solver iterations: red-black SGS (Sec. 3.1.2), the rpADMMI / rpADMMII /
Zach-pADMM updates (Sec. 3.1.1, appendix derivation of the y/s updates), pDR (Sec. 3.1.2), the
ALG1 primal-dual comparison solver (Sec. 4) and their common fixed point (Props. 3.1 and 3.2,
strong duality of Sec. 2.2).

The sparse operators come from tests/_mats.py, built entry by entry from the definitions, so
these checks share nothing with the oracle's C code."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from tests._mats import grad_matrix, neumann_laplacian


# ------------------------------------------------------------------------ helpers
def _ball(x, radius=1.0):
    """Pointwise projection of stacked components x[k] (k x N) onto the Euclidean ball."""
    n = np.sqrt(np.sum(x * x, axis=0))
    return x / np.maximum(1.0, n / radius)


def _random_problem(H, W, seed, beta=0.05, lam=0.3):
    rng = np.random.default_rng(seed)
    N = H * W
    data = dict(Ix=rng.normal(size=(H, W)) * 0.4, Iy=rng.normal(size=(H, W)) * 0.4,
                It=rng.normal(size=(H, W)) * 0.2)
    return rng, data, beta, lam


def _random_state(orc, rng, H, W, lam, beta):
    st = orc.State.zeros(H, W)
    p = _ball(rng.normal(size=(2, H * W)))
    q = _ball(rng.normal(size=(4, H * W)))
    # a vanishing boundary as the ADMM iterates keep it: x-components zero in the last column,
    # y-components zero in the last row
    for comp, arr in (("p1", p[0]), ("p2", p[1]), ("q11", q[0]), ("q12", q[1]), ("q21", q[2]), ("q22", q[3])):
        a = arr.reshape(H, W).copy()
        if comp in ("p1", "q11", "q21"):
            a[:, -1] = 0.0
        else:
            a[-1, :] = 0.0
        st[comp] = a
    st["s"] = rng.uniform(-lam, lam, size=(H, W))
    for k in ("w", "u", "v"):
        st[k] = rng.normal(size=(H, W))
    if beta == 0.0:
        st["w"] = np.zeros((H, W))
        st["p1"] = np.zeros((H, W))
        st["p2"] = np.zeros((H, W))
    return st


class _Ops:
    def __init__(self, H, W):
        Dx, Dy = grad_matrix(H, W)
        self.D = sp.vstack([Dx, Dy]).tocsr()         # 2N x N gradient
        self.N = H * W

    def grad(self, f):
        return (self.D @ f.ravel()).reshape(2, -1)

    def Bt(self, y2):
        """-div y = D^T y for a 2 x N dual field."""
        return self.D.T @ y2.ravel()


def _flat(st, *names):
    return np.stack([st[n].ravel() for n in names])


# ------------------------------------------------------------------------ SRBGS
def test_srbgs_red_equations_hold_after_a_sweep(orc):
    H, W, stau = 9, 7, 0.8
    rng = np.random.default_rng(0)
    x0, b = rng.normal(size=(H, W)), rng.normal(size=(H, W))
    T = sp.identity(H * W) - stau * neumann_laplacian(H, W)
    x = orc.srbgs(x0, b, stau, 1)
    r = (b.ravel() - T @ x.ravel()).reshape(H, W)
    red = (np.add.outer(np.arange(H), np.arange(W)) % 2) == 0
    assert np.max(np.abs(r[red])) < 1e-13            # the sweep ends with a red half-sweep
    assert np.max(np.abs(r[~red])) > 1e-6


def test_srbgs_decreases_quadratic_and_converges_to_direct_solve(orc):
    H, W, stau = 12, 10, 0.8
    rng = np.random.default_rng(1)
    x, b = rng.normal(size=(H, W)), rng.normal(size=(H, W))
    T = (sp.identity(H * W) - stau * neumann_laplacian(H, W)).tocsc()
    q = lambda z: 0.5 * z.ravel() @ (T @ z.ravel()) - b.ravel() @ z.ravel()
    prev = q(x)
    for _ in range(20):
        x = orc.srbgs(x, b, stau, 1)
        cur = q(x)
        assert cur <= prev + 1e-13
        prev = cur
    xs = spla.spsolve(T, b.ravel())
    x = orc.srbgs(x, b, stau, 400)
    np.testing.assert_allclose(x.ravel(), xs, atol=1e-12)


def test_srbgs_is_affine(orc):
    H, W, stau = 6, 5, 0.8
    rng = np.random.default_rng(2)
    x1, x2, b1, b2 = (rng.normal(size=(H, W)) for _ in range(4))
    lhs = orc.srbgs(x1 + 2 * x2, b1 + 2 * b2, stau, 2)
    rhs = orc.srbgs(x1, b1, stau, 2) + 2 * orc.srbgs(x2, b2, stau, 2)
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)


# ------------------------------------------------------------------------ ADMM updates
@pytest.mark.parametrize("beta", [0.05, 0.0])
@pytest.mark.parametrize("r", [1.0, 1.618])
@pytest.mark.parametrize("mode", [0, 1])
def test_rpadmm1_step_solves_its_subproblems(orc, beta, r, mode):
    """eq. (aug:pre1:vector): y^{k+1} maximises L_c(Lambda^k; y, s^k) - 1/2||y - y^k||^2_{acI - c grad grad^*}
    over |p|, |q| <= 1; s^{k+1} maximises L_c(Lambda^k; y^{k+1}, s) - 1/2||s - s^k||^2_{c(diag(a~) - M_s)}
    over |s| <= lambda (with <I_t, s> counted once), a~ one value (mode 0) or the per-pixel
    a~_ij = M_s(ij) (mode 1); Lambda^{k+1} = Lambda^k - rc(A s + B y)."""
    H, W = 7, 6
    rng, d, beta, lam = _random_problem(H, W, 11, beta=beta)
    Ix, Iy, It = (d[k].ravel() for k in ("Ix", "Iy", "It"))
    P = orc.Params(method=0, lam=lam, beta=beta, c=0.05, a=8.0, r=r, a_tilde_mode=mode)
    a, c = P.a, P.c
    st = _random_state(orc, rng, H, W, lam, beta)
    Ms = beta ** 2 + Ix ** 2 + Iy ** 2
    at = float(Ms.max()) * 1.1
    ops = _Ops(H, W)
    old = st.copy()
    orc.admm_step(st, d["Ix"], d["Iy"], d["It"], at, P)

    s0, w0, u0, v0 = (old[k].ravel() for k in ("s", "w", "u", "v"))
    blocks = [("u", ("q11", "q12"), Ix), ("v", ("q21", "q22"), Iy)]
    if beta != 0.0:
        blocks.insert(0, ("w", ("p1", "p2"), np.full_like(Ix, beta)))
    # --- y-update: grad of the concave objective at y^k; Hessian is -ac I, so
    # y^{k+1} = Proj(y^k + grad/(ac)); also check the variational inequality
    ystar, yk, gk = [], [], []
    for lam_name, comps, coef in blocks:
        yk_b = _flat(old, *comps)
        cons = coef * s0 + ops.Bt(yk_b)
        g = ops.grad(old[lam_name]) - c * ops.grad(cons.reshape(H, W))     # B^*(Lambda - c(A s + B y))
        yk.append(yk_b); gk.append(g); ystar.append(_flat(st, *comps))
    if beta != 0.0:
        pred = [_ball(yk[0] + gk[0] / (a * c))] + [None]
        qpred = _ball(np.vstack([yk[1] + gk[1] / (a * c), yk[2] + gk[2] / (a * c)]))
        np.testing.assert_allclose(ystar[0], pred[0], atol=1e-12)
        np.testing.assert_allclose(np.vstack(ystar[1:]), qpred, atol=1e-12)
    else:
        qpred = _ball(np.vstack([yk[0] + gk[0] / (a * c), yk[1] + gk[1] / (a * c)]))
        np.testing.assert_allclose(np.vstack(ystar), qpred, atol=1e-12)
    # variational inequality <grad Phi(y*), z - y*> <= 0 for feasible z
    def phi_grad(ys):
        out = []
        for (lam_name, comps, coef), yb, ykb in zip(blocks, ys, yk):
            cons = coef * s0 + ops.Bt(yb)
            prox = a * c * (yb - ykb).ravel() - c * (ops.D @ (ops.D.T @ (yb - ykb).ravel()))
            out.append(ops.grad(old[lam_name]).ravel() - c * (ops.D @ cons) - prox)
        return out
    gstar = phi_grad(ystar)
    for _ in range(20):
        z = [_ball(rng.normal(size=yb.shape) * 2) for yb in ystar]
        z[-2:] = list(np.split(_ball(np.vstack(z[-2:]) * 1.0), 2))
        vi = sum(g @ (zz - ys).ravel() for g, zz, ys in zip(gstar, z, ystar))
        assert vi <= 1e-10
    # --- s-update
    yn = {comps: _flat(st, *comps) for _, comps, _ in blocks}
    grad_s = It.copy()
    cons_tot = np.zeros_like(Ix)
    for lam_name, comps, coef in blocks:
        cons = coef * s0 + ops.Bt(yn[comps])
        grad_s += coef * (old[lam_name].ravel() - c * cons)
    at_px = np.maximum(Ms, 1e-12) if mode == 1 else at
    s_pred = np.clip(s0 + grad_s / (at_px * c), -lam, lam)
    np.testing.assert_allclose(st["s"].ravel(), s_pred, atol=1e-12)
    # --- multipliers
    s1 = st["s"].ravel()
    for lam_name, comps, coef in blocks:
        cons = coef * s1 + ops.Bt(yn[comps])
        np.testing.assert_allclose(st[lam_name].ravel(), old[lam_name].ravel() - r * c * cons, atol=1e-12)
    if beta == 0.0:
        for k in ("w", "p1", "p2"):
            assert np.all(st[k] == 0.0)


def test_rpadmm2_matches_its_generic_form(orc):
    """eq. (update:two:sun:lag) with N = acI, M = a~cI (and the multiplier scaled by c, as in
    the component form eq. rpADMMII)."""
    H, W = 6, 7
    rng, d, beta, lam = _random_problem(H, W, 12)
    Ix, Iy, It = (d[k].ravel() for k in ("Ix", "Iy", "It"))
    rho = 1.9
    P = orc.Params(method=1, lam=lam, beta=beta, c=0.05, a=8.0, rho=rho)
    a, c = P.a, P.c
    st = _random_state(orc, rng, H, W, lam, beta)
    at = float((beta ** 2 + Ix ** 2 + Iy ** 2).max())
    ops = _Ops(H, W)
    old = st.copy()
    orc.admm_step(st, d["Ix"], d["Iy"], d["It"], at, P)
    blocks = [("w", ("p1", "p2"), np.full_like(Ix, beta)), ("u", ("q11", "q12"), Ix), ("v", ("q21", "q22"), Iy)]
    s0 = old["s"].ravel()
    # y: (N + dH)^{-1}(B^*(-c A s^k + Lambda^k) + (N - c B^*B) y^k)
    args = []
    for lam_name, comps, coef in blocks:
        yk = _flat(old, *comps)
        arg = ops.grad((old[lam_name].ravel() - c * coef * s0).reshape(H, W)).ravel() \
            + a * c * yk.ravel() - c * (ops.D @ (ops.D.T @ yk.ravel()))
        args.append((arg / (a * c)).reshape(2, -1))
    np.testing.assert_allclose(_flat(st, "p1", "p2"), _ball(args[0]), atol=1e-12)
    np.testing.assert_allclose(np.vstack([_flat(st, "q11", "q12"), _flat(st, "q21", "q22")]),
                               _ball(np.vstack(args[1:])), atol=1e-12)
    # s: (M + dG)^{-1}(A^*(-c rho B y' + c(1-rho) A s^k + Lambda^k) + (M - c A^*A) s^k)
    arg = np.zeros_like(s0)
    Ms = np.zeros_like(s0)
    for lam_name, comps, coef in blocks:
        By = ops.Bt(_flat(st, *comps))
        arg += coef * (-c * rho * By + c * (1 - rho) * coef * s0 + old[lam_name].ravel())
        Ms += coef * coef
    arg += (a * 0 + at * c - c * Ms) * s0
    s_pred = np.clip((arg + It) / (at * c), -lam, lam)
    np.testing.assert_allclose(st["s"].ravel(), s_pred, atol=1e-12)
    s1 = st["s"].ravel()
    for lam_name, comps, coef in blocks:
        By = ops.Bt(_flat(st, *comps))
        pred = old[lam_name].ravel() - c * (coef * s1 - (1 - rho) * coef * s0 + rho * By)
        np.testing.assert_allclose(st[lam_name].ravel(), pred, atol=1e-12)


def test_rpadmm2_rho1_equals_padmm(orc):
    H, W = 9, 8
    rng, d, beta, lam = _random_problem(H, W, 13)
    st = _random_state(orc, rng, H, W, lam, beta)
    s1, s2 = st.copy(), st.copy()
    at = 2.0
    orc.admm_step(s1, d["Ix"], d["Iy"], d["It"], at, orc.Params(method=0, lam=lam, r=1.0))
    orc.admm_step(s2, d["Ix"], d["Iy"], d["It"], at, orc.Params(method=1, lam=lam, rho=1.0))
    for k in orc.STATE_FIELDS:
        np.testing.assert_allclose(s1[k], s2[k], atol=1e-14)


# ------------------------------------------------------------------------ pDR
def test_pdr_step_matches_generic_form_with_exact_inner_solve(orc):
    """Generic pDR: b = Xbar - sigma K^* ybar, X' solves T X = b (many SRBGS sweeps),
    Xbar' = Xbar + prox(2X' - Xbar) - X', ybar' = P(ybar + 2 tau K X') - tau K X'."""
    H, W = 6, 5
    rng, d, beta, lam = _random_problem(H, W, 14)
    P = orc.Params(method=2, lam=lam, beta=beta, sigma=2.0, tau=0.4, gs_sweeps=600)
    st = _random_state(orc, rng, H, W, lam, beta)
    for k in ("wb", "ub", "vb"):
        st[k] = rng.normal(size=(H, W))
    old = st.copy()
    orc.pdr_step(st, d["Ix"], d["Iy"], d["It"], P)
    ops = _Ops(H, W)
    T = (sp.identity(H * W) - P.sigma * P.tau * neumann_laplacian(H, W)).tocsc()
    Xn = {}
    for x, xb, comps in (("w", "wb", ("p1", "p2")), ("u", "ub", ("q11", "q12")), ("v", "vb", ("q21", "q22"))):
        b = old[xb].ravel() - P.sigma * ops.Bt(_flat(old, *comps))
        Xn[x] = spla.spsolve(T, b)
        np.testing.assert_allclose(st[x].ravel(), Xn[x], atol=1e-10)
    Z = [2 * st[x] - old[xb] for x, xb in (("w", "wb"), ("u", "ub"), ("v", "vb"))]
    pz = orc.prox_l1(*Z, d["Ix"], d["Iy"], d["It"], beta, lam, P.sigma)
    for (x, xb), pzc in zip((("w", "wb"), ("u", "ub"), ("v", "vb")), pz):
        np.testing.assert_allclose(st[xb], old[xb] + pzc - st[x], atol=1e-12)
    gw = ops.grad(st["w"])
    np.testing.assert_allclose(_flat(st, "p1", "p2"), _ball(_flat(old, "p1", "p2") + 2 * P.tau * gw) - P.tau * gw, atol=1e-12)
    gq = np.vstack([ops.grad(st["u"]), ops.grad(st["v"])])
    qo = np.vstack([_flat(old, "q11", "q12"), _flat(old, "q21", "q22")])
    np.testing.assert_allclose(np.vstack([_flat(st, "q11", "q12"), _flat(st, "q21", "q22")]),
                               _ball(qo + 2 * P.tau * gq) - P.tau * gq, atol=1e-12)


@pytest.mark.parametrize("beta", [0.05, 0.0])
def test_alg1_step_is_dual_projection_then_primal_prox(orc, beta):
    """ALG1 (Chambolle-Pock, theta = 1): y' is the projection of y + tau K Xbar (P_p, joint P_q);
    X' minimises sigma lambda |rho(X)| + |X - Z|^2 / 2 pointwise with Z = X - sigma K^* y'
    (checked against the objective at perturbed points and by a 1-D search along e);
    Xbar' = 2 X' - X."""
    H, W = 6, 7
    rng, d, _, lam = _random_problem(H, W, 31, beta=beta)
    P = orc.Params(method=3, lam=lam, beta=beta, cp_tau=0.1, cp_sigma=1.25)
    st = _random_state(orc, rng, H, W, lam, beta)
    for k in ("wb", "ub", "vb"):
        st[k] = rng.normal(size=(H, W)) if (beta != 0.0 or k != "wb") else np.zeros((H, W))
    old = st.copy()
    r2 = orc.cp_step(st, d["Ix"], d["Iy"], d["It"], P)
    ops = _Ops(H, W)
    # dual step
    if beta != 0.0:
        np.testing.assert_allclose(_flat(st, "p1", "p2"), _ball(_flat(old, "p1", "p2") + P.cp_tau * ops.grad(old["wb"])),
                                   atol=1e-13)
    qn = _ball(np.vstack([_flat(old, "q11", "q12") + P.cp_tau * ops.grad(old["ub"]),
                          _flat(old, "q21", "q22") + P.cp_tau * ops.grad(old["vb"])]))
    np.testing.assert_allclose(np.vstack([_flat(st, "q11", "q12"), _flat(st, "q21", "q22")]), qn, atol=1e-13)
    # primal step: pointwise minimiser of sigma lambda |rho(X)| + |X - Z|^2 / 2
    Z = [old[x].ravel() - P.cp_sigma * ops.Bt(_flat(st, *c)) for x, c in
         (("w", ("p1", "p2")), ("u", ("q11", "q12")), ("v", ("q21", "q22")))]
    if beta == 0.0:
        Z[0] = np.zeros(H * W)
    Xn = np.stack([st[x].ravel() for x in ("w", "u", "v")])
    Z = np.stack(Z)
    e = np.stack([np.full(H * W, beta), d["Ix"].ravel(), d["Iy"].ravel()])
    It = d["It"].ravel()

    def obj(X):
        return P.cp_sigma * lam * np.abs(It + np.sum(e * X, 0)) + 0.5 * np.sum((X - Z) ** 2, 0)

    f0 = obj(Xn)
    for _ in range(40):
        dX = rng.normal(size=Xn.shape) * 10.0 ** rng.uniform(-6, -1)
        if beta == 0.0:
            dX[0] = 0.0
        assert np.all(obj(Xn + dX) >= f0 - 1e-12)
    # the minimiser lies on the line Z + t e: no point of it does better
    ts = np.linspace(-3.0, 3.0, 6001)
    for k in range(H * W):
        ek = e[:, k]
        line = P.cp_sigma * lam * np.abs(It[k] + ek @ Z[:, k] + ts * (ek @ ek)) + 0.5 * ts ** 2 * (ek @ ek)
        assert f0[k] <= line.min() + 1e-12
    # extrapolation and the returned step size
    for x, xb in (("w", "wb"), ("u", "ub"), ("v", "vb")):
        np.testing.assert_allclose(st[xb], 2 * st[x] - old[x], atol=1e-13)
    assert r2 == pytest.approx(sum(np.sum((st[x] - old[x]) ** 2) for x in ("w", "u", "v")), rel=1e-12)


# ------------------------------------------------------------------------ fixed point
def _primal_energy_dense(H, W, X, d, beta, lam):
    ops = _Ops(H, W)
    w, u, v = (x.ravel() for x in X)
    gw, gu, gv = ops.grad(w.reshape(H, W)), ops.grad(u.reshape(H, W)), ops.grad(v.reshape(H, W))
    rho = d["Ix"].ravel() * u + d["Iy"].ravel() * v + beta * w + d["It"].ravel()
    E = np.sum(np.sqrt(np.sum(gu ** 2, 0) + np.sum(gv ** 2, 0))) + lam * np.sum(np.abs(rho))
    if beta != 0.0:
        E += np.sum(np.sqrt(np.sum(gw ** 2, 0)))
    return E


def _pdhg_bruteforce(H, W, d, beta, lam, iters=60000):
    """Generic first-order primal-dual solve of the discrete energy eq. (l1:finite) with dense
    matrices: min_X max_y <K X, y> - f^*(y), K = [grad w; grad u; grad v; A X]."""
    ops = _Ops(H, W)
    N = H * W
    D = ops.D.toarray()
    Z = np.zeros_like(D)
    Ix, Iy, It = (d[k].ravel() for k in ("Ix", "Iy", "It"))
    K = np.block([[D, Z[:, :N] * 0 + np.zeros((2 * N, N)), np.zeros((2 * N, N))],
                  [np.zeros((2 * N, N)), D, np.zeros((2 * N, N))],
                  [np.zeros((2 * N, N)), np.zeros((2 * N, N)), D],
                  [beta * np.eye(N), np.diag(Ix), np.diag(Iy)]])
    L = np.linalg.norm(K, 2)
    tau = sig = 0.99 / L
    X = np.zeros(3 * N); Xb = X.copy(); y = np.zeros(7 * N)
    Xsum = np.zeros(3 * N)
    for it in range(iters):
        y = y + sig * (K @ Xb)
        p = _ball(y[:2 * N].reshape(2, N)).ravel() if beta != 0.0 else np.zeros(2 * N)
        q = _ball(y[2 * N:6 * N].reshape(4, N)).ravel()
        s = np.clip(y[6 * N:] + sig * It, -lam, lam)
        y = np.concatenate([p, q, s])
        Xn = X - tau * (K.T @ y)
        if beta == 0.0:
            Xn[:N] = 0.0
        Xb = 2 * Xn - X
        X = Xn
    return X.reshape(3, H, W)


@pytest.mark.slow
def test_solvers_reach_the_same_minimum_with_a_dual_certificate(orc):
    """Props. 3.1 / 3.2: rpADMMI, rpADMMII and pDR converge to a saddle point.  At the limit the
    ADMM duals are feasible (A s + B y -> 0) and the primal energy equals the dual value
    <I_t, s> (strong duality), which certifies the minimum; pDR and an independent dense
    primal-dual solve reach the same energy."""
    H, W = 8, 8
    rng = np.random.default_rng(21)
    y_, x_ = np.mgrid[0:H, 0:W].astype(float)
    img = np.sin(0.9 * x_ + 0.3) + np.cos(0.7 * y_ - 0.2 * x_)
    d = dict(Ix=0.3 * np.cos(0.9 * x_ + 0.3), Iy=-0.2 * np.sin(0.7 * y_ - 0.2 * x_),
             It=0.15 * img + 0.05 * rng.normal(size=(H, W)))
    beta, lam = 0.05, 0.8
    at = float((beta ** 2 + d["Ix"] ** 2 + d["Iy"] ** 2).max())
    energies = {}
    for name, P in (("padmm", orc.Params(method=0, lam=lam, beta=beta, c=0.05)),
                    ("rpadmm1", orc.Params(method=0, lam=lam, beta=beta, c=0.05, r=1.618)),
                    ("rpadmm2", orc.Params(method=1, lam=lam, beta=beta, c=0.05, rho=1.9))):
        st = orc.State.zeros(H, W)
        n, res = orc.inner(st, d["Ix"], d["Iy"], d["It"], at, P, 150000)
        E = orc.energy(st["w"], st["u"], st["v"], d["Ix"], d["Iy"], d["It"], beta, lam)
        Ed = _primal_energy_dense(H, W, (st["w"], st["u"], st["v"]), d, beta, lam)
        dual = orc.dual_value(d["It"], st["s"])
        assert abs(E - Ed) < 1e-12 * E
        assert res < 1e-7, (name, res)
        assert abs(E - dual) < 1e-6 * E, (name, E, dual)
        energies[name] = E
    P = orc.Params(method=2, lam=lam, beta=beta, sigma=2.0, tau=0.4, gs_sweeps=1)
    st = orc.State.zeros(H, W)
    orc.inner(st, d["Ix"], d["Iy"], d["It"], at, P, 100000)
    energies["pdr"] = orc.energy(st["w"], st["u"], st["v"], d["Ix"], d["Iy"], d["It"], beta, lam)
    ref = energies["padmm"]
    for k, e in energies.items():
        assert abs(e - ref) < 1e-6 * ref, (k, energies)
    # ALG1 (constant steps tau = 0.1, sigma = 1.25) reaches the certified minimum as well
    P = orc.Params(method=3, lam=lam, beta=beta, cp_tau=0.1, cp_sigma=1.25)
    st = orc.State.zeros(H, W)
    orc.inner(st, d["Ix"], d["Iy"], d["It"], at, P, 200000)
    ecp = orc.energy(st["w"], st["u"], st["v"], d["Ix"], d["Iy"], d["It"], beta, lam)
    assert abs(ecp - ref) < 1e-7 * ref, (ecp, ref)
    # The dense generic solve converges slowly (O(1/k)); it must never find a lower energy than
    # the certified minimum and must approach it.
    Xbf = _pdhg_bruteforce(H, W, d, beta, lam)
    ebf = _primal_energy_dense(H, W, Xbf, d, beta, lam)
    assert ebf >= ref * (1 - 1e-9)
    assert ebf - ref < 5e-4 * ref


@pytest.mark.slow
def test_per_pixel_preconditioner_reaches_the_certified_minimum(orc):
    """The per-pixel s-preconditioner a~_ij = M_s(ij) keeps c(diag(a~) - M_s) >= 0 (M_s is
    diagonal), so pADMM and rpADMMII still converge to the saddle point: residual -> 0, primal
    energy = dual value (strong duality) = the scalar-a~ minimum.  On this problem pADMM needs
    about half the iterations of the scalar a~ = max M_s to reach a residual of 1e-6."""
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
    for kw in (dict(method=0), dict(method=1, rho=1.9)):
        st = orc.State.zeros(H, W)
        n, res = orc.inner(st, d["Ix"], d["Iy"], d["It"], at, orc.Params(lam=lam, beta=beta, a_tilde_mode=1, **kw), 150000)
        E = orc.energy(st["w"], st["u"], st["v"], d["Ix"], d["Iy"], d["It"], beta, lam)
        assert res < 1e-8, (kw, res)
        assert abs(E - ref) < 1e-7 * ref and abs(E - orc.dual_value(d["It"], st["s"])) < 1e-7 * E, (kw, E, ref)
    runs = {}
    for mode in (0, 1):
        st = orc.State.zeros(H, W)
        runs[mode], _ = orc.inner(st, d["Ix"], d["Iy"], d["It"], at,
                                  orc.Params(method=0, lam=lam, beta=beta, a_tilde_mode=mode, tol=1e-6), 200000)
    assert runs[1] < 0.7 * runs[0], runs


def test_zero_motion_pair_stays_zero(orc):
    """I1 = I0: at zero flow It = 0, every update keeps the whole state at exactly zero."""
    from paper_2011_10979_gb300 import synth
    pr = synth.sinusoid_pair(seed=5)
    for m in (0, 1, 2, 3):
        u, v, w, st = orc.solve(pr.I0, pr.I0, orc.Params(method=m, levels=2, warps=2, iters=20))
        assert np.all(u == 0.0) and np.all(v == 0.0) and np.all(w == 0.0)
