"""Pins of the oracle's discrete operators (Sec. 2.2) and projections / prox (Sec. 3.1)."""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from tests._mats import grad_matrix, neumann_laplacian

SHAPES = [(1, 1), (1, 9), (9, 1), (7, 5), (8, 8), (33, 17)]


@pytest.mark.parametrize("H,W", SHAPES)
def test_grad_div_adjoint(orc, H, W):
    """<grad u, p> = -<u, div p> exactly for arbitrary u, p (Sec. 2.2)."""
    rng = np.random.default_rng(H * 100 + W)
    for _ in range(5):
        u = rng.normal(size=(H, W))
        px, py = rng.normal(size=(H, W)), rng.normal(size=(H, W))
        gx, gy = orc.grad(u)
        lhs = np.sum(gx * px) + np.sum(gy * py)
        rhs = -np.sum(u * orc.div(px, py))
        assert abs(lhs - rhs) <= 1e-12 * (1 + abs(lhs))


@pytest.mark.parametrize("H,W", SHAPES)
def test_grad_matches_independent_matrix(orc, H, W):
    rng = np.random.default_rng(7)
    u = rng.normal(size=(H, W))
    Dx, Dy = grad_matrix(H, W)
    gx, gy = orc.grad(u)
    np.testing.assert_allclose(gx.ravel(), Dx @ u.ravel(), atol=1e-14)
    np.testing.assert_allclose(gy.ravel(), Dy @ u.ravel(), atol=1e-14)
    px, py = rng.normal(size=(H, W)), rng.normal(size=(H, W))
    np.testing.assert_allclose(orc.div(px, py).ravel(), -(Dx.T @ px.ravel() + Dy.T @ py.ravel()), atol=1e-13)


def test_grad_div_closed_forms(orc):
    H, W = 6, 9
    i, j = np.mgrid[0:H, 0:W].astype(float)
    gx, gy = orc.grad(2.5 * j - 1.25 * i + 3.0)
    assert np.all(gx[:, :-1] == 2.5) and np.all(gx[:, -1] == 0.0)
    assert np.all(gy[:-1, :] == -1.25) and np.all(gy[-1, :] == 0.0)
    d = orc.div(np.full((H, W), 2.0), np.zeros((H, W)))
    assert np.all(d[:, 0] == 2.0) and np.all(d[:, 1:-1] == 0.0) and np.all(d[:, -1] == -2.0)


def test_laplacian_is_div_grad(orc):
    H, W = 11, 7
    f = np.random.default_rng(3).normal(size=(H, W))
    lap = orc.div(*orc.grad(f))
    np.testing.assert_allclose(lap.ravel(), neumann_laplacian(H, W) @ f.ravel(), atol=1e-13)


def test_grad_norm_bound_8(orc):
    """||grad||^2 = ||grad^* grad|| <= 8, which justifies a = 8 (Prop. 3.1); near 8 on large grids."""
    rng = np.random.default_rng(0)
    for H, W, lo in ((5, 4, 0.0), (64, 64, 7.95)):
        x = rng.normal(size=(H, W))
        lam = 0.0
        for _ in range(3000 if H > 10 else 500):
            y = -orc.div(*orc.grad(x))
            lam = np.sqrt(np.sum(y * y) / np.sum(x * x))
            x = y / np.linalg.norm(y)
        assert lo <= lam <= 8.0 + 1e-12


# ------------------------------------------------------------------------- projections
def test_proj_p_invariants(orc):
    rng = np.random.default_rng(1)
    p1, p2 = 2 * rng.normal(size=500), 2 * rng.normal(size=500)
    q1, q2 = orc.proj_p(p1, p2)
    n_in, n_out = np.hypot(p1, p2), np.hypot(q1, q2)
    assert np.all(n_out <= 1 + 1e-15)
    inside = n_in <= 1
    assert np.all(q1[inside] == p1[inside]) and np.all(q2[inside] == p2[inside])
    np.testing.assert_allclose(n_out[~inside], 1.0, atol=1e-15)
    np.testing.assert_allclose(q1 * p2 - q2 * p1, 0.0, atol=1e-14)          # same direction
    assert np.all(q1 * p1 + q2 * p2 >= 0)
    r1, r2 = orc.proj_p(q1, q2)
    np.testing.assert_allclose(r1, q1, atol=1e-15)                          # idempotent
    np.testing.assert_allclose(r2, q2, atol=1e-15)
    # nearest point of the unit disc: no random disc point is closer
    z = rng.normal(size=(200, 2))
    z /= np.maximum(1, np.linalg.norm(z, axis=1))[:, None]
    for k in range(50):
        d_proj = np.hypot(p1[k] - q1[k], p2[k] - q2[k])
        assert np.all(np.hypot(p1[k] - z[:, 0], p2[k] - z[:, 1]) >= d_proj - 1e-14)


def test_proj_q_is_joint(orc):
    """P_q uses the joint 4-component norm (eq. euclid:norm), not two separate 2-norms."""
    q = [np.array([0.6]), np.array([0.6]), np.array([0.6]), np.array([0.6])]   # each pair 0.85 < 1
    out = orc.proj_q(*q)
    np.testing.assert_allclose([o[0] for o in out], [0.5, 0.5, 0.5, 0.5], atol=1e-15)
    rng = np.random.default_rng(2)
    qs = [rng.normal(size=300) for _ in range(4)]
    out = orc.proj_q(*qs)
    nin = np.sqrt(sum(x * x for x in qs))
    nout = np.sqrt(sum(x * x for x in out))
    assert np.all(nout <= 1 + 1e-15)
    np.testing.assert_allclose(nout[nin > 1], 1.0, atol=1e-15)
    for a, b in zip(qs, out):
        np.testing.assert_allclose(b, a / np.maximum(1.0, nin), rtol=0, atol=1e-15)


def test_proj_s_is_clip(orc):
    s = np.random.default_rng(3).normal(size=1000)
    for lam in (0.05, 1.0, 7.0):
        np.testing.assert_allclose(orc.proj_s(s, lam), np.clip(s, -lam, lam), atol=1e-16)


# ------------------------------------------------------------------------- L1 resolvent
def _prox_objective(X, Z, e, It, lam, sigma):
    rho = It + e @ X
    return lam * abs(rho) + np.sum((X - Z) ** 2) / (2 * sigma)


@pytest.mark.parametrize("beta", [0.05, 0.0])
def test_prox_l1_bruteforce(orc, beta):
    """Eq. (resolvent): compare with a brute-force minimisation of
    lambda|rho(X)| + |X - Z|^2 / (2 sigma), over the line Z + t e (where the minimiser lies)
    and against random off-line perturbations."""
    rng = np.random.default_rng(4)
    lam, sigma = 0.7, 2.0
    n = 300
    Ix, Iy = rng.normal(size=n) * 0.3, rng.normal(size=n) * 0.3
    It = rng.normal(size=n) * 0.5
    Z = rng.normal(size=(3, n))
    if beta == 0.0:
        Z[0] = 0.0
    zw, zu, zv = orc.prox_l1(Z[0], Z[1], Z[2], Ix, Iy, It, beta, lam, sigma)
    branches = set()
    for k in range(n):
        e = np.array([beta, Ix[k], Iy[k]])
        e2 = e @ e
        rho = It[k] + e @ Z[:, k]
        branches.add(0 if rho < -sigma * lam * e2 else (2 if rho > sigma * lam * e2 else 1))
        f = lambda t: _prox_objective(Z[:, k] + t * e, Z[:, k], e, It[k], lam, sigma)
        res = minimize_scalar(f, bounds=(-2 * sigma * lam - 1, 2 * sigma * lam + 1), method="bounded",
                              options={"xatol": 1e-13, "maxiter": 2000})
        Xbf = Z[:, k] + res.x * e
        Xo = np.array([zw[k], zu[k], zv[k]])
        assert f((Xo - Z[:, k]) @ e / e2) <= res.fun + 1e-12
        np.testing.assert_allclose(Xo, Xbf, atol=1e-6)
        fo = _prox_objective(Xo, Z[:, k], e, It[k], lam, sigma)
        for _ in range(5):
            Xp = Xo + rng.normal(size=3) * 1e-3
            assert _prox_objective(Xp, Z[:, k], e, It[k], lam, sigma) >= fo - 1e-14
    assert branches == {0, 1, 2}


def test_prox_l1_degenerate_and_nonexpansive(orc):
    rng = np.random.default_rng(5)
    z = [rng.normal(size=10) for _ in range(3)]
    zero = np.zeros(10)
    out = orc.prox_l1(*z, zero, zero, rng.normal(size=10), 0.0, 1.0, 2.0)   # |e| = 0: identity
    for a, b in zip(z, out):
        assert np.array_equal(a, b)
    Ix, Iy, It = rng.normal(size=400), rng.normal(size=400), rng.normal(size=400)
    A = [rng.normal(size=400) for _ in range(3)]
    B = [a + 0.1 * rng.normal(size=400) for a in A]
    PA, PB = orc.prox_l1(*A, Ix, Iy, It, 0.05, 0.5, 2.0), orc.prox_l1(*B, Ix, Iy, It, 0.05, 0.5, 2.0)
    dP = np.sqrt(sum((x - y) ** 2 for x, y in zip(PA, PB)))
    dZ = np.sqrt(sum((x - y) ** 2 for x, y in zip(A, B)))
    assert np.all(dP <= dZ + 1e-14)


def test_prox_l1_continuous_at_case_boundaries(orc):
    beta, lam, sigma = 0.05, 0.5, 2.0
    Ix, Iy, It = np.array([0.3]), np.array([-0.2]), np.array([0.0])
    e2 = beta ** 2 + 0.09 + 0.04
    for sgn in (-1, 1):
        for eps in (1e-9, -1e-9):
            rho = sgn * sigma * lam * e2 * (1 + eps)
            zu = np.array([rho / 0.3])
            out = orc.prox_l1(np.zeros(1), zu, np.zeros(1), Ix, Iy, It, beta, lam, sigma)
            t = (out[1][0] - zu[0]) / 0.3
            assert abs(t - (-sgn * sigma * lam)) < 1e-7
