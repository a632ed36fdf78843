"""Pins of the ADMM oracle (Sec. 2.2, Algorithm 1 on Eq. 3) against what the
mathematics fixes: an independent convolution routine, adjoint identities,
closed forms of TV and of its prox, and the optimum of the convex problem
solved by other methods (an exact LP when the constraint is a box, SQP when
the constraint has windows of several sides)."""
import numpy as np
import pytest

import oracle
from oracle import admm as A

scipy = pytest.importorskip("scipy")
from scipy import optimize, signal  # noqa: E402


def test_blur_matches_independent_convolution():
    # zero-boundary "same" convolution with the outer-product kernel
    rng = np.random.default_rng(0)
    x = rng.normal(size=(13, 17))
    for sigma, radius in ((0.6, 0), (1.5, 0), (2.0, 3)):
        w = A.gaussian_kernel(sigma, radius)
        assert abs(w.sum() - 1.0) < 1e-15 and np.allclose(w, w[::-1])
        ref = signal.convolve2d(x, np.outer(w, w), mode="same", boundary="fill")
        assert np.abs(A.blur(x, w) - ref).max() < 1e-13


def test_blur_is_self_adjoint_and_nonexpansive():
    rng = np.random.default_rng(1)
    w = A.gaussian_kernel(1.2)
    x, y = rng.normal(size=(2, 20, 11))
    assert abs((A.blur(x, w) * y).sum() - (x * A.blur(y, w)).sum()) < 1e-12
    assert np.sqrt((A.blur(x, w) ** 2).sum()) <= np.sqrt((x ** 2).sum())


def test_grad_adjoint_and_tv_closed_form():
    rng = np.random.default_rng(2)
    z = rng.normal(size=(9, 14))
    p1, p2 = rng.normal(size=(2, 9, 14))
    p1[-1, :] = 0.0   # entries D never produces
    p2[:, -1] = 0.0
    d1, d2 = A.grad(z)
    assert abs((d1 * p1 + d2 * p2).sum() - (z * A.grad_adj(p1, p2)).sum()) < 1e-12
    # a step of height h across a vertical edge of n rows: TV = h n; a ramp
    # along the rows: (W - 1) |slope| per row
    s = np.zeros((7, 10))
    s[:, 4:] = 2.5
    assert A.tv(s) == pytest.approx(2.5 * 7, abs=1e-12)
    r = np.tile(np.arange(10.0) * -0.75, (3, 1))
    assert A.tv(r) == pytest.approx(3 * 9 * 0.75, abs=1e-12)


@pytest.mark.parametrize("f1,f2,rho", [(3.0, 0.0, 1.0), (0.4, 0.0, 2.0), (-1.0, 2.5, 0.5)])
def test_tv_prox_two_pixels_closed_form(f1, f2, rho):
    # argmin |z1 - z2| + rho/2 ((z1 - f1)^2 + (z2 - f2)^2): the pair meets at
    # the mean when |f1 - f2| <= 2 / rho, else each moves 1/rho toward the other
    f = np.array([[f1, f2]])
    z, _, _ = A.tv_prox(f, rho, 4000)
    if abs(f1 - f2) <= 2.0 / rho:
        want = np.array([[(f1 + f2) / 2] * 2])
    else:
        s = np.sign(f1 - f2)
        want = np.array([[f1 - s / rho, f2 + s / rho]])
    assert np.abs(z - want).max() < 1e-9


def test_tv_prox_optimality_certificate():
    # rho (f - z) = D^T p with |p| <= 1 and p = sign(D z) where D z != 0
    rng = np.random.default_rng(3)
    f = rng.normal(size=(8, 9)) + np.where(np.arange(9) > 4, 2.0, 0.0)
    rho = 1.5
    z, p1, p2 = A.tv_prox(f, rho, 20000)
    assert np.abs(rho * (f - z) - A.grad_adj(p1, p2)).max() < 1e-12
    assert np.abs(p1).max() <= 1.0 and np.abs(p2).max() <= 1.0
    d1, d2 = A.grad(z)
    for d, p in ((d1, p1), (d2, p2)):
        big = np.abs(d) > 1e-6
        assert np.all(np.abs(p[big] - np.sign(d[big])) < 1e-6)
    # a constant image is its own prox
    c = np.full((5, 6), 3.25)
    assert np.abs(A.tv_prox(c, rho, 10)[0] - c).max() == 0.0


def _operators(H, W, w):
    n = H * W
    Am = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        Am[:, k] = A.blur(e.reshape(H, W), w).ravel()
    idx = np.arange(n).reshape(H, W)
    pairs = [(idx[i + 1, j], idx[i, j]) for i in range(H - 1) for j in range(W)]
    pairs += [(idx[i, j + 1], idx[i, j]) for i in range(H) for j in range(W - 1)]
    Dm = np.zeros((len(pairs), n))
    for k, (a, b) in enumerate(pairs):
        Dm[k, a], Dm[k, b] = 1.0, -1.0
    return Am, Dm, idx


def test_admm_reaches_the_lp_optimum_box_constraint():
    # sides {1}: the constraint is a box |I - A x|_i <= sqrt(c_1), so
    # min TV(x) is a linear program; its optimum value is unique
    rng = np.random.default_rng(1)
    H, W, sigma = 10, 12, 0.6
    truth = np.zeros((H, W))
    truth[3:7, 4:9] = 5.0
    w = A.gaussian_kernel(sigma)
    I = A.blur(truth, w) + rng.normal(size=(H, W))
    sides = [1]
    cS = oracle.bounds(sides, 0.9)
    Am, Dm, _ = _operators(H, W, w)
    n, m = Am.shape[0], Dm.shape[0]
    s = np.sqrt(cS[0])
    Z = np.zeros((n, m))
    lp = optimize.linprog(np.r_[np.zeros(n), np.ones(m)],
                          A_ub=np.block([[Dm, -np.eye(m)], [-Dm, -np.eye(m)], [Am, Z], [-Am, Z]]),
                          b_ub=np.r_[np.zeros(2 * m), I.ravel() + s, s - I.ravel()],
                          bounds=[(None, None)] * n + [(0, None)] * m, method="highs")
    assert lp.status == 0
    r = A.admm(I, sides, cS, sigma=sigma, rho1=1.0, rho2=1.0, tv_iters=30, max_iters=4000,
               delta=1e-10, dyk_cycles=2)
    assert A.tv(r.x) == pytest.approx(lp.fun, rel=2e-7)
    assert oracle.max_violation(I - A.blur(r.x, w), sides, cS) < 1e-6
    assert np.abs(r.x - r.z).max() < 1e-6


def test_admm_reaches_the_sqp_optimum_windows():
    # sides {1, 2}: quadratic window constraints; the optimum value of
    # min sum t s.t. -t <= D x <= t, sum_S (I - A x)^2 <= c_S from SLSQP
    rng = np.random.default_rng(2)
    H, W, sigma = 6, 7, 0.6
    truth = np.zeros((H, W))
    truth[2:5, 2:5] = 4.0
    w = A.gaussian_kernel(sigma)
    I = A.blur(truth, w) + rng.normal(size=(H, W))
    sides = [1, 2]
    cS = oracle.bounds(sides, 0.9)
    Am, Dm, idx = _operators(H, W, w)
    n, m = Am.shape[0], Dm.shape[0]
    wins = [(idx[i:i + L, j:j + L].ravel(), c) for L, c in zip(sides, cS)
            for i in range(H - L + 1) for j in range(W - L + 1)]

    def quad(v):
        e = I.ravel() - Am @ v[:n]
        return np.array([c - np.sum(e[s] ** 2) for s, c in wins])

    def quad_jac(v):
        e = I.ravel() - Am @ v[:n]
        J = np.zeros((len(wins), n + m))
        for k, (s, _) in enumerate(wins):
            g = np.zeros(n)
            g[s] = 2.0 * e[s]
            J[k, :n] = g @ Am
        return J

    Lin = np.block([[-Dm, np.eye(m)], [Dm, np.eye(m)]])
    v0 = np.r_[truth.ravel(), np.abs(Dm @ truth.ravel()) + 0.1]
    sqp = optimize.minimize(lambda v: v[n:].sum(), v0, jac=lambda v: np.r_[np.zeros(n), np.ones(m)],
                            constraints=[{"type": "ineq", "fun": lambda v: Lin @ v, "jac": lambda v: Lin},
                                         {"type": "ineq", "fun": quad, "jac": quad_jac}],
                            method="SLSQP", options={"maxiter": 2000, "ftol": 1e-12})
    assert sqp.status == 0
    r = A.admm(I, sides, cS, sigma=sigma, rho1=1.0, rho2=1.0, tv_iters=30, max_iters=3000,
               delta=1e-10, dyk_cycles=100, dyk_tol=1e-12)
    assert A.tv(r.x) == pytest.approx(sqp.fun, rel=1e-7)
    assert oracle.max_violation(I - A.blur(r.x, w), sides, cS) < 1e-6


def test_admm_fixed_point_conditions():
    # at convergence: A^T Y1 = Y2 (x-step stationary), x = z, I = A x + eps,
    # eps = P_G(eps + Y1 / rho1) (Y1 in the normal cone of the set at eps)
    rng = np.random.default_rng(4)
    H, W, sigma = 8, 9, 0.6
    w = A.gaussian_kernel(sigma)
    I = A.blur(np.where(rng.random((H, W)) < 0.2, 5.0, 0.0), w) + rng.normal(size=(H, W))
    sides = [1, 2]
    cS = oracle.bounds(sides, 0.9)
    rho = 1.0
    r = A.admm(I, sides, cS, sigma=sigma, rho1=rho, rho2=rho, tv_iters=30, max_iters=3000,
               delta=1e-11, dyk_cycles=200, dyk_tol=1e-13)
    assert np.abs(A.blur(r.Y1, w) - r.Y2).max() < 1e-6
    assert np.abs(r.x - r.z).max() < 1e-7
    assert np.abs(I - A.blur(r.x, w) - r.eps).max() < 1e-7
    back = oracle.dykstra(r.eps + r.Y1 / rho, sides, cS, max_cycles=2000, tol=1e-14).x
    assert np.abs(back - r.eps).max() < 1e-6
