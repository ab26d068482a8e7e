"""Pins of the oracle's L-BFGS: the two-loop recursion equals the textbook
dense BFGS inverse-Hessian update on the same pairs, and the method solves
a quadratic."""
import numpy as np

from oracle import lbfgs as L


def _dense_h(pairs, gamma, n):
    # H_{k+1} = (I - rho s y^T) H_k (I - rho y s^T) + rho s s^T  (Nocedal & Wright Eq. 6.17)
    h = gamma * np.eye(n)
    for s, y in pairs:
        rho = 1.0 / (s @ y)
        v = np.eye(n) - rho * np.outer(y, s)
        h = v.T @ h @ v + rho * np.outer(s, s)
    return h


def test_two_loop_equals_dense_bfgs():
    rng = np.random.default_rng(0)
    n = 40
    a = rng.standard_normal((n, n))
    a = a @ a.T + n * np.eye(n)
    opt = L.LBFGS(m=6)
    pairs = []
    for _ in range(9):
        s = rng.standard_normal(n)
        y = a @ s
        assert opt.push(s, y)
        pairs.append((s, y))
    kept = pairs[-6:]
    g = rng.standard_normal(n)
    gamma = kept[-1][0] @ kept[-1][1] / (kept[-1][1] @ kept[-1][1])
    np.testing.assert_allclose(opt.direction(g), -_dense_h(kept, gamma, n) @ g, rtol=1e-12, atol=1e-12)


def test_curvature_rule_and_reset():
    opt = L.LBFGS(m=3)
    assert not opt.push(np.array([1.0, 0.0]), np.array([-1.0, 0.0]))   # s.y < 0
    d, gd, pushed = opt.step(np.zeros(2), np.array([1.0, 2.0]))
    np.testing.assert_allclose(d, [-1.0, -2.0])
    assert gd == -5.0 and not pushed


def test_lbfgs_with_line_search_solves_quadratic():
    rng = np.random.default_rng(1)
    n = 30
    a = rng.standard_normal((n, n))
    a = a @ a.T / n + np.eye(n)
    b = rng.standard_normal(n)
    f = lambda x: 0.5 * x @ a @ x - b @ x
    grad = lambda x: a @ x - b
    x = np.zeros(n)
    opt = L.LBFGS(m=10)
    fx = f(x)
    for _ in range(100):
        d, gd, _ = opt.step(x, grad(x))
        res = L.line_search(f, x, fx, d, gd, lambda z, t: z, eps_max=10.0)
        x, fx = res[0], res[1]
        if np.linalg.norm(grad(x)) < 1e-10:
            break
    np.testing.assert_allclose(x, np.linalg.solve(a, b), atol=1e-8)
