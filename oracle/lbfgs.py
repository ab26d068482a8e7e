"""L-BFGS two-loop recursion and the projected backtracking line search.

Oracle (test infrastructure only).  FP64.

Sec. 2.3.1: L-BFGS supplies a direction; the line search evaluates
s' = P(s + eps p_hat) along the unit direction p_hat instead of s + eps p_hat.
Readings (the paper leaves them open): memory m = 10; H0 = gamma I with
gamma = s^T y / y^T y of the newest pair (1 with no pairs); a pair is stored
only if s^T y > 1e-10 |s| |y|; if g^T d >= 0 the history is cleared and
d = -g.  Line search: eps_0 = min(|d|, eps_max), Armijo sufficient decrease
f(s') <= f0 + c1 eps g^T p_hat with c1 = 1e-4, halving up to 30 times
(eps_max is the "max step size" of Appendix B Table 1).
"""
import numpy as np


class LBFGS:
    def __init__(self, m=10):
        self.m = m
        self.s = []
        self.y = []
        self.x_prev = None
        self.g_prev = None

    def reset(self):
        self.s, self.y = [], []

    def push(self, sv, yv):
        sy = float(np.dot(sv, yv))
        if sy > 1e-10 * np.linalg.norm(sv) * np.linalg.norm(yv):
            self.s.append(sv.copy())
            self.y.append(yv.copy())
            if len(self.s) > self.m:
                self.s.pop(0)
                self.y.pop(0)
            return True
        return False

    def direction(self, g):
        """d = -H g by the two-loop recursion (Nocedal & Wright Alg. 7.4)."""
        q = np.array(g, dtype=np.float64)
        k = len(self.s)
        alpha = np.zeros(k)
        rho = [1.0 / float(np.dot(self.s[i], self.y[i])) for i in range(k)]
        for i in range(k - 1, -1, -1):
            alpha[i] = rho[i] * float(np.dot(self.s[i], q))
            q -= alpha[i] * self.y[i]
        gamma = (float(np.dot(self.s[-1], self.y[-1])) / float(np.dot(self.y[-1], self.y[-1]))
                 if k else 1.0)
        r = gamma * q
        for i in range(k):
            beta = rho[i] * float(np.dot(self.y[i], r))
            r += self.s[i] * (alpha[i] - beta)
        return -r

    def step(self, x_new, g_new):
        """Push (x_new - x_prev, g_new - g_prev) when a previous point exists,
        then return (d, g.d, pushed); clears the history when g.d >= 0."""
        x_new = np.asarray(x_new, dtype=np.float64).reshape(-1)
        g_new = np.asarray(g_new, dtype=np.float64).reshape(-1)
        pushed = False
        if self.x_prev is not None:
            pushed = self.push(x_new - self.x_prev, g_new - self.g_prev)
        self.x_prev, self.g_prev = x_new.copy(), g_new.copy()
        d = self.direction(g_new)
        gd = float(np.dot(g_new, d))
        if gd >= 0.0:
            self.reset()
            d = -g_new
            gd = float(np.dot(g_new, d))
        return d, gd, pushed


def line_search(f, s0, f0, d, gd, project, eps_max=1.0, c1=1e-4, max_halvings=30):
    """Projected backtracking line search along p_hat = d/|d|.

    f(x) -> float; project(x, trial) -> projected point.  Returns
    (accepted point, its value, eps, halvings) or None on failure."""
    dn = float(np.linalg.norm(d))
    p_hat = d / dn
    slope = gd / dn
    eps = min(dn, eps_max)
    for t in range(max_halvings + 1):
        trial = project(s0 + eps * p_hat, t)
        ft = f(trial)
        if np.isfinite(ft) and ft <= f0 + c1 * eps * slope:
            return trial, ft, eps, t
        eps *= 0.5
    return None
