"""The MujicΛ forward model and its hand-derived adjoint (gradient wrt s).

Oracle (test infrastructure only).  FP64, single-threaded numpy.

Forward model (Sec. 2.2.1 items 1-5, Sec. 2.2.2):
  1. white noise s -> delta_L(k) = s(k) sqrt(P(|k|)/Delta^3), DC = 0
     (Sec. 2.2.1 item 1, Eq. for delta_ic: the complex Gaussian modes are
     built from real Gaussian variables s);
  2. 2LPT displacement of the Lagrangian lattice to a_init, then n leapfrog
     kick-drift-kick PM steps with FastPM factors to a = 1 (item 2);
  3. plane-parallel redshift-space shift along one axis (item 3, Eq. RSD with
     the line of sight fixed to a box axis);
  4. galaxy bias f(delta) (item 4): linear, b delta for the Gaussian and the
     rate 1 + b delta (floored) for the Poisson; or the power law + sigmoid
     of Eq. galaxy_bias, nbar g(delta) for the Gaussian and the rate g(delta)
     for the Poisson.  By default ("auto") the Gaussian takes the linear and
     the Poisson the power-law bias, the pairs Sec. 2.2.2 describes;
  5. survey response lambda_obs = R lambda (item 5);
  6. likelihood: Gaussian (1/2) sum R (f(delta) - d)^2 / sigma^2, or the
     Poisson log-likelihood of Sec. 2.2.2 without the constant log N!;
  plus the Gaussian prior (w/2) sum s^2 on the white noise.

The gradient is the reverse-mode chain through every step above, written by
hand: transposes of the spectral operators (conjugate multipliers), the CIC
weight derivative, the reverse of each kick and drift.
"""
from dataclasses import dataclass

import numpy as np

from . import cosmology as cosmo
from . import mesh as M


@dataclass
class Config:
    n: int                      # mesh cells = particles per side
    box: float                  # Mpc/h
    omega_m: float = 0.25
    a_init: float = 0.1
    n_steps: int = 5
    lpt_order: int = 2
    rsd_axis: int = -1          # -1: none, 0..2: plane-parallel shift along that axis, 3: radial
    observer: tuple = (0.0, 0.0, 0.0)   # Mpc/h, box coordinates (radial shift, lightcone)
    lightcone: bool = False     # observe each particle on the observer's past light cone (Appendix A)
    likelihood: str = "gaussian"   # "gaussian" | "poisson"
    bias: str = "auto"             # "auto" (gaussian: linear, poisson: power law) | "linear" | "powerlaw_sigmoid"
    bias_b: float = 1.5
    sigma: float = 1.0
    alpha: float = 0.7
    delta_th: float = 1.2
    K: float = 3.0
    nbar_cell: float = 1.0
    rho_floor: float = 1e-3
    prior_weight: float = 1.0

    @property
    def cell(self):
        return self.box / self.n


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def ic_amplitude(cfg, lnk, lnp):
    """A(k) = sqrt(P(|k|) / Delta^3) on the half spectrum, A(0) = 0."""
    k = np.sqrt(M.k_squared(cfg.n, cfg.box))
    amp = np.sqrt(cosmo.power_from_table(k, lnk, lnp) / cfg.cell ** 3)
    amp[0, 0, 0] = 0.0
    return amp


class _Ops:
    """The spectral multipliers of the model, each defined once; the adjoint
    applies their complex conjugates."""

    def __init__(self, cfg, lnk, lnp):
        n, box = cfg.n, cfg.box
        self.amp = ic_amplitude(cfg, lnk, lnp)
        self.ik2 = M.inv_k2(n, box)
        self.d = [M.deriv(n, box, i) for i in range(3)]
        # Psi1_i = -d_i phi1, lap phi1 = delta_L   ->  D_i / k^2 on delta_L
        self.psi1 = [self.d[i] * self.ik2 * self.amp for i in range(3)]
        # phi1_ij = d_i d_j phi1                   -> -D_i D_j / k^2 on delta_L
        self.pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
        self.phi = {(i, j): -self.d[i] * self.d[j] * self.ik2 * self.amp for (i, j) in self.pairs}
        # Psi2_i = +d_i phi2, lap phi2 = S          -> -D_i / k^2 on S
        self.psi2 = [-self.d[i] * self.ik2 for i in range(3)]
        # PM force F_i = -d_i phi, lap phi = 1.5 Om delta -> 1.5 Om D_i / k^2
        self.force = [1.5 * cfg.omega_m * self.d[i] * self.ik2 for i in range(3)]


def linear_field(s, cfg, lnk, lnp):
    """delta_L in real space (Sec. 2.2.1 item 1)."""
    ops = _Ops(cfg, lnk, lnp)
    return M.irfft3(ops.amp * M.rfft3(s), cfg.n)


def lpt(s, cfg, lnk, lnp, ops=None):
    """2LPT (or Zel'dovich) displacement and momentum at a_init, (M,3) in Mpc/h.

    x = q + D1 Psi1 + D2 Psi2,  p = a^3 E (D1' Psi1 + D2' Psi2),
    S = sum_{i<j} (phi_ii phi_jj - phi_ij^2)  (Sec. 2.2.1 item 2: 2LPT to a=0.1)."""
    ops = ops or _Ops(cfg, lnk, lnp)
    n = cfg.n
    sk = M.rfft3(np.asarray(s, dtype=np.float64))
    psi1 = np.stack([M.irfft3(ops.psi1[i] * sk, n).reshape(-1) for i in range(3)], axis=1)
    g = cosmo.growth([cfg.a_init], cfg.omega_m)
    disp = g["D1"][0] * psi1
    mom = g["Gp1"][0] * psi1
    phi = None
    psi2 = np.zeros_like(psi1)
    if cfg.lpt_order == 2:
        phi = {ij: M.irfft3(ops.phi[ij] * sk, n) for ij in ops.pairs}
        src = (phi[(0, 0)] * phi[(1, 1)] + phi[(0, 0)] * phi[(2, 2)] + phi[(1, 1)] * phi[(2, 2)]
               - phi[(0, 1)] ** 2 - phi[(0, 2)] ** 2 - phi[(1, 2)] ** 2)
        srck = M.rfft3(src)
        psi2 = np.stack([M.irfft3(ops.psi2[i] * srck, n).reshape(-1) for i in range(3)], axis=1)
        disp = disp + g["D2"][0] * psi2
        mom = mom + g["Gp2"][0] * psi2
    return disp, mom, {"psi1": psi1, "psi2": psi2, "phi": phi, "growth": g}


def positions_cells(disp, cfg):
    """u = q/Delta + disp/Delta (cell units)."""
    return M.lattice_cells(cfg.n) + disp / cfg.cell


def force(disp, cfg, ops):
    """PM force on every particle: CIC paint -> delta -> F_i = 1.5 Om D_i/k^2
    delta(k) -> CIC readout.  Returns (F (M,3) in Mpc/h, Phi list of meshes,
    delta mesh)."""
    u = positions_cells(disp, cfg)
    rho = M.cic_paint(u, cfg.n)
    delta = rho - 1.0            # (N_mesh^3 / N_part^3) rho - 1 with N_mesh = N_part
    dk = M.rfft3(delta)
    phi = [M.irfft3(ops.force[i] * dk, cfg.n) for i in range(3)]
    f = np.stack([M.cic_readout(u, phi[i]) for i in range(3)], axis=1)
    return f, phi, delta


def force_vjp(disp, fbar, cfg, ops):
    """Transpose of the Jacobian of ``force`` (wrt disp) applied to fbar.

    F_p,i = sum_c W(u_p - c) Phi_i(c),  Phi_i = G_i rho,  rho = sum_q W(u_q - c):
      (A) readout weights: sum_i fbar_p,i sum_c dW/du (u_p - c) Phi_i(c)
      (B) through rho: rhobar = sum_i G_i^T m_i, m_i = paint of fbar_i,
          then sum_c dW/du (u_p - c) rhobar(c).
    Result in 1/(Mpc/h) units of the cotangent (d/d disp = (1/Delta) d/du)."""
    u = positions_cells(disp, cfg)
    rho = M.cic_paint(u, cfg.n)
    dk = M.rfft3(rho - 1.0)
    phi = [M.irfft3(ops.force[i] * dk, cfg.n) for i in range(3)]
    grad = np.zeros_like(disp)
    for i in range(3):
        grad += fbar[:, i:i + 1] * M.cic_readout_grad(u, phi[i])
    rhobar = np.zeros((cfg.n,) * 3)
    for i in range(3):
        m_i = M.cic_paint(u, cfg.n, weights=fbar[:, i])
        rhobar += M.irfft3(np.conj(ops.force[i]) * M.rfft3(m_i), cfg.n)
    grad += M.cic_readout_grad(u, rhobar)
    return grad / cfg.cell


def evolve(s, cfg, lnk, lnp, keep=False):
    """2LPT + leapfrog KDK to a = 1.  Returns (disp, mom, info); with keep=True
    info["disp_k"] holds the displacement at each of the n+1 force
    evaluations (for the adjoint)."""
    ops = _Ops(cfg, lnk, lnp)
    disp, mom, lpt_info = lpt(s, cfg, lnk, lnp, ops)
    sch = cosmo.leapfrog_schedule(cfg.a_init, cfg.n_steps, cfg.omega_m)
    f, _, _ = force(disp, cfg, ops)
    disp_k = [disp.copy()] if keep else None
    snaps = snapshot_states(cfg) if cfg.lightcone else []
    snap_x, snap_p = [], []
    for k in range(cfg.n_steps):
        mom = mom + sch["Ka"][k] * f
        disp = disp + sch["Dr"][k] * mom
        f, _, _ = force(disp, cfg, ops)
        mom = mom + sch["Kb"][k] * f
        if keep:
            disp_k.append(disp.copy())
        if k + 1 in snaps:   # position and (synchronised) momentum at a snapshot
            snap_x.append(disp.copy())
            snap_p.append(mom.copy())
    return disp, mom, {"ops": ops, "sched": sch, "disp_k": disp_k, "lpt": lpt_info,
                       "snap_x": snap_x, "snap_p": snap_p}


# ---- lightcone (Sec. 2.2.1 item 3, Appendix A) -----------------------------
SNAP_A = (0.8, 0.9, 1.0)   # scale factors of the saved snapshots
LC_ITERATIONS = 3


def snapshot_states(cfg):
    """Indices k of the leapfrog states at the snapshot scale factors; the
    uniform a grid must contain them (e.g. a_init = 0.1 with 9 or 18 steps)."""
    a = cfg.a_init + (1.0 - cfg.a_init) / cfg.n_steps * np.arange(cfg.n_steps + 1)
    out = []
    for sa in SNAP_A:
        k = int(np.argmin(np.abs(a - sa)))
        if abs(a[k] - sa) > 1e-9:
            raise ValueError(f"the leapfrog grid has no state at a = {sa}")
        out.append(k)
    return out


def _interp_snapshots(Y, a):
    """Linear interpolation in a between the bracketing snapshots (a clamped to
    [0.8, 1]); returns (y, per-snapshot weights (3, M), dy/da)."""
    sa = np.asarray(SNAP_A)
    ac = np.clip(a, sa[0], sa[-1])
    j = np.where(ac <= sa[1], 0, 1)
    t = (ac - sa[j]) / (sa[j + 1] - sa[j])
    w = np.zeros((3, a.size))
    idx = np.arange(a.size)
    w[j, idx] += 1.0 - t
    w[j + 1, idx] += t
    y = np.einsum("sm,smc->mc", w, Y)
    inside = ((a >= sa[0]) & (a <= sa[-1]))[:, None]
    dy = np.where(inside, (Y[j + 1, idx] - Y[j, idx]) / (sa[j + 1] - sa[j])[:, None], 0.0)
    return y, w, dy


def _lightcone_forward(X, P, cfg, tab):
    q = M.lattice_cells(cfg.n) * cfg.cell
    o = np.asarray(cfg.observer, np.float64)
    a = np.ones(q.shape[0])
    hist = []
    for _ in range(LC_ITERATIONS):   # a^(n) = DistToScaleFactor(|x(a^(n-1)) - o|), a^(0) = 1
        x, w, dx = _interp_snapshots(X, a)
        r = q + x - o
        d = np.sqrt(np.sum(r * r, axis=1))
        a_new, slope = cosmo.dist_to_scale_factor(d, *tab)
        hist.append((w, dx, r, d, slope))
        a = a_new
    x, wx, dx = _interp_snapshots(X, a)
    p, _, dp = _interp_snapshots(P, a)
    r = q + x - o
    rn = np.sqrt(np.sum(r * r, axis=1))
    u = r / rn[:, None]
    e = cosmo.efunc(a, cfg.omega_m)
    s = 1.0 / (a * a * e)
    pu = np.sum(p * u, axis=1)
    obs = x + (s * pu)[:, None] * u
    return obs, {"a": a, "hist": hist, "wx": wx, "dx": dx, "dp": dp, "p": p, "u": u, "rn": rn, "s": s,
                 "pu": pu, "e": e}


def lightcone_observed(X, P, cfg, tab):
    """Displacement of each particle as observed on the light cone: scale
    factor a_i from three fixed-point iterations of DistToScaleFactor starting
    at a = 1, position and momentum interpolated to a_i between the snapshots,
    then the radial redshift-space shift (p . d) d / (a_i^2 E(a_i))."""
    return _lightcone_forward(np.asarray(X), np.asarray(P), cfg, tab)[0]


def lightcone_vjp(X, P, obsbar, cfg, tab):
    """Transpose of the Jacobian of lightcone_observed wrt the snapshots
    (X, P), applied to the cotangent of the observed displacement."""
    X, P = np.asarray(X), np.asarray(P)
    _, c = _lightcone_forward(X, P, cfg, tab)
    a, u, rn, s, pu, p = c["a"], c["u"], c["rn"], c["s"], c["pu"], c["p"]
    ux = np.sum(u * obsbar, axis=1)
    proj = lambda v: v - u * np.sum(u * v, axis=1)[:, None]
    pbar = (s * ux)[:, None] * u
    xbar = obsbar + (s / rn)[:, None] * (proj(p) * ux[:, None] + pu[:, None] * proj(obsbar))
    # d s / d a with s = 1/(a^2 E), dE/da = -1.5 Omega_m a^-4 / E
    e = c["e"]
    de = -1.5 * cfg.omega_m * a ** -4 / e
    ds = -2.0 / (a ** 3 * e) - de / (a * a * e * e)
    abar = ds * pu * ux + np.sum(xbar * c["dx"], axis=1) + np.sum(pbar * c["dp"], axis=1)
    Xbar = np.einsum("sm,mc->smc", c["wx"], xbar)
    Pbar = np.einsum("sm,mc->smc", c["wx"], pbar)
    for w, dx, r, d, slope in reversed(c["hist"]):
        rbar = (abar * slope / d)[:, None] * r
        Xbar += np.einsum("sm,mc->smc", w, rbar)
        abar = np.sum(rbar * dx, axis=1)
    return Xbar, Pbar



def rsd_coefficient(cfg):
    """Comoving redshift-space shift per unit canonical momentum at a = 1:
    v_pec / (a H) = p / (a^2 E(a)) (Sec. 2.2.1 item 3, Eq. RSD)."""
    a = 1.0
    return 1.0 / (a * a * float(cosmo.efunc(a, cfg.omega_m)))


def _line_of_sight(disp, cfg):
    """Unit vectors d = r/|r| from the observer to each particle, r = q + disp - o
    (unwrapped comoving position, Mpc/h), and |r|."""
    r = M.lattice_cells(cfg.n) * cfg.cell + disp - np.asarray(cfg.observer, np.float64)
    rn = np.sqrt(np.sum(r * r, axis=1))
    return r / rn[:, None], rn


def observed_positions(disp, mom, cfg):
    """Displacement after the RSD shift (Sec. 2.2.1 item 3): along a fixed box
    axis (plane parallel), or along the line of sight from the observer,
    x_s = x + c (p . d) d with d the unit vector from the observer (radial)."""
    out = disp.copy()
    if 0 <= cfg.rsd_axis <= 2:
        out[:, cfg.rsd_axis] += rsd_coefficient(cfg) * mom[:, cfg.rsd_axis]
    elif cfg.rsd_axis == 3:
        d, _ = _line_of_sight(disp, cfg)
        out += rsd_coefficient(cfg) * np.sum(mom * d, axis=1)[:, None] * d
    return out


def observed_positions_vjp(disp, mom, xsbar, cfg):
    """Transpose of the Jacobian of observed_positions applied to the cotangent
    xsbar of the shifted positions: returns (xbar, pbar).  Radial case, with
    P = I - d d^T and dd/dx = P/|r|:
      pbar = c d (d . xsbar),
      xbar = xsbar + (c/|r|) [P p (d . xsbar) + (p . d) P xsbar]."""
    c = rsd_coefficient(cfg)
    xbar = xsbar.copy()
    pbar = np.zeros_like(xsbar)
    if 0 <= cfg.rsd_axis <= 2:
        pbar[:, cfg.rsd_axis] = c * xsbar[:, cfg.rsd_axis]
    elif cfg.rsd_axis == 3:
        d, rn = _line_of_sight(disp, cfg)
        dxs = np.sum(d * xsbar, axis=1)[:, None]
        pd = np.sum(mom * d, axis=1)[:, None]
        proj = lambda v: v - d * np.sum(d * v, axis=1)[:, None]
        pbar = c * d * dxs
        xbar = xsbar + (c / rn)[:, None] * (proj(mom) * dxs + pd * proj(xsbar))
    return xbar, pbar


def final_density(disp_obs, cfg):
    return M.cic_paint(positions_cells(disp_obs, cfg), cfg.n) - 1.0


def bias_kind(cfg):
    """The bias model a configuration uses ("auto" resolves by likelihood)."""
    if cfg.bias == "auto":
        return "linear" if cfg.likelihood == "gaussian" else "powerlaw_sigmoid"
    if cfg.bias not in ("linear", "powerlaw_sigmoid"):
        raise ValueError(cfg.bias)
    return cfg.bias


def _powerlaw_sigmoid(delta, cfg):
    """g = max(1+delta, rho_floor)^alpha sigmoid(K (delta - delta_th))
    (Eq. galaxy_bias without its normalisation, with the floor that keeps the
    power law finite) and its derivative wrt delta (zero below the floor for
    the power-law factor)."""
    base = np.maximum(1.0 + delta, cfg.rho_floor)
    sig = _sigmoid(cfg.K * (delta - cfg.delta_th))
    g = base ** cfg.alpha * sig
    dpow = np.where(1.0 + delta > cfg.rho_floor, cfg.alpha * base ** (cfg.alpha - 1.0), 0.0)
    dg = dpow * sig + base ** cfg.alpha * cfg.K * sig * (1.0 - sig)
    return g, dg


def _linear_rate(delta, cfg):
    """g = max(1 + b delta, rho_floor): the mean galaxy density of the linear
    bias model per unit nbar, floored so that the Poisson rate stays positive
    where b delta < -1; derivative b above the floor, zero below it."""
    base = 1.0 + cfg.bias_b * delta
    g = np.maximum(base, cfg.rho_floor)
    dg = np.where(base > cfg.rho_floor, cfg.bias_b, 0.0)
    return g, dg


def likelihood_terms(delta, data, resp, cfg):
    """(-log L, d(-log L)/d delta) for the configured likelihood (Sec. 2.2.2)
    and bias model."""
    kind = bias_kind(cfg)
    if cfg.likelihood == "gaussian":
        if kind == "linear":
            f, df = cfg.bias_b * delta, cfg.bias_b
        else:
            g, dg = _powerlaw_sigmoid(delta, cfg)
            f, df = cfg.nbar_cell * g, cfg.nbar_cell * dg
        r = f - data
        val = 0.5 * np.sum(resp * r * r) / cfg.sigma ** 2
        grad = resp * df * r / cfg.sigma ** 2
        return val, grad
    if cfg.likelihood == "poisson":
        g, dg = (_linear_rate if kind == "linear" else _powerlaw_sigmoid)(delta, cfg)
        mask = resp > 0
        lam = np.where(mask, resp * cfg.nbar_cell * g, 1.0)
        val = np.sum(np.where(mask, lam - data * np.log(lam), 0.0))
        grad = np.where(mask, resp * cfg.nbar_cell * dg * (1.0 - data / lam), 0.0)
        return val, grad
    raise ValueError(cfg.likelihood)


def model_mean(delta, resp, cfg):
    """Mean of the data per cell, the rate mock data are drawn from: Poisson
    R nbar g(delta) on observed cells (zero elsewhere), Gaussian f(delta)."""
    kind = bias_kind(cfg)
    if cfg.likelihood == "poisson":
        g, _ = (_linear_rate if kind == "linear" else _powerlaw_sigmoid)(delta, cfg)
        return np.where(resp > 0, resp * cfg.nbar_cell * g, 0.0)
    if kind == "linear":
        return cfg.bias_b * delta
    return cfg.nbar_cell * _powerlaw_sigmoid(delta, cfg)[0]


def loss(s, cfg, lnk, lnp, data, resp):
    """Total loss = -log L + (w/2) sum s^2.  Returns (loss, parts dict)."""
    disp, mom, ev = evolve(s, cfg, lnk, lnp)
    if cfg.lightcone:
        obs = lightcone_observed(ev["snap_x"], ev["snap_p"], cfg, cosmo.distance_table(cfg.omega_m))
    else:
        obs = observed_positions(disp, mom, cfg)
    delta = final_density(obs, cfg)
    lik, _ = likelihood_terms(delta, data, resp, cfg)
    prior = 0.5 * cfg.prior_weight * float(np.sum(np.asarray(s, np.float64) ** 2))
    return lik + prior, {"likelihood": lik, "prior": prior, "delta": delta,
                         "disp": disp, "mom": mom}


def gradient(s, cfg, lnk, lnp, data, resp, loss_weight=1.0, cot_delta=None):
    """Value and gradient of loss_weight * loss + <cot_delta, delta_final> wrt s.

    Reverse of the forward model, step by step:
      likelihood -> final paint -> RSD -> for each leapfrog step in reverse:
      second half-kick, drift, first half-kick -> 2LPT -> linear field;
      plus the prior gradient."""
    s = np.asarray(s, dtype=np.float64)
    n = cfg.n
    disp, mom, info = evolve(s, cfg, lnk, lnp, keep=True)
    ops, sch, disp_k = info["ops"], info["sched"], info["disp_k"]
    if cfg.lightcone:
        tab = cosmo.distance_table(cfg.omega_m)
        obs = lightcone_observed(info["snap_x"], info["snap_p"], cfg, tab)
    else:
        obs = observed_positions(disp, mom, cfg)
    delta = final_density(obs, cfg)
    lik, dlik = likelihood_terms(delta, data, resp, cfg)
    prior = 0.5 * cfg.prior_weight * float(np.sum(s * s))
    total = lik + prior

    dbar = loss_weight * dlik
    if cot_delta is not None:
        dbar = dbar + cot_delta
    # final paint: delta = paint(u_obs) - 1
    xsbar = M.cic_readout_grad(positions_cells(obs, cfg), dbar) / cfg.cell
    if cfg.lightcone:
        # the observed field depends on the snapshot states: their cotangents
        # join the reverse sweep at those states
        Xbar, Pbar = lightcone_vjp(info["snap_x"], info["snap_p"], xsbar, cfg, tab)
        snaps = snapshot_states(cfg)
        xbar, pbar = np.zeros_like(xsbar), np.zeros_like(xsbar)
    else:
        xbar, pbar = observed_positions_vjp(disp, mom, xsbar, cfg)
        snaps = []
    # leapfrog steps in reverse
    for k in range(cfg.n_steps - 1, -1, -1):
        if k + 1 in snaps:
            j = snaps.index(k + 1)
            xbar = xbar + Xbar[j]
            pbar = pbar + Pbar[j]
        xbar = xbar + force_vjp(disp_k[k + 1], sch["Kb"][k] * pbar, cfg, ops)
        pbar = pbar + sch["Dr"][k] * xbar
        xbar = xbar + force_vjp(disp_k[k], sch["Ka"][k] * pbar, cfg, ops)
    # 2LPT:  disp = D1 Psi1 + D2 Psi2,  mom = Gp1 Psi1 + Gp2 Psi2
    g = info["lpt"]["growth"]
    psi1bar = g["D1"][0] * xbar + g["Gp1"][0] * pbar
    sbar_k = np.zeros_like(ops.amp, dtype=np.complex128)
    for i in range(3):
        sbar_k += np.conj(ops.psi1[i]) * M.rfft3(psi1bar[:, i].reshape(n, n, n))
    if cfg.lpt_order == 2:
        psi2bar = g["D2"][0] * xbar + g["Gp2"][0] * pbar
        srcbar = np.zeros((n, n, n))
        for i in range(3):
            srcbar += M.irfft3(np.conj(ops.psi2[i]) * M.rfft3(psi2bar[:, i].reshape(n, n, n)), n)
        phi = info["lpt"]["phi"]
        phibar = {
            (0, 0): srcbar * (phi[(1, 1)] + phi[(2, 2)]),
            (1, 1): srcbar * (phi[(0, 0)] + phi[(2, 2)]),
            (2, 2): srcbar * (phi[(0, 0)] + phi[(1, 1)]),
            (0, 1): -2.0 * srcbar * phi[(0, 1)],
            (0, 2): -2.0 * srcbar * phi[(0, 2)],
            (1, 2): -2.0 * srcbar * phi[(1, 2)],
        }
        for ij in ops.pairs:
            sbar_k += np.conj(ops.phi[ij]) * M.rfft3(phibar[ij])
    grad = M.irfft3(sbar_k, n) + loss_weight * cfg.prior_weight * s
    return total, grad, {"likelihood": lik, "prior": prior, "delta": delta,
                         "disp": disp, "mom": mom}
