"""Background cosmology, growth factors, leapfrog factors and the linear P(k).

Oracle (test infrastructure only).  FP64 throughout.

Units: comoving lengths in Mpc/h, wavenumbers in h/Mpc, time variable a, and
H0 = 1 so that E(a) = H(a)/H0.  With p the canonical momentum a^3 E dx/da,
the equations of motion of the particle-mesh solver are

    dx/da = p / (a^3 E),     dp/da = F / (a^2 E),     F = -grad(phi),
    lap(phi) = 1.5 Omega_m delta,

which is the system that the FastPM scheme the paper adopts (Sec. 2.2.1
item 2, FastPM of Feng et al. 2016) integrates.
"""
import functools
import warnings

import numpy as np
from scipy import integrate


def efunc(a, omega_m):
    """E(a) = H(a)/H0 for flat LCDM without radiation."""
    a = np.asarray(a, dtype=np.float64)
    return np.sqrt(omega_m * a ** -3 + (1.0 - omega_m))


def omega_m_of_a(a, omega_m):
    """Matter density parameter at scale factor a."""
    return omega_m * a ** -3 / efunc(a, omega_m) ** 2


def _growth_rhs(tau, y, omega_m):
    """Right-hand side in tau = ln a for y = (D1, dD1/dtau, D2, dD2/dtau).

    Linear growth:        D1'' + (2 - 1.5 Om(a)) D1' = 1.5 Om(a) D1
    Second order (2LPT):  D2'' + (2 - 1.5 Om(a)) D2' = 1.5 Om(a) (D2 - D1^2)
    (primes are d/dtau; these are the a-space equations
    D'' + (3/a + E'/E) D' = 1.5 Om / (a^5 E^2) (D [- D1^2]) rewritten in ln a).
    """
    a = np.exp(tau)
    om = omega_m_of_a(a, omega_m)
    d1, u1, d2, u2 = y
    return np.array([
        u1,
        -(2.0 - 1.5 * om) * u1 + 1.5 * om * d1,
        u2,
        -(2.0 - 1.5 * om) * u2 + 1.5 * om * (d2 - d1 * d1),
    ])


def growth(a_out, omega_m, a_start=1e-5, steps_per_efold=1000):
    """Growth factors at the scale factors ``a_out``.

    Classical RK4 in ln a from the Einstein-de Sitter growing mode at
    ``a_start`` (D1 = a, D2 = -3/7 a^2), then normalised so that D1(1) = 1
    with D2 scaled by the square of the same factor.

    Returns a dict of arrays (same shape as ``a_out``):
      D1, D2           growth factors
      dD1, dD2         derivatives d/da
      Gp1 = a^3 E dD1/da,  Gp2 = a^3 E dD2/da   (momentum growth)
    """
    a_out = np.atleast_1d(np.asarray(a_out, dtype=np.float64))
    res = _growth_cached(tuple(float(a) for a in a_out), float(omega_m), float(a_start),
                         int(steps_per_efold))
    return {k: v.copy() for k, v in res.items()}


@functools.lru_cache(maxsize=64)
def _growth_cached(a_tuple, omega_m, a_start, steps_per_efold):
    a_out = np.array(a_tuple, dtype=np.float64)
    pts = np.unique(np.concatenate([a_out, [1.0]]))
    if pts[0] <= a_start:
        raise ValueError("a_out must exceed a_start")
    tau = np.log(a_start)
    y = np.array([a_start, a_start, -3.0 / 7.0 * a_start ** 2, -6.0 / 7.0 * a_start ** 2])
    states = {}
    for a_t in pts:
        t_end = np.log(a_t)
        n = max(1, int(np.ceil((t_end - tau) * steps_per_efold)))
        h = (t_end - tau) / n
        for _ in range(n):
            k1 = _growth_rhs(tau, y, omega_m)
            k2 = _growth_rhs(tau + 0.5 * h, y + 0.5 * h * k1, omega_m)
            k3 = _growth_rhs(tau + 0.5 * h, y + 0.5 * h * k2, omega_m)
            k4 = _growth_rhs(tau + h, y + h * k3, omega_m)
            y = y + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
            tau = tau + h
        tau = t_end
        states[float(a_t)] = y.copy()
    norm = states[1.0][0]
    out = {k: np.empty_like(a_out) for k in ("D1", "D2", "dD1", "dD2", "Gp1", "Gp2")}
    for idx, a in enumerate(a_out):
        d1, u1, d2, u2 = states[float(a)]
        d1, u1 = d1 / norm, u1 / norm
        d2, u2 = d2 / norm ** 2, u2 / norm ** 2
        e = efunc(a, omega_m)
        out["D1"][idx] = d1
        out["D2"][idx] = d2
        out["dD1"][idx] = u1 / a
        out["dD2"][idx] = u2 / a
        out["Gp1"][idx] = a * a * e * u1
        out["Gp2"][idx] = a * a * e * u2
    return out


def leapfrog_schedule(a_init, n_steps, omega_m):
    """Scale factors and kick/drift factors of the FastPM leapfrog.

    Uniform grid a_k = a_init + k da, da = (1 - a_init)/n_steps, midpoints
    a_{k+1/2} = (a_k + a_{k+1})/2 (Sec. 2.2.1 item 2: leapfrog, constant da).
    Factors (FastPM):
      kick  K(a->b; c) = [Gp(b) - Gp(a)] / Gf(c),  Gf = 1.5 Omega_m D1
      drift Dr(a->b; c) = [D1(b) - D1(a)] / Gp(c),  Gp = a^3 E dD1/da
    Step k:  p += F(x_k) K(a_k -> a_{k+1/2}; a_k)
             x += p Dr(a_k -> a_{k+1}; a_{k+1/2})
             p += F(x_{k+1}) K(a_{k+1/2} -> a_{k+1}; a_{k+1})
    Both factors are exact for linear (Zel'dovich) growth.
    Returns dict with arrays a (n+1), ah (n), Ka (n), Kb (n), Dr (n).
    """
    da = (1.0 - a_init) / n_steps
    a = a_init + da * np.arange(n_steps + 1)
    a[-1] = 1.0
    ah = 0.5 * (a[:-1] + a[1:])
    g_a = growth(a, omega_m)
    g_h = growth(ah, omega_m)
    gf_a = 1.5 * omega_m * g_a["D1"]
    ka = (g_h["Gp1"] - g_a["Gp1"][:-1]) / gf_a[:-1]
    kb = (g_a["Gp1"][1:] - g_h["Gp1"]) / gf_a[1:]
    dr = (g_a["D1"][1:] - g_a["D1"][:-1]) / g_h["Gp1"]
    return {"a": a, "ah": ah, "Ka": ka, "Kb": kb, "Dr": dr}


def heath_growth(a, omega_m):
    """Closed-form linear growth of flat LCDM (Heath 1977), D1(1) = 1:
    D1(a) proportional to E(a) * int_0^a da' / (a' E(a'))^3.  Used as a pin."""
    def integral(x):
        val, _ = integrate.quad(lambda t: 1.0 / (t * efunc(t, omega_m)) ** 3, 0.0, x,
                                epsabs=0.0, epsrel=1e-13, limit=200)
        return val
    a = np.atleast_1d(np.asarray(a, dtype=np.float64))
    norm = efunc(1.0, omega_m) * integral(1.0)
    return np.array([efunc(x, omega_m) * integral(x) / norm for x in a])


# --- linear power spectrum (input table) -------------------------------------

def eh98_nowiggle_transfer(k, omega_m, omega_b, h, t_cmb=2.7255):
    """Eisenstein & Hu (1998) zero-baryon-oscillation ("no-wiggle") transfer
    function, k in h/Mpc (their Eqs. 26 and 28-31)."""
    k = np.asarray(k, dtype=np.float64)
    omh2 = omega_m * h * h
    obh2 = omega_b * h * h
    fb = omega_b / omega_m
    theta = t_cmb / 2.7
    s = 44.5 * np.log(9.83 / omh2) / np.sqrt(1.0 + 10.0 * obh2 ** 0.75)   # Mpc
    alpha = 1.0 - 0.328 * np.log(431.0 * omh2) * fb + 0.38 * np.log(22.3 * omh2) * fb * fb
    gamma_eff = omega_m * h * (alpha + (1.0 - alpha) / (1.0 + (0.43 * k * h * s) ** 4))
    q = k * theta * theta / gamma_eff
    l0 = np.log(2.0 * np.e + 1.8 * q)
    c0 = 14.2 + 731.0 / (1.0 + 62.5 * q)
    return l0 / (l0 + c0 * q * q)


def tophat_window(x):
    """Fourier transform of a unit-volume spherical top hat, W(x)=3(sin x - x cos x)/x^3."""
    x = np.asarray(x, dtype=np.float64)
    small = np.abs(x) < 1e-3
    xs = np.where(small, 1.0, x)
    w = 3.0 * (np.sin(xs) - xs * np.cos(xs)) / xs ** 3
    return np.where(small, 1.0 - x * x / 10.0, w)


def sigma_r(pk, r):
    """sigma(R)^2 = (1/2 pi^2) int k^3 P(k) W(kR)^2 dln k  for a callable pk."""
    def integrand(lnk):
        k = np.exp(lnk)
        return k ** 3 * pk(k) * tophat_window(k * r) ** 2
    with warnings.catch_warnings():
        # a tabulated, piecewise-interpolated pk trips quad's roundoff detector
        warnings.simplefilter("ignore", integrate.IntegrationWarning)
        val, _ = integrate.quad(integrand, np.log(1e-7), np.log(1e3), epsabs=0.0,
                                epsrel=1e-10, limit=2000)
    return np.sqrt(val / (2.0 * np.pi ** 2))


def linear_power_table(omega_m=0.25, omega_b=0.045, h=0.73, sigma8=0.9, n_s=1.0,
                       k_min=1e-4, k_max=1e2, n_k=512):
    """No-wiggle LCDM P(k) at z=0, normalised to sigma8 with an 8 Mpc/h top hat.

    Returns (ln k, ln P) on ``n_k`` log-spaced points; the model interpolates
    linearly in (ln k, ln P), clamping outside the table (Sec. 2.2.1 item 1:
    "linear power spectra come from fiducial cosmology")."""
    def shape(k):
        return k ** n_s * eh98_nowiggle_transfer(k, omega_m, omega_b, h) ** 2
    amp = (sigma8 / sigma_r(shape, 8.0)) ** 2
    k = np.logspace(np.log10(k_min), np.log10(k_max), n_k)
    return np.log(k), np.log(amp * shape(k))


def power_from_table(k, lnk_tab, lnp_tab):
    """P(k) by linear interpolation of the table in (ln k, ln P)."""
    k = np.asarray(k, dtype=np.float64)
    safe = np.where(k > 0, k, 1.0)
    return np.where(k > 0, np.exp(np.interp(np.log(safe), lnk_tab, lnp_tab)), 0.0)


C_OVER_H0 = 2997.92458  # speed of light / (100 km/s/Mpc), Mpc/h


def comoving_distance(a, omega_m):
    """chi(a) = (c/H0) int_a^1 da' / (a'^2 E(a')), Mpc/h, flat LCDM (adaptive
    quadrature, one integral per value)."""
    a = np.atleast_1d(np.asarray(a, dtype=np.float64))
    f = lambda x: 1.0 / (x * x * float(efunc(x, omega_m)))
    out = np.array([integrate.quad(f, ai, 1.0, epsabs=0.0, epsrel=1e-13, limit=200)[0] for ai in a])
    return C_OVER_H0 * out


def distance_table(omega_m, a_min=0.5, n=2049):
    """(a_j, chi_j) on a uniform grid of a in [a_min, 1]: the table from which
    the scale factor of a comoving distance is read (DistToScaleFactor of the
    lightcone construction, Appendix A)."""
    a = np.linspace(a_min, 1.0, n)
    return a, comoving_distance(a, omega_m)


def dist_to_scale_factor(d, a_tab, chi_tab):
    """a(d) by linear interpolation of the table (chi decreases with a),
    clamped to the table's ends; and da/dd of the interpolant (0 outside)."""
    d = np.asarray(d, dtype=np.float64)
    x, y = chi_tab[::-1], a_tab[::-1]          # increasing chi
    a = np.interp(d, x, y)
    j = np.clip(np.searchsorted(x, d, side="right") - 1, 0, len(x) - 2)
    slope = (y[j + 1] - y[j]) / (x[j + 1] - x[j])
    slope = np.where((d >= x[0]) & (d <= x[-1]), slope, 0.0)
    return a, slope
