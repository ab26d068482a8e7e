"""Annealing: the low-resolution reconstruction feeding the full-resolution
start (Sec. 3, opening: a first run at a coarser cell size whose result is
the initial condition of the full-resolution run).

Oracle (test infrastructure only).  FP64, single-threaded numpy.

The paper does not say how the coarse field becomes a fine one.  Reading:
the white noise s defines the linear density delta_L(k) = s(k) sqrt(P/Delta^3)
(Sec. 2.2.1 item 1), so the fine field keeps the coarse field's linear density
on every mode the coarse mesh resolves unambiguously (all |n_i| < n_c / 2; the
coarse Nyquist planes are shared by +-k and are left out) and is fresh unit
white noise on the others.  With r = n / n_c and Delta_f = Delta_c / r, the
unnormalised DFTs relate as s_f(k) = r^{3/2} s_c(k).

The coarse data are the fine counts summed over each r^3 block and the coarse
survey response the block mean of R.
"""
import numpy as np


def _signed(n):
    """Integer wave numbers of an n-point DFT, in numpy's index order."""
    return np.fft.fftfreq(n, 1.0 / n).astype(np.int64)


def refine_noise(s_coarse, fresh):
    """Fine white noise keeping the coarse field's modes (see module text)."""
    s_coarse = np.asarray(s_coarse, np.float64)
    fresh = np.asarray(fresh, np.float64)
    nc, n = s_coarse.shape[0], fresh.shape[0]
    r = n // nc
    S = np.fft.fftn(fresh)
    Sc = np.fft.fftn(s_coarse)
    kn = _signed(n)
    inside = np.abs(kn) < nc // 2
    for i in np.nonzero(inside)[0]:
        for j in np.nonzero(inside)[0]:
            for l in np.nonzero(inside)[0]:
                S[i, j, l] = r ** 1.5 * Sc[kn[i] % nc, kn[j] % nc, kn[l] % nc]
    return np.fft.ifftn(S).real


def coarsen(x, factor, mean=False):
    """Sum (or mean) of each factor^3 block of a cubic mesh."""
    x = np.asarray(x, np.float64)
    n = x.shape[0]
    nc = n // factor
    out = x.reshape(nc, factor, nc, factor, nc, factor).sum(axis=(1, 3, 5))
    return out / factor ** 3 if mean else out
