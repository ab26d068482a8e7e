"""Power spectrum and cross-correlation estimators (Sec. 3.2, Eq. r_c).

Oracle (test infrastructure only).  FP64.

P(k) = (V / N^6) <|delta(k)|^2> over shells of |k|; the half spectrum counts
modes with 0 < kz < N/2 twice (their conjugates are implicit).
r_c(k) = P_rt / sqrt(P_rr P_tt).
"""
import numpy as np

from . import mesh as M


def _mode_weights(n):
    w = np.full(n // 2 + 1, 2.0)
    w[0] = 1.0
    w[-1] = 1.0
    return np.broadcast_to(w[None, None, :], (n, n, n // 2 + 1))


def power_spectrum(a, box, edges, b=None):
    """Shell-averaged (cross) power; returns (k_mean, P, n_modes)."""
    n = a.shape[0]
    ak = M.rfft3(a)
    bk = ak if b is None else M.rfft3(b)
    prod = (ak * np.conj(bk)).real * box ** 3 / n ** 6
    kmag = np.sqrt(M.k_squared(n, box))
    w = _mode_weights(n)
    which = np.digitize(kmag.reshape(-1), edges) - 1
    ok = (which >= 0) & (which < len(edges) - 1)
    nb = len(edges) - 1
    wsum = np.bincount(which[ok], weights=w.reshape(-1)[ok], minlength=nb)
    psum = np.bincount(which[ok], weights=(w * prod).reshape(-1)[ok], minlength=nb)
    ksum = np.bincount(which[ok], weights=(w * kmag).reshape(-1)[ok], minlength=nb)
    with np.errstate(invalid="ignore", divide="ignore"):
        return ksum / wsum, psum / wsum, wsum


def cross_correlation(a, b, box, edges):
    """r_c(k) = P_ab / sqrt(P_aa P_bb)."""
    k, pab, nm = power_spectrum(a, box, edges, b)
    _, paa, _ = power_spectrum(a, box, edges)
    _, pbb, _ = power_spectrum(b, box, edges)
    with np.errstate(invalid="ignore", divide="ignore"):
        return k, pab / np.sqrt(paa * pbb), nm
