"""Analysis of reconstructed fields (Sec. 3.2, Eq. for r_c; Sec. 3.3, the
T-web): binned auto and cross power spectra, the correlation coefficient
r_c(k), Gaussian smoothing, the deformation-tensor (T-web) classification
with its eigenvectors, eigenvector cosine similarity and the confusion matrix
of two classifications.

Oracle (test infrastructure only).  FP64, single-threaded numpy.

Readings (the paper gives no binning, normalisation or derivative details):
  * DFT X(k) = sum_x x e^{-ikx} over all n^3 modes; P(k) = (V / n^6) sum |X|^2
    over the modes of a bin divided by their number (cross: Re(A conj B)),
    V = box^3; a mode of integer wave vector m, |k| = kf sqrt(m.m), falls in
    bin floor((|k| - k_min) / dk) when that lies in [0, n_bins);
  * r_c = P_ab / sqrt(P_aa P_bb) per bin;
  * smoothing multiplies by exp(-|k|^2 R^2 / 2), |k|^2 = kf^2 m.m;
  * psi_ij(k) = k_i k_j / |k|^2 G(k) delta(k) with k_i = 0 at axis i's
    Nyquist index (the spectral derivative convention of the forward model)
    and psi_ij(0) = 0; eigenvalues in increasing order
    lambda_1 <= lambda_2 <= lambda_3; the label is the number of eigenvalues
    above lambda_th: 0 void, 1 sheet, 2 filament, 3 knot;
  * cos theta_i = |e_i,a . e_i,b| per cell.
"""
import numpy as np


def _m(n):
    return np.fft.fftfreq(n, 1.0 / n).astype(np.int64)


def _grid_m(n):
    m = _m(n)
    return np.meshgrid(m, m, m, indexing="ij")


def power_spectra(a, b, box, n_bins, k_min, k_max):
    """(P_aa, P_bb, P_ab, counts) per bin; b may be None (then P_bb = P_ab = 0)."""
    a = np.asarray(a, np.float64)
    n = a.shape[0]
    kf = 2 * np.pi / box
    dk = (k_max - k_min) / n_bins
    mx, my, mz = _grid_m(n)
    n2 = (mx * mx + my * my + mz * mz).astype(np.float64)
    k = kf * np.sqrt(n2)
    idx = np.floor((k - k_min) / dk).astype(np.int64).ravel()
    ok = (idx >= 0) & (idx < n_bins)
    A = np.fft.fftn(a).ravel()
    B = np.fft.fftn(np.asarray(b, np.float64)).ravel() if b is not None else np.zeros_like(A)
    cnt = np.bincount(idx[ok], minlength=n_bins).astype(np.float64)
    norm = box ** 3 / float(n) ** 6
    paa = np.bincount(idx[ok], np.abs(A[ok]) ** 2, n_bins) * norm
    pbb = np.bincount(idx[ok], np.abs(B[ok]) ** 2, n_bins) * norm
    pab = np.bincount(idx[ok], (A[ok] * np.conj(B[ok])).real, n_bins) * norm
    with np.errstate(invalid="ignore", divide="ignore"):
        return paa / cnt, pbb / cnt, pab / cnt, cnt


def correlation_coefficient(paa, pbb, pab):
    return pab / np.sqrt(paa * pbb)


def smooth(x, box, r_sm):
    x = np.asarray(x, np.float64)
    n = x.shape[0]
    kf = 2 * np.pi / box
    mx, my, mz = _grid_m(n)
    k2 = kf * kf * (mx * mx + my * my + mz * mz)
    return np.fft.ifftn(np.fft.fftn(x) * np.exp(-0.5 * k2 * r_sm * r_sm)).real


def deformation_tensor(delta, box, r_sm):
    """psi_ij for (i, j) in (00, 11, 22, 01, 02, 12), each [n, n, n]."""
    delta = np.asarray(delta, np.float64)
    n = delta.shape[0]
    kf = 2 * np.pi / box
    mg = _grid_m(n)
    n2 = sum(m * m for m in mg)
    k2 = kf * kf * n2
    ki = [np.where(m == -(n // 2), 0.0, kf * m) for m in mg]   # k_i = 0 at the Nyquist index
    with np.errstate(invalid="ignore", divide="ignore"):
        base = np.where(n2 > 0, np.exp(-0.5 * k2 * r_sm * r_sm) / k2, 0.0) * np.fft.fftn(delta)
    pairs = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
    return [np.fft.ifftn(ki[i] * ki[j] * base).real for i, j in pairs]


def tweb(delta, box, r_sm, lambda_th):
    """(labels [n^3] int, eigenvalues [n^3, 3] increasing, eigenvectors
    [n^3, 3 (component), 3 (which)]) of the smoothed deformation tensor."""
    p = deformation_tensor(delta, box, r_sm)
    m = np.empty(p[0].shape + (3, 3))
    m[..., 0, 0], m[..., 1, 1], m[..., 2, 2] = p[0], p[1], p[2]
    m[..., 0, 1] = m[..., 1, 0] = p[3]
    m[..., 0, 2] = m[..., 2, 0] = p[4]
    m[..., 1, 2] = m[..., 2, 1] = p[5]
    lam, vec = np.linalg.eigh(m.reshape(-1, 3, 3))
    labels = np.sum(lam > lambda_th, axis=1)
    return labels, lam, vec


def eigvec_cosines(va, vb):
    """|cos theta_i| = |e_i,a . e_i,b| for i = 1, 2, 3 (columns of va, vb)."""
    return np.abs(np.sum(va * vb, axis=1))


def confusion(labels_truth, labels_rec, mask):
    """4 x 4 counts: row = truth label, column = reconstructed label, over mask."""
    out = np.zeros((4, 4), np.int64)
    t = np.asarray(labels_truth).ravel()[np.asarray(mask).ravel()]
    r = np.asarray(labels_rec).ravel()[np.asarray(mask).ravel()]
    np.add.at(out, (t, r), 1)
    return out
