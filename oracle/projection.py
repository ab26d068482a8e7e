"""Projection operator P and rank-order matching R (Sec. 2.3.1, Sec. 2.3.2).

Oracle (test infrastructure only).  FP64.

Random draws: the N(0,1) values that replace extreme modes in P are drawn
from a counter-based generator so that any implementation reproduces them:
  state0 = splitmix64 output for seed (see ``_stream_key``),
  h(i, j) = the (2 i + j + 1)-th output of the SplitMix64 generator started
            from state0 (Steele, Lea & Flood 2014; output function of Vigna's
            reference splitmix64), j in {0, 1},
  u1 = ((h(i,0) >> 11) + 1) 2^-53 in (0, 1],  u2 = (h(i,1) >> 11) 2^-53,
  z  = sqrt(-2 ln u1) cos(2 pi u2)           (Box & Muller 1958).
The rank-order-matching targets are supplied by the caller (already sorted
in descending order), as the paper's step 2 draws them at random.
"""
import numpy as np

from . import mesh as M

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    """SplitMix64 output function (xor-shift-multiply finaliser)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _stream_key(seed, counter):
    """Initial SplitMix64 state for one (seed, counter) pair: the first
    output of a SplitMix64 generator seeded with seed + counter * golden."""
    with np.errstate(over="ignore"):
        st = np.uint64(seed) + np.uint64(counter) * _GOLDEN
        return _mix(st + _GOLDEN)


def counter_normals(index, seed, counter):
    """N(0,1) draw for each flat element index (uint64 array)."""
    key = _stream_key(seed, counter)
    index = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        h0 = _mix(key + (np.uint64(2) * index + np.uint64(1)) * _GOLDEN)
        h1 = _mix(key + (np.uint64(2) * index + np.uint64(2)) * _GOLDEN)
    u1 = ((h0 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (h1 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def project(s, seed, counter, s_th=10.0):
    """P(s): z-score normalisation then reset of |s_hat| > s_th to fresh
    N(0,1) draws (Sec. 2.3.1, Eq. z-score and the reset rule).  Population
    standard deviation (ddof = 0); no renormalisation after the reset.
    Returns (projected array, number of reset elements)."""
    x = np.asarray(s, dtype=np.float64).reshape(-1)
    mu = np.mean(x)
    sd = np.sqrt(np.mean((x - mu) ** 2))
    z = (x - mu) / sd
    bad = np.abs(z) > s_th
    if np.any(bad):
        idx = np.nonzero(bad)[0].astype(np.uint64)
        z[bad] = counter_normals(idx, seed, counter)
    return z.reshape(np.shape(s)), int(np.count_nonzero(bad))


def rank_order_match(x, targets_desc):
    """R[x] (Sec. 2.3.2, steps 1-3): pi_i = descending rank of x_i (ties: the
    lower index ranks first), output x~_i = x'_{pi_i} with x' sorted in
    descending order."""
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(targets_desc, dtype=np.float64)
    if t.shape != x.shape:
        raise ValueError("targets must match the input length")
    order = np.argsort(-x, kind="stable")
    out = np.empty_like(x)
    out[order] = t
    return out


def rom_real(s, resp, targets_desc):
    """Real-space matching over the cells with R(q) > 0, in flat index order
    (Sec. 2.3.2: applied to the region with tracers)."""
    out = np.asarray(s, dtype=np.float64).copy().reshape(-1)
    sel = np.asarray(resp).reshape(-1) > 0
    out[sel] = rank_order_match(out[sel], targets_desc)
    return out.reshape(np.shape(s))


def rom_real_ranks(s, resp):
    """pi_i of Sec. 2.3.2 step 1 for real-space matching: each cell's
    descending rank among the cells with R(q) > 0 (0 = largest; ties: the
    lower flat index first), -1 for the cells outside that region."""
    x = np.asarray(s, dtype=np.float64).reshape(-1)
    sel = np.nonzero(np.asarray(resp).reshape(-1) > 0)[0]
    order = np.argsort(-x[sel], kind="stable")
    rank = np.full(x.size, -1, dtype=np.int64)
    rank[sel[order]] = np.arange(sel.size)
    return rank.reshape(np.shape(s))


N_BINS = 100
K_MIN = 0.1


def fourier_modes(n, box, n_bins=N_BINS, k_min=K_MIN):
    """Selection of the half-spectrum modes that Fourier matching touches.

    Returns (flat indices of the selected modes in increasing order, their
    bin, flat indices of their Hermitian partners on the kz=0 / kz=N/2
    planes (or -1)).  A mode is selected when it is the canonical member of
    its conjugate pair (kz in (0, N/2), or on a self-conjugate plane with a
    smaller flat index than its partner), is not its own conjugate, and has
    |k| >= k_min.  Bins: n_bins equal-width |k| bins over [0, sqrt(3) k_Nyq]
    (Sec. 2.3.2: 100 bins of equal size, k < 0.1 h/cMpc left unchanged)."""
    h = n // 2 + 1
    ix, iy, iz = np.meshgrid(np.arange(n), np.arange(n), np.arange(h), indexing="ij")
    flat = (ix * n + iy) * h + iz
    px, py = (-ix) % n, (-iy) % n
    partner = (px * n + py) * h + iz
    plane = (iz == 0) | (iz == n // 2)
    canonical = np.where(plane, flat < partner, True)
    kmag = np.sqrt(M.k_squared(n, box))
    # floor(|k| / (sqrt(3) k_Nyq) * n_bins) with |k| = 2 pi |m| / L for the
    # integer mode vector m: the largest b with 3 n^2 b^2 <= 4 n_bins^2 |m|^2,
    # evaluated in integers so that modes exactly on a bin edge are binned
    # without rounding
    mx = np.where(ix < n // 2, ix, ix - n).astype(np.int64)
    my = np.where(iy < n // 2, iy, iy - n).astype(np.int64)
    m2 = mx * mx + my * my + iz.astype(np.int64) ** 2
    lhs = 4 * n_bins * n_bins * m2
    c = 3 * n * n
    binid = np.floor(np.sqrt(lhs / c)).astype(np.int64)
    binid = np.where(c * binid * binid > lhs, binid - 1, binid)
    binid = np.where(c * (binid + 1) ** 2 <= lhs, binid + 1, binid)
    binid = np.minimum(binid, n_bins - 1)
    sel = canonical & (kmag >= k_min)
    idx = flat[sel]
    order = np.argsort(idx)
    part = np.where(plane, partner, -1)[sel]
    return idx[order], binid[sel][order], part[order]


def fourier_bin_counts(n, box, n_bins=N_BINS, k_min=K_MIN):
    """Number of matched real values (2 per selected mode) in each bin."""
    _, b, _ = fourier_modes(n, box, n_bins, k_min)
    return 2 * np.bincount(b, minlength=n_bins)


def rom_fourier(s, box, targets_desc_concat, n_bins=N_BINS, k_min=K_MIN):
    """Fourier-space matching: z = sqrt(2/N^3) s(k) on the selected modes,
    Re and Im pooled per bin (element order: modes in increasing flat index,
    Re before Im), matched to the caller's N(0,1) targets (concatenated per
    bin, each bin sorted descending), written back with Hermitian symmetry,
    then back to real space."""
    s = np.asarray(s, dtype=np.float64)
    n = s.shape[0]
    sk = M.rfft3(s).reshape(-1)
    idx, b, part = fourier_modes(n, box, n_bins, k_min)
    scale = np.sqrt(2.0 / n ** 3)
    vals = np.empty(2 * idx.size)
    vals[0::2] = sk[idx].real * scale
    vals[1::2] = sk[idx].imag * scale
    ebin = np.repeat(b, 2)
    counts = np.bincount(ebin, minlength=n_bins)
    t = np.asarray(targets_desc_concat, dtype=np.float64)
    if t.size != vals.size:
        raise ValueError("targets length must equal the matched value count")
    offs = np.concatenate([[0], np.cumsum(counts)])
    out = vals.copy()
    for bb in range(n_bins):
        m = np.nonzero(ebin == bb)[0]
        if m.size:
            out[m] = rank_order_match(vals[m], t[offs[bb]:offs[bb + 1]])
    newk = (out[0::2] + 1j * out[1::2]) / scale
    sk[idx] = newk
    has = part >= 0
    sk[part[has]] = np.conj(newk[has])
    return M.irfft3(sk.reshape(n, n, n // 2 + 1), n)


def project_rank_match(s, box, resp, mode, targets_real=None, targets_fourier=None,
                       seed=0, counter=0, s_th=10.0):
    """Composite operator in the order Fourier matching -> real-space matching
    -> projection (each step only when its bit is set: 1 project, 2 Fourier,
    4 real)."""
    out = np.asarray(s, dtype=np.float64)
    if mode & 2:
        out = rom_fourier(out, box, targets_fourier)
    if mode & 4:
        out = rom_real(out, resp, targets_real)
    nreset = 0
    if mode & 1:
        out, nreset = project(out, seed, counter, s_th)
    return out, nreset
