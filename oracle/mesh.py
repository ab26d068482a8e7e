"""Mesh conventions, spectral operators and cloud-in-cell assignment.

Oracle (test infrastructure only).  FP64, numpy library FFTs.

Conventions
-----------
* Meshes are (N, N, N) arrays in C order, axis 0 = x slowest, axis 2 = z
  fastest; cell / node (i, j, l) sits at (i, j, l) * Delta, Delta = L / N.
* DFT: X(k) = sum_x x e^{-i k.x}; inverse carries 1/N^3 (numpy's rfftn /
  irfftn).  k_n = 2 pi n / L with n in [-N/2, N/2) on the full axes and
  n in [0, N/2] on the halved last axis.
* First-derivative multiplier D_i(k) = i k_i, set to 0 where the i-th index
  is the Nyquist index N/2 (there i k_i has no real-valued counterpart).
  Every multiplier used by the model is Hermitian, h(-k) = conj h(k), so
  irfftn(h * rfftn(f)) is an exact real linear operator whose transpose is
  irfftn(conj(h) * rfftn(.)).
* Particles carry the index of their Lagrangian node: particle p = (i*N+j)*N+l
  starts from q = (i, j, l) * Delta.
"""
import numpy as np


def wavenumbers(n, box):
    """Return (kx, ky, kz) broadcastable to the half-spectrum shape and the
    Nyquist masks (True where that axis is at index N/2)."""
    nfull = np.fft.fftfreq(n, d=1.0 / n)          # 0..N/2-1, -N/2..-1
    nhalf = np.arange(n // 2 + 1, dtype=np.float64)
    kf = 2.0 * np.pi / box * nfull
    kh = 2.0 * np.pi / box * nhalf
    kx = kf[:, None, None]
    ky = kf[None, :, None]
    kz = kh[None, None, :]
    nyq_x = (np.abs(nfull) == n // 2)[:, None, None]
    nyq_y = (np.abs(nfull) == n // 2)[None, :, None]
    nyq_z = (nhalf == n // 2)[None, None, :]
    return (kx, ky, kz), (nyq_x, nyq_y, nyq_z)


def k_squared(n, box):
    (kx, ky, kz), _ = wavenumbers(n, box)
    return kx * kx + ky * ky + kz * kz


def deriv(n, box, axis):
    """First-derivative multiplier D_axis = i k_axis (0 at that axis' Nyquist)."""
    (k, nyq) = wavenumbers(n, box)
    return np.where(nyq[axis], 0.0, 1j * k[axis])


def inv_k2(n, box):
    """1/k^2 with the k = 0 mode set to 0."""
    k2 = k_squared(n, box)
    out = np.zeros_like(k2)
    np.divide(1.0, k2, out=out, where=k2 > 0)
    return out


def rfft3(f):
    return np.fft.rfftn(f)


def irfft3(fk, n):
    return np.fft.irfftn(fk, s=(n, n, n), axes=(0, 1, 2))


def apply_multiplier(f, mult):
    """Real linear operator irfftn(mult * rfftn(f))."""
    return irfft3(mult * rfft3(f), f.shape[0])


# --- cloud in cell -----------------------------------------------------------

def lattice_cells(n):
    """Lagrangian node coordinates of every particle, in cell units, (M, 3)."""
    idx = np.arange(n ** 3, dtype=np.int64)
    i = idx // (n * n)
    j = (idx // n) % n
    l = idx % n
    return np.stack([i, j, l], axis=1).astype(np.float64)


def _corners(u, n):
    """Base node, fractional offsets and 1-D weights of the CIC kernel.

    u: (M, 3) positions in cell units.  The particle at u deposits
    prod_d (1 - |u_d - c_d|) on the 8 nodes c with floor(u_d) <= c_d <=
    floor(u_d)+1 (periodic)."""
    base = np.floor(u)
    frac = u - base
    base = base.astype(np.int64) % n
    return base, frac


def _corner_index(base, n, ox, oy, oz):
    return ((((base[:, 0] + ox) % n) * n + (base[:, 1] + oy) % n) * n
            + (base[:, 2] + oz) % n)


def cic_paint(u, n, weights=None):
    """rho(c) = sum_p w_p W(u_p - c), summed with np.bincount in particle
    order (deterministic).  Returns an (n, n, n) mesh."""
    base, frac = _corners(u, n)
    out = np.zeros(n ** 3)
    for ox in (0, 1):
        wx = frac[:, 0] if ox else 1.0 - frac[:, 0]
        for oy in (0, 1):
            wy = frac[:, 1] if oy else 1.0 - frac[:, 1]
            for oz in (0, 1):
                wz = frac[:, 2] if oz else 1.0 - frac[:, 2]
                w = wx * wy * wz
                if weights is not None:
                    w = w * weights
                out += np.bincount(_corner_index(base, n, ox, oy, oz), weights=w,
                                   minlength=n ** 3)
    return out.reshape(n, n, n)


def cic_readout(u, mesh):
    """value_p = sum_c W(u_p - c) mesh(c), the transpose of ``cic_paint``."""
    n = mesh.shape[0]
    flat = mesh.reshape(-1)
    base, frac = _corners(u, n)
    out = np.zeros(u.shape[0])
    for ox in (0, 1):
        wx = frac[:, 0] if ox else 1.0 - frac[:, 0]
        for oy in (0, 1):
            wy = frac[:, 1] if oy else 1.0 - frac[:, 1]
            for oz in (0, 1):
                wz = frac[:, 2] if oz else 1.0 - frac[:, 2]
                out += wx * wy * wz * flat[_corner_index(base, n, ox, oy, oz)]
    return out


def cic_readout_grad(u, mesh):
    """d/du_d of sum_c W(u_p - c) mesh(c), (M, 3), in 1/cell units.

    dW/du_d = -sgn(u_d - c_d) prod_{e != d} (1 - |u_e - c_e|) with the
    floor-based convention: the lower node of each axis gets -1, the upper +1
    (so u_d exactly on a node counts as inside the cell above it)."""
    n = mesh.shape[0]
    flat = mesh.reshape(-1)
    base, frac = _corners(u, n)
    out = np.zeros((u.shape[0], 3))
    for ox in (0, 1):
        wx = frac[:, 0] if ox else 1.0 - frac[:, 0]
        gx = 1.0 if ox else -1.0
        for oy in (0, 1):
            wy = frac[:, 1] if oy else 1.0 - frac[:, 1]
            gy = 1.0 if oy else -1.0
            for oz in (0, 1):
                wz = frac[:, 2] if oz else 1.0 - frac[:, 2]
                gz = 1.0 if oz else -1.0
                m = flat[_corner_index(base, n, ox, oy, oz)]
                out[:, 0] += gx * wy * wz * m
                out[:, 1] += wx * gy * wz * m
                out[:, 2] += wx * wy * gz * m
    return out
