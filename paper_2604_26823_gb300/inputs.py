"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests
and the benchmark.

This module holds no arithmetic of the method: it only draws random numbers
and builds the survey geometry that the model reads as input (white noise,
noise fields, Poisson draws at a given rate, the selection mesh R, sorted
targets for rank-order matching, random directions).

The paper's mock catalogue (a Millennium-based lightcone) is not available;
the survey geometry here stands in for it with the paper's proportions: a
cube of side L, an observer outside the box looking along +z, a cone of
galaxies with a radial number density and angular holes (Sec. 2.1).
"""
import numpy as np


def white_noise(n, seed, dtype=np.float32):
    """s ~ N(0, 1) on an (n, n, n) grid (C order, x slowest)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, n, n)).astype(dtype)


def normal_field(n, seed, scale=1.0, dtype=np.float32):
    rng = np.random.default_rng(seed)
    return (scale * rng.standard_normal((n, n, n))).astype(dtype)


def uniform_field(n, seed, lo, hi, dtype=np.float32):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, (n, n, n)).astype(dtype)


def poisson_counts(rate, seed, dtype=np.float32):
    """N ~ Poisson(rate) per cell (rate >= 0 array)."""
    rng = np.random.default_rng(seed)
    return rng.poisson(np.maximum(np.asarray(rate, dtype=np.float64), 0.0)).astype(dtype)


def sorted_normal_targets(count, seed, dtype=np.float32):
    """``count`` N(0,1) draws sorted in descending order."""
    rng = np.random.default_rng(seed)
    t = rng.standard_normal(count)
    return np.sort(t)[::-1].astype(dtype).copy()


def sorted_normal_targets_per_bin(counts, seed, dtype=np.float32):
    """Concatenation over bins of ``sorted_normal_targets(counts[b])``, drawn
    from one generator in bin order."""
    rng = np.random.default_rng(seed)
    parts = []
    for c in counts:
        t = rng.standard_normal(int(c))
        parts.append(np.sort(t)[::-1])
    if not parts:
        return np.zeros(0, dtype=dtype)
    return np.concatenate(parts).astype(dtype)


def random_unit_directions(n, count, seed, dtype=np.float64):
    """``count`` directions u_j = g_j / |g_j|, g_j ~ N(0,1)^(n^3)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        g = rng.standard_normal((n, n, n))
        out.append((g / np.linalg.norm(g)).astype(dtype))
    return out


def survey_selection(n, box, seed, observer=(250.0, 250.0, -150.0), half_angle_deg=40.0,
                     r_scale=300.0, n_patches=16, completeness=(0.3, 0.9), dtype=np.float32):
    """Selection mesh R on the nodes (i, j, l) * L / n.

    Inside a cone around +z from ``observer`` with the given half angle:
    R = C(patch) n(r) / max n, with n(r) = r^2 exp(-(r / r_scale)^1.5) and
    C drawn U(lo, hi) on an n_patches x n_patches grid of (cos theta, phi)
    patches of the cone; outside the cone R = 0."""
    rng = np.random.default_rng(seed)
    comp = rng.uniform(completeness[0], completeness[1], (n_patches, n_patches))
    cell = box / n
    coords = np.arange(n) * cell
    x = coords[:, None, None] - observer[0]
    y = coords[None, :, None] - observer[1]
    z = coords[None, None, :] - observer[2]
    r = np.sqrt(x * x + y * y + z * z)
    cos_t = np.where(r > 0, z / np.where(r > 0, r, 1.0), 1.0)
    cmin = np.cos(np.deg2rad(half_angle_deg))
    inside = cos_t >= cmin
    phi = np.arctan2(y, x) % (2.0 * np.pi)
    it = np.clip(((cos_t - cmin) / (1.0 - cmin) * n_patches).astype(np.int64), 0, n_patches - 1)
    ip = np.clip((phi / (2.0 * np.pi) * n_patches).astype(np.int64), 0, n_patches - 1)
    rpeak = r_scale * (4.0 / 3.0) ** (1.0 / 1.5)       # maximum of r^2 exp(-(r/r_s)^1.5)
    nr = (r / rpeak) ** 2 * np.exp(-(r / r_scale) ** 1.5 + (rpeak / r_scale) ** 1.5)
    sel = np.where(inside, comp[it, ip] * nr, 0.0)
    return sel.astype(dtype)
