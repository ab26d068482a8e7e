"""Pins of the projection operator and rank-order matching (Sec. 2.3.1,
Sec. 2.3.2): published generator test vector, closed forms, invariants and
hand-worked examples."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import mesh as M
from oracle import projection as P
from paper_2604_26823_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line)
    return rows


def test_splitmix64_published_vector():
    expect = [int(x) for x in _golden("splitmix64_seed1234567.txt")]
    state = np.uint64(1234567)
    got = []
    with np.errstate(over="ignore"):
        for _ in range(5):
            state = state + P._GOLDEN
            got.append(int(P._mix(state)))
    assert got == expect


def test_counter_normals_are_standard_normal_and_reproducible():
    idx = np.arange(200000, dtype=np.uint64)
    z = P.counter_normals(idx, seed=6, counter=3)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    assert stats.kstest(z, "norm").pvalue > 1e-3
    np.testing.assert_array_equal(z[1234:1240], P.counter_normals(idx[1234:1240], 6, 3))
    assert not np.allclose(z[:100], P.counter_normals(idx[:100], 6, 4))


def test_projection_zscore_closed_form_and_idempotence():
    rng = np.random.default_rng(0)
    s = 3.0 + 2.5 * rng.standard_normal(10000)
    out, nreset = P.project(s, seed=1, counter=0)
    assert nreset == 0
    assert abs(out.mean()) < 1e-14 and abs(out.std() - 1.0) < 1e-14
    np.testing.assert_allclose(out, (s - s.mean()) / s.std(), rtol=1e-14, atol=1e-14)
    again, n2 = P.project(out, seed=1, counter=1)
    assert n2 == 0
    np.testing.assert_allclose(again, out, atol=1e-13)
    # a Gaussian vector is almost a fixed point: P(s) = s + O(1/sqrt(d)) per element
    g = rng.standard_normal(100000)
    pg, _ = P.project(g, 1, 0)
    assert np.max(np.abs(pg - g)) < 0.05


def test_projection_resets_extreme_values():
    rng = np.random.default_rng(1)
    s = rng.standard_normal(100000)
    s[[5, 77, 999]] = [400.0, -500.0, 450.0]
    mu, sd = s.mean(), s.std()
    zhat = (s - mu) / sd
    expect_bad = np.nonzero(np.abs(zhat) > 10.0)[0]
    out, nreset = P.project(s, seed=9, counter=2)
    assert nreset == expect_bad.size == 3
    np.testing.assert_allclose(out[expect_bad],
                               P.counter_normals(expect_bad.astype(np.uint64), 9, 2), rtol=0, atol=0)
    keep = np.ones(s.size, bool)
    keep[expect_bad] = False
    np.testing.assert_allclose(out[keep], zhat[keep], rtol=1e-14)
    assert np.all(np.abs(out) <= 10.0)


def test_rom_hand_worked_example():
    x, t, expect = (np.array([float(v) for v in row.split()]) for row in _golden("rom_tiny.txt"))
    np.testing.assert_array_equal(P.rank_order_match(x, t), expect)


def test_rom_invariants_and_quantiles():
    rng = np.random.default_rng(2)
    x = rng.standard_normal(5000) ** 3
    t = np.sort(rng.standard_normal(5000))[::-1]
    out = P.rank_order_match(x, t)
    np.testing.assert_array_equal(np.sort(out), np.sort(t))          # multiset
    assert stats.spearmanr(x, out).correlation == pytest.approx(1.0)  # order kept
    # quantile targets: the k-th largest input gets Phi^-1(1 - (k - 1/2)/n)
    n = 1000
    xq = rng.standard_normal(n)
    q = stats.norm.ppf((np.arange(n) + 0.5) / n)[::-1]
    outq = P.rank_order_match(xq, q)
    order = np.argsort(-xq)
    np.testing.assert_allclose(outq[order], q)
    # Gaussian input: the change scales like 1/sqrt(n) (Sec. 2.3.2)
    big = rng.standard_normal(200000)
    tb = np.sort(rng.standard_normal(200000))[::-1]
    assert np.mean(np.abs(P.rank_order_match(big, tb) - big)) < 5.0 / np.sqrt(200000)


def test_rom_real_touches_only_selected_cells():
    n = 8
    s = inputs.white_noise(n, 3).astype(np.float64)
    resp = inputs.uniform_field(n, 4, -1.0, 1.0).astype(np.float64)
    sel = resp > 0
    t = inputs.sorted_normal_targets(int(sel.sum()), 5).astype(np.float64)
    out = P.rom_real(s, resp, t)
    np.testing.assert_array_equal(out[~sel], s[~sel])
    np.testing.assert_array_equal(np.sort(out[sel]), np.sort(t))


def test_rom_real_ranks_brute_force():
    """Rank by direct counting: the number of selected cells with a larger
    value, or an equal value at a lower index."""
    n = 8
    s = inputs.white_noise(n, 6).astype(np.float64).reshape(-1)
    s[10:40] = 0.25                     # ties
    resp = inputs.uniform_field(n, 7, -1.0, 1.0).astype(np.float64).reshape(-1)
    rank = P.rom_real_ranks(s, resp)
    sel = np.nonzero(resp > 0)[0]
    for i in range(s.size):
        if resp[i] > 0:
            assert rank[i] == sum(1 for j in sel if s[j] > s[i] or (s[j] == s[i] and j < i))
        else:
            assert rank[i] == -1
    # real-space matching puts the rank-r target at the rank-r cell
    t = inputs.sorted_normal_targets(sel.size, 8).astype(np.float64)
    out = P.rom_real(s, resp, t)
    np.testing.assert_array_equal(out[sel], t[rank[sel]])


def test_fourier_mode_selection_brute_force():
    # canonical half-space modes by direct enumeration of conjugate pairs
    n, box = 8, 20.0
    idx, b, part = P.fourier_modes(n, box, n_bins=10, k_min=0.0)
    h = n // 2 + 1
    seen, expect = set(), []
    for i in range(n):
        for j in range(n):
            for l in range(h):
                key = (i, j, l)
                conj = ((-i) % n, (-j) % n, (-l) % n)
                if conj[2] >= h:       # partner lives in the implicit half
                    expect.append(key)
                    continue
                if conj == key:        # self-conjugate: never matched
                    continue
                if conj in seen:
                    continue
                seen.add(key)
                expect.append(key)
    flat = sorted((i * n + j) * h + l for (i, j, l) in expect)
    np.testing.assert_array_equal(idx, flat)
    # 2 * (number of canonical non-self-conjugate modes) = n^3 - (# self-conjugate real dofs)
    assert 2 * idx.size == n ** 3 - 8


def test_rom_fourier_invariants():
    n, box = 16, 100.0
    s = inputs.white_noise(n, 6).astype(np.float64)
    counts = P.fourier_bin_counts(n, box)
    t = inputs.sorted_normal_targets_per_bin(counts, 7).astype(np.float64)
    out = P.rom_fourier(s, box, t)
    assert out.shape == s.shape and np.isrealobj(out)
    sk, ok = M.rfft3(s), M.rfft3(out)
    kmag = np.sqrt(M.k_squared(n, box))
    low = kmag < P.K_MIN
    np.testing.assert_allclose(ok[low], sk[low], atol=1e-9)
    # per-bin multiset of the matched values equals the targets
    idx, b, _ = P.fourier_modes(n, box)
    z = ok.reshape(-1)[idx] * np.sqrt(2.0 / n ** 3)
    vals = np.empty(2 * idx.size)
    vals[0::2], vals[1::2] = z.real, z.imag
    eb = np.repeat(b, 2)
    offs = np.concatenate([[0], np.cumsum(counts)])
    for bb in range(P.N_BINS):
        np.testing.assert_allclose(np.sort(vals[eb == bb]), np.sort(t[offs[bb]:offs[bb + 1]]),
                                   atol=1e-12)
    # matching a field to its own sorted values is the identity
    z0 = M.rfft3(s).reshape(-1)[idx] * np.sqrt(2.0 / n ** 3)
    v0 = np.empty(2 * idx.size)
    v0[0::2], v0[1::2] = z0.real, z0.imag
    own = np.concatenate([np.sort(v0[eb == bb])[::-1] for bb in range(P.N_BINS)])
    np.testing.assert_allclose(P.rom_fourier(s, box, own), s, atol=1e-12)


def test_composite_order():
    n, box = 8, 40.0
    s = inputs.white_noise(n, 8).astype(np.float64) * 2 + 1
    resp = inputs.uniform_field(n, 9, -1.0, 1.0).astype(np.float64)
    tr = inputs.sorted_normal_targets(int((resp > 0).sum()), 10).astype(np.float64)
    tf = inputs.sorted_normal_targets_per_bin(P.fourier_bin_counts(n, box), 11).astype(np.float64)
    out, _ = P.project_rank_match(s, box, resp, 7, tr, tf, seed=3, counter=4)
    step = P.rom_fourier(s, box, tf)
    step = P.rom_real(step, resp, tr)
    step, _ = P.project(step, 3, 4)
    np.testing.assert_array_equal(out, step)


def test_fourier_bins_exact_on_edges():
    # m = (32, 32, 32) at n = 256 lies exactly on the edge between bins 24
    # and 25: |m| / (sqrt(3) n / 2) * 100 = 25
    n, box = 256, 500.0
    idx, b, _ = P.fourier_modes(n, box)
    h = n // 2 + 1
    flat = (32 * n + 32) * h + 32
    assert b[np.searchsorted(idx, flat)] == 25
    # and the bin of every mode agrees with a brute-force exact rational test
    rng = np.random.default_rng(0)
    pick = rng.choice(idx.size, 2000, replace=False)
    for q in pick:
        f = idx[q]
        ix, iy, iz = f // (n * h), (f // h) % n, f % h
        mx = ix if ix < n // 2 else ix - n
        my = iy if iy < n // 2 else iy - n
        m2 = mx * mx + my * my + iz * iz
        bb = 0
        while 3 * n * n * (bb + 1) ** 2 <= 4 * 100 * 100 * m2:
            bb += 1
        assert b[q] == min(bb, 99)
