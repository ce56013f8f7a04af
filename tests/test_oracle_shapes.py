"""Pins of the oracle's general particle shapes, frame-2 variation and hiding.

The paper's single-particle model (Eq. 1) has sigma_x, sigma_y and rho drawn
per particle from configured intervals; frame-2 parameters vary by a
zero-mean Gaussian of configured variance (text after Eq. 1), and a particle
may be hidden from either image ("aggregation of the particle contributions").
Each test checks the oracle against something other than itself: a library
routine (scipy's bivariate normal), brute-force integration of Eq. 1,
closed forms, symmetries, or sampling statistics.  No GPU needed.
"""
import math

import numpy as np
import pytest
from scipy import special, stats

import oracle
from paper_2512_09664_b300 import workloads as W


def _eq1_pixel_bruteforce(x0, y0, sx, sy, rho, j, i, n=600):
    """Midpoint rule of the normalised Eq. 1 density over pixel (i, j) on
    n x n and 2n x 2n grids, Richardson-extrapolated (error O(h^4))."""
    def mid(m):
        t = (np.arange(m) + 0.5) / m
        X, Y = np.meshgrid(j + t, i + t, indexing="xy")
        tx, ty = (X - x0) / sx, (Y - y0) / sy
        q = (tx * tx - 2 * rho * tx * ty + ty * ty) / (2 * (1 - rho * rho))
        return float((np.exp(-q) / (2 * math.pi * sx * sy * math.sqrt(1 - rho * rho))).mean())
    return (4.0 * mid(2 * n) - mid(n)) / 3.0


def _bvn_rect(x0, y0, sx, sy, rho, j, i):
    """scipy's bivariate normal probability of [j, j+1) x [i, i+1)."""
    cov = [[sx * sx, rho * sx * sy], [rho * sx * sy, sy * sy]]
    mvn = stats.multivariate_normal(mean=[x0, y0], cov=cov)
    return float(mvn.cdf([j + 1, i + 1], lower_limit=[j, i]))


SHAPES = [(0.25, 0.25, 0.0), (0.25, 0.9, 0.6), (0.75, 0.4, -0.85), (1.0, 1.0, 0.9), (0.5, 2.0, 0.3)]


@pytest.mark.parametrize("sx,sy,rho", SHAPES)
def test_oracle_pixel_mass2_matches_bruteforce_eq1(sx, sy, rho):
    x0, y0 = 0.37, 0.81
    for j in (-1, 0, 1):
        for i in (-1, 0, 1):
            got = oracle.pixel_mass2(x0, y0, sx, sy, rho, j, i)
            want = _eq1_pixel_bruteforce(x0, y0, sx, sy, rho, j, i)
            assert abs(got - want) <= 2e-6 * max(want, 1e-3), (j, i, got, want)


@pytest.mark.parametrize("sx,sy,rho", SHAPES)
def test_oracle_pixel_mass2_matches_scipy_bivariate_normal(sx, sy, rho):
    x0, y0 = -0.2, 0.45
    for j, i in ((0, 0), (-1, 0), (0, 1), (1, -1), (-2, 1)):
        got = oracle.pixel_mass2(x0, y0, sx, sy, rho, j, i)
        want = _bvn_rect(x0, y0, sx, sy, rho, j, i)
        assert abs(got - want) < 1e-7, (j, i, got, want)


def test_oracle_pixel_mass2_rho0_is_product_of_ndtr_differences():
    x0, y0, sx, sy = 0.3, 0.6, 0.5, 0.7
    for j in range(-3, 4):
        for i in range(-3, 4):
            want = ((special.ndtr((j + 1 - x0) / sx) - special.ndtr((j - x0) / sx))
                    * (special.ndtr((i + 1 - y0) / sy) - special.ndtr((i - y0) / sy)))
            assert abs(oracle.pixel_mass2(x0, y0, sx, sy, 0.0, j, i) - want) < 1e-15


@pytest.mark.parametrize("sx,sy,rho", SHAPES)
def test_oracle_pixel_mass2_sums_to_one(sx, sy, rho):
    x0, y0 = 0.5, 0.5
    rx, ry = int(math.ceil(9 * sx)) + 1, int(math.ceil(9 * sy)) + 1
    tot = sum(oracle.pixel_mass2(x0, y0, sx, sy, rho, j, i)
              for j in range(-rx, rx + 1) for i in range(-ry, ry + 1))
    assert abs(tot - 1.0) < 1e-10


def test_oracle_pixel_mass2_symmetries():
    x0, y0, sx, sy, rho = 0.3, 0.7, 0.6, 0.35, 0.55
    for j in range(-2, 3):
        for i in range(-2, 3):
            m = oracle.pixel_mass2(x0, y0, sx, sy, rho, j, i)
            # transpose: swap the axes (x <-> y, sigma_x <-> sigma_y)
            assert abs(m - oracle.pixel_mass2(y0, x0, sy, sx, rho, i, j)) < 1e-13
            # mirror x about 0: x0 -> -x0, pixel j -> -j - 1, rho -> -rho
            assert abs(m - oracle.pixel_mass2(-x0, y0, sx, sy, -rho, -j - 1, i)) < 1e-13


def test_oracle_splat_shapes_window_matches_bruteforce_and_total():
    H = W_ = 32
    parts = np.array([[15.3, 16.8, 3.2, 2.0, 0.7, 0.9],
                      [9.6, 10.1, 1.5, 3.6, -0.4, 0.6]])
    win = oracle.splat_shapes(H, W_, parts, mode=0)
    brute = oracle.splat_shapes(H, W_, parts, mode=1)
    assert np.abs(win - brute).max() < 1e-8
    amp = parts[:, 5] * 2 * math.pi * (parts[:, 2] / 4) * (parts[:, 3] / 4) * np.sqrt(1 - parts[:, 4] ** 2)
    assert abs(brute.sum() / amp.sum() - 1.0) < 1e-9


def test_oracle_splat_shapes_round_equals_separable_splat():
    H, W_ = 24, 40
    rng = np.random.default_rng(4)
    n = 30
    x = rng.uniform(0, W_, n)
    y = rng.uniform(0, H, n)
    d = rng.uniform(1, 4, n)
    ie = rng.uniform(0.5, 1, n)
    a = oracle.splat(H, W_, np.stack([x, y, d, ie], 1))
    b = oracle.splat_shapes(H, W_, np.stack([x, y, d, d, np.zeros(n), ie], 1))
    assert np.abs(a - b).max() <= 1e-15 * max(1.0, a.max())


def test_oracle_splat_shapes_point_sampled_is_eq1():
    H = W_ = 20
    x, y, dx, dy, rho, ie = 10.2, 9.7, 6.0, 4.0, -0.5, 0.8
    S = oracle.splat_shapes(H, W_, np.array([[x, y, dx, dy, rho, ie]]), mode=2)
    sx, sy = dx / 4, dy / 4
    for (i, j) in ((9, 10), (7, 12), (12, 8)):
        tx, ty = (j + 0.5 - x) / sx, (i + 0.5 - y) / sy
        want = ie * math.exp(-(tx * tx - 2 * rho * tx * ty + ty * ty) / (2 * (1 - rho * rho)))
        assert abs(S[i, j] - want) < 1e-14


def test_oracle_integrated_tends_to_point_sampled_for_wide_particles():
    # the pixel average of a smooth density is its centre value plus
    # (f_xx + f_yy) / 24: at the peak of Eq. 1 a relative gap of
    # (1 / sigma_x^2 + 1 / sigma_y^2) / (24 (1 - rho^2))
    H = W_ = 64
    x, y, dx, dy, rho = 31.5, 32.5, 40.0, 28.0, 0.4
    row = np.array([[x, y, dx, dy, rho, 1.0]])
    integ = oracle.splat_shapes(H, W_, row, mode=0)
    point = oracle.splat_shapes(H, W_, row, mode=2)
    gap = (point[32, 31] - integ[32, 31]) / point[32, 31]
    pred = (1 / (dx / 4) ** 2 + 1 / (dy / 4) ** 2) / (24 * (1 - rho * rho))
    assert abs(gap / pred - 1.0) < 0.02


# ----------------------------------------------------------------------------
# per-particle shapes, frame-2 variation and hiding
# ----------------------------------------------------------------------------

def _spec(**kw):
    base = dict(height=64, width=64, n_particles=40000, pair_id=3, d_min=1.0, d_max=4.0)
    base.update(kw)
    return W.PairSpec(**base)


def test_oracle_default_shapes_are_round_and_unchanged_between_frames():
    spec = _spec(n_particles=3000)
    pr = oracle.make_pair(spec, seed=7)
    t = oracle.particles(pr, W.zero_flow(64, 64))
    s = oracle.particle_shapes(pr)
    for f in range(2):
        assert np.array_equal(s[:, f, 0], t[:, 2]) and np.array_equal(s[:, f, 1], t[:, 2])
        assert np.all(s[:, f, 2] == 0.0) and np.array_equal(s[:, f, 3], t[:, 5])
        assert np.all(s[:, f, 4] == 1.0)


@pytest.mark.parametrize("p", [0.0, 0.3, 1.0])
def test_oracle_hiding_frequency_and_independence(p):
    spec = _spec()
    s = oracle.particle_shapes(oracle.make_pair(spec, seed=9, hide_prob=p))
    n = s.shape[0]
    p32 = float(np.float32(p))
    h1, h2 = s[:, 0, 4] == 0.0, s[:, 1, 4] == 0.0
    tol = 5 * math.sqrt(max(p32 * (1 - p32), 1e-12) / n)
    assert abs(h1.mean() - p32) <= tol and abs(h2.mean() - p32) <= tol
    assert abs((h1 & h2).mean() - p32 * p32) <= tol


def test_oracle_hiding_uses_stream_2_words():
    # hide from frame f when u24(word f of stream 2) < hide_prob
    spec = _spec(n_particles=200)
    pr = oracle.make_pair(spec, seed=21, hide_prob=0.5)
    s = oracle.particle_shapes(pr)
    for i in range(200):
        w = oracle.stream_words(21, spec.pair_id, i, 2)
        for f in range(2):
            assert (s[i, f, 4] == 0.0) == (((int(w[f]) >> 8) / 2.0 ** 24) < 0.5)


def test_oracle_frame2_variation_statistics():
    jd, ji, jr = 0.1, 0.02, 0.05
    spec = _spec(d_min=1.0, d_max=5.0, i_min=0.2, i_max=1.0, dy_min=1.0, dy_max=5.0,
                 rho_min=-0.8, rho_max=0.8, jitter_d=jd, jitter_i=ji, jitter_rho=jr,
                 sheet_sigma=0.0)
    pr = oracle.make_pair(spec, seed=13)
    s = oracle.particle_shapes(pr)
    t = oracle.particles(pr, W.zero_flow(64, 64))
    # frame-1 draws: uniform over their intervals
    assert stats.kstest((s[:, 0, 1] - 1.0) / 4.0, "uniform").pvalue > 1e-3
    assert stats.kstest((s[:, 0, 2] + float(np.float32(0.8))) / (2 * float(np.float32(0.8))),
                        "uniform").pvalue > 1e-3
    for col, j, lo, hi, f1 in ((0, jd, 1.0, 5.0, s[:, 0, 0]), (1, jd, 1.0, 5.0, s[:, 0, 1]),
                               (2, jr, -0.8, 0.8, s[:, 0, 2]), (3, ji, 0.2, 1.0, t[:, 3])):
        f2 = s[:, 1, col] if col < 3 else s[:, 1, 3]  # Ieff = I with the sheet off
        inner = (f1 > lo + 6 * j) & (f1 < hi - 6 * j)
        dlt = (f2 - f1)[inner]
        assert abs(dlt.mean()) < 5 * j / math.sqrt(inner.sum())
        assert abs(dlt.std() / j - 1.0) < 0.03
        assert stats.kstest(dlt / j, "norm").pvalue > 1e-3
        assert f2.min() >= float(np.float32(lo)) - 1e-12 and f2.max() <= float(np.float32(hi)) + 1e-12
    # the four normals are independent of each other
    c = np.corrcoef(np.stack([s[:, 1, k] - s[:, 0, k] for k in range(3)]))
    assert np.abs(c - np.eye(3)).max() < 0.05


def test_oracle_render_hidden_everywhere_is_blank():
    wl = W.Workload("hide_all", 5, [_spec(height=32, width=32, n_particles=50)],
                    [W.zero_flow(32, 32)], hide_prob=1.0)
    r = oracle.render_workload(wl)[0]
    assert np.all(r["S"] == 0.0)


def test_oracle_render_general_zero_flow_frames_identical():
    spec = _spec(height=40, width=48, n_particles=120, dy_min=1.5, dy_max=3.5, rho_min=-0.6, rho_max=0.6)
    wl = W.Workload("aniso", 17, [spec], [W.zero_flow(40, 48)])
    r = oracle.render_workload(wl)[0]
    assert np.array_equal(r["S"][0], r["S"][1])
    assert r["S"][0].max() > 0.1
