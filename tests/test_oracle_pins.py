"""Pins of the FP64 oracle against things other than itself.

Each test checks one part of the oracle against a published known answer,
a closed form, an invariant, a library routine (scipy / torch) or brute
force, so that a dropped term, wrong sign, wrong index or transposed operand
anywhere in it fails at least one test.  No GPU needed.
"""
import math
import os

import numpy as np
import pytest
from scipy import ndimage, special, stats

import oracle
from paper_2512_09664_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# Philox4x32-10 (known answers published with the generator)
# ----------------------------------------------------------------------------

def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t, 16) for t in line.split()])
    return rows


@pytest.mark.parametrize("row", _kat_rows())
def test_oracle_philox_known_answers(row):
    ctr, key, want = row[0:4], row[4:6], row[6:10]
    assert list(oracle.philox4x32_10(ctr, key)) == want


def test_oracle_stream_counter_layout():
    # counter = (index, tag, pair_id lo, pair_id hi), key = (seed lo, seed hi)
    seed, pid = 0x0123456789ABCDEF, 0xFEDCBA9876543210
    got = oracle.stream_words(seed, pid, 77, 0x101)
    want = oracle.philox4x32_10([77, 0x101, pid & 0xFFFFFFFF, pid >> 32],
                                [seed & 0xFFFFFFFF, seed >> 32])
    assert list(got) == list(want)


# ----------------------------------------------------------------------------
# attribute sampling (Section 2: uniform positions and parameters)
# ----------------------------------------------------------------------------

def _pair(**kw):
    base = dict(height=64, width=96, n_particles=20000, pair_id=5)
    base.update(kw)
    return W.PairSpec(**base)


def test_oracle_positions_uniform_over_image():
    spec = _pair()
    pr = oracle.make_pair(spec, seed=11)
    t = oracle.particles(pr, W.zero_flow(64, 96))
    x, y = t[:, 0], t[:, 1]
    assert x.min() >= 0 and x.max() < 96 and y.min() >= 0 and y.max() < 64
    assert stats.kstest(x / 96.0, "uniform").pvalue > 1e-3
    assert stats.kstest(y / 64.0, "uniform").pvalue > 1e-3
    # x and y come from different words: no correlation
    assert abs(np.corrcoef(x, y)[0, 1]) < 0.05


def test_oracle_uniform_diameter_and_intensity_ranges():
    spec = _pair(d_dist=0, d_min=1.0, d_max=4.0, i_min=0.8, i_max=1.0)
    t = oracle.particles(oracle.make_pair(spec, seed=3), W.zero_flow(64, 96))
    d, I = t[:, 2], t[:, 3]
    assert d.min() >= 1.0 and d.max() < 4.0
    assert stats.kstest((d - 1.0) / 3.0, "uniform").pvalue > 1e-3
    assert I.min() >= np.float32(0.8) - 1e-12 and I.max() < 1.0
    assert stats.kstest((I - float(np.float32(0.8))) / (1 - float(np.float32(0.8))), "uniform").pvalue > 1e-3


def test_oracle_clipped_normal_diameter_is_box_muller_normal():
    spec = _pair(d_dist=1, d_min=1.0, d_max=4.0, d_mu=2.5, d_sigma=0.3)
    t = oracle.particles(oracle.make_pair(spec, seed=9), W.zero_flow(64, 96))
    d = t[:, 2]
    mu, s = float(np.float32(2.5)), float(np.float32(0.3))
    assert stats.kstest((d - mu) / s, "norm").pvalue > 1e-3
    # clipping: a wide normal hits both bounds with the closed-form probabilities
    spec2 = _pair(d_dist=1, d_min=2.0, d_max=3.0, d_mu=2.5, d_sigma=0.5)
    d2 = oracle.particles(oracle.make_pair(spec2, seed=9), W.zero_flow(64, 96))[:, 2]
    assert d2.min() == 2.0 and d2.max() == 3.0
    p_lo = special.ndtr(-1.0)  # P(N(2.5, .5) < 2)
    n = len(d2)
    assert abs(np.mean(d2 == 2.0) - p_lo) < 4 * math.sqrt(p_lo * (1 - p_lo) / n)
    assert abs(np.mean(d2 == 3.0) - p_lo) < 4 * math.sqrt(p_lo * (1 - p_lo) / n)


def test_oracle_sheet_gain_expectation_closed_form():
    # E[Ieff / I] for z ~ U[z0, z1] under exp(-z^2 / (2 s^2)):
    #   sqrt(pi/2) s (erf(z1 / (sqrt2 s)) - erf(z0 / (sqrt2 s))) / (z1 - z0)
    spec = _pair(z_min=-1.0, z_max=1.0, sheet_sigma=0.5)
    t = oracle.particles(oracle.make_pair(spec, seed=21), W.zero_flow(64, 96))
    g = t[:, 5] / t[:, 3]
    s = 0.5
    want = math.sqrt(math.pi / 2) * s * (math.erf(1 / (math.sqrt(2) * s)) - math.erf(-1 / (math.sqrt(2) * s))) / 2
    se = g.std() / math.sqrt(len(g))
    assert abs(g.mean() - want) < 4 * se
    # z = 0 everywhere -> no attenuation; no sheet -> no attenuation
    t0 = oracle.particles(oracle.make_pair(_pair(z_min=0.0, z_max=0.0), seed=1), W.zero_flow(64, 96))
    assert np.array_equal(t0[:, 5], t0[:, 3])
    t1 = oracle.particles(oracle.make_pair(_pair(sheet_sigma=0.0), seed=1), W.zero_flow(64, 96))
    assert np.array_equal(t1[:, 5], t1[:, 3])


def test_oracle_particle_count_recipe():
    # frame particle counts of the workloads: floor(ppp H W)
    assert W.single_pair_256().pairs[0].n_particles == 1310
    assert W.n_particles_for(0.05, 512, 512) == 13107
    assert W.n_particles_for(0.1, 2048, 2048) == 419430


# ----------------------------------------------------------------------------
# noise (additive Gaussian, Box-Muller on the per-frame noise stream)
# ----------------------------------------------------------------------------

def test_oracle_noise_standard_normal_and_frames_independent():
    n0 = np.array([oracle.noise(7, 3, 0, p) for p in range(40000)])
    n1 = np.array([oracle.noise(7, 3, 1, p) for p in range(40000)])
    assert stats.kstest(n0, "norm").pvalue > 1e-3
    assert stats.kstest(n1, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(n0, n1)[0, 1]) < 0.03
    assert abs(np.corrcoef(n0[:-1], n0[1:])[0, 1]) < 0.03


def test_oracle_noise_quad_is_one_box_muller_pair_each():
    # pixels 4q, 4q+1 share a radius: n^2 + n'^2 = -2 ln(u)
    for q in (0, 5, 1000):
        w = oracle.stream_words(7, 3, q, 0x100)
        a = [oracle.noise(7, 3, 0, 4 * q + k) for k in range(4)]
        r0 = -2 * math.log(((int(w[0]) >> 8) + 1) / 2 ** 24)
        r1 = -2 * math.log(((int(w[2]) >> 8) + 1) / 2 ** 24)
        assert math.isclose(a[0] ** 2 + a[1] ** 2, r0, rel_tol=1e-12)
        assert math.isclose(a[2] ** 2 + a[3] ** 2, r1, rel_tol=1e-12)


# ----------------------------------------------------------------------------
# bilinear interpolation on the cell-centred grid
# ----------------------------------------------------------------------------

def test_oracle_bilinear_matches_torch_grid_sample():
    import torch
    rng = np.random.default_rng(0)
    gh, gw, H, Wd = 13, 17, 40, 52  # grid coarser than the image, odd sizes
    flow = rng.standard_normal((gh, gw, 2)).astype(np.float32)
    pts = np.stack([rng.uniform(-8, Wd + 8, 400), rng.uniform(-8, H + 8, 400)], 1)
    ft = torch.from_numpy(flow.astype(np.float64)).permute(2, 0, 1)[None]
    g = torch.from_numpy(np.stack([2 * pts[:, 0] / Wd - 1, 2 * pts[:, 1] / H - 1], 1))[None, None]
    ref = torch.nn.functional.grid_sample(ft, g, mode="bilinear", padding_mode="border",
                                          align_corners=False)[0, :, 0].numpy().T
    got = np.array([oracle.velocity(flow, H, Wd, x, y) for x, y in pts])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


def test_oracle_bilinear_reproduces_affine_field_inside_hull():
    a = np.array([[0.01, -0.02], [0.03, 0.005]])
    flow = W.linear_flow(32, 32, 32, 32, a, (16.0, 16.0))
    rng = np.random.default_rng(1)
    for x, y in rng.uniform(0.5, 31.5, (100, 2)):
        u, v = oracle.velocity(flow, 32, 32, x, y)
        want = a @ np.array([x - 16, y - 16])
        # the grid holds FP32 values of the affine field
        assert abs(u - want[0]) < 1e-6 and abs(v - want[1]) < 1e-6


# ----------------------------------------------------------------------------
# advection (displacement map; RK4 / Euler substeps)
# ----------------------------------------------------------------------------

def _adv_pair(integrator="rk4", n=4, dt=1.0, H=64, Wd=64):
    return oracle.make_pair(_pair(height=H, width=Wd, n_particles=0), seed=0,
                            integrator=integrator, n_substeps=n, dt=dt)


def test_oracle_advect_uniform_field_exact():
    flow = W.uniform_flow(64, 64, 1.75, -2.5)
    for integ in ("rk4", "euler"):
        pr = _adv_pair(integ, n=4, dt=2.0)
        x, y = oracle.advect(pr, flow, 10.125, 20.5)
        assert x == 10.125 + 3.5 and y == 20.5 - 5.0


def test_oracle_advect_linear_field_rk4_closed_form():
    # inside the node hull the bilinear field of U = A (p - c) is exact, so one
    # RK4 step maps p - c by the degree-4 Taylor polynomial of exp(hA).
    a = np.array([[0.02, -0.05], [0.04, -0.01]])
    c = np.array([32.0, 32.0])
    flow = W.linear_flow(64, 64, 64, 64, a, c)
    af = np.array([[np.float32(0.02), np.float32(-0.05)], [np.float32(0.04), np.float32(-0.01)]])
    for n, dt in ((1, 1.0), (4, 2.0), (3, 1.5)):
        pr = _adv_pair("rk4", n=n, dt=dt)
        p0 = np.array([30.3, 35.1])
        x, y = oracle.advect(pr, flow, *p0)
        h = dt / n
        hA = h * af
        R = np.eye(2) + hA + hA @ hA / 2 + hA @ hA @ hA / 6 + hA @ hA @ hA @ hA / 24
        want = c + np.linalg.matrix_power(R, n) @ (p0 - c)
        assert np.allclose([x, y], want, atol=2e-5)  # FP32 flow storage
        # and RK4 is within its error bound of the exact flow map exp(dt A)
        from scipy.linalg import expm
        exact = c + expm(dt * af) @ (p0 - c)
        assert np.allclose([x, y], exact, atol=1e-4)


def test_oracle_euler_single_step_is_paper_displacement_map():
    # Euler, one substep, dt = 1: (x, y) -> (x + u(x, y), y + v(x, y))
    import torch
    flow = W.fourier_flow(48, 48, 48, 48, rms=2.0, seed=5)
    pr = _adv_pair("euler", n=1, dt=1.0, H=48, Wd=48)
    rng = np.random.default_rng(2)
    pts = rng.uniform(0, 48, (50, 2))
    ft = torch.from_numpy(flow.astype(np.float64)).permute(2, 0, 1)[None]
    g = torch.from_numpy(np.stack([2 * pts[:, 0] / 48 - 1, 2 * pts[:, 1] / 48 - 1], 1))[None, None]
    uv = torch.nn.functional.grid_sample(ft, g, mode="bilinear", padding_mode="border",
                                         align_corners=False)[0, :, 0].numpy().T
    for (x, y), (u, v) in zip(pts, uv):
        xo, yo = oracle.advect(pr, flow, x, y)
        assert abs(xo - (x + u)) < 1e-12 and abs(yo - (y + v)) < 1e-12


def test_oracle_advect_lamb_oseen_preserves_radius():
    H = Wd = 256
    flow = W.lamb_oseen_flow(H, Wd, H, Wd)
    pr = _adv_pair("rk4", n=4, dt=1.0, H=H, Wd=Wd)
    for r0 in (10.0, 22.4, 40.0, 80.0):
        x, y = oracle.advect(pr, flow, 128 + r0, 128.0)
        r1 = math.hypot(x - 128, y - 128)
        # analytic angular speed of the vortex: Gamma / (2 pi r^2) (1 - exp(-r^2 / rc^2))
        om = 200.0 / (2 * math.pi * r0 * r0) * (1 - math.exp(-r0 * r0 / 400.0))
        assert abs(r1 - r0) < 2e-3
        assert abs(math.atan2(y - 128, x - 128) - om) < 2e-3


# ----------------------------------------------------------------------------
# splat: pixel integration of Eq. 1
# ----------------------------------------------------------------------------

def test_oracle_pixel_mass_matches_scipy_ndtr():
    rng = np.random.default_rng(3)
    for _ in range(300):
        c = rng.uniform(-3, 20)
        s = rng.uniform(0.2, 3)
        j = int(rng.integers(-4, 24))
        want = special.ndtr((j + 1 - c) / s) - special.ndtr((j - c) / s)
        got = oracle.pixel_mass(c, s, j)
        assert abs(got - want) < 1e-15 + 1e-12 * want


def test_oracle_isolated_particle_total_is_pi_d2_over_8():
    # the integrated particle image is pi d^2 / 8 * I0 (times the window mass
    # m^2 of the 3d+1 patch, m >= 1 - 4e-9)
    for x, y, d, I in ((40.3, 33.7, 2.5, 0.9), (50.0, 50.0, 4.0, 1.0), (20.61, 61.2, 1.0, 0.5)):
        S = oracle.splat(100, 100, np.array([[x, y, d, I]]))
        s = d / 4
        mx = special.ndtr((math.floor(x + 1.5 * d) + 1 - x) / s) - special.ndtr((math.floor(x - 1.5 * d) - x) / s)
        my = special.ndtr((math.floor(y + 1.5 * d) + 1 - y) / s) - special.ndtr((math.floor(y - 1.5 * d) - y) / s)
        assert abs(S.sum() - math.pi * d * d / 8 * I * mx * my) < 1e-12
        assert abs(S.sum() / (math.pi * d * d / 8 * I) - 1) < 1e-8


def _gauss_legendre_pixel_integral(x, y, d, I, H, Wd, n=48):
    # Eq. 1 with rho = 0, sigma_x = sigma_y = d / 4, integrated over each pixel
    # by tensor Gauss-Legendre quadrature (independent of erf)
    t, w = np.polynomial.legendre.leggauss(n)
    t = 0.5 * (t + 1)
    w = 0.5 * w
    s = d / 4
    out = np.zeros((H, Wd))
    gx = np.exp(-((np.arange(Wd)[:, None] + t[None, :] - x) ** 2) / (2 * s * s)) @ w
    gy = np.exp(-((np.arange(H)[:, None] + t[None, :] - y) ** 2) / (2 * s * s)) @ w
    out += I * np.outer(gy, gx)
    return out


def test_oracle_bruteforce_16x16_matches_window_and_quadrature():
    rng = np.random.default_rng(4)
    n = 12
    parts = np.stack([rng.uniform(-2, 18, n), rng.uniform(-2, 18, n), rng.uniform(1, 4, n),
                      rng.uniform(0.5, 1, n)], 1)
    win = oracle.splat(16, 16, parts, mode=0)
    brute = oracle.splat(16, 16, parts, mode=1)
    assert np.abs(win - brute).max() < 1e-8
    quad = sum(_gauss_legendre_pixel_integral(*p, 16, 16) for p in parts)
    assert np.abs(brute - quad).max() < 1e-11


def test_oracle_point_sampled_mode_is_eq1_at_pixel_centres():
    x, y, d, I = 7.3, 8.9, 3.0, 0.8
    S = oracle.splat(16, 16, np.array([[x, y, d, I]]), mode=2)
    jj, ii = np.meshgrid(np.arange(16), np.arange(16))
    s = d / 4
    ref = I * np.exp(-((jj + 0.5 - x) ** 2 + (ii + 0.5 - y) ** 2) / (2 * s * s))
    inside = (jj >= math.floor(x - 1.5 * d)) & (jj <= math.floor(x + 1.5 * d)) & \
             (ii >= math.floor(y - 1.5 * d)) & (ii <= math.floor(y + 1.5 * d))
    np.testing.assert_allclose(S, np.where(inside, ref, 0.0), atol=1e-15)


def test_oracle_splat_symmetry_and_separability():
    # x +- 1.5 d not an integer, so the window [floor(x - 1.5d), floor(x + 1.5d)]
    # is mirror-symmetric about the particle
    S = oracle.splat(21, 21, np.array([[10.5, 10.5, 2.9, 1.0]]))
    np.testing.assert_allclose(S, S[::-1, :], atol=1e-16)
    np.testing.assert_allclose(S, S[:, ::-1], atol=1e-16)
    np.testing.assert_allclose(S, S.T, atol=1e-16)
    # rank one (separable) for a single particle
    sv = np.linalg.svd(S, compute_uv=False)
    assert sv[1] < 1e-14 * sv[0]


def test_oracle_window_clip_at_image_border():
    # a particle partly outside loses exactly the mass of the clipped pixels
    S = oracle.splat(30, 30, np.array([[0.4, 15.2, 3.0, 1.0]]))
    s = 0.75
    mx = special.ndtr((math.floor(0.4 + 4.5) + 1 - 0.4) / s) - special.ndtr((0 - 0.4) / s)
    my = special.ndtr((math.floor(15.2 + 4.5) + 1 - 15.2) / s) - special.ndtr((math.floor(15.2 - 4.5) - 15.2) / s)
    assert abs(S.sum() - math.pi * 9 / 8 * mx * my) < 1e-12


# ----------------------------------------------------------------------------
# whole-pair invariants
# ----------------------------------------------------------------------------

def _spec(H=48, Wd=40, n=150, **kw):
    return W.PairSpec(height=H, width=Wd, n_particles=n, pair_id=kw.pop("pair_id", 2), **kw)


def test_oracle_zero_flow_frames_identical():
    spec = _spec(d_min=1.0, d_max=4.0, illum_min=0.7, illum_max=1.0, blur_sigma=0.7)
    pr = oracle.make_pair(spec, seed=5)
    out = oracle.render_pair(pr, W.zero_flow(48, 40))
    assert np.array_equal(out["S"][0], out["S"][1])
    assert np.array_equal(out["B"][0], out["B"][1])


@pytest.mark.parametrize("a,b", [(3, 0), (0, -2), (2, 5), (-4, -1)])
def test_oracle_integer_translation_shifts_frames_exactly(a, b):
    H, Wd = 64, 72
    spec = _spec(H, Wd, 400, d_min=1.0, d_max=4.0)
    for integ in ("rk4", "euler"):
        pr = oracle.make_pair(spec, seed=6, integrator=integ, n_substeps=4)
        S = oracle.render_pair(pr, W.uniform_flow(H, Wd, a, b))["S"]
        m = abs(a) + math.ceil(1.5 * 4) + 1, abs(b) + math.ceil(1.5 * 4) + 1
        i0, i1 = m[1], H - m[1]
        j0, j1 = m[0], Wd - m[0]
        s2 = S[1][i0:i1, j0:j1]
        s1 = S[0][i0 - b:i1 - b, j0 - a:j1 - a]
        assert np.array_equal(s2, s1)


def test_oracle_render_is_superposition_of_particles():
    spec = _spec(n=30, d_min=1.0, d_max=4.0)
    pr = oracle.make_pair(spec, seed=8)
    flow = W.fourier_flow(48, 40, 48, 40, rms=1.5, seed=3)
    out = oracle.render_pair(pr, flow, want_particles=True)
    t = out["parts"]
    for f, (cx, cy) in enumerate(((0, 1), (6, 7))):
        S = oracle.splat(48, 40, np.stack([t[:, cx], t[:, cy], t[:, 2], t[:, 5]], 1))
        np.testing.assert_allclose(out["S"][f], S, rtol=0, atol=1e-15)
        # positions of frame 2 are the advected positions
    for row in t[:5]:
        x1, y1 = oracle.advect(pr, flow, row[0], row[1])
        assert x1 == row[6] and y1 == row[7]


def test_oracle_no_particles_gives_blank_frames():
    pr = oracle.make_pair(_spec(n=0), seed=1)
    out = oracle.render_pair(pr, W.zero_flow(48, 40))
    assert not out["S"].any() and not out["B"].any()


# ----------------------------------------------------------------------------
# epilogue: illumination, blur, quantisation
# ----------------------------------------------------------------------------

def test_oracle_illumination_field_properties():
    H, Wd = 33, 45  # odd: a centre pixel exists
    pr = oracle.make_pair(_spec(H, Wd, 0, illum_min=0.7, illum_max=1.0), seed=0)
    L = np.array([[oracle.illumination(pr, i, j) for j in range(Wd)] for i in range(H)])
    lo, hi = float(np.float32(0.7)), 1.0
    assert L.min() >= lo and L.max() <= hi
    assert L[H // 2, Wd // 2] == pytest.approx(hi, abs=1e-15)
    np.testing.assert_allclose(L, L[::-1, ::-1], atol=1e-15)
    # mean of sin^2 over the midpoint grid is exactly 1/2 per axis
    assert L.mean() == pytest.approx(lo + (hi - lo) / 4, abs=1e-14)
    # the epilogue multiplies S by L (no noise / blur): constant S reproduces L
    B, _ = oracle.epilogue(pr, 0, np.ones((H, Wd)))
    np.testing.assert_allclose(B, L, atol=1e-15)


@pytest.mark.parametrize("sb", [0.7, 1.0, 1.6])
def test_oracle_blur_matches_scipy_gaussian_filter(sb):
    rng = np.random.default_rng(5)
    H, Wd = 23, 31
    S = rng.uniform(0, 1, (H, Wd))
    pr = oracle.make_pair(_spec(H, Wd, 0, blur_sigma=sb), seed=0)
    B, _ = oracle.epilogue(pr, 1, S)
    s = float(np.float32(sb))
    R = math.ceil(3 * s)
    assert oracle.blur_radius(s) == R
    ref = ndimage.gaussian_filter1d(S, s, axis=1, mode="nearest", truncate=R / s)
    ref = ndimage.gaussian_filter1d(ref, s, axis=0, mode="nearest", truncate=R / s)
    np.testing.assert_allclose(B, ref, atol=1e-14)
    # a constant image is unchanged
    B1, _ = oracle.epilogue(pr, 1, np.full((H, Wd), 0.37))
    np.testing.assert_allclose(B1, 0.37, atol=1e-15)


def test_oracle_noise_enters_additively_with_sigma():
    H, Wd = 64, 64
    pr = oracle.make_pair(_spec(H, Wd, 0, noise_sigma=0.02), seed=4)
    B, _ = oracle.epilogue(pr, 0, np.zeros((H, Wd)))
    n = np.array([oracle.noise(4, pr.pair_id, 0, p) for p in range(H * Wd)]).reshape(H, Wd)
    np.testing.assert_allclose(B, float(np.float32(0.02)) * n, atol=1e-16)
    assert abs(B.std() - 0.02) < 0.02 * 0.05


@pytest.mark.parametrize("bits", [8, 12, 16])
def test_oracle_quantisation_round_half_even_and_clamp(bits):
    # Q = clamp(round-half-even(B M), 0, M) on the FP64 value B.  The expected
    # codes are written from that definition with integers: a value a fixed
    # 1e-9 (in units of B M) above or below the boundary k + 1/2 must give
    # k + 1 or k.  The FP64 product is exact to ~1e-12 there, so the decision
    # is unambiguous in FP64; an FP32 decision (relative error 6e-8 of B M)
    # misrounds some of these and fails the test.
    M = 2 ** bits - 1
    ks = [0, 1, 2, 3, 100, M // 3, M // 2, M - 2, M - 1]
    delta = 1e-9
    above = np.array([(k + 0.5 + delta) / M for k in ks])
    below = np.array([(k + 0.5 - delta) / M for k in ks])
    want_above = [k + 1 for k in ks]
    want_below = [k for k in ks]
    # B = 1/2 is the one exact half step in [0, 1]: B M = (M - 1) / 2 + 1/2
    # exactly; (M - 1) / 2 = 2^(bits-1) - 1 is odd, so round-half-even picks
    # the upper neighbour 2^(bits-1).  Then zero, full scale and the clamps.
    special = np.array([0.5, 0.0, 1.0, -0.3, -1e-9, 1.2, 2.0, 1.0 + 0.4 / M, 1.0 - 0.4 / M])
    want_special = [2 ** (bits - 1), 0, M, 0, 0, M, M, M, M]
    n = len(ks)
    S = np.zeros((3, n))
    S[0], S[1], S[2] = above, below, special
    pr = oracle.make_pair(_spec(3, n, 0), seed=0, quant_bits=bits)
    B, Q = oracle.epilogue(pr, 0, S)
    assert np.array_equal(B, S)  # no illumination, noise or blur: B is S
    assert Q[0].tolist() == want_above
    assert Q[1].tolist() == want_below
    assert Q[2].tolist() == want_special
    # the same values decided in FP32 disagree somewhere: the test tells the two apart
    f32 = np.clip(np.rint(S[:2].astype(np.float32) * np.float32(M)), 0, M).astype(np.int64)
    assert (f32 != np.array([want_above, want_below])).any()
