"""Pins of the oracle's out-of-focus intensity (Remark "out-of-focus") and
out-of-plane motion: closed forms, reduction to the Gaussian sheet, and
exactly integrable fields."""
import math

import numpy as np
import pytest

import oracle
from paper_2512_09664_b300 import workloads as W


def _pair(**kw):
    base = dict(height=48, width=64, n_particles=150, pair_id=2, d_min=1.0, d_max=4.0, sheet_sigma=0.5)
    base.update(kw)
    return W.PairSpec(**base)


@pytest.mark.parametrize("s", [0.5, 1.0, 2.0, 4.0])
def test_remark_gain_closed_form(s):
    pr = oracle.make_pair(_pair(sheet_model=1, sheet_shape=s, sheet_sigma=0.8), seed=1)
    dz0 = float(np.float32(0.8))
    for z in (0.0, 0.1, -0.3, 0.8, 1.5):
        want = math.exp(-abs(2 * z * z / dz0 ** 2) ** s / math.sqrt(2 * math.pi))
        assert abs(oracle.sheet_gain(pr, z) - want) < 1e-15
    assert oracle.sheet_gain(pr, 0.0) == 1.0
    assert oracle.sheet_gain(pr, 0.37) == oracle.sheet_gain(pr, -0.37)


def test_remark_shape_one_is_a_gaussian_sheet():
    # s = 1: exp(-2 z^2 / (dz0^2 sqrt(2 pi))) = exp(-z^2 / (2 sigma^2)) with sigma^2 = dz0^2 sqrt(2 pi) / 4
    dz0 = 0.75
    sig = math.sqrt(dz0 ** 2 * math.sqrt(2 * math.pi) / 4)
    rem = oracle.make_pair(_pair(sheet_model=1, sheet_shape=1.0, sheet_sigma=dz0), seed=1)
    gau = oracle.make_pair(_pair(sheet_sigma=sig), seed=1)
    for z in np.linspace(-2, 2, 9):
        assert abs(oracle.sheet_gain(rem, z) - math.exp(-z * z / (2 * gau.sheet_sigma ** 2))) < 1e-6


def test_remark_shape_factor_flattens_the_top():
    a = oracle.make_pair(_pair(sheet_model=1, sheet_shape=1.0), seed=1)
    b = oracle.make_pair(_pair(sheet_model=1, sheet_shape=4.0), seed=1)
    inner, outer = 0.2, 0.6  # 2 z^2 / dz0^2 below / above 1
    assert oracle.sheet_gain(b, inner) > oracle.sheet_gain(a, inner)
    assert oracle.sheet_gain(b, outer) < oracle.sheet_gain(a, outer)


def test_particle_intensity_uses_the_sheet_model():
    spec = _pair(sheet_model=1, sheet_shape=2.0, sheet_sigma=0.6, z_min=-1.0, z_max=1.0)
    pr = oracle.make_pair(spec, seed=4)
    t = oracle.particles(pr, W.zero_flow(48, 64))
    for row in t[:20]:
        assert abs(row[5] - row[3] * oracle.sheet_gain(pr, row[4])) < 1e-15


def test_scalar_grid_is_the_flow_bilinear():
    rng = np.random.default_rng(0)
    w = rng.normal(size=(13, 17)).astype(np.float32)
    flow = np.stack([w, np.zeros_like(w)], axis=-1)
    for x, y in rng.uniform(-5, 70, size=(30, 2)):
        assert oracle.scalar_at(w, 48, 64, x, y) == oracle.velocity(flow, 48, 64, x, y)[0]


def test_advect3_positions_match_advect_and_depth_is_exact():
    # w = c x on a uniform in-plane flow (a, b): z(t) = z0 + c (x0 t + a t^2 / 2), which RK4 integrates exactly
    H, Wd = 48, 64
    a, b, c = 1.25, -0.5, 0.01
    flow = W.uniform_flow(H, Wd, a, b)
    xs, _ = W.node_centres(H, Wd, H, Wd)
    w = np.tile((c * xs)[None, :], (H, 1)).astype(np.float32)
    for integ, n in (("rk4", 4), ("rk4", 1), ("euler", 1)):
        pr = oracle.make_pair(_pair(), seed=1, integrator=integ, n_substeps=n, dt=2.0)
        x0, y0, z0 = 20.3, 24.1, 0.2
        x1, y1, z1 = oracle.advect3(pr, flow, w, x0, y0, z0)
        assert (x1, y1) == oracle.advect(pr, flow, x0, y0)
        cw = float(np.float32(c * xs[1])) / xs[1]  # the stored node values carry FP32 rounding
        want = z0 + c * (x0 * 2.0 + a * 2.0 ** 2 / 2) if integ == "rk4" else z0 + 2.0 * float(
            oracle.scalar_at(w, H, Wd, x0, y0))
        assert abs(z1 - want) < 1e-6 * (1 + abs(cw))


def test_render_zero_w_equals_render_without_and_large_w_empties_frame2():
    spec = _pair(n_particles=200, noise_sigma=0.0, z_min=-0.2, z_max=0.2)
    flow = W.fourier_flow(48, 64, 48, 64, rms=1.0, seed=3)
    pr = oracle.make_pair(spec, seed=6)
    base = oracle.render_pair(pr, flow)
    zero = oracle.render_pair(pr, flow, wgrid=np.zeros((48, 64), np.float32))
    assert np.allclose(base["S"], zero["S"], rtol=0, atol=1e-13)
    far = oracle.render_pair(pr, flow, wgrid=np.full((48, 64), 5.0, np.float32))  # 5 sheet widths per frame
    assert np.allclose(far["S"][0], base["S"][0], rtol=0, atol=1e-13)  # general vs separable splat rounding
    assert far["S"][1].max() < 1e-20 * base["S"][1].max()


# ----------------------------------------------------------------------------
# intensity-histogram matching of quantised frames
# ----------------------------------------------------------------------------

def _match_fractions(codes, n_codes, target):
    """Brute force with exact rationals: code c -> min t with C_t(t)/T >= C_s(c)/N."""
    from fractions import Fraction
    N, T = codes.size, int(sum(int(x) for x in target))
    hs = np.bincount(codes, minlength=n_codes)
    cs, out = 0, {}
    for c in range(n_codes):
        cs += int(hs[c])
        p = Fraction(cs, N)
        ct = 0
        for t in range(n_codes):
            ct += int(target[t])
            if Fraction(ct, T) >= p:
                break
        out[c] = t
    return np.array([out[c] for c in codes], dtype=np.uint32)


@pytest.mark.parametrize("n_codes,seed", [(16, 0), (256, 1), (64, 2)])
def test_histogram_matching_equals_exact_quantile_mapping(n_codes, seed):
    rng = np.random.default_rng(seed)
    codes = np.minimum(rng.gamma(2.0, n_codes / 8, size=3000).astype(np.int64), n_codes - 1).astype(np.uint32)
    target = rng.integers(0, 50, size=n_codes).astype(np.uint64)
    target[rng.integers(0, n_codes)] += 1  # non-empty
    got = oracle.match_histogram(codes, n_codes, target)
    assert np.array_equal(got, _match_fractions(codes, n_codes, target))


def test_histogram_matching_properties():
    rng = np.random.default_rng(5)
    n_codes = 256
    codes = rng.integers(0, 200, size=5000).astype(np.uint32)
    # identity when the target is the frame's own histogram
    own = np.bincount(codes, minlength=n_codes).astype(np.uint64)
    assert np.array_equal(oracle.match_histogram(codes, n_codes, own), codes)
    # monotone mapping, and the output follows the target's CDF within one source bin
    target = np.exp(-np.arange(n_codes) / 30.0) * 1000
    target = target.astype(np.uint64) + 1
    out = oracle.match_histogram(codes, n_codes, target)
    order = np.argsort(codes, kind="stable")
    assert np.all(np.diff(out[order].astype(np.int64)) >= 0)
    cdf_out = np.cumsum(np.bincount(out, minlength=n_codes)) / codes.size
    cdf_t = np.cumsum(target) / target.sum()
    max_bin = np.bincount(codes).max() / codes.size
    assert np.all(cdf_out >= cdf_t - max_bin - 1e-12)
