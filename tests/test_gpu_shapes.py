"""CUDA path vs the FP64 oracle for the shape options of Eq. 1: general
particles (sigma_x != sigma_y, rho != 0), frame-2 parameter variation and
hiding (Section 2, text after Eq. 1 and the aggregation paragraph).

Same tolerances as the other parity tests: float images within 1e-4 of full
scale, quantised codes bit-exact away from the 1e-6 rounding band.  Hiding
decisions compare a 24-bit uniform with hide_prob on both sides, so they
agree exactly; a disagreement would move a whole particle image and fail the
float tolerance.
"""
import numpy as np
import pytest

from paper_2512_09664_b300 import workloads as W

from parity import compare, gpu_render, oracle_render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")


def _wl(pairs, flows, seed=7, **kw):
    return W.Workload(name="t", seed=seed, pairs=pairs, flows=flows, **kw)


def _spec(H, Wd, n, **kw):
    args = dict(height=H, width=Wd, n_particles=n, pair_id=0, d_min=1.0, d_max=4.0)
    args.update(kw)
    return W.PairSpec(**args)


FLOW = W.fourier_flow(96, 136, 96, 136, rms=2.5, seed=31)


@pytest.mark.parametrize("tile", [16, 32, 64, 128])
def test_general_shapes_float(tile):
    p = _spec(96, 136, 650, dy_min=1.0, dy_max=5.0, rho_min=-0.8, rho_max=0.8)
    wl = _wl([p], [FLOW])
    st = compare(wl, gpu_render(wl, tile=tile), oracle_render(wl))
    print("general float", tile, st)
    assert st["max_abs"] < 2e-6


def test_axis_aligned_elliptical_float():
    # rho = 0: separable pixel masses with sigma_x != sigma_y
    p = _spec(96, 136, 650, dy_min=2.0, dy_max=6.0)
    wl = _wl([p], [FLOW])
    st = compare(wl, gpu_render(wl, tile=32), oracle_render(wl))
    assert st["max_abs"] < 2e-6


def test_round_correlated_fixed_rho():
    # d_y = d but rho fixed at 0.9 (a 45-degree ellipse); small particles
    # need the most quadrature sub-intervals
    p = _spec(64, 80, 300, rho_min=0.9, rho_max=0.9, d_min=1.0, d_max=1.5)
    wl = _wl([p], [W.fourier_flow(64, 80, 64, 80, rms=2.0, seed=3)])
    st = compare(wl, gpu_render(wl, tile=32), oracle_render(wl))
    assert st["max_abs"] < 2e-6


@pytest.mark.parametrize("p_hide", [0.0, 0.3, 1.0])
def test_hiding_round_particles(p_hide):
    p = _spec(96, 136, 650)
    wl = _wl([p], [FLOW], hide_prob=p_hide)
    g = gpu_render(wl, tile=32)
    st = compare(wl, g, oracle_render(wl))
    if p_hide == 1.0:
        assert all(np.all(x == 0) for x in g)
    print("hide", p_hide, st)


def test_frame2_variation_round_particles():
    p = _spec(96, 136, 650, jitter_d=0.3, jitter_i=0.1)
    wl = _wl([p], [FLOW])
    compare(wl, gpu_render(wl, tile=64), oracle_render(wl))


def test_zero_flow_general_frames_identical():
    p = _spec(64, 72, 200, dy_min=1.0, dy_max=3.0, rho_min=-0.5, rho_max=0.5)
    wl = _wl([p], [W.zero_flow(64, 72)])
    g = gpu_render(wl, tile=32)[0]
    assert np.array_equal(g[0], g[1])
    compare(wl, [g], oracle_render(wl))


def test_shapes_batch_u8_epilogue_all_options():
    wl = W.shapes_batch(n_pairs=2, size=192)
    for tile in (32, 64, 128):
        st = compare(wl, gpu_render(wl, tile=tile), oracle_render(wl))
        print("shapes u8", tile, st)


def test_shapes_batch_round_u8():
    wl = W.shapes_batch(n_pairs=2, size=192, general=False, hide_prob=0.1)
    st = compare(wl, gpu_render(wl), oracle_render(wl))
    print("shapes round u8", st)


def test_general_shapes_fp16_intermediates():
    # 16-bit intermediate frames: compared as in the precision tests (max / RMS in LSB)
    wl = W.shapes_batch(n_pairs=2, size=128)
    wl.out_dtype, wl.quant_bits = "u16", 16
    g = gpu_render(wl, tile=32, inter_dtype="f16")
    ref = oracle_render(wl)
    err = np.concatenate([(gg.astype(np.float64) - r["Q"].astype(np.float64)).ravel() for gg, r in zip(g, ref)])
    lsb_max, lsb_rms = float(np.abs(err).max()), float(np.sqrt(np.mean(err ** 2)))
    print("general f16 intermediates: max", lsb_max, "rms", lsb_rms, "LSB")
    assert lsb_max <= 64 and lsb_rms <= 4.0


def test_render_is_independent_of_tile_and_batch():
    # exact fixed-point sums: the same pair renders bit-identically at every
    # tile edge and alone or inside a batch
    wl = W.shapes_batch(n_pairs=3, size=160)
    ref = gpu_render(wl, tile=32)
    for tile in (16, 64, 128):
        g = gpu_render(wl, tile=tile)
        assert all(np.array_equal(a, b) for a, b in zip(g, ref))
    one = gpu_render(wl.subset([1]), tile=64)[0]
    assert np.array_equal(one, ref[1])


def test_general_dense_overlap_and_carries():
    # general shapes with sums above 64 i_max: the checked adds and carries of the general splat
    p = _spec(32, 32, 3000, d_min=8.0, d_max=10.0, dy_min=6.0, dy_max=12.0, rho_min=-0.5, rho_max=0.5,
              sheet_sigma=0.0)
    wl = _wl([p], [W.zero_flow(32, 32)])
    ref = oracle_render(wl)
    assert ref[0]["S"].max() > 64.0
    outs = [gpu_render(wl, tile=t) for t in (16, 32, 128)]
    st = compare(wl, outs[0], ref)
    print("general carries", st, "max S", float(ref[0]["S"].max()))
    assert all(np.array_equal(outs[0][0], o[0]) for o in outs[1:])


def test_general_wide_windows_both_paths():
    # windows wider than the lanes' edge budget (separable fallback) and many
    # quadrature columns (correlated), large and thin particles mixed
    for rho in ((0.0, 0.0), (-0.9, 0.9)):
        p = _spec(96, 120, 120, d_min=2.0, d_max=14.0, dy_min=0.6, dy_max=20.0, rho_min=rho[0], rho_max=rho[1])
        wl = _wl([p], [W.fourier_flow(96, 120, 96, 120, rms=2.0, seed=5)])
        st = compare(wl, gpu_render(wl, tile=32), oracle_render(wl))
        print("wide", rho, st)
        assert st["max_abs"] < 4e-6


def test_general_batch_with_empty_and_tiny_pairs():
    flows = [W.fourier_flow(40, 56, 40, 56, rms=1.5, seed=6), W.fourier_flow(9, 7, 9, 7, rms=1.0, seed=7)]
    pairs = [_spec(40, 56, 0, dy_min=1.0, dy_max=3.0, rho_min=0.2, rho_max=0.2),
             _spec(9, 7, 5, pair_id=1, flow_index=1, dy_min=1.0, dy_max=3.0, rho_min=-0.3, rho_max=0.3),
             _spec(40, 56, 90, pair_id=2, dy_min=1.0, dy_max=3.0, rho_min=-0.3, rho_max=0.3)]
    wl = _wl(pairs, flows, hide_prob=0.2)
    for tile in (16, 64):
        compare(wl, gpu_render(wl, tile=tile), oracle_render(wl))
