"""16-bit intermediate storage (FP16 / BF16 splatted frames, exact fixed-point
accumulation inside each tile) against the FP64 oracle.

The intermediate S is rounded once to the storage type (relative error at most
2^-11 for FP16, 2^-8 for BF16).  Illumination (L <= 1) and the normalised blur
are convex, so |B - B_oracle| <= 1e-4 + u * max(S) with u the storage unit
roundoff; the measured max and RMS errors are printed.
"""
import numpy as np
import pytest

from paper_2512_09664_b300 import workloads as W

from parity import gpu_render, oracle_render

pytestmark = pytest.mark.gpu

UNIT = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")


def _mixed(inter):
    # a reduced large-mixed batch: dense small tracers and sparse large tracers
    flows = [W.fourier_flow(256, 256, 256, 256, rms=8.0, seed=4000),
             W.fourier_flow(135, 240, 135, 240, rms=8.0, seed=4100)]
    pairs = [W.PairSpec(height=256, width=256, n_particles=W.n_particles_for(0.1, 256, 256), pair_id=0,
                        flow_index=0, d_min=1.0, d_max=4.0, illum_min=0.7, illum_max=1.0, noise_sigma=0.02,
                        blur_sigma=0.7),
             W.PairSpec(height=135, width=240, n_particles=W.n_particles_for(0.002, 135, 240) + 20, pair_id=1,
                        flow_index=1, d_min=4.0, d_max=10.0, illum_min=0.7, illum_max=1.0, noise_sigma=0.02,
                        blur_sigma=0.7)]
    return W.Workload(name="mixed_small", seed=4, pairs=pairs, flows=flows, out_dtype="f32", quant_bits=0,
                      inter_dtype=inter)


@pytest.mark.parametrize("inter", ["f16", "bf16"])
def test_16bit_intermediate_float_output_error_bound(inter):
    wl = _mixed(inter)
    ref = oracle_render(wl)
    for tile in (32, 64):
        g = gpu_render(wl, tile=tile)
        for b, (gi, r) in enumerate(zip(g, ref)):
            err = np.abs(gi.astype(np.float64) - r["B"])
            bound = 1e-4 + UNIT[inter] * r["S"].max()
            print(f"{inter} tile {tile} pair {b}: max {err.max():.3e} rms {np.sqrt((err ** 2).mean()):.3e} "
                  f"bound {bound:.3e}")
            assert err.max() <= bound


@pytest.mark.parametrize("inter", ["f16", "bf16"])
def test_16bit_intermediate_16bit_codes(inter):
    wl = _mixed(inter)
    wl.out_dtype, wl.quant_bits = "u16", 16
    ref = oracle_render(wl)
    g = gpu_render(wl)
    M = 65535.0
    for gi, r in zip(g, ref):
        d = np.abs(gi.astype(np.int64) - r["Q"].astype(np.int64))
        lim = int(np.ceil((1e-4 + UNIT[inter] * r["S"].max()) * M)) + 1
        print(f"{inter}: max code error {d.max()} LSB, rms {np.sqrt((d ** 2).mean()):.2f} LSB (limit {lim})")
        assert d.max() <= lim


def test_f32_fused_and_16bit_paths_agree_with_each_other():
    wl = _mixed("f32")
    a = gpu_render(wl)
    wl.inter_dtype = "f16"
    b = gpu_render(wl)
    for x, y in zip(a, b):
        assert np.abs(x - y).max() < 2.0 ** -10 * 4
