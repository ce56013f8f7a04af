"""CUDA path vs the oracle for the out-of-focus intensity of the Remark form
and out-of-plane motion (a w grid moving z along the particle path)."""
import dataclasses

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


def _wl(**kw):
    H, Wd = 96, 136
    flows = [W.fourier_flow(H, Wd, H, Wd, rms=2.5, seed=41)]
    spec = W.PairSpec(height=H, width=Wd, n_particles=650, pair_id=0, d_min=1.0, d_max=4.0, sheet_sigma=0.5,
                      **kw.pop("spec", {}))
    return W.Workload(name="t", seed=9, pairs=[spec], flows=flows, **kw)


def _wgrid(scale, seed=43):
    g = W.fourier_flow(96, 136, 96, 136, rms=1.0, seed=seed)[..., 0]
    return (g * scale).astype(np.float32)


@pytest.mark.parametrize("s", [0.7, 2.0])
def test_remark_sheet_float(s):
    wl = _wl(spec=dict(sheet_model=1, sheet_shape=s))
    st = compare(wl, gpu_render(wl, tile=32), oracle_render(wl))
    assert st["max_abs"] < 2e-6


@pytest.mark.parametrize("integ,n", [("rk4", 4), ("euler", 1)])
def test_out_of_plane_motion_float(integ, n):
    wl = _wl(flows_w=[_wgrid(0.3)], integrator=integ, n_substeps=n, spec=dict(sheet_model=1, sheet_shape=2.0))
    st = compare(wl, gpu_render(wl, tile=64), oracle_render(wl))
    print("out of plane", integ, st)
    assert st["max_abs"] < 2e-6


def test_zero_w_renders_as_without_out_of_plane_motion():
    a = _wl()
    b = _wl(flows_w=[np.zeros((96, 136), np.float32)])
    ga, gb = gpu_render(a, tile=32)[0], gpu_render(b, tile=32)[0]
    assert np.array_equal(ga, gb)


def test_focus_batch_u8_epilogue():
    wl = W.focus_batch(n_pairs=2, size=160)
    for tile in (32, 128):
        st = compare(wl, gpu_render(wl, tile=tile), oracle_render(wl))
        print("focus u8", tile, st)
