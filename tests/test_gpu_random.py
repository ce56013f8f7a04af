"""Randomised parity: seeded small configurations across the option space.

Each case draws frame sizes (ragged, down to one pixel), particle counts
(zero included), diameter ranges, blur, noise, illumination, output type,
integrator, substeps, dt, flow-grid resolution (one node up to finer than
the frame), general shapes, frame-2 variation, hiding, the sheet model,
out-of-plane motion and the tile edge,
and compares the CUDA path with the oracle element by element.
"""
import numpy as np
import pytest

from paper_2512_09664_b300 import workloads as W

from parity import compare, gpu_render, oracle_render

pytestmark = pytest.mark.gpu

F32 = np.float32


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")


def _case(seed: int):
    rng = np.random.default_rng(seed)
    general = rng.random() < 0.35
    variation = rng.random() < 0.3
    n_pairs = int(rng.integers(1, 4))
    pairs, flows = [], []
    for b in range(n_pairs):
        H, Wd = int(rng.integers(1, 91)), int(rng.integers(1, 91))
        gh, gw = int(rng.integers(1, H + 11)), int(rng.integers(1, Wd + 11))
        flows.append(W.fourier_flow(gh, gw, H, Wd, rms=float(rng.uniform(0.0, 4.0)), seed=seed * 7 + b))
        d_min = float(rng.uniform(0.6, 6.0))
        kw = dict(height=H, width=Wd, n_particles=int(round(rng.uniform(0.0, 0.1) * H * Wd)), pair_id=b,
                  flow_index=b, d_min=F32(d_min), d_max=F32(d_min + rng.uniform(0.0, 6.0)),
                  illum_min=F32(rng.uniform(0.6, 1.0)), illum_max=F32(1.0),
                  noise_sigma=F32(rng.choice([0.0, 0.02])), blur_sigma=F32(rng.choice([0.0, 0.5, 1.3, 2.6])))
        if general:
            dy = float(rng.uniform(0.6, 4.0))
            r0 = float(rng.uniform(-0.9, 0.9))
            kw.update(dy_min=F32(dy), dy_max=F32(dy + rng.uniform(0.0, 4.0)), rho_min=F32(min(r0, 0.0)),
                      rho_max=F32(max(r0, 0.0)))
        if variation:
            kw.update(jitter_d=F32(rng.uniform(0.0, 0.3)), jitter_i=F32(rng.uniform(0.0, 0.1)))
        pairs.append(W.PairSpec(**kw))
    # the out-of-focus sheet and out-of-plane motion, from a stream of their own
    xr = np.random.default_rng(10_000 + seed)
    if xr.random() < 0.3:
        for p in pairs:
            p.sheet_model, p.sheet_shape = 1, F32(xr.uniform(1.0, 3.0))
    flows_w = None
    if xr.random() < 0.3:
        flows_w = [xr.normal(0.0, 0.2, size=f.shape[:2]).astype(np.float32) for f in flows]
    out = str(rng.choice(["f32", "u8", "u16", "f16", "bf16"]))
    bits = {"u8": 8, "u16": int(rng.choice([10, 12, 16]))}.get(out, 0)
    wl = W.Workload(name=f"random{seed}", seed=1000 + seed, pairs=pairs, flows=flows, out_dtype=out,
                    quant_bits=bits, integrator=str(rng.choice(["rk4", "euler"])),
                    n_substeps=int(rng.integers(1, 5)), dt=F32(rng.uniform(0.5, 1.5)),
                    hide_prob=F32(rng.uniform(0.0, 0.3)) if variation else F32(0.0), flows_w=flows_w)
    tile = int(rng.choice([16, 32, 64, 128]))
    return wl, tile


@pytest.mark.parametrize("seed", range(32))
def test_random_configuration_matches_oracle(seed):
    wl, tile = _case(seed)
    compare(wl, gpu_render(wl, tile=tile), oracle_render(wl))
