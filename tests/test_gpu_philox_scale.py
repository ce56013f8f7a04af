"""Philox4x32-10 streams of the GPU against the oracle at scale.

* Particle stream: the full headline batch (64 pairs of 512 x 512, 13107
  particles each, 838 848 particles, two Philox calls = 8 words per
  particle) exported by synthpix_seed_particles.  With a power-of-two frame
  x0 = u24 W and y0 = u24 H are exact in FP32, so they must equal the
  oracle's bit for bit; d (one FP32 multiply-add of the interval) within
  2e-7 relative.
* Noise stream: 64 noise-only pairs (no particles, noise sigma 1, no
  illumination or blur, FP32 output): every pixel is one Box-Muller value of
  its Philox words, 33.5 M words in all; each must match the oracle's FP64
  value within the FP32 Box-Muller error bound (hardware log2 and sine,
  below 2e-6 on the deviate; asserted at 5e-6).
"""
import numpy as np
import pytest

import oracle
from paper_2512_09664_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")


def test_particle_stream_full_headline_batch_bit_exact():
    from paper_2512_09664_b300.binding import Renderer
    wl = W.batch_512_u8(n_pairs=64, seed=1)
    r = Renderer(wl)
    parts = r.seed_particles().cpu().numpy().astype(np.float64)
    assert parts.shape[0] == 64 * 13107
    off, words = 0, 0
    for b, spec in enumerate(wl.pairs):
        ref = oracle.particles(oracle.pair_from_workload(wl, b), wl.flows[spec.flow_index])
        got = parts[off:off + spec.n_particles]
        np.testing.assert_array_equal(got[:, :2], ref[:, :2])
        np.testing.assert_allclose(got[:, 2], ref[:, 2], rtol=2e-7)
        off += spec.n_particles
        words += 8 * spec.n_particles
    assert words >= 6_000_000


def test_noise_stream_every_pixel_of_64_frames_pairs():
    import torch

    from paper_2512_09664_b300.binding import Renderer
    pairs = [W.PairSpec(height=512, width=512, n_particles=0, pair_id=1000 + b, flow_index=0,
                        noise_sigma=1.0) for b in range(64)]
    wl = W.Workload(name="noise", seed=77, pairs=pairs, flows=[W.zero_flow(4, 4)], out_dtype="f32", quant_bits=0)
    r = Renderer(wl)
    r.render()
    torch.cuda.synchronize()
    ref = oracle.render_workload(wl)
    n, worst = 0, 0.0
    for b in range(wl.n_pairs):
        g = r.frames(b).cpu().numpy().astype(np.float64)
        err = np.abs(g - ref[b]["B"])
        worst = max(worst, float(err.max()))
        n += g.size
        # a standard normal sample: mean and variance within their sampling error
        assert abs(g.mean()) < 5 * (1.0 / np.sqrt(g.size)) and abs(g.var() - 1.0) < 5 * np.sqrt(2.0 / g.size)
    print("noise words", n, "max |gpu - oracle|", worst)
    assert n >= 10_000_000
    assert worst < 5e-6
