"""The three advection and binning paths of a seeded render: per particle
while seeding with fixed-capacity bins (the default), tile by tile from flow
nodes staged on chip (TILED_ADVECT), and per particle with a counting sort
(GATHER_ADVECT).  The lookups use the same nodes and arithmetic and the
splat's sums are exact, so whole batches must render bit-identically, including
flows coarser and finer than the image, displacements that leave the
staged window and the frame-2 tile neighbourhood, Euler and RK4, and all
tile edges.  One case is also compared with the FP64 oracle."""
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


def _both(wl, tile):
    """The default render and the gather render; the tiled render must equal the default."""
    import torch

    from paper_2512_09664_b300.binding import FLAG_GATHER_ADVECT, FLAG_TILED_ADVECT, Renderer
    a = Renderer(wl, tile=tile).render().clone()
    t = Renderer(wl, tile=tile, flags=FLAG_TILED_ADVECT).render().clone()
    b = Renderer(wl, tile=tile, flags=FLAG_GATHER_ADVECT).render().clone()
    torch.cuda.synchronize()
    assert torch.equal(a, t), ("tiled", wl.pairs[0].height, tile)
    return a, b


def _workload(size, grid, rms, integ="rk4", n_sub=4, n_pairs=3, ppp=0.05, seed=21):
    flows = [W.fourier_flow(grid[0], grid[1], size[0], size[1], rms=rms, seed=seed + b) for b in range(n_pairs)]
    pairs = [W.PairSpec(height=size[0], width=size[1], n_particles=W.n_particles_for(ppp, *size), pair_id=b,
                        flow_index=b, illum_min=0.7, illum_max=1.0, noise_sigma=0.02, blur_sigma=0.7)
             for b in range(n_pairs)]
    return W.Workload(name="adv", seed=seed, pairs=pairs, flows=flows, out_dtype="f32", quant_bits=0,
                      integrator=integ, n_substeps=n_sub, dt=1.0)


@pytest.mark.parametrize("tile", [16, 32, 64, 128])
def test_tiled_and_gather_advection_render_identically(tile):
    import torch
    cases = [
        _workload((200, 296), (200, 296), rms=3.0),               # grid = image
        _workload((256, 256), (40, 56), rms=6.0, integ="euler", n_sub=3),  # coarser grid
        _workload((128, 160), (256, 320), rms=2.0),               # finer grid: window larger than staged
        _workload((256, 256), (256, 256), rms=40.0, n_sub=8),     # leaves the window and the +-3 tile band
    ]
    for wl in cases:
        a, b = _both(wl, tile)
        assert torch.equal(a, b), (wl.pairs[0].height, tile)


def test_tiled_advection_batch_512_u8_identical_and_matches_oracle():
    import torch
    wl = W.batch_512_u8(n_pairs=4)
    a, b = _both(wl, 64)
    assert torch.equal(a, b)
    compare(wl, gpu_render(wl), oracle_render(wl))


def test_batch_of_more_chunks_than_one_wave_renders_identically():
    # 12 pairs of 13 107 particles: 312 chunks of 512, more than two per SM, so
    # the seeding kernel runs two particles a thread (one a thread below that)
    import torch
    wl = W.batch_512_u8(n_pairs=12)
    n_chunks = sum(-(-p.n_particles // 512) for p in wl.pairs)
    assert n_chunks > 2 * torch.cuda.get_device_properties(0).multi_processor_count
    a, b = _both(wl, 128)
    assert torch.equal(a, b)
