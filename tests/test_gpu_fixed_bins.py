"""Fixed-capacity bins of seeded renders and the exact rebinning after an
overflow, on the GPU.

Seeded renders place each record straight into a bin of fixed capacity
while seeding and advecting each particle (both frames; with TILED_ADVECT,
frame 1 while seeding and frame 2 in the tiled advection).  A bin that overflows
flags its frame, and k_rebin then bins the frame again exactly.  The splat
sums in exact fixed point, so the record order in a bin does not matter and
both layouts must give bit-identical frames:

* libsynthpix_smallbins.so is built from the same sources with bins of half
  the expected count, so nearly every bin of both frames overflows there;
  its renders must equal the product library's bit for bit;
* a converging flow overflows frame 2 in the product library itself (the
  count it piles into the centre tile, from the oracle's positions, exceeds
  the bin capacity); that render must match the oracle;
* frame-1 bins of more records than the tiled advection examines per pass
  (a dense 1024^2 pair at tile 128) place frame 2 over several passes; the
  render must equal the undersized-bin library's exact rebinning.
"""
import contextlib
import os

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


@contextlib.contextmanager
def _library(path):
    """Route the binding's calls to another build of the library."""
    from paper_2512_09664_b300 import binding as B
    saved = (B.LIB_PATH, B._lib)
    B.LIB_PATH, B._lib = path, None
    try:
        yield
    finally:
        B.LIB_PATH, B._lib = saved


def _smallbins_path():
    from paper_2512_09664_b300 import build
    if not os.path.exists(build.SMALLBINS_LIB):
        pytest.fail(f"{build.SMALLBINS_LIB} is missing: python -m paper_2512_09664_b300.build")
    return build.SMALLBINS_LIB


def _window_max(d_max):
    return int(np.floor(3.0 * float(d_max))) + 5


def _cap2(p, tile, halo):
    """The frame-2 bin capacity of the library's fixed layout (integer arithmetic)."""
    reach = tile + 2 * halo + _window_max(max(p.d_max, p.dy_max))
    sx, sy = min(reach, p.width), min(reach, p.height)
    e = (p.n_particles * sx * sy + p.width * p.height - 1) // (p.width * p.height)
    ntiles = -(-p.width // tile) * -(-p.height // tile)
    if p.n_particles * ntiles <= 1 << 16:  # small pairs: capacity N, no overflow
        return p.n_particles
    return min(e + e // 2 + 64, p.n_particles)


@pytest.mark.parametrize("out,tile,tiled,n_pairs", [("u8", 128, False, 3), ("u8", 64, False, 3),
                                                    ("f32", 128, False, 3), ("u8", 128, False, 12),
                                                    ("u8", 128, True, 3), ("u8", 32, True, 3)])
def test_overflowing_bins_render_the_same_bits(out, tile, tiled, n_pairs):
    # 12 pairs: more seeding chunks than one wave (two particles a thread)
    import torch

    from paper_2512_09664_b300.binding import FLAG_TILED_ADVECT, Renderer
    wl = W.batch_512_u8(n_pairs=n_pairs)
    if out == "f32":
        wl.out_dtype, wl.quant_bits = "f32", 0
    flags = FLAG_TILED_ADVECT if tiled else 0
    ref = Renderer(wl, tile=tile, flags=flags).render().clone()
    torch.cuda.synchronize()
    with _library(_smallbins_path()):
        got = Renderer(wl, tile=tile, flags=flags).render().clone()
        torch.cuda.synchronize()
    assert torch.equal(got, ref)
    assert int((ref != 0).sum()) > 0


def test_converging_flow_overflows_frame2_and_matches_the_oracle():
    import oracle

    h = w = 256
    tile = 64
    # (u, v) = -(p - c), c the middle of tile (2, 2): RK4 over dt = 1 contracts distances to c by
    # about e^-1, so the tile receives the particles of a 174 px square around it (up to 100 px away)
    c = 2.5 * tile
    flow = W.linear_flow(h, w, h, w, [[-1.0, 0.0], [0.0, -1.0]], (c, c))
    pair = W.PairSpec(height=h, width=w, n_particles=W.n_particles_for(0.08, h, w), pair_id=7,
                      d_dist=0, d_min=1.0, d_max=3.0, noise_sigma=0.02, blur_sigma=0.7,
                      illum_min=0.8, illum_max=1.0)
    wl = W.Workload(name="converging_256", seed=11, pairs=[pair], flows=[flow], out_dtype="u8", quant_bits=8)
    # the precondition: the centre tile's frame-2 bin holds more records than fit
    parts = oracle.particles(oracle.pair_from_workload(wl, 0), flow)
    x1, y1 = parts[:, 6], parts[:, 7]
    t0 = 2 * tile
    inside = int(((x1 >= t0) & (x1 < t0 + tile) & (y1 >= t0) & (y1 < t0 + tile)).sum())
    halo = int(np.ceil(3.0 * float(pair.blur_sigma)))
    assert inside > _cap2(pair, tile, halo), (inside, _cap2(pair, tile, halo))
    from paper_2512_09664_b300.binding import FLAG_TILED_ADVECT, Renderer
    ref = oracle_render(wl)
    for flags in (0, FLAG_TILED_ADVECT):
        st = compare(wl, gpu_render(wl, renderer=Renderer(wl, tile=tile, flags=flags)), ref)
        print("converging", flags, st)
        assert st["pixels"] == 2 * h * w


def test_dense_bins_placed_over_several_passes_render_the_same_bits():
    import torch

    from paper_2512_09664_b300.binding import FLAG_TILED_ADVECT, Renderer
    h = w = 1024
    flow = W.fourier_flow(h, w, h, w, rms=3.0, seed=2251)
    pair = W.PairSpec(height=h, width=w, n_particles=W.n_particles_for(0.099, h, w), pair_id=251,
                      d_dist=0, d_min=1.0, d_max=5.0, illum_min=0.7, illum_max=1.0, noise_sigma=0.02,
                      blur_sigma=0.7)
    wl = W.Workload(name="dense_1024", seed=2, pairs=[pair], flows=[flow], out_dtype="u16", quant_bits=12)
    # a frame-1 bin of tile 128 holds about 2300 records: more than one pass of 2048
    ref = Renderer(wl, tile=128, flags=FLAG_TILED_ADVECT).render().clone()
    torch.cuda.synchronize()
    with _library(_smallbins_path()):
        got = Renderer(wl, tile=128, flags=FLAG_TILED_ADVECT).render().clone()
        torch.cuda.synchronize()
    assert torch.equal(got, ref)
    assert torch.equal(Renderer(wl, tile=128).render(), ref)  # advected while seeding



def test_launch_count_of_each_binning_mode():
    import torch

    from paper_2512_09664_b300.binding import FLAG_TILED_ADVECT, Renderer, launch_count
    wl = W.batch_512_u8(n_pairs=2)

    def launches(r):
        r.render()
        torch.cuda.synchronize()
        n0 = launch_count()
        r.render()
        torch.cuda.synchronize()
        return launch_count() - n0

    # fixed bins: plan, seeding + advection + both frames' placement, one rebin check of both
    # frames, splat
    assert launches(Renderer(wl, tile=128)) == 4
    assert launches(Renderer(wl, tile=32)) == 4
    empty = W.batch_512_u8(n_pairs=2)  # an empty pair: one empty chunk writes its work items
    empty.pairs[1].n_particles = 0
    assert launches(Renderer(empty, tile=128)) == 4
    # tiled advection: plan, seeding + frame-1 placement, rebin check, advection + frame-2
    # placement, rebin check, splat
    assert launches(Renderer(wl, tile=128, flags=FLAG_TILED_ADVECT)) == 6
    assert launches(Renderer(empty, tile=32, flags=FLAG_TILED_ADVECT)) == 6
    # per-particle advection (hiding): plan, seed + advect, scan, scatter, splat
    hidden = W.batch_512_u8(n_pairs=2)
    hidden.hide_prob = np.float32(0.1)
    assert launches(Renderer(hidden, tile=128)) == 5
    # a small pair (N x tiles <= 2^16): bins of capacity N cannot overflow, no rebinning launches
    assert launches(Renderer(W.single_pair_256(seed=0), tile=64)) == 3
    assert launches(Renderer(W.single_pair_256(seed=0), tile=64, flags=FLAG_TILED_ADVECT)) == 4


def test_a_batch_with_an_empty_pair_matches_the_oracle():
    # the empty pair has bins of capacity 0 and one empty seeding chunk, which writes its work
    # items; its frames hold noise only, the other pairs render as the oracle does
    h = w = 256
    flows = [W.fourier_flow(h, w, h, w, rms=3.0, seed=1500 + b) for b in range(3)]
    pairs = [W.PairSpec(height=h, width=w, n_particles=W.n_particles_for(0.05, h, w) if b != 1 else 0,
                        pair_id=b, flow_index=b, d_min=1.0, d_max=4.0, illum_min=0.7, illum_max=1.0,
                        noise_sigma=0.02, blur_sigma=0.7) for b in range(3)]
    wl = W.Workload(name="empty_pair", seed=5, pairs=pairs, flows=flows, out_dtype="u8", quant_bits=8)
    for tile in (64, 128):
        st = compare(wl, gpu_render(wl, tile=tile), oracle_render(wl))
        assert st["pixels"] == 3 * 2 * h * w
