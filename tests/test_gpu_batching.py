"""Batching and scheduling: the persistent work queue over uneven batches,
the tile autotuner and CUDA-graph replay."""
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


def test_autotuner_picks_a_candidate_and_results_do_not_depend_on_it():
    import torch

    from paper_2512_09664_b300.binding import Renderer
    wl = W.uneven_batch(n_pairs=12, sizes=(64, 128, 256))
    r = Renderer(wl)
    tile, ms = r.autotune(reps=2)
    assert tile in (16, 32, 64, 128) and ms > 0
    img = r.render().clone()
    torch.cuda.synchronize()
    for t in (16, 32, 64, 128):
        r.pk.batch.tile = t
        assert torch.equal(r.render(), img)
    compare(wl, gpu_render(wl, renderer=r), oracle_render(wl))


def test_graph_replay_matches_eager():
    import torch

    from paper_2512_09664_b300.binding import Renderer
    wl = W.uneven_batch(n_pairs=8, sizes=(96, 160))
    r = Renderer(wl, tile=32)
    eager = r.render().clone()
    r.images.zero_()
    r.capture()
    for _ in range(3):
        r.images.zero_()
        r.replay()
        torch.cuda.synchronize()
        assert torch.equal(r.images, eager)


def test_renders_submitted_as_graphs_match_kernel_by_kernel_launches():
    """From a launch sequence's second use on, a render goes to the GPU as one
    CUDA graph whose nodes' arguments are set for each render; a render with
    an events array launches kernel by kernel.  Both give the same bits, seed
    after seed, and a second renderer of the same shapes (other buffers)
    reuses the graph with its own arguments."""
    import torch

    from paper_2512_09664_b300.binding import Renderer, launch_count
    wl = W.batch_512_u8(n_pairs=3)
    r = Renderer(wl, tile=64)
    first = {}
    for seed in (11, 12, 13, 11):
        r.pk.batch.seed = seed
        n0 = launch_count()
        via_graph = r.render().clone()
        torch.cuda.synchronize()
        assert launch_count() - n0 == 4
        r.images.zero_()
        direct = r.render_staged([None] * 6).clone()
        torch.cuda.synchronize()
        assert torch.equal(via_graph, direct)
        first.setdefault(seed, via_graph)
    assert torch.equal(first[11], via_graph) and not torch.equal(first[11], first[12])
    r2 = Renderer(wl, tile=64)
    r2.pk.batch.seed = 12
    assert torch.equal(r2.render(), first[12])


def test_uneven_batch_full_size_mix_sampled_against_oracle():
    # the uneven workload's size mix (128..1024) with fewer pairs; every pair
    # of the batch is compared in full
    wl = W.uneven_batch(n_pairs=6, sizes=(128, 256, 512, 1024))
    st = compare(wl, gpu_render(wl), oracle_render(wl))
    print("uneven full-size mix", st)


def test_host_pipeline_steps_match_plain_renders():
    # a stream of steps from pinned host flows to pinned host images, copies
    # overlapped with rendering: each step's images equal a plain render of
    # its flows, whatever the steps before it left in the other buffer set
    import torch

    from paper_2512_09664_b300.binding import HostPipeline, Renderer
    wl = W.uneven_batch(n_pairs=3, sizes=(64, 128))
    r = Renderer(wl, tile=32)
    base = torch.from_numpy(r.pk.flows_host)
    scales = (1.0, -0.6, 0.35)
    flows_host = [(base * s).pin_memory() for s in scales]
    pipe = HostPipeline(r, depth=2)
    outs, events = [], []
    for k in range(5):
        out = torch.empty(r.images.shape, dtype=r.images.dtype).pin_memory()
        events.append(pipe.submit(flows_host[k % 3], out))
        outs.append(out)
    pipe.synchronize()
    torch.cuda.synchronize()
    with pytest.raises(ValueError):  # the steps share the renderer's workspace: one stream only
        pipe.submit(flows_host[0], outs[0], torch.cuda.Stream())
    ref = Renderer(wl, tile=32)
    for k, out in enumerate(outs):
        img = ref.render_from(flows=flows_host[k % 3].to(ref.device)).cpu()
        torch.cuda.synchronize()
        assert torch.equal(out.view(torch.uint8), img.view(torch.uint8)), k
    # the unscaled step against the oracle
    pipe_frames = []
    for b in range(wl.n_pairs):
        h, w = r.pk.shapes[b]
        o = r.pk.image_offsets[b]
        t = outs[3][o:o + 2 * h * w].view(2, h, w)
        pipe_frames.append(t.view(torch.int16).numpy().view(np.uint16) if t.dtype == torch.uint16 else t.numpy())
    compare(wl, pipe_frames, oracle_render(wl))
