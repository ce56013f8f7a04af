"""Particle reuse across consecutive frames (the paper's Conclusions: the
flow applied for a second dt' to the frame-2 positions gives the frame-1
positions of the next batch), through synthpix_advect_particles and
synthpix_render_pairs_from, against the FP64 oracle.

Positions cross the C ABI as FP32 triples (x, y, d); the oracle's chain
rounds its FP64 positions to FP32 at the same hand-offs, so both sides
render the next batch from positions that agree to an FP32 ulp."""
import numpy as np
import pytest

import oracle
from paper_2512_09664_b300 import workloads as W

from parity import FLOAT_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")


def _workload():
    H, Wd = 96, 128
    flows = [W.fourier_flow(H, Wd, H, Wd, rms=2.5, seed=60 + b) for b in range(2)]
    pairs = [W.PairSpec(height=H, width=Wd, n_particles=W.n_particles_for(0.05, H, Wd), pair_id=b,
                        flow_index=b, d_min=1.0, d_max=4.0, illum_min=0.7, illum_max=1.0) for b in range(2)]
    return W.Workload(name="seq", seed=11, pairs=pairs, flows=flows, out_dtype="f32", quant_bits=0,
                      n_substeps=4, dt=1.0)


def _oracle_chain(wl, b, dt2):
    """FP32 (x, y, d) of frame 2 and of the next batch's frame 1, for pair b."""
    spec, flow = wl.pairs[b], wl.flows[wl.pairs[b].flow_index]
    pair = oracle.pair_from_workload(wl, b)
    parts = oracle.particles(pair, flow)
    f32 = lambda a: a.astype(np.float32).astype(np.float64)  # noqa: E731
    p1 = np.stack([f32(parts[:, 6]), f32(parts[:, 7]), parts[:, 2]], axis=1)
    pair2 = oracle.make_pair(spec, wl.seed, wl.integrator, wl.n_substeps, dt2, wl.quant_bits,
                             flow_shape=flow.shape[:2])
    nxt = np.array([oracle.advect(pair2, flow, x, y) for x, y in p1[:, :2]])
    p2 = np.stack([f32(nxt[:, 0]), f32(nxt[:, 1]), p1[:, 2]], axis=1)
    return p1, p2


def test_advected_positions_match_the_oracle_and_chain_into_the_next_batch():
    import torch

    from paper_2512_09664_b300.binding import Renderer
    wl = _workload()
    dt2 = 0.75
    r = Renderer(wl)
    p1 = r.advect_particles()                     # frame-2 positions over dt
    p2 = r.advect_particles(particles=p1, dt=dt2)  # next batch's frame-1 positions over dt'
    nxt = r.render_from(particles=p2).clone()
    torch.cuda.synchronize()
    g1, g2, gi = p1.cpu().numpy(), p2.cpu().numpy(), nxt.cpu().numpy()
    off = 0
    for b, spec in enumerate(wl.pairs):
        o1, o2 = _oracle_chain(wl, b, dt2)
        n = spec.n_particles
        # positions: within one FP32 ulp of the oracle's rounded values (1/32768 px at < 512 px)
        assert np.abs(g1[off:off + n] - o1).max() <= 2.0 ** -15
        assert np.abs(g2[off:off + n] - o2).max() <= 2.0 ** -14
        assert np.array_equal(g1[off:off + n, 2], o1[:, 2].astype(np.float32))
        # the next batch rendered from its reused particles
        pair = oracle.pair_from_workload(wl, b)
        ref = oracle.render_from(pair, wl.flows[spec.flow_index], parts_in=o2)
        io = r.pk.image_offsets[b]
        got = gi[io:io + 2 * spec.height * spec.width].reshape(2, spec.height, spec.width)
        assert np.abs(got - ref).max() <= FLOAT_TOL
        off += n


def test_frame_two_repeats_as_the_next_frame_one():
    import torch

    from paper_2512_09664_b300.binding import Renderer
    wl = _workload()
    r = Renderer(wl)
    cur = r.render().clone()
    p1 = r.advect_particles()
    nxt = r.render_from(particles=p1).clone()  # dt' = 0: the next batch starts where this one ends
    torch.cuda.synchronize()
    for b, spec in enumerate(wl.pairs):
        io, hw = r.pk.image_offsets[b], spec.height * spec.width
        f2 = cur[io + hw:io + 2 * hw].cpu().numpy()
        f1n = nxt[io:io + hw].cpu().numpy()
        # equal up to the FP32 rounding of the positions (< 2^-17 px at < 128 px)
        assert np.abs(f2 - f1n).max() <= 1e-5
