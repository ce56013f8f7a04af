"""Histogram matching of rendered frames on the GPU against the oracle's
integer histogram specification (bit-exact: integer work)."""
import numpy as np
import pytest

from paper_2512_09664_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")


def _uneven(out_dtype, bits):
    sizes = [(96, 128), (200, 160), (64, 64)]
    flows = [W.fourier_flow(h, w, h, w, rms=2.0, seed=80 + k) for k, (h, w) in enumerate(sizes)]
    pairs = [W.PairSpec(height=h, width=w, n_particles=int(0.04 * h * w), pair_id=k, flow_index=k,
                        illum_min=0.7, illum_max=1.0, noise_sigma=0.02, blur_sigma=0.7)
             for k, (h, w) in enumerate(sizes)]
    return W.Workload(name="hist", seed=3, pairs=pairs, flows=flows, out_dtype=out_dtype, quant_bits=bits)


def _target(n_codes, seed=0):
    rng = np.random.default_rng(seed)
    t = (np.exp(-np.arange(n_codes) / (n_codes / 6.0)) * 1e6).astype(np.uint64)
    t += rng.integers(0, 1000, size=n_codes).astype(np.uint64)
    return t


@pytest.mark.parametrize("out_dtype,bits", [("u8", 8), ("u16", 12), ("u16", 16), ("u8", 5)])
def test_histogram_matching_matches_oracle(out_dtype, bits):
    import torch

    import oracle
    from paper_2512_09664_b300 import binding as B
    wl = _uneven(out_dtype, bits)
    r = B.Renderer(wl)
    r.render()
    n_codes = 1 << bits
    before = [r.frames(b).view(torch.int16 if out_dtype == "u16" else torch.uint8).cpu().numpy()
              for b in range(wl.n_pairs)]
    target = _target(n_codes)
    B.match_histogram(r.pk, r.images, torch.from_numpy(target).cuda())
    for b in range(wl.n_pairs):
        got = r.frames(b).view(torch.int16 if out_dtype == "u16" else torch.uint8).cpu().numpy()
        for f in range(2):
            src = before[b][f].view(np.uint16 if out_dtype == "u16" else np.uint8).astype(np.uint32)
            want = oracle.match_histogram(src.ravel(), n_codes, target).reshape(src.shape)
            g = got[f].view(np.uint16 if out_dtype == "u16" else np.uint8).astype(np.uint32)
            assert np.array_equal(g, want), (b, f)


def test_matching_to_own_histogram_is_identity():
    import torch

    from paper_2512_09664_b300 import binding as B
    wl = _uneven("u8", 8).subset([0])
    r = B.Renderer(wl)
    r.render()
    f0 = r.frames(0)[0].cpu().numpy()
    own = np.bincount(f0.ravel(), minlength=256).astype(np.uint64)
    B.match_histogram(r.pk, r.images, torch.from_numpy(own).cuda())
    assert np.array_equal(r.frames(0)[0].cpu().numpy(), f0)
