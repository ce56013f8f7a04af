"""The streaming sampler and the device flow generator on the GPU."""
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


@pytest.mark.parametrize("gh,gw,H,Wd,nm", [(96, 128, 96, 128, 64), (33, 47, 96, 128, 16), (512, 512, 512, 512, 64)])
def test_fourier_flows_match_host_fp64(gh, gw, H, Wd, nm):
    import torch

    from paper_2512_09664_b300 import binding as B
    F = 3
    modes = np.stack([W.fourier_modes(100 + f, H, Wd, nm) for f in range(F)])
    want = np.stack([W.fourier_flow_from_modes(m, gh, gw, H, Wd, rms=3.0) for m in modes])
    md = torch.from_numpy(modes).cuda()
    out = torch.empty((F, gh, gw, 2), dtype=torch.float32, device="cuda")
    ws = torch.empty(B.fourier_flows_workspace_bytes(F, nm, gh, gw), dtype=torch.uint8, device="cuda")
    B.fourier_flows(md, gh, gw, H, Wd, 3.0, out, ws)
    got = out.cpu().numpy()
    err = np.abs(got.astype(np.float64) - want).max()
    print("fourier flows", gh, gw, "max |err|", err)
    assert err < 5e-5
    assert np.allclose(np.sqrt((got.astype(np.float64) ** 2).sum(-1).mean(axis=(1, 2))), 3.0, rtol=1e-5)


def _cfg(**kw):
    cfg = {"image_shape": [96, 128], "batch_size": 4, "flows_per_batch": 2, "batches_per_flow": 2, "seed": 3,
           "seeding_density": [0.02, 0.06], "output": "u8", "noise_sigma": 0.02, "blur_sigma": 0.7,
           "illumination": [0.7, 1.0], "flow": {"kind": "fourier", "rms": 2.0}}
    cfg.update(kw)
    return cfg


def test_sampler_batches_equal_direct_renders_and_reuse_flows():
    import torch

    from paper_2512_09664_b300 import sampler as S
    smp = S.make(_cfg())
    seen = []
    for k in range(3):
        batch = next(smp)
        assert batch.params.batch_index == k and batch.params.flow_set == k // 2
        imgs = batch.images.clone()
        flows = batch.flows.clone()
        wl = smp.workload(k)  # the resident device flows of this batch's set
        direct = gpu_render(wl)
        for b in range(4):
            assert np.array_equal(imgs[b].cpu().numpy(), direct[b]), (k, b)
        assert torch.equal(batch.flow_fields, flows[batch.flow_index])
        seen.append(flows)
    assert torch.equal(seen[0], seen[1]) and not torch.equal(seen[1], seen[2])


def test_sampler_batch_matches_oracle():
    from paper_2512_09664_b300 import sampler as S
    smp = S.make(_cfg(jitter={"diameter": 0.1, "intensity": 0.05}, hide_prob=0.05, diameter_y=[1.0, 3.0],
                      rho=[-0.5, 0.5]))
    batch = next(smp)
    got = [x.cpu().numpy() for x in batch.images]
    wl = smp.workload(0)
    st = compare(wl, got, oracle_render(wl))
    print("sampler vs oracle", st)


def test_sampler_double_buffers_images():
    from paper_2512_09664_b300 import sampler as S
    smp = S.make(_cfg(batches_per_flow=1))
    b0 = next(smp)
    keep = b0.images.clone()
    b1 = next(smp)
    assert b1.images.data_ptr() != b0.images.data_ptr()
    assert np.array_equal(b0.images.cpu().numpy(), keep.cpu().numpy())  # untouched by the next batch


def test_sampler_flow_providers():
    import torch

    from paper_2512_09664_b300 import sampler as S
    smp = S.make(_cfg(flow={"kind": "uniform", "u": 1.0, "v": -0.5}))
    b = next(smp)
    assert torch.all(b.flows[..., 0] == 1.0) and torch.all(b.flows[..., 1] == -0.5)
    calls = []

    def provider(set_index, n, shape):
        calls.append(set_index)
        return np.full((n, *shape, 2), 0.25 * (set_index + 1), dtype=np.float32)
    smp = S.make(_cfg(), flow_provider=provider)
    b0 = next(smp)
    b1 = next(smp)
    b2 = next(smp)
    assert float(b2.flows[0, 0, 0, 0]) == 0.5 and calls[:2] == [0, 1]


def test_sampler_target_histogram_and_remark_sheet():
    import oracle
    from paper_2512_09664_b300 import sampler as S
    target = (np.exp(-np.arange(256) / 40.0) * 1e5).astype(np.uint64) + 1
    cfg = _cfg(sheet_model="remark", sheet_shape=2.0, sheet_sigma=0.5, target_histogram=target.tolist())
    smp = S.make(cfg)
    batch = next(smp)
    got = batch.images.cpu().numpy()
    wl = smp.workload(0)
    assert wl.pairs[0].sheet_model == 1
    direct = gpu_render(wl)
    for b in range(4):
        for f in range(2):
            want = oracle.match_histogram(direct[b][f].astype(np.uint32).ravel(), 256, target)
            assert np.array_equal(got[b, f].astype(np.uint32).ravel(), want)
