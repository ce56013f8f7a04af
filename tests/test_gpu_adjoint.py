"""The adjoint of the render on the GPU (synthpix_render_backward) against the
FP64 oracle gradient and against central finite differences of the GPU
forward, and the differentiable workload (flow from a bilinearly upsampled
32x32 control grid, MSE against a target rendered from a perturbed grid)
through torch.autograd."""
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


def _small_batch(n_pairs=2, size=64, integ="rk4", n_sub=4, illum=(0.7, 1.0)):
    flows = [W.fourier_flow(size, size, size, size, rms=2.0, seed=50 + b) for b in range(n_pairs)]
    pairs = [W.PairSpec(height=size, width=size, n_particles=W.n_particles_for(0.04, size, size), pair_id=b,
                        flow_index=b, d_min=1.5, d_max=3.5, illum_min=illum[0], illum_max=illum[1])
             for b in range(n_pairs)]
    return W.Workload(name="adj", seed=3, pairs=pairs, flows=flows, out_dtype="f32", quant_bits=0,
                      integrator=integ, n_substeps=n_sub, dt=1.0)


def _renderer(wl):
    from paper_2512_09664_b300.binding import Renderer
    return Renderer(wl, tile=32)


def test_seeded_particles_match_oracle_and_render_from_reproduces_render():
    import torch
    wl = _small_batch()
    r = _renderer(wl)
    parts = r.seed_particles().cpu().numpy().astype(np.float64)
    off = 0
    for b, spec in enumerate(wl.pairs):
        ref = oracle.particles(oracle.pair_from_workload(wl, b), wl.flows[b])
        got = parts[off:off + spec.n_particles]
        np.testing.assert_array_equal(got[:, :2], ref[:, :2])  # power-of-two frames: exact
        np.testing.assert_allclose(got[:, 2], ref[:, 2], rtol=2e-7)
        off += spec.n_particles
    a = r.render().clone()
    b_ = r.render_from(particles=r.seed_particles()).clone()
    torch.cuda.synchronize()
    assert torch.equal(a, b_)


@pytest.mark.parametrize("integ,n_sub", [("rk4", 4), ("euler", 2)])
def test_backward_matches_oracle_gradient(integ, n_sub):
    import torch
    wl = _small_batch(integ=integ, n_sub=n_sub)
    r = _renderer(wl)
    G = torch.randn(r.images.shape, device="cuda", dtype=torch.float32, generator=torch.Generator("cuda").manual_seed(1))
    gf = torch.zeros_like(r.flows)
    n = sum(p.n_particles for p in wl.pairs)
    gp = torch.empty((n, 3), device="cuda")
    r.backward(G, grad_flows=gf, grad_particles=gp)
    torch.cuda.synchronize()
    Gh, gfh, gph = G.cpu().numpy(), gf.cpu().numpy(), gp.cpu().numpy()
    off_p, off_f = 0, 0
    for b, spec in enumerate(wl.pairs):
        pr = oracle.pair_from_workload(wl, b)
        io = r.pk.image_offsets[b]
        Gb = Gh[io:io + 2 * spec.height * spec.width].reshape(2, spec.height, spec.width).astype(np.float64)
        rf, rp = oracle.backward(pr, wl.flows[b], Gb)
        sp = gph[off_p:off_p + spec.n_particles]
        scale = np.abs(rp).max(0)
        assert np.all(np.abs(sp - rp) <= 1e-4 * scale + 1e-6), np.abs(sp - rp).max(0) / scale
        nf = wl.flows[b].size
        sf = gfh[off_f:off_f + nf].reshape(wl.flows[b].shape)
        assert np.abs(sf - rf).max() <= 1e-4 * np.abs(rf).max()
        off_p += spec.n_particles
        off_f += nf


def test_backward_matches_central_differences_of_gpu_forward():
    import torch
    wl = _small_batch(n_pairs=1)
    r = _renderer(wl)
    G = torch.randn(r.images.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(2))
    parts = r.seed_particles().clone()
    n = parts.shape[0]
    gf = torch.zeros_like(r.flows)
    gp = torch.empty((n, 3), device="cuda")
    r.backward(G, particles=parts, grad_flows=gf, grad_particles=gp)

    def loss(p=None, f=None):
        img = r.render_from(flows=f, particles=parts if p is None else p)
        return float((G.double() * img.double()).sum())

    h = 1e-3
    rng = np.random.default_rng(0)
    gscale = gp.abs().max(0).values.cpu().numpy()
    for k in rng.choice(n, size=12, replace=False):
        for c in range(3):
            pp, pm = parts.clone(), parts.clone()
            pp[k, c] += h
            pm[k, c] -= h
            fd = (loss(pp) - loss(pm)) / (2 * h)
            g = float(gp[k, c])
            assert abs(fd - g) <= 2e-2 * abs(g) + 2e-3 * gscale[c], (k, c, fd, g)
    # flow nodes with sizeable gradients
    gfv = gf.cpu().numpy()
    idx = np.argsort(-np.abs(gfv))[:8]
    for j in idx:
        fp, fm = r.flows.clone(), r.flows.clone()
        fp[j] += h
        fm[j] -= h
        fd = (loss(f=fp) - loss(f=fm)) / (2 * h)
        assert abs(fd - gfv[j]) <= 2e-2 * abs(gfv[j]) + 2e-3 * np.abs(gfv).max(), (j, fd, gfv[j])


def _control_workload(n_pairs, size=256, n_ctrl=32):
    import torch
    wl = W.differentiable_batch(n_pairs=n_pairs, size=size, n_ctrl=n_ctrl)
    ctrl = torch.tensor(np.stack(wl.meta["control"]), dtype=torch.float32)  # [B, n, n, 2]
    return wl, ctrl


def _upsample(ctrl, size):
    import torch.nn.functional as F
    x = ctrl.permute(0, 3, 1, 2)  # [B, 2, n, n]
    up = F.interpolate(x, size=(size, size), mode="bilinear", align_corners=False)
    return up.permute(0, 2, 3, 1).contiguous()  # [B, size, size, 2]


def test_control_grid_workload_gradients_vs_oracle_and_fd():
    import torch

    from paper_2512_09664_b300.binding import Renderer, render
    wl, ctrl = _control_workload(n_pairs=3)
    size = wl.pairs[0].height
    flows0 = _upsample(ctrl.double(), size).float()
    wl.flows = [f.numpy() for f in flows0]
    r = Renderer(wl, tile=32)
    # target: the same particles under a perturbed control grid (+ N(0, 0.1) px)
    gen = torch.Generator().manual_seed(7)
    tgt_ctrl = ctrl + 0.1 * torch.randn(ctrl.shape, generator=gen)
    target = render(r, _upsample(tgt_ctrl, size).reshape(-1).cuda()).detach().clone()

    c = ctrl.clone().cuda().requires_grad_(True)
    img = render(r, _upsample(c, size).reshape(-1))
    loss = ((img - target) ** 2).mean()
    loss.backward()
    g_gpu = c.grad.cpu().double()

    # oracle: dL/dflow per pair in FP64, chained through the upsampling by torch (FP64)
    G = (2.0 / img.numel() * (img - target)).detach().cpu().numpy().astype(np.float64)
    gflow = []
    for b, spec in enumerate(wl.pairs):
        io = r.pk.image_offsets[b]
        Gb = G[io:io + 2 * size * size].reshape(2, size, size)
        gflow.append(oracle.backward(oracle.pair_from_workload(wl, b), wl.flows[b], Gb)[0])
    cd = ctrl.double().requires_grad_(True)
    up = _upsample(cd, size)
    (up * torch.tensor(np.stack(gflow))).sum().backward()
    g_ref = cd.grad
    assert torch.abs(g_gpu - g_ref).max() <= 1e-3 * torch.abs(g_ref).max()

    # central differences of the GPU forward on the largest control entries
    def L(cc):
        with torch.no_grad():
            im = render(r, _upsample(cc, size).reshape(-1))
            return float(((im.double() - target.double()) ** 2).mean())
    h = 1e-3
    flat = torch.argsort(-g_ref.abs().reshape(-1))[:6]
    for j in flat.tolist():
        cp, cm = ctrl.clone().cuda(), ctrl.clone().cuda()
        cp.view(-1)[j] += h
        cm.view(-1)[j] -= h
        fd = (L(cp) - L(cm)) / (2 * h)
        g = float(g_gpu.view(-1)[j])
        assert abs(fd - g) <= 3e-2 * abs(g) + 1e-3 * float(g_ref.abs().max()), (j, fd, g)


def test_backward_rejects_quantised_and_blurred_batches():
    import torch

    from paper_2512_09664_b300 import binding as B
    wl = W.batch_512_u8(n_pairs=1)
    r = B.Renderer(wl.subset([0]))
    G = torch.zeros(r.images.shape, dtype=torch.float32, device="cuda")
    with pytest.raises(B.SynthpixError) as e:
        r.backward(G)
    assert e.value.code == B.EUNSUPPORTED
