"""Pins of the oracle's gradients (the differentiable render: frames
B_f = L * S_f, no noise or blur; loss sum(G * B)).

* central finite differences of the FP64 oracle forward (h = 1e-6);
* an independent re-expression of the forward in torch FP64 (grid_sample for
  the bilinear flow, torch.special.ndtr for the pixel masses) differentiated
  by torch autograd.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2512_09664_b300 import workloads as W


def _case(integ="rk4", n_sub=4, illum=(0.7, 1.0), H=24, Wd=28, n=7, seed=3):
    spec = W.PairSpec(height=H, width=Wd, n_particles=n, pair_id=1, d_min=1.5, d_max=3.5,
                      illum_min=illum[0], illum_max=illum[1])
    pr = oracle.make_pair(spec, seed=seed, integrator=integ, n_substeps=n_sub, dt=1.0, flow_shape=(H, Wd))
    flow = W.fourier_flow(H, Wd, H, Wd, rms=1.5, seed=2)
    G = np.random.default_rng(seed).standard_normal((2, H, Wd))
    parts = oracle.particles(pr, flow)[:, [0, 1, 2]].copy()
    return pr, flow, G, parts


def _loss(pr, flow, G, parts):
    return float((G * oracle.render_from(pr, flow, parts)).sum())


@pytest.mark.parametrize("integ,n_sub", [("rk4", 4), ("rk4", 1), ("euler", 3)])
def test_oracle_gradients_match_central_differences(integ, n_sub):
    pr, flow, G, parts = _case(integ, n_sub)
    gf, gp = oracle.backward(pr, flow, G, parts)
    h = 1e-6
    for k in range(len(parts)):
        for c in range(3):
            pp, pm = parts.copy(), parts.copy()
            pp[k, c] += h
            pm[k, c] -= h
            fd = (_loss(pr, flow, G, pp) - _loss(pr, flow, G, pm)) / (2 * h)
            assert abs(fd - gp[k, c]) <= 1e-6 * max(1.0, abs(fd)), (k, c, fd, gp[k, c])
    # flow nodes: the FP32 grid is perturbed in FP64 through a float64 copy
    rng = np.random.default_rng(1)
    nz = np.argwhere(np.abs(gf).sum(-1) > 1e-8)
    for k, l in nz[rng.choice(len(nz), size=min(12, len(nz)), replace=False)]:
        for c in range(2):
            hf = 2.0 ** -12  # exact in FP32 near O(1) flow values
            fp, fm = flow.copy(), flow.copy()
            fp[k, l, c] += np.float32(hf)
            fm[k, l, c] -= np.float32(hf)
            step = float(fp[k, l, c]) - float(fm[k, l, c])
            fd = (_loss(pr, fp, G, parts) - _loss(pr, fm, G, parts)) / step
            # the loss is smooth but not linear in the flow: O(h^2) curvature
            assert abs(fd - gf[k, l, c]) <= 1e-5 * max(1.0, abs(fd)), (k, l, c, fd, gf[k, l, c])


def _torch_forward(pr, flow, parts, integ, n_sub):
    """The differentiable render re-expressed with torch ops (FP64)."""
    H, Wd = pr.height, pr.width
    fl = torch.tensor(flow, dtype=torch.float64, requires_grad=True)
    pt = torch.tensor(parts, dtype=torch.float64, requires_grad=True)
    ieff = torch.tensor(oracle.particles(pr, flow)[:, 5], dtype=torch.float64)
    inp = fl.permute(2, 0, 1)[None]

    def vel(x, y):
        g = torch.stack([2 * x / Wd - 1, 2 * y / H - 1], -1)[None, None]
        uv = torch.nn.functional.grid_sample(inp, g, mode="bilinear", padding_mode="border", align_corners=False)
        return uv[0, 0, 0], uv[0, 1, 0]

    x, y = pt[:, 0], pt[:, 1]
    h = float(pr.dt) / n_sub
    pos = [(x, y)]
    for _ in range(n_sub):
        u1, v1 = vel(x, y)
        if integ == "euler":
            x, y = x + h * u1, y + h * v1
            continue
        u2, v2 = vel(x + h / 2 * u1, y + h / 2 * v1)
        u3, v3 = vel(x + h / 2 * u2, y + h / 2 * v2)
        u4, v4 = vel(x + h * u3, y + h * v3)
        x, y = x + h / 6 * (u1 + 2 * u2 + 2 * u3 + u4), y + h / 6 * (v1 + 2 * v2 + 2 * v3 + v4)
    pos.append((x, y))
    d = pt[:, 2]
    sig = d / 4
    amp = ieff * 2 * math.pi * sig * sig
    frames = []
    jj, ii = np.arange(Wd), np.arange(H)
    L = torch.tensor([[oracle.illumination(pr, i, j) for j in range(Wd)] for i in range(H)], dtype=torch.float64)
    for (xf, yf) in pos:
        S = torch.zeros(H, Wd, dtype=torch.float64)
        for k in range(len(parts)):
            xv, yv, dv = float(xf[k].detach()), float(yf[k].detach()), float(d[k].detach())
            cols = jj[(jj >= math.floor(xv - 1.5 * dv)) & (jj <= math.floor(xv + 1.5 * dv))]
            rows = ii[(ii >= math.floor(yv - 1.5 * dv)) & (ii <= math.floor(yv + 1.5 * dv))]
            if len(cols) == 0 or len(rows) == 0:
                continue
            ct = torch.tensor(cols, dtype=torch.float64)
            rt = torch.tensor(rows, dtype=torch.float64)
            ex = torch.special.ndtr((ct + 1 - xf[k]) / sig[k]) - torch.special.ndtr((ct - xf[k]) / sig[k])
            ey = torch.special.ndtr((rt + 1 - yf[k]) / sig[k]) - torch.special.ndtr((rt - yf[k]) / sig[k])
            blk = amp[k] * ey[:, None] * ex[None, :]
            S = S.index_put((torch.tensor(rows)[:, None].expand_as(blk), torch.tensor(cols)[None, :].expand_as(blk)),
                            blk, accumulate=True)
        frames.append(L * S)
    return torch.stack(frames), fl, pt


@pytest.mark.parametrize("integ,n_sub", [("rk4", 4), ("euler", 2)])
def test_oracle_gradients_match_torch_autograd_reexpression(integ, n_sub):
    pr, flow, G, parts = _case(integ, n_sub, n=5)
    B, fl, pt = _torch_forward(pr, flow, parts, integ, n_sub)
    np.testing.assert_allclose(B.detach().numpy(), oracle.render_from(pr, flow, parts), atol=1e-12)
    (torch.tensor(G) * B).sum().backward()
    gf, gp = oracle.backward(pr, flow, G, parts)
    np.testing.assert_allclose(gp, pt.grad.numpy(), rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(gf, fl.grad.numpy(), rtol=1e-9, atol=1e-11)


def test_oracle_seeded_particles_default():
    pr, flow, G, parts = _case()
    np.testing.assert_array_equal(oracle.render_from(pr, flow, None), oracle.render_from(pr, flow, parts))
    g1 = oracle.backward(pr, flow, G, None)
    g2 = oracle.backward(pr, flow, G, parts)
    np.testing.assert_array_equal(g1[1], g2[1])
