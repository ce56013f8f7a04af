"""Seeded synthetic inputs for the PIV image-pair renderer.

This module only *generates inputs*: flow grids, per-pair acquisition
parameters and batch settings shaped like the paper's workloads (512x512
pairs in the throughput study of Section 3.1; batches of 64-256 pairs and
1024x1024 frames in Section 2 "Configuration file"; the ablation defaults
of Section 3.3).  It contains none of the rendering arithmetic: the CUDA
library and the FP64 oracle both receive exactly the numbers produced here
and implement the method independently.

Every floating-point parameter is stored as ``np.float32`` because the
library's descriptors hold FP32 values; the oracle is handed the same FP32
values (widened to FP64) so both sides start from identical inputs.

Flow grids are ``float32`` arrays of shape ``[Gh, Gw, 2]`` holding
``(u, v)`` in pixels per frame, nodes at cell centres
``((l + 1/2) W / Gw, (k + 1/2) H / Gh)``.  Paper Section 2 ("Data loaders")
lists file-based flow providers (JHTDB .hdf5, .mat, .npy); those datasets
are not available here, so analytic and random procedural flows stand in
for them, which the paper also allows ("supplied procedurally").
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

F32 = np.float32

# output / intermediate dtype names shared by the Python bindings and tests
OUT_DTYPES = ("f32", "f16", "bf16", "u8", "u16")
INTER_DTYPES = ("f32", "f16", "bf16")


@dataclass
class PairSpec:
    """Acquisition parameters of one image pair (all FP32 where real)."""

    height: int
    width: int
    n_particles: int
    pair_id: int
    flow_index: int = 0
    d_dist: int = 0  # 0: uniform [d_min, d_max]; 1: normal(d_mu, d_sigma) clipped
    d_min: np.float32 = F32(1.0)
    d_max: np.float32 = F32(4.0)
    d_mu: np.float32 = F32(2.5)
    d_sigma: np.float32 = F32(0.3)
    i_min: np.float32 = F32(0.8)
    i_max: np.float32 = F32(1.0)
    z_min: np.float32 = F32(-1.0)
    z_max: np.float32 = F32(1.0)
    sheet_sigma: np.float32 = F32(0.5)
    illum_min: np.float32 = F32(1.0)
    illum_max: np.float32 = F32(1.0)
    noise_sigma: np.float32 = F32(0.0)
    blur_sigma: np.float32 = F32(0.0)
    # general particle shapes and frame-2 variation (all 0: round particles,
    # identical parameters in both frames)
    dy_min: np.float32 = F32(0.0)   # diameter along y ~ U[dy_min, dy_max]; 0, 0: d_y = d
    dy_max: np.float32 = F32(0.0)
    rho_min: np.float32 = F32(0.0)  # correlation of Eq. 1 ~ U[rho_min, rho_max]
    rho_max: np.float32 = F32(0.0)
    jitter_d: np.float32 = F32(0.0)    # std of the frame-2 change of each diameter (px)
    jitter_i: np.float32 = F32(0.0)    # std of the frame-2 change of I0
    jitter_rho: np.float32 = F32(0.0)  # std of the frame-2 change of rho
    sheet_model: int = 0               # 0: Gaussian sheet; 1: the out-of-focus Remark form
    sheet_shape: np.float32 = F32(0.0)  # shape factor s of the Remark form

    def __post_init__(self):
        for k in ("d_min", "d_max", "d_mu", "d_sigma", "i_min", "i_max", "z_min",
                  "z_max", "sheet_sigma", "illum_min", "illum_max", "noise_sigma",
                  "blur_sigma", "dy_min", "dy_max", "rho_min", "rho_max", "jitter_d",
                  "jitter_i", "jitter_rho", "sheet_shape"):
            setattr(self, k, F32(getattr(self, k)))


@dataclass
class Workload:
    """A batch: shared settings, per-pair parameters and the flow grids."""

    name: str
    seed: int
    pairs: List[PairSpec]
    flows: List[np.ndarray]
    out_dtype: str = "f32"
    quant_bits: int = 0
    inter_dtype: str = "f32"
    integrator: str = "rk4"  # or "euler"
    n_substeps: int = 4
    dt: np.float32 = F32(1.0)
    description: str = ""
    meta: dict = field(default_factory=dict)
    hide_prob: np.float32 = F32(0.0)  # probability of hiding a particle from each frame
    flows_w: Optional[List[np.ndarray]] = None  # per flow grid: out-of-plane velocity [gh, gw] (moves z)

    def __post_init__(self):
        self.dt = F32(self.dt)
        self.hide_prob = F32(self.hide_prob)

    @property
    def n_pairs(self) -> int:
        return len(self.pairs)

    def subset(self, idx) -> "Workload":
        """A workload of the selected pairs; flows are re-indexed compactly."""
        idx = list(idx)
        used = sorted({self.pairs[i].flow_index for i in idx})
        remap = {f: n for n, f in enumerate(used)}
        pairs = [replace(self.pairs[i], flow_index=remap[self.pairs[i].flow_index]) for i in idx]
        fw = None if self.flows_w is None else [self.flows_w[f] for f in used]
        return replace(self, pairs=pairs, flows=[self.flows[f] for f in used], flows_w=fw,
                       name=f"{self.name}[{len(idx)}]")

    def image_elems(self) -> int:
        return sum(2 * p.height * p.width for p in self.pairs)


def n_particles_for(ppp: float, height: int, width: int) -> int:
    """Workload recipe: the particle count of a frame seeded at density ppp."""
    return int(math.floor(ppp * height * width))


# ----------------------------------------------------------------------------
# flow grids
# ----------------------------------------------------------------------------

def node_centres(gh: int, gw: int, height: int, width: int):
    xs = (np.arange(gw, dtype=np.float64) + 0.5) * (width / gw)
    ys = (np.arange(gh, dtype=np.float64) + 0.5) * (height / gh)
    return xs, ys


def zero_flow(gh: int, gw: int) -> np.ndarray:
    return np.zeros((gh, gw, 2), dtype=np.float32)


def uniform_flow(gh: int, gw: int, u: float, v: float) -> np.ndarray:
    f = np.empty((gh, gw, 2), dtype=np.float32)
    f[..., 0] = u
    f[..., 1] = v
    return f


def linear_flow(gh: int, gw: int, height: int, width: int, a, centre) -> np.ndarray:
    """(u, v) = a @ (p - centre) sampled at the nodes; a is 2x2."""
    xs, ys = node_centres(gh, gw, height, width)
    X, Y = np.meshgrid(xs - centre[0], ys - centre[1])
    a = np.asarray(a, dtype=np.float64)
    f = np.empty((gh, gw, 2), dtype=np.float64)
    f[..., 0] = a[0, 0] * X + a[0, 1] * Y
    f[..., 1] = a[1, 0] * X + a[1, 1] * Y
    return f.astype(np.float32)


def lamb_oseen_flow(gh: int, gw: int, height: int, width: int,
                    gamma: float = 200.0, core: float = 20.0) -> np.ndarray:
    """Lamb-Oseen vortex centred on the image (circulation gamma px^2/frame)."""
    xs, ys = node_centres(gh, gw, height, width)
    X, Y = np.meshgrid(xs - width / 2.0, ys - height / 2.0)
    r2 = X * X + Y * Y
    with np.errstate(invalid="ignore", divide="ignore"):
        g = gamma / (2.0 * math.pi * r2) * (1.0 - np.exp(-r2 / (core * core)))
    g = np.where(r2 > 0, g, 0.0)
    f = np.empty((gh, gw, 2), dtype=np.float64)
    f[..., 0] = -g * Y
    f[..., 1] = g * X
    return f.astype(np.float32)


def fourier_modes(seed: int, height: int, width: int, n_modes: int = 64,
                  k_max_wavelength: float = 16.0) -> np.ndarray:
    """[n_modes, 4] float64 (kx, ky, phi, a) of the stream function of fourier_flow.

    |k_m| log-spaced between 2 pi / max(H, W) and 2 pi / k_max_wavelength,
    directions and phases uniform from the seeded generator, a_m ~ |k_m|^(-4/3).
    """
    rng = np.random.default_rng(seed)
    kmin = 2.0 * math.pi / max(height, width)
    kmax = 2.0 * math.pi / k_max_wavelength
    kmag = np.exp(np.linspace(math.log(kmin), math.log(kmax), n_modes))
    theta = rng.uniform(0.0, 2.0 * math.pi, n_modes)
    phi = rng.uniform(0.0, 2.0 * math.pi, n_modes)
    amp = kmag ** (-4.0 / 3.0)
    return np.stack([kmag * np.cos(theta), kmag * np.sin(theta), phi, amp], axis=1)


def fourier_modes_set(key, n_flows: int, height: int, width: int, n_modes: int = 64,
                      k_max_wavelength: float = 16.0) -> np.ndarray:
    """[n_flows, n_modes, 4] modes (kx, ky, phi, a) of n_flows fields from one generator keyed by key.

    The same spectrum as fourier_modes; directions and phases of all the
    fields are drawn at once (a [n_flows, n_modes] array each).
    """
    rng = np.random.default_rng(key)
    kmin = 2.0 * math.pi / max(height, width)
    kmax = 2.0 * math.pi / k_max_wavelength
    kmag = np.exp(np.linspace(math.log(kmin), math.log(kmax), n_modes))[None, :]
    theta = rng.uniform(0.0, 2.0 * math.pi, (n_flows, n_modes))
    phi = rng.uniform(0.0, 2.0 * math.pi, (n_flows, n_modes))
    amp = np.broadcast_to(kmag ** (-4.0 / 3.0), (n_flows, n_modes))
    return np.stack([kmag * np.cos(theta), kmag * np.sin(theta), phi, amp], axis=2)


def fourier_flow(gh: int, gw: int, height: int, width: int, rms: float,
                 seed: int, n_modes: int = 64, k_max_wavelength: float = 16.0) -> np.ndarray:
    """Divergence-free random flow from a streamfunction of n_modes plane waves.

    psi = sum_m a_m sin(k_m . x + phi_m) with |k_m| log-spaced between
    2 pi / max(H, W) and 2 pi / 16, directions and phases uniform, and
    a_m ~ |k_m|^(-4/3) so that the energy per log-spaced mode follows
    E(k) ~ k^(-5/3).  u = d psi / dy, v = -d psi / dx; rescaled to the
    requested RMS speed (px/frame).
    """
    return fourier_flow_from_modes(fourier_modes(seed, height, width, n_modes, k_max_wavelength),
                                   gh, gw, height, width, rms)


def fourier_flow_from_modes(modes: np.ndarray, gh: int, gw: int, height: int, width: int,
                            rms: float) -> np.ndarray:
    """The field of fourier_modes' stream function on a gh x gw cell-centred grid (FP64, stored FP32)."""
    kx, ky, phi, amp = modes[:, 0], modes[:, 1], modes[:, 2], modes[:, 3]
    xs, ys = node_centres(gh, gw, height, width)
    # cos(kx x + phi + ky y) = cos(ky y) cos(kx x + phi) - sin(ky y) sin(kx x + phi),
    # summed over the modes as two matrix products
    ax = np.outer(xs, kx) + phi[None, :]          # [gw, M]
    ay = np.outer(ys, ky)                         # [gh, M]
    cx, sx, cy, sy = np.cos(ax), np.sin(ax), np.cos(ay), np.sin(ay)
    wu, wv = amp * ky, -amp * kx
    u = (cy * wu) @ cx.T - (sy * wu) @ sx.T
    v = (cy * wv) @ cx.T - (sy * wv) @ sx.T
    scale = rms / math.sqrt(np.mean(u * u + v * v))
    f = np.empty((gh, gw, 2), dtype=np.float64)
    f[..., 0] = u * scale
    f[..., 1] = v * scale
    return f.astype(np.float32)


# ----------------------------------------------------------------------------
# the five workloads (shapes, sizes and distributions of the paper's setups)
# ----------------------------------------------------------------------------

def single_pair_256(seed: int = 0) -> Workload:
    """One 256x256 pair, FP32 output, Lamb-Oseen vortex, RK4 x4, no epilogue."""
    h = w = 256
    pair = PairSpec(height=h, width=w, n_particles=n_particles_for(0.02, h, w), pair_id=0,
                    d_dist=1, d_min=1.0, d_max=4.0, d_mu=2.5, d_sigma=0.3,
                    i_min=0.8, i_max=1.0, z_min=-1.0, z_max=1.0, sheet_sigma=0.5)
    return Workload(name="single_pair_256", seed=seed, pairs=[pair],
                    flows=[lamb_oseen_flow(h, w, h, w)], out_dtype="f32", quant_bits=0,
                    n_substeps=4, dt=1.0,
                    description="1 pair 256x256 ppp 0.02, d~N(2.5,0.3) in [1,4], Lamb-Oseen, RK4x4, f32")


def batch_512_u8(n_pairs: int = 64, seed: int = 1, shared_flow: bool = False,
                 out_dtype: str = "u8", quant_bits: int = 8) -> Workload:
    """n_pairs 512x512 pairs, ppp 0.05, d~U[1,4], Fourier flow rms 3, full epilogue, 8 bit."""
    h = w = 512
    n_flows = 1 if shared_flow else n_pairs
    flows = [fourier_flow(h, w, h, w, rms=3.0, seed=1000 + b) for b in range(n_flows)]
    pairs = [PairSpec(height=h, width=w, n_particles=n_particles_for(0.05, h, w), pair_id=b,
                      flow_index=0 if shared_flow else b, d_dist=0, d_min=1.0, d_max=4.0,
                      illum_min=0.7, illum_max=1.0, noise_sigma=0.02, blur_sigma=0.7)
             for b in range(n_pairs)]
    return Workload(name=f"batch{n_pairs}_512_{out_dtype}", seed=seed, pairs=pairs, flows=flows,
                    out_dtype=out_dtype, quant_bits=quant_bits, n_substeps=4, dt=1.0,
                    description=f"{n_pairs} pairs 512x512 ppp 0.05, d~U[1,4], Fourier rms 3 "
                                f"(F={n_flows}), illum 0.7-1, noise 0.02, blur 0.7, {quant_bits}-bit")


def uneven_batch(n_pairs: int = 256, seed: int = 2, quant_bits: int = 12,
                 sizes=(128, 256, 512, 1024)) -> Workload:
    """Uneven batch: sizes uniform over `sizes`, ppp~U[0.005,0.1], d~U[1,5], 12-bit in u16."""
    rng = np.random.default_rng(seed)
    side = rng.choice(np.asarray(sizes), size=n_pairs)
    ppp = rng.uniform(0.005, 0.1, size=n_pairs)
    pairs, flows = [], []
    for b in range(n_pairs):
        s = int(side[b])
        flows.append(fourier_flow(s, s, s, s, rms=3.0, seed=2000 + b))
        pairs.append(PairSpec(height=s, width=s, n_particles=n_particles_for(float(ppp[b]), s, s),
                              pair_id=b, flow_index=b, d_dist=0, d_min=1.0, d_max=5.0,
                              illum_min=0.7, illum_max=1.0, noise_sigma=0.02, blur_sigma=0.7))
    return Workload(name=f"uneven{n_pairs}", seed=seed, pairs=pairs, flows=flows, out_dtype="u16",
                    quant_bits=quant_bits, n_substeps=4, dt=1.0,
                    description=f"{n_pairs} pairs, sides from {sizes}, ppp~U[0.005,0.1], d~U[1,5], "
                                f"Fourier rms 3, epilogue, {quant_bits}-bit in u16",
                    meta={"ppp": ppp})


def control_grid_flow(n_ctrl: int, size: int, rms: float, seed: int) -> np.ndarray:
    """A coarse Fourier-mode control grid [n_ctrl, n_ctrl, 2] (upsampled by the caller)."""
    return fourier_flow(n_ctrl, n_ctrl, size, size, rms=rms, seed=seed, n_modes=16,
                        k_max_wavelength=size / 4.0)


def differentiable_batch(n_pairs: int = 32, seed: int = 3, size: int = 256,
                         n_ctrl: int = 32) -> Workload:
    """32 pairs 256x256, ppp 0.04, d~U[1.5,3.5], FP32 output, no epilogue.

    The flows are left empty: the differentiable workload builds them by
    upsampling a control grid (``control_grid_flow``) inside torch.
    """
    pairs = [PairSpec(height=size, width=size, n_particles=n_particles_for(0.04, size, size),
                      pair_id=b, flow_index=b, d_dist=0, d_min=1.5, d_max=3.5)
             for b in range(n_pairs)]
    ctrl = [control_grid_flow(n_ctrl, size, rms=2.0, seed=3000 + b) for b in range(n_pairs)]
    return Workload(name=f"diff{n_pairs}_{size}", seed=seed, pairs=pairs, flows=[], out_dtype="f32",
                    quant_bits=0, n_substeps=4, dt=1.0, meta={"control": ctrl, "n_ctrl": n_ctrl},
                    description=f"{n_pairs} pairs {size}x{size}, ppp 0.04, d~U[1.5,3.5], "
                                f"flow = {n_ctrl}^2 control grid upsampled")


def large_mixed_batch(n_big: int = 16, n_hd: int = 16, seed: int = 4,
                      inter_dtype: str = "f16") -> Workload:
    """16x 2048^2 (ppp 0.1, d~U[1,4]) + 16x 1920x1080 (ppp 0.002, d~U[4,10]), 16-bit out."""
    pairs, flows = [], []
    for b in range(n_big):
        flows.append(fourier_flow(2048, 2048, 2048, 2048, rms=8.0, seed=4000 + b))
        pairs.append(PairSpec(height=2048, width=2048, n_particles=n_particles_for(0.1, 2048, 2048),
                              pair_id=b, flow_index=len(flows) - 1, d_min=1.0, d_max=4.0,
                              illum_min=0.7, illum_max=1.0, noise_sigma=0.02, blur_sigma=0.7))
    for b in range(n_hd):
        flows.append(fourier_flow(1080, 1920, 1080, 1920, rms=8.0, seed=4100 + b))
        pairs.append(PairSpec(height=1080, width=1920, n_particles=n_particles_for(0.002, 1080, 1920),
                              pair_id=n_big + b, flow_index=len(flows) - 1, d_min=4.0, d_max=10.0,
                              illum_min=0.7, illum_max=1.0, noise_sigma=0.02, blur_sigma=0.7))
    return Workload(name="large_mixed", seed=seed, pairs=pairs, flows=flows, out_dtype="u16",
                    quant_bits=16, inter_dtype=inter_dtype, n_substeps=4, dt=1.0,
                    description="16x 2048^2 ppp 0.1 d~U[1,4] + 16x 1920x1080 ppp 0.002 d~U[4,10], "
                                f"Fourier rms 8, {inter_dtype} intermediates, 16-bit")


def shapes_batch(n_pairs: int = 64, seed: int = 5, size: int = 512, general: bool = True,
                 hide_prob: float = 0.05) -> Workload:
    """The 512x512 u8 workload with the Eq. 1 shape options of Section 2.

    d~U[1,4] (sigma_x = d/4); with `general`, d_y~U[1,4] and rho~U[-0.6,0.6]
    (axis-misaligned elliptical particles), else round particles; frame-2
    changes of std 0.1 px (each diameter), 0.05 (I0) and 0.05 (rho); each
    particle hidden from each frame with probability hide_prob.
    """
    h = w = size
    flows = [fourier_flow(h, w, h, w, rms=3.0, seed=5000 + b) for b in range(n_pairs)]
    extra = dict(dy_min=1.0, dy_max=4.0, rho_min=-0.6, rho_max=0.6) if general else {}
    pairs = [PairSpec(height=h, width=w, n_particles=n_particles_for(0.05, h, w), pair_id=b,
                      flow_index=b, d_dist=0, d_min=1.0, d_max=4.0, illum_min=0.7, illum_max=1.0,
                      noise_sigma=0.02, blur_sigma=0.7, jitter_d=0.1, jitter_i=0.05,
                      jitter_rho=0.05 if general else 0.0, **extra)
             for b in range(n_pairs)]
    kind = "elliptical d_y~U[1,4] rho~U[-0.6,0.6]" if general else "round"
    return Workload(name=f"shapes{n_pairs}_{size}_{'general' if general else 'round'}", seed=seed,
                    pairs=pairs, flows=flows, out_dtype="u8", quant_bits=8, n_substeps=4, dt=1.0,
                    hide_prob=hide_prob,
                    description=f"{n_pairs} pairs {size}x{size} ppp 0.05, d~U[1,4], {kind}, frame-2 "
                                f"jitter (d 0.1, I0 0.05, rho 0.05), hide {hide_prob}, Fourier rms 3, "
                                f"illum 0.7-1, noise 0.02, blur 0.7, 8-bit")


def ablation_batch(size: int = 512, ppp: float = 0.06, d_min: float = 0.8, d_max: float = 1.2,
                   n_pairs: int = 64, n_flows: int = 1, ppp_min=None, seed: int = 6) -> Workload:
    """One point of the throughput ablations of Section 3.3.

    Defaults are the paper's fixed parameters: 512x512, seeding density 0.06,
    d~U[0.8, 1.2], B = 64 pairs, F = 1 flow field per batch.  With ppp_min,
    each pair's density is drawn from U[ppp_min, ppp] (the spread study).
    Fourier flows (rms 3), RK4 x4, no epilogue, FP32 output.
    """
    rng = np.random.default_rng(seed)
    flows = [fourier_flow(size, size, size, size, rms=3.0, seed=6000 + f) for f in range(n_flows)]
    dens = rng.uniform(ppp_min, ppp, size=n_pairs) if ppp_min is not None else np.full(n_pairs, ppp)
    pairs = [PairSpec(height=size, width=size, n_particles=n_particles_for(float(dens[b]), size, size),
                      pair_id=b, flow_index=b % n_flows, d_dist=0, d_min=d_min, d_max=d_max)
             for b in range(n_pairs)]
    return Workload(name=f"ablation_{size}_{ppp}_{d_max}_{n_pairs}_{n_flows}", seed=seed, pairs=pairs,
                    flows=flows, out_dtype="f32", quant_bits=0, n_substeps=4, dt=1.0,
                    description=f"{n_pairs} pairs {size}x{size}, ppp {ppp if ppp_min is None else (ppp_min, ppp)}, "
                                f"d~U[{d_min},{d_max}], F={n_flows}, f32")


def focus_batch(n_pairs: int = 64, seed: int = 7, size: int = 512, w_rms: float = 0.15,
                sheet_shape: float = 2.0) -> Workload:
    """The 512x512 u8 workload with the Remark's out-of-focus intensity and out-of-plane motion.

    Sheet thickness dz0 = 0.5 (z~U[-1,1]) with shape factor sheet_shape; an
    out-of-plane velocity grid w per pair: the u component of an independent
    Fourier field, rescaled to RMS w_rms (z units per frame).
    """
    h = w = size
    flows = [fourier_flow(h, w, h, w, rms=3.0, seed=7000 + b) for b in range(n_pairs)]
    ws = []
    for b in range(n_pairs):
        g = fourier_flow(h, w, h, w, rms=1.0, seed=7500 + b)[..., 0].astype(np.float64)
        ws.append((g * (w_rms / math.sqrt(np.mean(g * g)))).astype(np.float32))
    pairs = [PairSpec(height=h, width=w, n_particles=n_particles_for(0.05, h, w), pair_id=b, flow_index=b,
                      d_dist=0, d_min=1.0, d_max=4.0, illum_min=0.7, illum_max=1.0, noise_sigma=0.02,
                      blur_sigma=0.7, sheet_sigma=0.5, sheet_model=1, sheet_shape=sheet_shape)
             for b in range(n_pairs)]
    return Workload(name=f"focus{n_pairs}_{size}", seed=seed, pairs=pairs, flows=flows, flows_w=ws,
                    out_dtype="u8", quant_bits=8, n_substeps=4, dt=1.0,
                    description=f"{n_pairs} pairs {size}x{size} ppp 0.05, d~U[1,4], Remark out-of-focus "
                                f"(dz0 0.5, s {sheet_shape}), out-of-plane w rms {w_rms}, Fourier rms 3, "
                                f"illum 0.7-1, noise 0.02, blur 0.7, 8-bit")
