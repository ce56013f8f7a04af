"""Streaming sampler: batches of PIV image pairs, generated on the GPU on demand.

The paper's package is used as an iterator built from a configuration file
(Section 2, "Usage" and "Configuration file"): each step yields a batch of
image pairs, the flow fields they were rendered from and the sampled
parameters.  The configuration fixes the image shape, the batch size B, the
number of flow fields per batch F (B / F pairs share a field) and for how
many consecutive batches a set of flow fields is reused.

    sampler = make("config.yaml")        # or a dict, or a .json file
    batch = next(sampler)
    batch.images1, batch.images2         # [B, H, W] device tensors (views)
    batch.flows                          # [F, gh, gw, 2] velocity grids, px/frame
    batch.flow_fields                    # [B, gh, gw, 2]: each pair's grid (a gather)
    batch.params.seeding_densities       # [B] densities drawn for this batch

Every render goes through the C ABI (synthpix_render_pairs); procedural
flows come from synthpix_fourier_flows on a side stream, one set ahead, so
the next set is generated while the current batch renders (double
buffering).  A batch's tensors stay valid until two further next() calls
(the sampler alternates between two image buffers); a flow set stays valid
while it is in use and for the following set's batches.

Configuration keys (all optional except image_shape):

    image_shape: [H, W]
    batch_size: 64                 flows_per_batch: 1        batches_per_flow: 1
    seed: 0                        device: cuda              tile: 0 (library default)
    seeding_density: [0.05, 0.05]  (a number: fixed; per pair U[min, max], N = floor(ppp H W))
    diameter: [1.0, 4.0]           diameter_distribution: uniform | normal
    diameter_mean: 2.5             diameter_std: 0.3
    intensity: [0.8, 1.0]          out_of_plane: [-1.0, 1.0]  sheet_sigma: 0.5
    illumination: [1.0, 1.0]       noise_sigma: 0.0           blur_sigma: 0.0
    diameter_y: [0, 0]             rho: [0, 0]                hide_prob: 0.0
    jitter: {diameter: 0, intensity: 0, rho: 0}
    output: f32 | f16 | bf16 | u8 | u16     bits: 8           intermediate: f32 | f16 | bf16
    integrator: rk4 | euler        substeps: 4                dt: 1.0
    sheet_model: gaussian | remark  sheet_shape: 2.0 (the Remark's out-of-focus form)
    target_histogram: [counts per code]  (quantised outputs: frames matched to it after each render)
    flow: {kind: fourier, rms: 3.0, modes: 64, min_wavelength: 16.0, grid: [gh, gw]}
          {kind: uniform, u: 1.0, v: 0.0} | {kind: lamb_oseen, gamma: 200.0, core: 20.0}
          or a callable passed to make(): provider(set_index, n_flows, (gh, gw)) -> [F, gh, gw, 2]

YAML files are read with a small parser for the subset above (nested
mappings by indentation, [a, b] lists, numbers, booleans, strings,
comments); JSON files and dicts are accepted as they are.
"""
from __future__ import annotations

import ctypes as C
import json
import os
from dataclasses import dataclass
from typing import Callable, Optional

import numpy as np

from . import binding as B
from . import workloads as W

# ----------------------------------------------------------------------------
# configuration
# ----------------------------------------------------------------------------

DEFAULTS = {
    "batch_size": 64, "flows_per_batch": 1, "batches_per_flow": 1, "seed": 0, "device": "cuda", "tile": 0,
    "seeding_density": [0.05, 0.05], "diameter": [1.0, 4.0], "diameter_distribution": "uniform",
    "diameter_mean": 2.5, "diameter_std": 0.3, "intensity": [0.8, 1.0], "out_of_plane": [-1.0, 1.0],
    "sheet_sigma": 0.5, "illumination": [1.0, 1.0], "noise_sigma": 0.0, "blur_sigma": 0.0,
    "diameter_y": [0.0, 0.0], "rho": [0.0, 0.0], "hide_prob": 0.0,
    "jitter": {"diameter": 0.0, "intensity": 0.0, "rho": 0.0},
    "output": "f32", "bits": 8, "intermediate": "f32", "integrator": "rk4", "substeps": 4, "dt": 1.0,
    "sheet_model": "gaussian", "sheet_shape": 0.0, "target_histogram": None,
    "flow": {"kind": "fourier", "rms": 3.0, "modes": 64, "min_wavelength": 16.0},
}


def _scalar(tok: str):
    t = tok.strip()
    if t == "" or t in ("~", "null", "None"):
        return None
    if t[0] in "'\"" and t[-1] == t[0] and len(t) >= 2:
        return t[1:-1]
    low = t.lower()
    if low in ("true", "yes", "on"):
        return True
    if low in ("false", "no", "off"):
        return False
    if t.startswith("[") and t.endswith("]"):
        inner = t[1:-1].strip()
        return [] if not inner else [_scalar(x) for x in inner.split(",")]
    if t.startswith("{") and t.endswith("}"):
        inner = t[1:-1].strip()
        out = {}
        for item in filter(None, (x.strip() for x in inner.split(","))):
            k, _, v = item.partition(":")
            out[k.strip()] = _scalar(v)
        return out
    for cast in (int, float):
        try:
            return cast(t)
        except ValueError:
            pass
    return t


def parse_yaml_subset(text: str) -> dict:
    """Nested mappings by indentation with scalar, [list] and {map} values."""
    root: dict = {}
    stack = [(-1, root)]
    for raw in text.splitlines():
        line = raw.split(" #")[0].rstrip() if not raw.lstrip().startswith("#") else ""
        if not line.strip():
            continue
        indent = len(line) - len(line.lstrip(" "))
        key, sep, val = line.strip().partition(":")
        if not sep:
            raise ValueError(f"config line without 'key:' -> {raw!r}")
        while stack and indent <= stack[-1][0]:
            stack.pop()
        parent = stack[-1][1]
        if val.strip() == "":
            child: dict = {}
            parent[key.strip()] = child
            stack.append((indent, child))
        else:
            parent[key.strip()] = _scalar(val)
    return root


def load_config(config) -> dict:
    """A configuration dict from a dict, a .json file or a YAML-subset file, defaults filled in."""
    if isinstance(config, (str, os.PathLike)):
        with open(config) as f:
            text = f.read()
        cfg = json.loads(text) if str(config).endswith(".json") else parse_yaml_subset(text)
    else:
        cfg = dict(config)
    out = json.loads(json.dumps(DEFAULTS))
    for k, v in cfg.items():
        if isinstance(v, dict) and isinstance(out.get(k), dict):
            out[k].update(v)
        else:
            out[k] = v
    if "image_shape" not in out:
        raise ValueError("the configuration needs image_shape: [H, W]")
    H, Wd = (int(x) for x in out["image_shape"])
    if H < 1 or Wd < 1:
        raise ValueError("image_shape must be positive")
    Bn, F, R = int(out["batch_size"]), int(out["flows_per_batch"]), int(out["batches_per_flow"])
    if Bn < 1 or F < 1 or F > Bn or R < 1:
        raise ValueError("need batch_size >= 1, 1 <= flows_per_batch <= batch_size, batches_per_flow >= 1")
    out["image_shape"] = [H, Wd]
    for k in ("seeding_density", "diameter", "intensity", "out_of_plane", "illumination", "diameter_y", "rho"):
        v = out[k]
        out[k] = [float(v), float(v)] if not isinstance(v, (list, tuple)) else [float(v[0]), float(v[1])]
    if out["seeding_density"][0] > out["seeding_density"][1] or out["seeding_density"][0] < 0:
        raise ValueError("seeding_density needs 0 <= min <= max")
    return out


# ----------------------------------------------------------------------------
# the sampler
# ----------------------------------------------------------------------------

def pair_spec(cfg: dict, density: float, pair_id: int, flow_index: int) -> W.PairSpec:
    """The pair parameters a configuration gives one pair of a batch."""
    H, Wd = cfg["image_shape"]
    jit = cfg["jitter"]
    return W.PairSpec(
        height=H, width=Wd, n_particles=W.n_particles_for(float(density), H, Wd), pair_id=pair_id,
        flow_index=flow_index, d_dist=1 if cfg["diameter_distribution"] == "normal" else 0,
        d_min=cfg["diameter"][0], d_max=cfg["diameter"][1], d_mu=cfg["diameter_mean"], d_sigma=cfg["diameter_std"],
        i_min=cfg["intensity"][0], i_max=cfg["intensity"][1], z_min=cfg["out_of_plane"][0],
        z_max=cfg["out_of_plane"][1], sheet_sigma=cfg["sheet_sigma"], illum_min=cfg["illumination"][0],
        illum_max=cfg["illumination"][1], noise_sigma=cfg["noise_sigma"], blur_sigma=cfg["blur_sigma"],
        dy_min=cfg["diameter_y"][0], dy_max=cfg["diameter_y"][1], rho_min=cfg["rho"][0], rho_max=cfg["rho"][1],
        jitter_d=jit.get("diameter", 0.0), jitter_i=jit.get("intensity", 0.0), jitter_rho=jit.get("rho", 0.0),
        sheet_model=1 if cfg["sheet_model"] == "remark" else 0, sheet_shape=cfg["sheet_shape"])


def batch_specs(cfg: dict, densities, batch_index: int) -> list:
    """PairSpecs of batch batch_index: pair b has Philox pair id batch_index * B + b and
    uses field b * F // B of the batch's flow set."""
    Bn, F = int(cfg["batch_size"]), int(cfg["flows_per_batch"])
    return [pair_spec(cfg, densities[b], batch_index * Bn + b, b * F // Bn) for b in range(Bn)]


def batch_densities(cfg: dict, batch_index: int) -> np.ndarray:
    """Seeding densities of a batch: U[min, max] per pair from a generator keyed by (seed, batch)."""
    lo, hi = cfg["seeding_density"]
    Bn = int(cfg["batch_size"])
    rng = np.random.default_rng([int(cfg["seed"]), batch_index])
    return rng.uniform(lo, hi, Bn) if hi > lo else np.full(Bn, lo)


def flow_set_of(cfg: dict, batch_index: int) -> int:
    """The flow set a batch renders from: sets change every batches_per_flow batches."""
    return batch_index // int(cfg["batches_per_flow"])


def flow_set_key(seed: int, set_index: int) -> list:
    """Generator key of flow set set_index (all its fields' modes are drawn from it)."""
    return [int(seed), 0x5E7, int(set_index)]


@dataclass
class SampledParams:
    """What was drawn for one batch (host arrays)."""

    seeding_densities: np.ndarray  # [B]
    n_particles: np.ndarray        # [B]
    pair_ids: np.ndarray           # [B] Philox counter words of each pair
    flow_index: np.ndarray         # [B] field of the batch's set used by each pair
    flow_set: int                  # index of the flow set (batch // batches_per_flow)
    batch_index: int


class Batch:
    def __init__(self, images, flows, flow_index_dev, params: SampledParams):
        self.images = images            # [B, 2, H, W]
        self.images1 = images[:, 0]
        self.images2 = images[:, 1]
        self.flows = flows              # [F, gh, gw, 2]
        self.flow_index = flow_index_dev
        self.params = params

    @property
    def flow_fields(self):
        """Each pair's flow grid, [B, gh, gw, 2] (a gather of flows)."""
        return self.flows.index_select(0, self.flow_index)


class Sampler:
    """Iterator over rendered batches; see the module docstring."""

    def __init__(self, config, flow_provider: Optional[Callable] = None):
        import torch
        self.cfg = cfg = load_config(config)
        self.device = torch.device(cfg["device"])
        self.H, self.W = cfg["image_shape"]
        self.B, self.F, self.R = int(cfg["batch_size"]), int(cfg["flows_per_batch"]), int(cfg["batches_per_flow"])
        fl = cfg["flow"]
        self.gh, self.gw = (int(x) for x in fl.get("grid", [self.H, self.W]))
        self.provider = flow_provider
        self.out_dtype = cfg["output"]
        bits = int(cfg["bits"]) if self.out_dtype in ("u8", "u16") else 0
        self.batch = B.batch_desc(int(cfg["seed"]), self.out_dtype, bits, cfg["intermediate"], cfg["integrator"],
                                  int(cfg["substeps"]), float(cfg["dt"]), int(cfg["tile"]), float(cfg["hide_prob"]))
        self.rng_seed = int(cfg["seed"])
        # workspace for the densest batch the configuration can draw
        self.pairs = (B.PairDesc * self.B)()
        self._fill_pairs(np.full(self.B, self.cfg["seeding_density"][1]), 0)
        ws = B.lib().synthpix_workspace_bytes(C.byref(self.batch), self.pairs, self.B)
        if ws == 0:
            raise B.SynthpixError(B.EINVAL, B.last_error())
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=self.device)
        td = B.torch_dtype(self.out_dtype)
        self.images = [torch.empty((self.B, 2, self.H, self.W), dtype=td, device=self.device) for _ in range(2)]
        self.flows = [torch.empty((self.F, self.gh, self.gw, 2), dtype=torch.float32, device=self.device)
                      for _ in range(2)]
        self.flow_stream = torch.cuda.Stream(device=self.device)
        self.flow_ready = [torch.cuda.Event() for _ in range(2)]
        self.flow_free = [torch.cuda.Event() for _ in range(2)]
        self.set_in = [-1, -1]  # flow set held by each flow buffer
        self.kind = fl.get("kind", "fourier") if flow_provider is None else "callable"
        if self.kind == "fourier":
            self.n_modes = int(fl.get("modes", 64))
            self.modes = [torch.empty((self.F, self.n_modes, 4), dtype=torch.float64, device=self.device)
                          for _ in range(2)]
            self.modes_host = [torch.empty((self.F, self.n_modes, 4), dtype=torch.float64).pin_memory()
                               for _ in range(2)]
            fws = B.fourier_flows_workspace_bytes(self.F, self.n_modes, self.gh, self.gw)
            self.flow_ws = torch.empty(fws, dtype=torch.uint8, device=self.device)
        self._flow_index_host = np.array([b * self.F // self.B for b in range(self.B)])
        self.flow_index = torch.from_numpy(self._flow_index_host).to(self.device)
        self.target = None
        if cfg["target_histogram"] is not None:
            if self.out_dtype not in ("u8", "u16"):
                raise ValueError("target_histogram needs a quantised output (u8 / u16)")
            t = np.asarray(cfg["target_histogram"], dtype=np.uint64)
            if t.size != 1 << bits or t.sum() == 0:
                raise ValueError(f"target_histogram needs {1 << bits} counts with a positive total")
            self.target = torch.from_numpy(t).to(self.device)
            self.match_ws = None
        self.k = 0
        self._generate(0)

    # -- descriptors ---------------------------------------------------------
    def _fill_pairs(self, densities, batch_index: int):
        """Descriptors of a batch: built once, then only the particle counts and
        pair ids change (numpy views of the descriptor array's fields)."""
        H, Wd, gh, gw = self.H, self.W, self.gh, self.gw
        if not getattr(self, "_built", False):
            for b, spec in enumerate(batch_specs(self.cfg, densities, batch_index)):
                self.pairs[b] = B.pair_desc(spec, b * 2 * H * Wd, spec.flow_index * gh * gw * 2, (gh, gw))
            raw = np.frombuffer(self.pairs, dtype=np.uint8).reshape(self.B, C.sizeof(B.PairDesc))
            o_n, o_id = B.PairDesc.n_particles.offset, B.PairDesc.pair_id.offset
            self._n_view = raw[:, o_n:o_n + 4].view(np.uint32)[:, 0]
            self._id_view = raw[:, o_id:o_id + 8].view(np.uint64)[:, 0]
            self._built = True
        self._n_view[:] = np.floor(np.asarray(densities, dtype=np.float64) * H * Wd).astype(np.uint32)
        self._id_view[:] = np.arange(self.B, dtype=np.uint64) + np.uint64(batch_index * self.B)

    def densities(self, batch_index: int) -> np.ndarray:
        return batch_densities(self.cfg, batch_index)

    # -- flows ---------------------------------------------------------------
    def flow_set_modes(self, set_index: int) -> np.ndarray:
        """[F, M, 4] stream-function modes of a flow set (host, FP64)."""
        fl = self.cfg["flow"]
        return W.fourier_modes_set(flow_set_key(self.rng_seed, set_index), self.F, self.H, self.W, self.n_modes,
                                   float(fl.get("min_wavelength", 16.0)))

    def _generate(self, set_index: int):
        """Enqueue flow set set_index into buffer set_index % 2 on the flow stream."""
        import torch
        j = set_index % 2
        if self.set_in[j] == set_index:
            return
        fl = self.cfg["flow"]
        st = self.flow_stream
        st.wait_event(self.flow_free[j])  # the renders reading this buffer's previous set are done
        with torch.cuda.stream(st):
            if self.kind == "fourier":
                self.flow_ready[j].synchronize()  # the last copy out of this pinned buffer has completed
                self.modes_host[j].copy_(torch.from_numpy(self.flow_set_modes(set_index)))
                self.modes[j].copy_(self.modes_host[j], non_blocking=True)
                B.fourier_flows(self.modes[j], self.gh, self.gw, self.H, self.W, float(fl.get("rms", 3.0)),
                                self.flows[j], self.flow_ws, stream=st)
            elif self.kind == "callable":
                v = self.provider(set_index, self.F, (self.gh, self.gw))
                self.flows[j].copy_(torch.as_tensor(v, dtype=torch.float32), non_blocking=False)
            elif self.kind == "uniform":
                self.flows[j][..., 0] = float(fl.get("u", 0.0))
                self.flows[j][..., 1] = float(fl.get("v", 0.0))
            elif self.kind == "lamb_oseen":
                g = W.lamb_oseen_flow(self.gh, self.gw, self.H, self.W, float(fl.get("gamma", 200.0)),
                                      float(fl.get("core", 20.0)))
                self.flows[j].copy_(torch.from_numpy(np.broadcast_to(g, self.flows[j].shape).copy()))
            else:
                raise ValueError(f"unknown flow kind {self.kind!r}")
            self.flow_ready[j].record(st)
        self.set_in[j] = set_index

    # -- iteration -----------------------------------------------------------
    def __iter__(self):
        return self

    def __next__(self) -> Batch:
        import torch
        k = self.k
        s = flow_set_of(self.cfg, k)
        j = s % 2
        self._generate(s)  # normally prefetched during the previous batch
        main = torch.cuda.current_stream(self.device)
        main.wait_event(self.flow_ready[j])
        dens = self.densities(k)
        self._fill_pairs(dens, k)
        out = self.images[k % 2]
        rc = B.lib().synthpix_render_pairs(
            C.byref(self.batch), self.pairs, None, self.B, C.c_void_p(self.flows[j].data_ptr()),
            C.c_void_p(out.data_ptr()), C.c_void_p(self.workspace.data_ptr()), self.workspace.numel(),
            C.c_void_p(main.cuda_stream))
        B._check(rc)
        if self.target is not None:  # frames matched to the target histogram, in place
            self.match_ws = B.match_histogram_desc(self.batch, self.pairs, self.B, out, self.target, self.match_ws,
                                                   stream=main)
        self.flow_free[j].record(main)
        self.k += 1
        if (k + 1) // self.R != s:  # the next batch starts a new set: generate it while this one renders
            self._generate(s + 1)
        params = SampledParams(seeding_densities=dens, n_particles=self._n_view.astype(np.int64),
                               pair_ids=self._id_view.copy(), flow_index=self._flow_index_host,
                               flow_set=s, batch_index=k)
        return Batch(out, self.flows[j], self.flow_index, params)

    def workload(self, batch_index: int, device_flows: bool = True) -> W.Workload:
        """The same batch as a Workload of host arrays (checks against the oracle or a Renderer).

        device_flows: take the flow set from the device buffer (it must still
        be resident: the batch's set or the next one); else recompute it on
        the host in FP64 (procedural flows only).
        """
        import torch
        s = flow_set_of(self.cfg, batch_index)
        if device_flows or self.kind != "fourier":
            j = s % 2
            if self.set_in[j] != s:
                raise RuntimeError(f"flow set {s} is no longer resident")
            torch.cuda.synchronize(self.device)
            flows = [f.cpu().numpy() for f in self.flows[j]]
        else:
            fl = self.cfg["flow"]
            flows = [W.fourier_flow_from_modes(m, self.gh, self.gw, self.H, self.W, float(fl.get("rms", 3.0)))
                     for m in self.flow_set_modes(s)]
        cfg = self.cfg
        return W.Workload(name=f"sampler[{batch_index}]", seed=self.rng_seed,
                          pairs=batch_specs(cfg, batch_densities(cfg, batch_index), batch_index), flows=flows,
                          out_dtype=self.out_dtype, quant_bits=int(cfg["bits"]) if self.out_dtype in ("u8", "u16")
                          else 0, inter_dtype=cfg["intermediate"], integrator=cfg["integrator"],
                          n_substeps=int(cfg["substeps"]), dt=float(cfg["dt"]), hide_prob=float(cfg["hide_prob"]))


def make(config, flow_provider: Optional[Callable] = None) -> Sampler:
    """A sampler from a configuration (dict, .json or YAML-subset file)."""
    return Sampler(config, flow_provider)
