"""Thin Python binding of ``libsynthpix.so`` (the C ABI in include/synthpix.h).

Argument marshalling only: descriptors become ctypes structures, tensors
become raw device pointers and the current torch stream is passed through.
Every step of the rendering runs in the library's CUDA kernels; if the
library is missing or fails to load this module raises — there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsynthpix.so")

OK, EINVAL, EWORKSPACE, ECUDA, EUNSUPPORTED = 0, -1, -2, -3, -4
FLAG_GATHER_ADVECT = 1  # advect per particle by direct flow gathers, bin by a counting sort
FLAG_OUT_OF_PLANE = 2   # a w grid follows each flow grid; particles move in z (set by pack for flows_w)
FLAG_TILED_ADVECT = 4   # advect tile by tile from on-chip flow windows (default: per particle while seeding)
DTYPE_CODE = {"f32": 0, "f16": 1, "bf16": 2, "u8": 3, "u16": 4}
INTEGRATOR_CODE = {"rk4": 0, "euler": 1}
_EXPORTS = ("synthpix_workspace_bytes", "synthpix_render_pairs", "synthpix_render_pairs_staged",
            "synthpix_render_pairs_from", "synthpix_seed_particles", "synthpix_advect_particles",
            "synthpix_render_backward", "synthpix_autotune_tile", "synthpix_autotune", "synthpix_tuning_lookup",
            "synthpix_tuning_set", "synthpix_tuning_clear", "synthpix_render_pairs_noalloc",
            "synthpix_fourier_flows", "synthpix_fourier_flows_workspace_bytes", "synthpix_match_histogram",
            "synthpix_match_histogram_workspace_bytes", "synthpix_last_error", "synthpix_version",
            "synthpix_launch_count")
STAGES = ("plan", "seed_advect", "bin_scan", "bin_scatter", "splat_epilogue")


class PairDesc(C.Structure):
    _fields_ = [
        ("height", C.c_int32), ("width", C.c_int32),
        ("image_offset", C.c_int64), ("flow_offset", C.c_int64),
        ("flow_h", C.c_int32), ("flow_w", C.c_int32),
        ("pair_id", C.c_uint64),
        ("n_particles", C.c_uint32), ("d_dist", C.c_int32),
        ("d_min", C.c_float), ("d_max", C.c_float), ("d_mu", C.c_float), ("d_sigma", C.c_float),
        ("i_min", C.c_float), ("i_max", C.c_float), ("z_min", C.c_float), ("z_max", C.c_float),
        ("sheet_sigma", C.c_float), ("illum_min", C.c_float), ("illum_max", C.c_float),
        ("noise_sigma", C.c_float), ("blur_sigma", C.c_float),
        ("dy_min", C.c_float), ("dy_max", C.c_float), ("rho_min", C.c_float), ("rho_max", C.c_float),
        ("jitter_d", C.c_float), ("jitter_i", C.c_float), ("jitter_rho", C.c_float),
        ("sheet_model", C.c_int32), ("sheet_shape", C.c_float), ("reserved", C.c_int32 * 6),
    ]


class BatchDesc(C.Structure):
    _fields_ = [
        ("seed", C.c_uint64), ("out_dtype", C.c_int32), ("quant_bits", C.c_int32),
        ("inter_dtype", C.c_int32), ("integrator", C.c_int32), ("n_substeps", C.c_int32),
        ("dt", C.c_float), ("tile", C.c_int32), ("flags", C.c_int32), ("hide_prob", C.c_float),
        ("reserved", C.c_int32 * 5),
    ]


class Tuning(C.Structure):
    _fields_ = [("tile", C.c_int32 * 4), ("records_per_stage", C.c_int32), ("register_epilogue", C.c_int32),
                ("ms", C.c_float), ("reserved", C.c_int32 * 2)]

    def as_dict(self):
        return {"tile": list(self.tile), "records_per_stage": self.records_per_stage,
                "register_epilogue": self.register_epilogue, "ms": self.ms}


assert C.sizeof(PairDesc) == 160 and C.sizeof(BatchDesc) == 64 and C.sizeof(Tuning) == 36

_lib = None


class SynthpixError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"synthpix error {code}: {msg}")
        self.code = code


def lib():
    """Load the CUDA library (raises if it is absent: no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing; build it with `python -m paper_2512_09664_b300.build`")
        L = C.CDLL(LIB_PATH)
        vp, sz = C.c_void_p, C.c_size_t
        L.synthpix_workspace_bytes.argtypes = [C.POINTER(BatchDesc), C.POINTER(PairDesc), C.c_int32]
        L.synthpix_workspace_bytes.restype = sz
        L.synthpix_render_pairs.argtypes = [C.POINTER(BatchDesc), C.POINTER(PairDesc), vp, C.c_int32,
                                            vp, vp, vp, sz, vp]
        L.synthpix_render_pairs.restype = C.c_int
        L.synthpix_render_pairs_staged.argtypes = [C.POINTER(BatchDesc), C.POINTER(PairDesc), vp, C.c_int32,
                                                   vp, vp, vp, sz, vp, C.POINTER(C.c_void_p)]
        L.synthpix_render_pairs_staged.restype = C.c_int
        L.synthpix_render_pairs_from.argtypes = [C.POINTER(BatchDesc), C.POINTER(PairDesc), vp, C.c_int32,
                                                 vp, vp, vp, vp, sz, vp]
        L.synthpix_render_pairs_from.restype = C.c_int
        L.synthpix_seed_particles.argtypes = [C.POINTER(BatchDesc), C.POINTER(PairDesc), vp, C.c_int32, vp, vp,
                                              sz, vp]
        L.synthpix_seed_particles.restype = C.c_int
        L.synthpix_advect_particles.argtypes = [C.POINTER(BatchDesc), C.POINTER(PairDesc), vp, C.c_int32, vp, vp,
                                                vp, vp, sz, vp]
        L.synthpix_advect_particles.restype = C.c_int
        L.synthpix_render_backward.argtypes = [C.POINTER(BatchDesc), C.POINTER(PairDesc), vp, C.c_int32,
                                               vp, vp, vp, vp, vp, vp, sz, vp]
        L.synthpix_render_backward.restype = C.c_int
        L.synthpix_autotune_tile.argtypes = [C.POINTER(BatchDesc), C.POINTER(PairDesc), vp, C.c_int32,
                                             vp, vp, vp, sz, vp, C.c_int32, C.POINTER(C.c_int32),
                                             C.POINTER(C.c_float)]
        L.synthpix_autotune_tile.restype = C.c_int
        L.synthpix_autotune.argtypes = [C.POINTER(BatchDesc), C.POINTER(PairDesc), vp, C.c_int32,
                                        vp, vp, vp, sz, vp, C.c_int32, C.POINTER(Tuning)]
        L.synthpix_autotune.restype = C.c_int
        L.synthpix_tuning_lookup.argtypes = [C.POINTER(BatchDesc), C.POINTER(PairDesc), C.c_int32, C.POINTER(Tuning)]
        L.synthpix_tuning_lookup.restype = C.c_int
        L.synthpix_tuning_set.argtypes = [C.POINTER(BatchDesc), C.POINTER(PairDesc), C.c_int32, C.POINTER(Tuning)]
        L.synthpix_tuning_set.restype = C.c_int
        L.synthpix_tuning_clear.argtypes = []
        L.synthpix_tuning_clear.restype = None
        L.synthpix_fourier_flows_workspace_bytes.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32]
        L.synthpix_fourier_flows_workspace_bytes.restype = sz
        L.synthpix_fourier_flows.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                             vp, C.c_float, vp, vp, sz, vp]
        L.synthpix_fourier_flows.restype = C.c_int
        L.synthpix_match_histogram_workspace_bytes.argtypes = [C.POINTER(BatchDesc), C.POINTER(PairDesc), C.c_int32]
        L.synthpix_match_histogram_workspace_bytes.restype = sz
        L.synthpix_match_histogram.argtypes = [C.POINTER(BatchDesc), C.POINTER(PairDesc), C.c_int32, vp, vp, vp, sz,
                                               vp]
        L.synthpix_match_histogram.restype = C.c_int
        L.synthpix_last_error.argtypes = []
        L.synthpix_last_error.restype = C.c_char_p
        L.synthpix_version.argtypes = []
        L.synthpix_version.restype = C.c_int
        L.synthpix_launch_count.argtypes = []
        L.synthpix_launch_count.restype = C.c_uint64
        _lib = L
    return _lib


def launch_count() -> int:
    """Kernel launches the library has issued in this process (synthpix_launch_count)."""
    return int(lib().synthpix_launch_count())


def exported_symbols() -> List[str]:
    L = lib()
    return [s for s in _EXPORTS if hasattr(L, s)]


def last_error() -> str:
    return lib().synthpix_last_error().decode()


def _check(rc: int):
    if rc != OK:
        raise SynthpixError(rc, last_error())


# ----------------------------------------------------------------------------
# descriptor marshalling
# ----------------------------------------------------------------------------

def batch_desc(seed: int, out_dtype="f32", quant_bits=0, inter_dtype="f32", integrator="rk4",
               n_substeps=4, dt=1.0, tile=0, hide_prob=0.0) -> BatchDesc:
    b = BatchDesc()
    b.seed = seed
    b.out_dtype = DTYPE_CODE[out_dtype]
    b.quant_bits = quant_bits
    b.inter_dtype = DTYPE_CODE[inter_dtype]
    b.integrator = INTEGRATOR_CODE[integrator]
    b.n_substeps = n_substeps
    b.dt = float(np.float32(dt))
    b.tile = tile
    b.hide_prob = float(np.float32(hide_prob))
    return b


def pair_desc(spec, image_offset: int, flow_offset: int, flow_shape) -> PairDesc:
    p = PairDesc()
    p.height, p.width = spec.height, spec.width
    p.image_offset, p.flow_offset = image_offset, flow_offset
    p.flow_h, p.flow_w = int(flow_shape[0]), int(flow_shape[1])
    p.pair_id = spec.pair_id
    p.n_particles = spec.n_particles
    p.d_dist = spec.d_dist
    for k in ("d_min", "d_max", "d_mu", "d_sigma", "i_min", "i_max", "z_min", "z_max", "sheet_sigma",
              "illum_min", "illum_max", "noise_sigma", "blur_sigma"):
        setattr(p, k, float(getattr(spec, k)))
    for k in ("dy_min", "dy_max", "rho_min", "rho_max", "jitter_d", "jitter_i", "jitter_rho", "sheet_shape"):
        setattr(p, k, float(getattr(spec, k, 0.0)))
    p.sheet_model = int(getattr(spec, "sheet_model", 0))
    return p


def torch_dtype(name: str):
    import torch
    return {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16, "u8": torch.uint8,
            "u16": torch.uint16}[name]


@dataclass
class Packed:
    """A workload laid out for the library: descriptors, flat flows, offsets."""

    batch: BatchDesc
    pairs: C.Array
    n_pairs: int
    flows_host: np.ndarray       # flat float32
    image_offsets: List[int]
    image_elems: int
    out_dtype: str
    shapes: List[tuple]


def pack(wl, tile: int = 0, out_dtype: Optional[str] = None, inter_dtype: Optional[str] = None) -> Packed:
    out_dtype = out_dtype or wl.out_dtype
    flat, flow_off = [], []
    off = 0
    fw = getattr(wl, "flows_w", None)
    for i, f in enumerate(wl.flows):  # each grid's (u, v), then its w when the batch moves particles in z
        flow_off.append(off)
        flat.append(np.ascontiguousarray(f, dtype=np.float32).reshape(-1))
        off += f.size
        if fw is not None:
            w = np.ascontiguousarray(fw[i], dtype=np.float32).reshape(-1)
            assert w.size * 2 == f.size, "w grid must have the flow grid's nodes"
            flat.append(w)
            off += w.size
            if w.size & 1:  # the next grid must start on an even float (8-byte float2 nodes)
                flat.append(np.zeros(1, np.float32))
                off += 1
    arr = (PairDesc * max(wl.n_pairs, 1))()
    img_off, io = [], 0
    for b, spec in enumerate(wl.pairs):
        img_off.append(io)
        arr[b] = pair_desc(spec, io, flow_off[spec.flow_index], wl.flows[spec.flow_index].shape[:2])
        io += 2 * spec.height * spec.width
    bd = batch_desc(wl.seed, out_dtype, wl.quant_bits if out_dtype in ("u8", "u16") else 0,
                    inter_dtype or wl.inter_dtype, wl.integrator, wl.n_substeps, wl.dt, tile,
                    getattr(wl, "hide_prob", 0.0))
    if fw is not None:
        bd.flags |= FLAG_OUT_OF_PLANE
    flows = np.concatenate(flat) if flat else np.zeros(2, np.float32)
    return Packed(bd, arr, wl.n_pairs, flows, img_off, io, out_dtype,
                  [(p.height, p.width) for p in wl.pairs])


def workspace_bytes(pk: Packed) -> int:
    n = lib().synthpix_workspace_bytes(C.byref(pk.batch), pk.pairs, pk.n_pairs)
    if n == 0 and pk.n_pairs > 0:
        raise SynthpixError(EINVAL, last_error())
    return n


def render_pairs(pk: Packed, flows_dev, images_dev, workspace_dev, pairs_dev=None, stream=None) -> None:
    """synthpix_render_pairs on torch tensors (device pointers) and the current stream."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = lib().synthpix_render_pairs(
        C.byref(pk.batch), pk.pairs, C.c_void_p(pairs_dev.data_ptr()) if pairs_dev is not None else None,
        pk.n_pairs, C.c_void_p(flows_dev.data_ptr()), C.c_void_p(images_dev.data_ptr()),
        C.c_void_p(workspace_dev.data_ptr()), workspace_dev.numel() * workspace_dev.element_size(),
        C.c_void_p(st.cuda_stream))
    _check(rc)


def render_pairs_staged(pk: Packed, flows_dev, images_dev, workspace_dev, events, pairs_dev=None,
                        stream=None) -> None:
    """render_pairs recording 6 torch.cuda.Events (already created) at the stage boundaries."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    arr = (C.c_void_p * 6)(*[C.c_void_p(e.cuda_event) if e is not None else None for e in events])
    rc = lib().synthpix_render_pairs_staged(
        C.byref(pk.batch), pk.pairs, C.c_void_p(pairs_dev.data_ptr()) if pairs_dev is not None else None,
        pk.n_pairs, C.c_void_p(flows_dev.data_ptr()), C.c_void_p(images_dev.data_ptr()),
        C.c_void_p(workspace_dev.data_ptr()), workspace_dev.numel() * workspace_dev.element_size(),
        C.c_void_p(st.cuda_stream), arr)
    _check(rc)


def fourier_flows(modes_dev, flow_h: int, flow_w: int, height: int, width: int, rms: float, flows_dev,
                  workspace_dev, stream=None) -> None:
    """synthpix_fourier_flows: modes_dev float64 [F, M, 4] -> flows_dev float32 [F, flow_h, flow_w, 2]."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    F, M = int(modes_dev.shape[0]), int(modes_dev.shape[1])
    rc = lib().synthpix_fourier_flows(F, M, flow_h, flow_w, height, width, C.c_void_p(modes_dev.data_ptr()),
                                      float(rms), C.c_void_p(flows_dev.data_ptr()),
                                      C.c_void_p(workspace_dev.data_ptr()),
                                      workspace_dev.numel() * workspace_dev.element_size(), C.c_void_p(st.cuda_stream))
    _check(rc)


def fourier_flows_workspace_bytes(n_flows: int, n_modes: int, flow_h: int, flow_w: int) -> int:
    n = lib().synthpix_fourier_flows_workspace_bytes(n_flows, n_modes, flow_h, flow_w)
    if n == 0:
        raise SynthpixError(EINVAL, last_error())
    return n


def match_histogram_desc(batch: BatchDesc, pairs, n_pairs: int, images_dev, target_dev, workspace_dev=None,
                         stream=None):
    """synthpix_match_histogram on rendered images (in place) from raw descriptors; returns the workspace."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    if workspace_dev is None:
        n = lib().synthpix_match_histogram_workspace_bytes(C.byref(batch), pairs, n_pairs)
        if n == 0 and n_pairs > 0:
            raise SynthpixError(EINVAL, last_error())
        workspace_dev = torch.empty(max(n, 256), dtype=torch.uint8, device=images_dev.device)
    rc = lib().synthpix_match_histogram(C.byref(batch), pairs, n_pairs, C.c_void_p(images_dev.data_ptr()),
                                        C.c_void_p(target_dev.data_ptr()), C.c_void_p(workspace_dev.data_ptr()),
                                        workspace_dev.numel(), C.c_void_p(st.cuda_stream))
    _check(rc)
    return workspace_dev


def match_histogram(pk: Packed, images_dev, target_dev, workspace_dev=None, stream=None):
    """synthpix_match_histogram on a packed batch's rendered images (in place); returns the workspace."""
    return match_histogram_desc(pk.batch, pk.pairs, pk.n_pairs, images_dev, target_dev, workspace_dev, stream)


def size_class(height: int, width: int) -> int:
    """Frame size class of the tuning table (the library's rule): area < 2^15, < 2^17, < 2^19, larger."""
    a = height * width
    return 0 if a < (1 << 15) else (1 if a < (1 << 17) else (2 if a < (1 << 19) else 3))


def tuning_clear():
    """Empty the library's tuning table (synthpix_tuning_clear)."""
    lib().synthpix_tuning_clear()


class Renderer:
    """Device buffers for repeated rendering of one packed workload."""

    def __init__(self, wl, device="cuda", tile: int = 0, out_dtype=None, inter_dtype=None,
                 device_descriptors: bool = True, flags: int = 0):
        import torch
        self.pk = pack(wl, tile=tile, out_dtype=out_dtype, inter_dtype=inter_dtype)
        self.pk.batch.flags |= flags
        self.device = torch.device(device)
        self.flows = torch.from_numpy(self.pk.flows_host).to(self.device)
        ws = workspace_bytes(self.pk)
        self.workspace = torch.empty(max(ws, 256), dtype=torch.uint8, device=self.device)
        self.images = torch.empty(max(self.pk.image_elems, 1), dtype=torch_dtype(self.pk.out_dtype),
                                  device=self.device)
        self.pairs_dev = None
        if device_descriptors and self.pk.n_pairs > 0:
            raw = np.frombuffer(C.string_at(C.addressof(self.pk.pairs), C.sizeof(PairDesc) * self.pk.n_pairs),
                                dtype=np.uint8)
            self.pairs_dev = torch.from_numpy(raw.copy()).to(self.device)

    def render(self, stream=None):
        render_pairs(self.pk, self.flows, self.images, self.workspace, self.pairs_dev, stream)
        return self.images

    def render_staged(self, events, stream=None):
        render_pairs_staged(self.pk, self.flows, self.images, self.workspace, events, self.pairs_dev, stream)
        return self.images

    def autotune(self, reps: int = 3, stream=None):
        """Pick one tile edge for the whole batch with synthpix_autotune_tile; later renders use it."""
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        best, ms = C.c_int32(0), C.c_float(0.0)
        saved = self.pk.batch.tile
        self.pk.batch.tile = 0
        rc = lib().synthpix_autotune_tile(
            C.byref(self.pk.batch), self.pk.pairs,
            C.c_void_p(self.pairs_dev.data_ptr()) if self.pairs_dev is not None else None, self.pk.n_pairs,
            C.c_void_p(self.flows.data_ptr()), C.c_void_p(self.images.data_ptr()),
            C.c_void_p(self.workspace.data_ptr()), self.workspace.numel(), C.c_void_p(st.cuda_stream), reps,
            C.byref(best), C.byref(ms))
        if rc != OK:
            self.pk.batch.tile = saved
            _check(rc)
        self.pk.batch.tile = best.value
        return best.value, ms.value

    def _tile0(self):
        """Switch to tile 0 (per-class edges from the tuning table), growing the workspace if needed."""
        import torch
        self.pk.batch.tile = 0
        ws = workspace_bytes(self.pk)
        if ws > self.workspace.numel():
            self.workspace = torch.empty(ws, dtype=torch.uint8, device=self.device)

    def tune(self, reps: int = 3, stream=None) -> dict:
        """synthpix_autotune: tile edge per size class, records per stage and epilogue path.

        The result goes into the library's table; this renderer switches to
        tile 0, so its later renders use it (as does any batch of the same
        classes).  Returns the chosen parameters and their time per render.
        """
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        self._tile0()
        t = Tuning()
        _check(lib().synthpix_autotune(
            C.byref(self.pk.batch), self.pk.pairs,
            C.c_void_p(self.pairs_dev.data_ptr()) if self.pairs_dev is not None else None, self.pk.n_pairs,
            C.c_void_p(self.flows.data_ptr()), C.c_void_p(self.images.data_ptr()),
            C.c_void_p(self.workspace.data_ptr()), self.workspace.numel(), C.c_void_p(st.cuda_stream), reps,
            C.byref(t)))
        return t.as_dict()

    def tuning(self) -> dict:
        """The parameters this renderer's next render runs with (synthpix_tuning_lookup)."""
        t = Tuning()
        _check(lib().synthpix_tuning_lookup(C.byref(self.pk.batch), self.pk.pairs, self.pk.n_pairs, C.byref(t)))
        return t.as_dict()

    def set_tuning(self, tile, records_per_stage: int, register_epilogue: int):
        """Write parameters into the tuning table for this batch's classes and switch to tile 0."""
        self._tile0()
        t = Tuning()
        for k in range(4):
            t.tile[k] = int(tile[k])
        t.records_per_stage, t.register_epilogue = int(records_per_stage), int(register_epilogue)
        _check(lib().synthpix_tuning_set(C.byref(self.pk.batch), self.pk.pairs, self.pk.n_pairs, C.byref(t)))

    def capture(self):
        """Capture one render into a CUDA graph (descriptors must be on the device)."""
        import torch
        assert self.pairs_dev is not None or self.pk.n_pairs == 0
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.render()
        torch.cuda.current_stream().wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.render()
        return self.graph

    def replay(self):
        self.graph.replay()
        return self.images

    # --- differentiable use -------------------------------------------------
    def _ptrs(self, stream):
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        pd = C.c_void_p(self.pairs_dev.data_ptr()) if self.pairs_dev is not None else None
        return pd, C.c_void_p(self.workspace.data_ptr()), self.workspace.numel(), C.c_void_p(st.cuda_stream)

    @staticmethod
    def _vp(t):
        return C.c_void_p(t.data_ptr()) if t is not None else None

    def seed_particles(self, stream=None):
        """[sum N, 3] float32 device tensor of the seeded (x0, y0, d)."""
        import torch
        n = sum(p.n_particles for p in self.pk.pairs[:self.pk.n_pairs])
        out = torch.empty((max(n, 1), 3), dtype=torch.float32, device=self.device)
        pd, ws, wsn, st = self._ptrs(stream)
        _check(lib().synthpix_seed_particles(C.byref(self.pk.batch), self.pk.pairs, pd, self.pk.n_pairs,
                                             self._vp(out), ws, wsn, st))
        return out[:n]

    def advect_particles(self, particles=None, dt=None, flows=None, stream=None):
        """[sum N, 3] float32 device tensor: (x, y, d) advected over dt (default: the batch's dt)
        from the given frame-1 particles (default: the seeded ones)."""
        import torch
        flows = self.flows if flows is None else flows
        n = sum(p.n_particles for p in self.pk.pairs[:self.pk.n_pairs])
        out = torch.empty((max(n, 1), 3), dtype=torch.float32, device=self.device)
        saved = self.pk.batch.dt
        if dt is not None:
            self.pk.batch.dt = float(dt)
        try:
            pd, ws, wsn, st = self._ptrs(stream)
            _check(lib().synthpix_advect_particles(C.byref(self.pk.batch), self.pk.pairs, pd, self.pk.n_pairs,
                                                   self._vp(particles), self._vp(flows), self._vp(out), ws, wsn,
                                                   st))
        finally:
            self.pk.batch.dt = saved
        return out[:n]

    def render_from(self, flows=None, particles=None, stream=None):
        """Render with the given flow tensor (default: the packed flows) and particles (or seeded)."""
        flows = self.flows if flows is None else flows
        pd, ws, wsn, st = self._ptrs(stream)
        _check(lib().synthpix_render_pairs_from(C.byref(self.pk.batch), self.pk.pairs, pd, self.pk.n_pairs,
                                                self._vp(particles), self._vp(flows), self._vp(self.images),
                                                ws, wsn, st))
        return self.images

    def backward(self, grad_images, flows=None, particles=None, grad_flows=None, grad_particles=None, stream=None):
        """synthpix_render_backward: grad_flows is accumulated, grad_particles overwritten."""
        flows = self.flows if flows is None else flows
        pd, ws, wsn, st = self._ptrs(stream)
        _check(lib().synthpix_render_backward(C.byref(self.pk.batch), self.pk.pairs, pd, self.pk.n_pairs,
                                              self._vp(particles), self._vp(flows), self._vp(grad_images),
                                              self._vp(grad_flows), self._vp(grad_particles), ws, wsn, st))

    def frames(self, b: int):
        """[2, H, W] view of pair b in the output buffer."""
        h, w = self.pk.shapes[b]
        o = self.pk.image_offsets[b]
        return self.images[o:o + 2 * h * w].view(2, h, w)


class HostPipeline:
    """Batches rendered from pinned host flow grids into pinned host images.

    A step copies its flow grids in on an upload stream, renders them with
    synthpix_render_pairs on the caller's stream and copies the images out on
    a download stream.  `depth` device sets of (flows, images) let the upload
    of step k+1 and the download of step k-1 run on the copy engines while
    step k renders, so in steady state a step costs its longest part, not the
    sum of the three.  Every step uses the renderer's packed batch (pair
    descriptors and sizes); only the flows differ.  The caller must not
    overwrite a step's host flows before its `uploaded` event nor read its
    host images before the event submit() returns.  Every step must render
    on the same stream: the renders share the renderer's workspace, so two
    of them must never overlap.
    """

    def __init__(self, renderer: "Renderer", depth: int = 2):
        import torch
        if depth < 1:
            raise ValueError("depth must be at least 1")
        self.r = renderer
        self.depth = depth
        self.flows = [renderer.flows] + [torch.empty_like(renderer.flows) for _ in range(depth - 1)]
        self.images = [renderer.images] + [torch.empty_like(renderer.images) for _ in range(depth - 1)]
        self.up = torch.cuda.Stream(renderer.device)
        self.down = torch.cuda.Stream(renderer.device)
        self.uploaded = [torch.cuda.Event() for _ in range(depth)]
        self.rendered = [torch.cuda.Event() for _ in range(depth)]
        self.downloaded = [torch.cuda.Event() for _ in range(depth)]
        self.used = [False] * depth
        self.k = 0
        self.stream = None  # the render stream, fixed by the first step

    def submit(self, flows_host, images_host, stream=None):
        """Queue one step; returns the event after which images_host holds its images."""
        import torch
        st = stream if stream is not None else torch.cuda.current_stream(self.r.device)
        if self.stream is None:
            self.stream = st
        elif st.cuda_stream != self.stream.cuda_stream:
            raise ValueError("every step must render on the stream of the first one (shared workspace)")
        if flows_host.numel() != self.flows[0].numel() or images_host.numel() != self.images[0].numel():
            raise ValueError("host buffers do not match the packed batch")
        s = self.k % self.depth
        if self.used[s]:
            self.up.wait_event(self.rendered[s])  # the render that last read this flow set
        with torch.cuda.stream(self.up):
            self.flows[s].copy_(flows_host, non_blocking=True)
        self.uploaded[s].record(self.up)
        st.wait_event(self.uploaded[s])
        if self.used[s]:
            st.wait_event(self.downloaded[s])  # the download that last read this image set
        render_pairs(self.r.pk, self.flows[s], self.images[s], self.r.workspace, self.r.pairs_dev, st)
        self.rendered[s].record(st)
        self.down.wait_event(self.rendered[s])
        with torch.cuda.stream(self.down):
            images_host.copy_(self.images[s], non_blocking=True)
        self.downloaded[s].record(self.down)
        self.used[s] = True
        self.k += 1
        return self.downloaded[s]

    def synchronize(self, stream=None):
        """Make `stream` (default: the current one) wait for every queued copy."""
        import torch
        st = stream if stream is not None else torch.cuda.current_stream(self.r.device)
        st.wait_stream(self.up)
        st.wait_stream(self.down)


def _render_fn():
    import torch

    class RenderFunction(torch.autograd.Function):
        """images = render(flows, particles); differentiable in both (float output)."""

        @staticmethod
        def forward(ctx, flows, particles, renderer):
            renderer.render_from(flows, particles)
            ctx.renderer = renderer
            ctx.save_for_backward(flows, particles)
            return renderer.images.clone()

        @staticmethod
        def backward(ctx, grad):
            flows, particles = ctx.saved_tensors
            r = ctx.renderer
            gf = torch.zeros_like(flows) if ctx.needs_input_grad[0] else None
            gp = torch.empty_like(particles) if (particles is not None and ctx.needs_input_grad[1]) else None
            r.backward(grad.contiguous().float(), flows, particles, gf, gp)
            return gf, gp, None

    return RenderFunction


_RENDER_FN = None


def render(renderer: "Renderer", flows, particles=None):
    """Differentiable render through the C ABI (torch.autograd.Function).

    flows: flat float32 device tensor laid out like ``renderer.flows``;
    particles: None (seeded) or a [sum N, 3] float32 device tensor (x0, y0, d).
    Returns the flat image buffer (FP32 output workloads).
    """
    global _RENDER_FN
    if _RENDER_FN is None:
        _RENDER_FN = _render_fn()
    return _RENDER_FN.apply(flows, particles, renderer)
