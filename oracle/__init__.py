"""FP64 CPU oracle for PIV image-pair rendering — TEST INFRASTRUCTURE ONLY.

A plain, slow, step-by-step restatement of the method of SynthPix
(arXiv 2512.09664, Section 2) in C (``synthpix_oracle.c``), compiled with
gcc and called through ctypes.  It exists to check the CUDA library; it
shares no code with it, and only the tests, the smoke check and the
CPU-baseline leg of the benchmark may load it.

Parity status: every function here is pinned by CPU tests against closed
forms, library routines (scipy, torch) or brute force; see the tests named
``test_oracle_*``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synthpix_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class OraclePair(C.Structure):
    _fields_ = [
        ("height", C.c_int32), ("width", C.c_int32),
        ("flow_h", C.c_int32), ("flow_w", C.c_int32),
        ("n_particles", C.c_int64),
        ("seed", C.c_uint64), ("pair_id", C.c_uint64),
        ("d_dist", C.c_int32), ("integrator", C.c_int32),
        ("n_substeps", C.c_int32), ("quant_bits", C.c_int32),
        ("d_min", C.c_double), ("d_max", C.c_double), ("d_mu", C.c_double), ("d_sigma", C.c_double),
        ("i_min", C.c_double), ("i_max", C.c_double), ("z_min", C.c_double), ("z_max", C.c_double),
        ("sheet_sigma", C.c_double),
        ("illum_min", C.c_double), ("illum_max", C.c_double),
        ("noise_sigma", C.c_double), ("blur_sigma", C.c_double),
        ("dt", C.c_double),
        ("dy_min", C.c_double), ("dy_max", C.c_double), ("rho_min", C.c_double), ("rho_max", C.c_double),
        ("jitter_d", C.c_double), ("jitter_i", C.c_double), ("jitter_rho", C.c_double),
        ("hide_prob", C.c_double),
        ("sheet_model", C.c_int32), ("sheet_shape", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, FP64, no fast-math, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                                   "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        dp, fp, up = C.POINTER(C.c_double), C.POINTER(C.c_float), C.POINTER(C.c_uint32)
        L.oracle_philox4x32_10.argtypes = [up, up, up]
        L.oracle_stream_words.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, up]
        L.oracle_velocity.argtypes = [fp, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                      C.c_double, C.c_double, dp, dp]
        L.oracle_advect.argtypes = [C.POINTER(OraclePair), fp, C.c_double, C.c_double, dp, dp]
        L.oracle_particles.argtypes = [C.POINTER(OraclePair), fp, dp]
        L.oracle_particles.restype = C.c_int
        L.oracle_pixel_mass.argtypes = [C.c_double, C.c_double, C.c_int64]
        L.oracle_pixel_mass.restype = C.c_double
        L.oracle_pixel_mass2.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                         C.c_int64, C.c_int64]
        L.oracle_pixel_mass2.restype = C.c_double
        L.oracle_splat_shapes.argtypes = [C.c_int32, C.c_int32, dp, C.c_int64, C.c_int32, dp]
        L.oracle_splat_shapes.restype = C.c_int
        L.oracle_particle_shapes.argtypes = [C.POINTER(OraclePair), dp]
        L.oracle_particle_shapes.restype = C.c_int
        L.oracle_round_particles.argtypes = [C.POINTER(OraclePair)]
        L.oracle_round_particles.restype = C.c_int
        L.oracle_splat.argtypes = [C.c_int32, C.c_int32, dp, C.c_int64, C.c_int32, dp]
        L.oracle_splat.restype = C.c_int
        L.oracle_noise.argtypes = [C.c_uint64, C.c_uint64, C.c_int32, C.c_int64]
        L.oracle_noise.restype = C.c_double
        L.oracle_illumination.argtypes = [C.POINTER(OraclePair), C.c_int64, C.c_int64]
        L.oracle_illumination.restype = C.c_double
        L.oracle_blur_radius.argtypes = [C.c_double]
        L.oracle_blur_radius.restype = C.c_int32
        L.oracle_epilogue.argtypes = [C.POINTER(OraclePair), C.c_int32, dp, dp, up]
        L.oracle_epilogue.restype = C.c_int
        L.oracle_render_pair.argtypes = [C.POINTER(OraclePair), fp, dp, dp, up, dp, C.c_int32]
        L.oracle_render_pair.restype = C.c_int
        L.oracle_render_pair3.argtypes = [C.POINTER(OraclePair), fp, fp, dp, dp, up, dp, C.c_int32]
        L.oracle_render_pair3.restype = C.c_int
        L.oracle_match_histogram.argtypes = [up, C.c_int64, C.c_int32, C.POINTER(C.c_uint64)]
        L.oracle_match_histogram.restype = C.c_int
        L.oracle_sheet_gain.argtypes = [C.POINTER(OraclePair), C.c_double]
        L.oracle_sheet_gain.restype = C.c_double
        L.oracle_scalar_at.argtypes = [fp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double]
        L.oracle_scalar_at.restype = C.c_double
        L.oracle_advect3.argtypes = [C.POINTER(OraclePair), fp, fp, C.c_double, C.c_double, C.c_double, dp, dp, dp]
        L.oracle_render_from.argtypes = [C.POINTER(OraclePair), fp, dp, dp]
        L.oracle_render_from.restype = C.c_int
        L.oracle_backward.argtypes = [C.POINTER(OraclePair), fp, dp, dp, dp, dp]
        L.oracle_backward.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


# ----------------------------------------------------------------------------
# parameter marshalling
# ----------------------------------------------------------------------------

def make_pair(spec, seed: int, integrator: str = "rk4", n_substeps: int = 4, dt=1.0,
              quant_bits: int = 0, flow_shape=None, hide_prob=0.0) -> OraclePair:
    """Oracle parameters from a workload PairSpec (FP32 values widened to FP64)."""
    gh, gw = flow_shape if flow_shape is not None else (spec.height, spec.width)
    f = lambda v: float(np.float32(v))  # noqa: E731
    g = lambda k: f(getattr(spec, k, 0.0))  # noqa: E731
    return OraclePair(
        dy_min=g("dy_min"), dy_max=g("dy_max"), rho_min=g("rho_min"), rho_max=g("rho_max"),
        jitter_d=g("jitter_d"), jitter_i=g("jitter_i"), jitter_rho=g("jitter_rho"), hide_prob=f(hide_prob),
        sheet_model=int(getattr(spec, "sheet_model", 0)), sheet_shape=g("sheet_shape"),
        height=spec.height, width=spec.width, flow_h=gh, flow_w=gw,
        n_particles=spec.n_particles, seed=seed, pair_id=spec.pair_id,
        d_dist=spec.d_dist, integrator=0 if integrator == "rk4" else 1,
        n_substeps=n_substeps, quant_bits=quant_bits,
        d_min=f(spec.d_min), d_max=f(spec.d_max), d_mu=f(spec.d_mu), d_sigma=f(spec.d_sigma),
        i_min=f(spec.i_min), i_max=f(spec.i_max), z_min=f(spec.z_min), z_max=f(spec.z_max),
        sheet_sigma=f(spec.sheet_sigma), illum_min=f(spec.illum_min), illum_max=f(spec.illum_max),
        noise_sigma=f(spec.noise_sigma), blur_sigma=f(spec.blur_sigma), dt=f(dt))


def pair_from_workload(wl, b: int) -> OraclePair:
    spec = wl.pairs[b]
    flow = wl.flows[spec.flow_index]
    return make_pair(spec, wl.seed, wl.integrator, wl.n_substeps, wl.dt, wl.quant_bits,
                     flow_shape=flow.shape[:2], hide_prob=getattr(wl, "hide_prob", 0.0))


# ----------------------------------------------------------------------------
# functions
# ----------------------------------------------------------------------------

def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def stream_words(seed: int, pair_id: int, idx: int, tag: int) -> np.ndarray:
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_stream_words(seed, pair_id, idx, tag, _ptr(out, C.c_uint32))
    return out


def velocity(flow: np.ndarray, height: int, width: int, x: float, y: float):
    flow = np.ascontiguousarray(flow, dtype=np.float32)
    u, v = C.c_double(), C.c_double()
    lib().oracle_velocity(_ptr(flow, C.c_float), flow.shape[0], flow.shape[1], height, width,
                          x, y, C.byref(u), C.byref(v))
    return u.value, v.value


def advect(pair: OraclePair, flow: np.ndarray, x: float, y: float):
    flow = np.ascontiguousarray(flow, dtype=np.float32)
    xo, yo = C.c_double(), C.c_double()
    lib().oracle_advect(C.byref(pair), _ptr(flow, C.c_float), x, y, C.byref(xo), C.byref(yo))
    return xo.value, yo.value


PARTICLE_COLUMNS = ("x0", "y0", "d", "I", "z", "Ieff", "x1", "y1")


def particles(pair: OraclePair, flow: np.ndarray) -> np.ndarray:
    """[N, 8] table: x0, y0, d, I, z, Ieff, x1, y1."""
    flow = np.ascontiguousarray(flow, dtype=np.float32)
    out = np.zeros((max(pair.n_particles, 0), 8), dtype=np.float64)
    lib().oracle_particles(C.byref(pair), _ptr(flow, C.c_float), _ptr(out, C.c_double))
    return out


def pixel_mass(c: float, sigma: float, j: int) -> float:
    return lib().oracle_pixel_mass(c, sigma, j)


def pixel_mass2(x0: float, y0: float, sx: float, sy: float, rho: float, j: int, i: int) -> float:
    """Probability of pixel (i, j) under the normal density of Eq. 1 (general shape)."""
    return lib().oracle_pixel_mass2(x0, y0, sx, sy, rho, j, i)


SHAPE_COLUMNS = ("dx", "dy", "rho", "Ieff", "visible")


def particle_shapes(pair: OraclePair) -> np.ndarray:
    """[N, 2, 5] per particle and frame: d_x, d_y, rho, Ieff, visible (1.0 / 0.0)."""
    out = np.zeros((max(pair.n_particles, 0), 2, 5), dtype=np.float64)
    lib().oracle_particle_shapes(C.byref(pair), _ptr(out, C.c_double))
    return out


def splat_shapes(height: int, width: int, parts: np.ndarray, mode: int = 0) -> np.ndarray:
    """Splat rows (x, y, d_x, d_y, rho, Ieff) into a fresh [H, W] frame (modes as splat())."""
    p = np.ascontiguousarray(parts, dtype=np.float64).reshape(-1, 6)
    S = np.zeros((height, width), dtype=np.float64)
    lib().oracle_splat_shapes(height, width, _ptr(p, C.c_double), p.shape[0], mode, _ptr(S, C.c_double))
    return S


def splat(height: int, width: int, parts: np.ndarray, mode: int = 0) -> np.ndarray:
    """Splat rows (x, y, d, Ieff) into a fresh [H, W] frame. mode 0 window, 1 brute, 2 point."""
    p = np.ascontiguousarray(parts, dtype=np.float64).reshape(-1, 4)
    S = np.zeros((height, width), dtype=np.float64)
    lib().oracle_splat(height, width, _ptr(p, C.c_double), p.shape[0], mode, _ptr(S, C.c_double))
    return S


def noise(seed: int, pair_id: int, frame: int, pix: int) -> float:
    return lib().oracle_noise(seed, pair_id, frame, pix)


def illumination(pair: OraclePair, i: int, j: int) -> float:
    return lib().oracle_illumination(C.byref(pair), i, j)


def blur_radius(blur_sigma: float) -> int:
    return lib().oracle_blur_radius(blur_sigma)


def epilogue(pair: OraclePair, frame: int, S: np.ndarray):
    S = np.ascontiguousarray(S, dtype=np.float64)
    B = np.zeros_like(S)
    Q = np.zeros(S.shape, dtype=np.uint32)
    lib().oracle_epilogue(C.byref(pair), frame, _ptr(S, C.c_double), _ptr(B, C.c_double),
                          _ptr(Q, C.c_uint32))
    return B, Q


def match_histogram(codes: np.ndarray, n_codes: int, target) -> np.ndarray:
    """Histogram specification of one quantised frame to target counts (a new array)."""
    c = np.ascontiguousarray(codes, dtype=np.uint32).copy()
    t = np.ascontiguousarray(target, dtype=np.uint64)
    assert t.size == n_codes and int(c.max(initial=0)) < n_codes
    if lib().oracle_match_histogram(_ptr(c, C.c_uint32), c.size, n_codes, t.ctypes.data_as(C.POINTER(C.c_uint64))):
        raise MemoryError("oracle_match_histogram failed")
    return c


def sheet_gain(pair: OraclePair, z: float) -> float:
    return lib().oracle_sheet_gain(C.byref(pair), z)


def scalar_at(w: np.ndarray, height: int, width: int, x: float, y: float) -> float:
    w = np.ascontiguousarray(w, dtype=np.float32)
    return lib().oracle_scalar_at(_ptr(w, C.c_float), w.shape[0], w.shape[1], height, width, x, y)


def advect3(pair: OraclePair, flow: np.ndarray, w: np.ndarray, x: float, y: float, z: float):
    flow = np.ascontiguousarray(flow, dtype=np.float32)
    w = np.ascontiguousarray(w, dtype=np.float32)
    xo, yo, zo = C.c_double(), C.c_double(), C.c_double()
    lib().oracle_advect3(C.byref(pair), _ptr(flow, C.c_float), _ptr(w, C.c_float), x, y, z, C.byref(xo),
                         C.byref(yo), C.byref(zo))
    return xo.value, yo.value, zo.value


def render_pair(pair: OraclePair, flow: np.ndarray, splat_mode: int = 0, want_particles=False, wgrid=None):
    """Returns dict with S [2,H,W], B [2,H,W], Q [2,H,W] (uint32 codes) and parts.
    wgrid: optional [flow_h, flow_w] out-of-plane velocity (moves z along the path)."""
    flow = np.ascontiguousarray(flow, dtype=np.float32)
    wg = None if wgrid is None else np.ascontiguousarray(wgrid, dtype=np.float32)
    H, W = pair.height, pair.width
    S = np.zeros((2, H, W), dtype=np.float64)
    B = np.zeros((2, H, W), dtype=np.float64)
    Q = np.zeros((2, H, W), dtype=np.uint32)
    parts = np.zeros((max(pair.n_particles, 0), 8), dtype=np.float64) if want_particles else None
    rc = lib().oracle_render_pair3(C.byref(pair), _ptr(flow, C.c_float), _ptr(wg, C.c_float), _ptr(S, C.c_double),
                                   _ptr(B, C.c_double), _ptr(Q, C.c_uint32),
                                   _ptr(parts, C.c_double), splat_mode)
    if rc != 0:
        raise MemoryError("oracle_render_pair failed")
    return {"S": S, "B": B, "Q": Q, "parts": parts}


def render_from(pair: OraclePair, flow: np.ndarray, parts_in=None) -> np.ndarray:
    """[2, H, W] = L * S for particles (x0, y0, d) given as [N, 3] (None: seeded)."""
    flow = np.ascontiguousarray(flow, dtype=np.float32)
    pin = None if parts_in is None else np.ascontiguousarray(parts_in, dtype=np.float64).reshape(-1, 3)
    B = np.zeros((2, pair.height, pair.width), dtype=np.float64)
    if lib().oracle_render_from(C.byref(pair), _ptr(flow, C.c_float), _ptr(pin, C.c_double),
                                _ptr(B, C.c_double)) != 0:
        raise MemoryError("oracle_render_from failed")
    return B


def backward(pair: OraclePair, flow: np.ndarray, G: np.ndarray, parts_in=None):
    """Gradients of sum(G * render_from(...)): (grad_flow [gh, gw, 2], grad_parts [N, 3])."""
    flow = np.ascontiguousarray(flow, dtype=np.float32)
    pin = None if parts_in is None else np.ascontiguousarray(parts_in, dtype=np.float64).reshape(-1, 3)
    Gd = np.ascontiguousarray(G, dtype=np.float64)
    gf = np.zeros(flow.shape, dtype=np.float64)
    gp = np.zeros((max(pair.n_particles, 0), 3), dtype=np.float64)
    if lib().oracle_backward(C.byref(pair), _ptr(flow, C.c_float), _ptr(pin, C.c_double), _ptr(Gd, C.c_double),
                             _ptr(gf, C.c_double), _ptr(gp, C.c_double)) != 0:
        raise MemoryError("oracle_backward failed")
    return gf, gp


def render_workload(wl, pairs=None, threads: int | None = None, want_particles=False):
    """Render the selected pairs of a workload on host threads (ctypes releases the GIL)."""
    idx = list(range(wl.n_pairs)) if pairs is None else list(pairs)
    lib()
    fw = getattr(wl, "flows_w", None)

    def one(b):
        fi = wl.pairs[b].flow_index
        return render_pair(pair_from_workload(wl, b), wl.flows[fi], want_particles=want_particles,
                           wgrid=None if fw is None else fw[fi])
    n = threads or min(len(idx), os.cpu_count() or 1)
    if n <= 1:
        return [one(b) for b in idx]
    with ThreadPoolExecutor(max_workers=n) as ex:
        return list(ex.map(one, idx))
