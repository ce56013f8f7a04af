"""Helpers shared by the parity tests: run the CUDA path and the oracle on the
same seeded workload and compare them element by element.

Tolerances (stated per the method's arithmetic):
  * float outputs: |GPU - oracle| <= 1e-4 of full scale (1.0);
  * quantised outputs: codes bit-exact, except pixels whose FP64 oracle value
    lies within 1e-6 (full scale) of a rounding boundary (k + 1/2) / M; those
    are counted and returned, never asserted on;
  * 16-bit float outputs: the oracle value rounded to the storage type, plus
    the float tolerance and one storage ulp (two values within 1e-6 of each
    other can round to neighbouring 16-bit codes).
"""
from __future__ import annotations

import numpy as np

FLOAT_TOL = 1e-4
BAND = 1e-6


def gpu_render(wl, tile: int = 0, out_dtype=None, renderer=None, inter_dtype=None):
    import torch

    from paper_2512_09664_b300.binding import Renderer
    r = renderer or Renderer(wl, tile=tile, out_dtype=out_dtype, inter_dtype=inter_dtype)
    r.render()
    torch.cuda.synchronize()
    outs = []
    for b in range(wl.n_pairs):
        t = r.frames(b)
        if t.dtype == torch.uint16:
            outs.append(t.view(torch.int16).cpu().numpy().view(np.uint16))
        elif t.dtype in (torch.float16, torch.bfloat16):
            outs.append(t.float().cpu().numpy())
        else:
            outs.append(t.cpu().numpy())
    return outs


def oracle_render(wl, pairs=None):
    import oracle
    return oracle.render_workload(wl, pairs=pairs)


def compare(wl, gpu, ref, out_dtype=None):
    """Assert parity; returns a dict of statistics."""
    out_dtype = out_dtype or wl.out_dtype
    stats = {"max_abs": 0.0, "band": 0, "mismatch": 0, "pixels": 0}
    for g, r in zip(gpu, ref):
        B = r["B"]
        stats["pixels"] += B.size
        if out_dtype in ("u8", "u16"):
            M = float(2 ** wl.quant_bits - 1)
            q = r["Q"].astype(np.int64)
            gq = g.astype(np.int64)
            frac = B * M - np.floor(B * M)
            near = np.abs(frac - 0.5) < BAND * M
            bad = gq != q
            stats["band"] += int(near.sum())
            stats["mismatch"] += int(bad.sum())
            outside = bad & ~near
            assert not outside.any(), (
                f"{int(outside.sum())} quantised codes differ away from rounding boundaries; "
                f"first at {np.argwhere(outside)[0]}: gpu {gq[outside][0]} oracle {q[outside][0]} "
                f"B={B[outside][0]!r}")
            assert int(np.abs(gq - q).max(initial=0)) <= 1
        else:
            ref_v = B
            tol = FLOAT_TOL
            if out_dtype == "f16":
                # both sides round a value within 1e-6 of the other: at most one
                # storage ulp (<= |B| 2^-10) apart
                ref_v = B.astype(np.float16).astype(np.float64)
                tol = FLOAT_TOL + np.abs(B) * 2.0 ** -10
            elif out_dtype == "bf16":
                import torch
                ref_v = torch.from_numpy(B).to(torch.bfloat16).double().numpy()
                tol = FLOAT_TOL + np.abs(B) * 2.0 ** -7
            err = np.abs(g.astype(np.float64) - ref_v)
            stats["max_abs"] = max(stats["max_abs"], float(err.max(initial=0.0)))
            assert np.all(err <= tol), f"max |gpu - oracle| = {err.max()} > {FLOAT_TOL}"
    return stats
