"""Generate phi_table.cuh: the upper tail Q(t) = erfc(t / sqrt 2) / 2 of the
standard normal on [0, 8] as 129 cubic pieces.

Method: Chebyshev interpolation (Trefethen, "Approximation Theory and
Approximation Practice", ch. 4) of Q on each interval [k/16 - 1/32, k/16 +
1/32], k = 0..128, at 25 Chebyshev points, truncated to degree 3 and converted
to powers of s = t - k/16; coefficients rounded to FP32.  Q is evaluated with
scipy.special.erfc in FP64.  The kernels clamp t to 8 (Q(8) = 6.2e-16) and
select the piece k = rint(16 t), so each piece is used on its own interval.

    python -m paper_2512_09664_b300.csrc.gen_phi_table   # rewrites phi_table.cuh

The script checks the FP32 Horner evaluation of the rounded coefficients
(each step rounded separately, a bound on the FMA evaluation) against FP64 Q
on a dense grid and refuses to write a table whose absolute error exceeds
4e-8 (0.7 FP32 ulp at Q = 1/2; the pixel masses are differences of Q values,
so absolute accuracy is what matters).  The truncation error alone is below
1e-9; the rest is FP32 rounding.
"""
from __future__ import annotations

import os

import numpy as np
from numpy.polynomial import chebyshev as Ch
from scipy.special import erfc

PIECES_PER_UNIT = 16
T_MAX = 8.0
N_PIECES = int(T_MAX * PIECES_PER_UNIT) + 1
DEGREE = 3
HERE = os.path.dirname(os.path.abspath(__file__))


def q_tail(t):
    return 0.5 * erfc(np.asarray(t, dtype=np.float64) / np.sqrt(2.0))


def piece_coefficients(k: int) -> np.ndarray:
    c = k / PIECES_PER_UNIT
    half = 0.5 / PIECES_PER_UNIT
    # Chebyshev interpolant in x in [-1, 1], t = c + half x
    cheb = Ch.chebinterpolate(lambda x: q_tail(c + half * x), 24)
    cheb = cheb[:DEGREE + 1]
    mono_x = Ch.cheb2poly(cheb)                      # powers of x
    return mono_x / half ** np.arange(DEGREE + 1)    # powers of s = half x


def horner32(coef32: np.ndarray, s: np.ndarray) -> np.ndarray:
    acc = np.full(s.shape, coef32[-1], dtype=np.float32)
    s32 = s.astype(np.float32)
    for a in coef32[-2::-1]:
        acc = (acc * s32 + a).astype(np.float32)  # separate rounding: an upper bound on FMA error
    return acc


def build():
    table = np.zeros((N_PIECES, DEGREE + 1), dtype=np.float32)
    worst = 0.0
    half = 0.5 / PIECES_PER_UNIT
    for k in range(N_PIECES):
        c = k / PIECES_PER_UNIT
        coef = piece_coefficients(k).astype(np.float32)
        table[k] = coef
        t = np.linspace(max(c - half, 0.0), min(c + half, T_MAX), 2001).astype(np.float32)
        s = (t.astype(np.float64) - c).astype(np.float32)  # exact in the kernels (Sterbenz)
        exact = q_tail(t.astype(np.float64))
        err = np.abs(horner32(coef, s).astype(np.float64) - exact)
        worst = max(worst, float(err.max()))
    return table, worst


def write(path=os.path.join(HERE, "phi_table.cuh")):
    table, worst = build()
    if worst > 4e-8:
        raise SystemExit(f"table error {worst:.3e} too large")
    lines = ["// Generated by gen_phi_table.py: upper normal tail Q(t) = erfc(t / sqrt 2) / 2 on [0, 8]",
             f"// as {N_PIECES} Chebyshev-interpolated cubic pieces in s = t - k/{PIECES_PER_UNIT}, "
             f"k = rint({PIECES_PER_UNIT} t);",
             "// piece k = (c0, c1, c2, c3) at kPhiTable[4 k ..].  Max |error| of FP32 Horner",
             f"// on a dense grid: {worst:.2e}.",
             "#pragma once", "", "namespace spx {", "",
             f"constexpr int kPhiPieces = {N_PIECES};", f"constexpr int kPhiDegree = {DEGREE};",
             f"constexpr float kPhiPerUnit = {float(PIECES_PER_UNIT):.1f}f;",
             f"constexpr float kPhiTMax = {T_MAX:.1f}f;",
             f"static __device__ __constant__ float kPhiTable[{(DEGREE + 1) * N_PIECES}] = {{"]
    for k in range(N_PIECES):
        vals = ", ".join(f"{float(v):.9e}f" for v in table[k])
        lines.append(f"    {vals},")
    lines += ["};", "", "}  // namespace spx", ""]
    with open(path, "w") as f:
        f.write("\n".join(lines))
    return worst


if __name__ == "__main__":
    print(f"max abs error {write():.3e}")
