"""Write plk_quad_consts.inc: the kappa-independent constants of the Matern
rho table builder, correctly rounded from 60-digit arithmetic (mpmath).

  QUAD_E1[k]        cosh(t_k) - 1 = 2 sinh^2(t_k / 2), t_k = k QH, k < QNODES (FP64)
  QUAD_E1F[k]       the same as a double-float pair (hi = nearest float,
                    lo = nearest float to the remainder)
  QUAD_CT[k][m]     cos(pi k (m + 1/2) / NC), the Chebyshev nodes' cosines (FP64)
  QUAD_TM[k][m]     coefficient of t^m in the Chebyshev polynomial T_k (integers)

The trapezoid rule for rho(u) = c u^kappa int_0^inf cosh(kappa t) e^{-u cosh t} dt
runs on the fixed nodes t_k; its terms and the Chebyshev fit of each table
sub-interval use these.  Run from this directory: python gen_quad_consts.py
(the values only change with QH, QNODES or NC, which must match plk_common.cuh).
"""
import os
import struct

import mpmath

QH = mpmath.mpf(1) / 8
QNODES = 256
NC = 10

mpmath.mp.dps = 60


def f64(x):
    """Nearest double to the mpf x; values that are zero exactly (cos of an odd
    multiple of pi / 2) come out of 60-digit arithmetic as ~1e-60 and are 0."""
    return 0.0 if abs(x) < mpmath.mpf(10) ** -40 else float(mpmath.nstr(x, 40, strip_zeros=False))


def f32(x):
    return struct.unpack("f", struct.pack("f", x))[0]


def f32_nearest(x):
    """Nearest float to the mpf x (ties cannot occur at these values)."""
    d = f64(x)
    a = f32(d)
    # pick the float closest to x among a and its neighbours
    best = a
    bits = struct.unpack("I", struct.pack("f", a))[0]
    for nb in (bits - 1, bits + 1):
        c = struct.unpack("f", struct.pack("I", nb & 0xFFFFFFFF))[0]
        if abs(mpmath.mpf(c) - x) < abs(mpmath.mpf(best) - x):
            best = c
    return best


def hexd(v):
    return float.hex(v)


def hexf(v):
    return float.hex(v) + "f" if v != 0.0 else "0.0f"


def main():
    e1 = [2 * mpmath.sinh(k * QH / 2) ** 2 for k in range(QNODES)]
    e1d = [f64(v) for v in e1]
    e1h = [f32_nearest(v) for v in e1]
    e1l = [f32_nearest(v - mpmath.mpf(h)) for v, h in zip(e1, e1h)]
    ct = [[f64(mpmath.cos(mpmath.pi * k * (m + mpmath.mpf(1) / 2) / NC)) for m in range(NC)] for k in range(NC)]
    tm = [[0] * NC for _ in range(NC)]
    for k in range(NC):
        for m in range(NC):
            if k == 0:
                tm[k][m] = 1 if m == 0 else 0
            elif k == 1:
                tm[k][m] = 1 if m == 1 else 0
            else:
                tm[k][m] = (2 * tm[k - 1][m - 1] if m > 0 else 0) - tm[k - 2][m]
    out = ["// Generated by gen_quad_consts.py: kappa-independent constants of the rho",
           "// table builder (quadrature nodes t_k = k / 8, k < 256; Chebyshev degree 10).",
           "// Do not edit.", ""]
    out.append("__device__ const double QUAD_E1[QNODES] = {")
    out += ["    " + ", ".join(hexd(v) for v in e1d[i:i + 4]) + "," for i in range(0, QNODES, 4)]
    out.append("};")
    out.append("__device__ const float QUAD_E1F_HI[QNODES] = {")
    out += ["    " + ", ".join(hexf(v) for v in e1h[i:i + 4]) + "," for i in range(0, QNODES, 4)]
    out.append("};")
    out.append("__device__ const float QUAD_E1F_LO[QNODES] = {")
    out += ["    " + ", ".join(hexf(v) for v in e1l[i:i + 4]) + "," for i in range(0, QNODES, 4)]
    out.append("};")
    out.append("__device__ const double QUAD_CT[TAB_NC * TAB_NC] = {")
    out += ["    " + ", ".join(hexd(v) for v in row) + "," for row in ct]
    out.append("};")
    out.append("__device__ const int QUAD_TM[TAB_NC * TAB_NC] = {")
    out += ["    " + ", ".join(str(v) for v in row) + "," for row in tm]
    out.append("};")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "plk_quad_consts.inc")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
