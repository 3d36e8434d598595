"""The generated constants of the rho table builder (plk_quad_consts.inc):
the committed file is what its generator writes, and its values agree with
independent FP64 evaluations of their definitions (cosh(t) - 1 at the
trapezoid nodes t_k = k / 8, the Chebyshev nodes' cosines, the monomial
coefficients of T_k from their closed form)."""
import math
import os
import re
import subprocess
import sys
from math import comb

import numpy as np

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2305_04318_b300", "csrc")
INC = os.path.join(CSRC, "plk_quad_consts.inc")


def _arrays(text):
    out = {}
    for m in re.finditer(r"const (double|float|int) (\w+)\[[^\]]*\] = \{(.*?)\};", text, re.S):
        kind, name, body = m.groups()
        vals = [v.strip() for v in body.replace("\n", " ").split(",") if v.strip()]
        if kind == "int":
            out[name] = np.array([int(v) for v in vals])
        else:
            out[name] = np.array([float.fromhex(v.rstrip("f")) for v in vals])
    return out


def test_generator_reproduces_committed_file(tmp_path):
    import shutil
    shutil.copy(os.path.join(CSRC, "gen_quad_consts.py"), tmp_path / "gen_quad_consts.py")
    subprocess.run([sys.executable, str(tmp_path / "gen_quad_consts.py")], check=True, cwd=tmp_path)
    assert (tmp_path / "plk_quad_consts.inc").read_text() == open(INC).read()


def test_values_against_their_definitions():
    a = _arrays(open(INC).read())
    t = np.arange(256) / 8.0
    e1 = np.array([2.0 * math.sinh(x / 2.0) ** 2 for x in t])           # cosh t - 1
    np.testing.assert_allclose(a["QUAD_E1"], e1, rtol=1e-15, atol=0)   # e1 itself: ~3 roundings
    np.testing.assert_allclose(a["QUAD_E1"][1:], np.cosh(t[1:]) - 1.0, rtol=1e-13)
    hi, lo = a["QUAD_E1F_HI"], a["QUAD_E1F_LO"]
    assert np.all(hi.astype(np.float32) == hi) and np.all(lo.astype(np.float32) == lo)
    assert np.all(np.abs(lo) <= np.abs(hi) * 2.0 ** -24)                 # normalised pairs
    np.testing.assert_allclose(hi + lo, e1, rtol=2.0 ** -46, atol=0)
    # cos(pi x), x = k (m + 1/2) / 10 reduced exactly to [0, 2) first (so that
    # the FP64 reference carries ~1 rounding of pi x, not k (m + 1/2) of them)
    from fractions import Fraction
    ct = np.array([[math.cos(math.pi * float(Fraction(kk * (2 * mm + 1), 20) % 2)) for mm in range(10)]
                   for kk in range(10)])
    np.testing.assert_allclose(a["QUAD_CT"].reshape(10, 10), ct, rtol=0, atol=8e-16)
    # T_k(x) = (k/2) sum_j (-1)^j / (k - j) C(k - j, j) (2x)^(k - 2j), k >= 1
    tm = np.zeros((10, 10), dtype=np.int64)
    tm[0, 0] = 1
    for kk in range(1, 10):
        for j in range(kk // 2 + 1):
            c = kk * (-1) ** j * comb(kk - j, j) * 2 ** (kk - 2 * j) // (2 * (kk - j))
            tm[kk, kk - 2 * j] += c
    np.testing.assert_array_equal(a["QUAD_TM"].reshape(10, 10), tm)
