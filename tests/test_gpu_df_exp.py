"""The double-float exponential of the mixed path's first-pass Matern table
against CUDA's FP64 exp, through plk_selftest_df_exp: relative error within
2^-44 for arguments in [-50, 86] (the stated ~2^-45 with a factor-2 margin),
within 2^-20 in [-86, -50) (there the low float becomes subnormal), exactly 0
below -86 and +inf above 86; double-float inputs with a nonzero low part
included."""
import numpy as np
import pytest
import torch

from paper_2305_04318_b300 import native as nv

pytestmark = pytest.mark.gpu


def _case(x):
    """Double-float arguments xh + xl around the FP32 grid x: xl up to 2^-25 |xh|."""
    rng = np.random.default_rng(7)
    xh = x.astype(np.float32)
    xl = (xh.astype(np.float64) * rng.uniform(-2.0 ** -25, 2.0 ** -25, size=x.shape)).astype(np.float32)
    return xh, xl


def _run(xh, xl):
    th, tl = torch.as_tensor(xh, device="cuda"), torch.as_tensor(xl, device="cuda")
    yh, yl = nv.selftest_df_exp(th, tl)
    ref = torch.exp(th.double() + tl.double())
    torch.cuda.synchronize()
    return (yh.double() + yl.double()).cpu().numpy(), ref.cpu().numpy()


def test_df_exp_against_fp64_exp():
    x = np.concatenate([np.linspace(-86.0, 86.0, 400001), np.linspace(-1.0, 1.0, 100001),
                        np.array([0.0, -0.0, 1e-30, -1e-30, 0.34657359, -0.34657359])])
    xh, xl = _case(x)
    got, ref = _run(xh, xl)
    xd = xh.astype(np.float64) + xl.astype(np.float64)
    rel = np.abs(got / ref - 1.0)
    main = xd >= -50.0
    tail = (xd >= -86.0) & ~main
    print(f"max rel err on [-50, 86]: {rel[main].max():.3e} (2^{np.log2(rel[main].max() + 1e-300):.1f}); "
          f"on [-86, -50): {rel[tail].max():.3e}")
    assert rel[main].max() <= 2.0 ** -44
    assert rel[tail].max() <= 2.0 ** -20


def test_df_exp_range_ends():
    xh = np.array([-86.5, -100.0, -1e30, 86.5, 100.0, np.inf, -np.inf], dtype=np.float32)
    got, _ = _run(xh, np.zeros_like(xh))
    assert np.all(got[:3] == 0.0) and got[6] == 0.0
    assert np.all(np.isposinf(got[3:6]))
    nan, _ = _run(np.array([np.nan], dtype=np.float32), np.zeros(1, dtype=np.float32))
    assert np.isnan(nan[0])
