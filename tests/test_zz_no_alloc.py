"""The allocation-free entry point, plk_eval_device_static.

It exists for callers that must not allocate device memory while they
evaluate (a plugin whose host application owns the device-memory budget, a
latency-critical loop that cannot afford cudaMalloc/cudaFree stalling other
work).  This file is named so that pytest collects it last.  It checks, on two
calls in a row with different problem sizes, that the entry point agrees with
plk_eval_device (same tolerance as the other GPU tests), and that a size too
large for its fixed scratch array is refused before any work is queued.
"""
import math

import numpy as np
import pytest
import torch

from paper_2305_04318_b300 import native as nv, synth
from gpu_util import RTOL_LOGL, compare, gpu_eval, oracle_eval, to_dev

pytestmark = pytest.mark.gpu


def _static(ds, params, lambdas, reml=False):
    out = nv.eval_device_static(to_dev(ds.coords), to_dev(ds.y), to_dev(ds.X), to_dev(lambdas), to_dev(params),
                                reml=reml)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_static_scratch_matches_workspace_entry_point_twice():
    """Calls in a row share the scratch array.  The third case has n = 1000
    sites, for which 8 points fit in the array at once: its 23 points run as
    batches of 8, 8 and 7 at different offsets of the same array; that case is
    also compared with the oracle directly."""
    cases = [
        (synth.aniso_dataset(501, 300, math.sqrt(30), 3), 23, synth.LAMBDA_GRID_9, False),
        (synth.aniso_dataset(502, 129, math.sqrt(12.9), 2), 9, np.array([0.0, 0.5]), True),
        (synth.aniso_dataset(504, 1000, 10.0, 3), 23, synth.LAMBDA_GRID_9, False),
    ]
    assert nv.workspace_bytes(1000, 3, 9, 8) <= nv.STATIC_SCRATCH_BYTES < nv.workspace_bytes(1000, 3, 9, 16)   # several batches
    for ds, K, lams, reml in cases:
        P = synth.omega_from_unit(np.random.default_rng(K + ds.n).uniform(size=(K, 5)))
        got = _static(ds, P, lams, reml=reml)
        ref = gpu_eval(ds, P, lams, reml=reml)
        compare(got, ref, rtol=RTOL_LOGL, what=f"static vs workspace, n={ds.n}")
        if ds.n == 1000:
            compare(got, oracle_eval(ds, P, lams), rtol=RTOL_LOGL, what="static vs oracle, n=1000")


def test_static_scratch_rejects_too_large_n():
    ds = synth.aniso_dataset(503, 4000, 20.0, 3)
    P = np.array([[1.0, 1.0, 0.1, 1.0, 0.0]])
    with pytest.raises(nv.PlkError) as e:
        _static(ds, P, np.array([0.0]))
    assert e.value.status == nv.PLK_E_NOMEM
    assert "static scratch" in str(e.value)
