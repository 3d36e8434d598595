"""Host-side checks of libplk.so that need no GPU: it loads, exports every
function include/plk.h declares, sizes workspaces, validates arguments."""
import ctypes as C

import pytest
import scipy.stats as st

from paper_2305_04318_b300 import build, native as nv


@pytest.fixture(scope="module")
def L():
    build.build()
    return nv.lib()


def test_exports_every_declared_symbol(L):
    names = nv.declared_symbols()
    assert len(names) >= 13
    for n in names:
        assert hasattr(L, n), n


def test_workspace_sizes(L):
    assert nv.workspace_bytes(4000, 3, 9, 1) > 0
    assert nv.workspace_bytes(4000, 3, 9, 8) > 7 * nv.workspace_bytes(4000, 3, 9, 1) * 0.9
    # tiles: (nb + 1)(nb + 2)/2 tiles of 128 x 128 doubles per point
    nb = 32
    assert nv.workspace_bytes(4000, 3, 9, 1) >= (nb + 1) * (nb + 2) // 2 * 128 * 128 * 8
    for bad in [(3, 3, 1), (10, 0, 1), (10, 17, 1), (100, 3, 0), (100, 10, 60)]:
        assert nv.workspace_bytes(*bad, 1) == 0
    assert nv.workspace_bytes(100, 2, 1, 1, precision=7) == 0


def test_chi2_quantile(L):
    for lev in (0.5, 0.9, 0.95, 0.999):
        assert abs(nv.chi2_1_quantile(lev) - st.chi2.ppf(lev, 1)) < 1e-11


def test_eval_device_rejects_bad_arguments_without_touching_the_gpu(L):
    a = nv.EvalArgs(n=10, p=2, M=1)   # NULL input pointers
    o = nv.Options(0, 0, 1, 0)
    assert L.plk_eval_device(C.byref(a), C.byref(o), None, 0, None) == nv.PLK_E_INVALID
    assert b"NULL" in L.plk_last_error()
    a = nv.EvalArgs(n=2, p=2, M=1)
    assert L.plk_eval_device(C.byref(a), C.byref(o), None, 0, None) == nv.PLK_E_INVALID
    assert L.plk_eval_device(None, C.byref(o), None, 0, None) == nv.PLK_E_INVALID


def test_profile_ci_rejects_bad_level(L):
    assert L.plk_profile_ci_device(None, None, 5, 0.95, None, None) == nv.PLK_E_INVALID
    assert L.plk_profile_max_device(None, 3, 0, None, None) == nv.PLK_E_INVALID


def test_post_processing_rejects_bad_arguments_without_touching_the_gpu(L):
    a = nv.StatsArgs(n=10, p=2, M=1, K=4)   # NULL input pointers
    assert L.plk_profile_beta_device(C.byref(a), 0, None, 3, None, None) == nv.PLK_E_INVALID
    assert L.plk_profile_sigma_device(None, None, 3, None, None) == nv.PLK_E_INVALID
    a = nv.StatsArgs(n=10, p=17, M=1, K=4)
    assert L.plk_profile_sigma_device(C.byref(a), None, 3, None, None) == nv.PLK_E_INVALID
    assert b"bad sizes" in L.plk_last_error()
    assert L.plk_profile_lambda_device(None, 5, 0, None, None) == nv.PLK_E_INVALID
    assert L.plk_profile_hull_device(None, 0, None, 5, None, 0, None, None, None) == nv.PLK_E_INVALID
    assert L.plk_internal_params_device(None, 3, 0, None, None) == nv.PLK_E_INVALID
    # nothing to do is not an error and launches nothing
    assert L.plk_internal_params_device(None, 0, 0, None, None) == nv.PLK_OK


def test_binding_constants_match_header():
    """Every PLK_FLAG_* and PLK_POINT_* value of include/plk.h has the same
    value in the Python binding (the binding restates them by hand)."""
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(nv.__file__), os.pardir, "include", "plk.h")).read()
    defs = dict(re.findall(r"^#define PLK_((?:FLAG|POINT|FAULT|SCHED)_\w+)\s+(\d+)", hdr, re.M))
    assert len(defs) >= 10
    for name, value in defs.items():
        assert getattr(nv, name) == int(value), name


def test_static_scratch_size_matches_header():
    """The binding's size of the allocation-free entry point's scratch array
    equals PLK_STATIC_SCRATCH_BYTES of include/plk.h."""
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(nv.__file__), os.pardir, "include", "plk.h")).read()
    m = re.search(r"#define PLK_STATIC_SCRATCH_BYTES \(\(size_t\)(\d+) << (\d+)\)", hdr)
    assert m, "PLK_STATIC_SCRATCH_BYTES not found"
    assert nv.STATIC_SCRATCH_BYTES == int(m.group(1)) << int(m.group(2))


def test_mixed_tolerance_setting(L):
    """plk_set_mixed_tolerance: default 1e-3, values in (0, 1] taken, others
    refused with the setting unchanged (no GPU needed)."""
    from paper_2305_04318_b300 import native as nv
    assert nv.get_mixed_tolerance() == 1e-3
    try:
        nv.set_mixed_tolerance(1e-4)
        assert nv.get_mixed_tolerance() == 1e-4
        for bad in (0.0, -1e-3, 2.0, float("nan"), float("inf")):
            with pytest.raises(RuntimeError):
                nv.set_mixed_tolerance(bad)
            assert nv.get_mixed_tolerance() == 1e-4
    finally:
        nv.set_mixed_tolerance(1e-3)


def test_pipe_counters_absent_from_the_plain_build(L):
    """plk_pipe_counters exists in every build; without -DPLK_PIPE_COUNTERS it
    refuses (no GPU needed)."""
    buf = (C.c_uint64 * 27)()
    assert L.plk_pipe_counters(C.cast(buf, C.c_void_p), 0) == nv.PLK_E_INVALID
    assert b"PLK_PIPE_COUNTERS" in L.plk_last_error()
