"""Context API on the GPU: device-resident datasets, asynchronous jobs,
continuous batching; results equal the stateless path's and are the same
alone and in the mix."""
import math

import numpy as np
import pytest
import torch

from paper_2305_04318_b300 import native as nv, synth
from gpu_util import gpu_eval

pytestmark = pytest.mark.gpu


def test_jobs_match_stateless_and_mix():
    dsets = [synth.aniso_dataset(40 + i, n, math.sqrt(n / 10), p) for i, (n, p) in enumerate([(300, 3), (700, 2), (150, 5)])]
    lams = synth.LAMBDA_GRID_9
    grids = [synth.omega_from_unit(np.random.default_rng(i).uniform(size=(K, 5))) for i, K in enumerate([37, 20, 50])]
    ref = [gpu_eval(d, g, lams, batch=8) for d, g in zip(dsets, grids)]
    arena = torch.empty(6 << 30, dtype=torch.uint8, device="cuda")
    with nv.Context(arena.numel(), arena=arena, n_streams=3) as ctx:
        ids = [ctx.create_dataset(d.coords, d.y, d.X) for d in dsets]
        # alone
        alone = []
        for i, d in enumerate(dsets):
            j = ctx.submit(ids[i], grids[i], lams, batch=8)
            alone.append(ctx.poll(j, d.p))
        # all at once (interleaved on 3 streams)
        jobs = [ctx.submit(ids[i], grids[i], lams, batch=8) for i in range(3)]
        mix = [ctx.poll(j, dsets[i].p) for i, j in enumerate(jobs)]
        used, high = ctx.memory_stats()
        assert high > used > 0
        for i in range(3):
            for k in ("logL", "sigma2", "beta", "logdet", "status"):
                np.testing.assert_array_equal(alone[i][k], ref[i][k])
                np.testing.assert_array_equal(mix[i][k], ref[i][k])
            assert mix[i]["t_done"] >= mix[i]["t_start"] >= mix[i]["t_submit"]
        for i in ids:
            ctx.release_dataset(i)


def test_context_validation_and_nomem():
    with nv.Context(64 << 20, n_streams=1) as ctx:
        d = synth.aniso_dataset(1, 50, 2.0, 2)
        with pytest.raises(nv.PlkError):
            ctx.create_dataset(d.coords, -d.y, d.X)
        big = synth.aniso_dataset(2, 4000, 20.0, 3)
        ds = ctx.create_dataset(big.coords, big.y, big.X)
        with pytest.raises(nv.PlkError) as e:
            ctx.submit(ds, np.array([[1.0, 1.0, 0.1, 1.0, 0.0]]), [0.0])
        assert e.value.status == nv.PLK_E_NOMEM
        ds2 = ctx.create_dataset(d.coords, d.y, d.X)
        j = ctx.submit(ds2, np.array([[0.5, 1.0, 0.1, 1.0, 0.0]]), [0.0, 1.0])
        r = ctx.poll(j, 2)
        assert r["status"][0] == 0 and np.all(np.isfinite(r["logL"]))
        j = ctx.submit(ds2, np.zeros((0, 5)), [0.0])
        assert ctx.poll(j, 2)["logL"].shape == (0, 1)


def test_mixed_jobs_same_alone_and_in_the_mix():
    """Continuous batching in mixed precision: three jobs run alone, then
    submitted together over three streams; every result is identical."""
    dsets = [synth.aniso_dataset(70 + i, n, math.sqrt(n / 10), 3) for i, n in enumerate([500, 900, 260])]
    lams = synth.LAMBDA_GRID_9
    grids = [synth.omega_from_unit(np.random.default_rng(10 + i).uniform(size=(K, 5))) for i, K in enumerate([30, 18, 41])]
    arena = torch.empty(8 << 30, dtype=torch.uint8, device="cuda")
    with nv.Context(arena.numel(), arena=arena, n_streams=3) as ctx:
        ids = [ctx.create_dataset(d.coords, d.y, d.X) for d in dsets]
        alone = [ctx.poll(ctx.submit(ids[i], grids[i], lams, precision=nv.MIXED, batch=8), 3) for i in range(3)]
        jobs = [ctx.submit(ids[i], grids[i], lams, precision=nv.MIXED, batch=8) for i in range(3)]
        mix = [ctx.poll(j, 3) for j in jobs]
    for i in range(3):
        for k in ("logL", "sigma2", "beta", "logdet", "status"):
            np.testing.assert_array_equal(alone[i][k], mix[i][k])
        ref = gpu_eval(dsets[i], grids[i], lams, precision=nv.MIXED, batch=8)
        np.testing.assert_array_equal(alone[i]["logL"], ref["logL"])


@pytest.mark.parametrize("precision", [nv.FP64, nv.MIXED])
def test_autotuned_batch_is_used_and_results_unchanged(precision):
    """plk_autotune picks one of the candidate batch sizes for n's half-octave
    bucket; jobs submitted with batch = 0 on a dataset in that bucket use it,
    and their results equal those of an explicit batch size bit for bit (each
    point's arithmetic depends only on its own data)."""
    ds = synth.aniso_dataset(61, 300, math.sqrt(30.0), 3)
    lams = synth.LAMBDA_GRID_9
    P = synth.omega_from_unit(np.random.default_rng(61).uniform(size=(45, 5)))
    arena = torch.empty(4 << 30, dtype=torch.uint8, device="cuda")
    with nv.Context(arena.numel(), arena=arena, n_streams=2) as ctx:
        assert ctx.scheduled_batch(300, precision)[1] is False
        b, rate = ctx.autotune(300, 3, len(lams), precision, candidates=[4, 8, 16])
        assert b in (4, 8, 16) and rate > 0
        assert ctx.scheduled_batch(300, precision) == (b, True)
        assert ctx.scheduled_batch(330, precision) == (b, True)      # same or neighbouring bucket
        assert ctx.scheduled_batch(2000, precision)[1] is False      # far away: library default
        d = ctx.create_dataset(ds.coords, ds.y, ds.X)
        tuned = ctx.poll(ctx.submit(d, P, lams, precision=precision), ds.p)
        explicit = ctx.poll(ctx.submit(d, P, lams, precision=precision, batch=7), ds.p)
        for k in ("logL", "sigma2", "beta", "logdet", "status"):
            np.testing.assert_array_equal(tuned[k], explicit[k], err_msg=k)
        ctx.release_dataset(d)


def test_bounded_wait_gives_up_and_device_stays_usable():
    """Failure detection without a fault: a bounded wait on a barrier that
    nothing completes gives up, the call reports PLK_E_TIMEOUT, and the device
    keeps working (an evaluation right after matches the oracle)."""
    import oracle
    assert nv.selftest_bounded_wait(1000) == nv.PLK_E_TIMEOUT
    assert nv.selftest_bounded_wait(50) == nv.PLK_E_TIMEOUT
    with pytest.raises(nv.PlkError):
        nv._check(nv.lib().plk_selftest_bounded_wait(0, None))
    ds = synth.aniso_dataset(62, 140, math.sqrt(14.0), 2)
    P = synth.omega_from_unit(np.random.default_rng(62).uniform(size=(6, 5)))
    lams = synth.LAMBDA_GRID_9
    g = gpu_eval(ds, P, lams, precision=nv.MIXED)
    o = oracle.profile_batch(ds.coords, ds.y, ds.X, P, lams)
    ok = o["status"] == 0
    assert np.max(np.abs(g["logL"][ok] - o["logL"][ok])) <= 1e-3


def test_cancel_and_fault_hooks_on_a_gpu_context(tmp_path):
    """plk_cancel on a running GPU job (its in-flight batches finish, the rest
    are dropped), an injected batch failure and arena-allocation failures,
    all made on the host; the context keeps producing the stateless path's
    results afterwards; every job leaves one metrics line."""
    import json
    ds = synth.aniso_dataset(63, 1500, math.sqrt(150.0), 3)
    lams = synth.LAMBDA_GRID_9
    P = synth.omega_from_unit(np.random.default_rng(63).uniform(size=(400, 5)))
    small = P[:12]
    ref = gpu_eval(ds, small, lams, batch=4)
    log = tmp_path / "jobs.jsonl"
    arena = torch.empty(6 << 30, dtype=torch.uint8, device="cuda")
    with nv.Context(arena.numel(), arena=arena, n_streams=1) as ctx:
        ctx.set_metrics_log(str(log))
        d = ctx.create_dataset(ds.coords, ds.y, ds.X)
        big = ctx.submit(d, P, lams, batch=4)           # 100 batches
        assert ctx.poll(big, ds.p, timeout_ms=200) is None
        ctx.cancel(big)
        with pytest.raises(nv.PlkError) as e:
            ctx.poll(big, ds.p)
        assert e.value.status == nv.PLK_E_CANCELLED
        ctx.inject_fault(nv.FAULT_BATCH, 1)
        with pytest.raises(nv.PlkError) as e:
            ctx.poll(ctx.submit(d, small, lams, batch=4), ds.p)
        assert "injected batch failure" in str(e.value)
        ctx.inject_fault(nv.FAULT_ARENA_ALLOC, 3)
        r = ctx.poll(ctx.submit(d, small, lams, batch=4), ds.p)
        for k in ("logL", "sigma2", "beta", "logdet", "status"):
            np.testing.assert_array_equal(r[k], ref[k], err_msg=k)
        ctx.release_dataset(d)
    lines = [json.loads(x) for x in log.read_text().splitlines()]
    assert [x["outcome"] for x in lines] == ["cancelled", "failed", "ok"]
    assert 1 <= lines[0]["items"] < 100
