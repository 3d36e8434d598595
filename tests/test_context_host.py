"""The context's scheduler without a GPU: plk_create_with_evaluator runs the
same admission, continuous batching, cancellation, fault hooks and metrics
log as a GPU context, with every batch evaluated on the host by a callback
(here the FP64 oracle).  Failures are made on the host (fault hooks, an
evaluator that raises); nothing here touches a GPU."""
import json
import threading
import time

import numpy as np
import pytest

from paper_2305_04318_b300 import native as nv, synth


def oracle_fn(delay=0.0, fail_on=None):
    import oracle

    def fn(coords, y, X, params, lambdas):
        if delay:
            time.sleep(delay)
        if fail_on is not None and np.any(np.all(np.isclose(params, fail_on), axis=1)):
            raise RuntimeError("evaluator failure")
        return oracle.profile_batch(coords, y, X, params, lambdas, nthreads=1)
    return fn


def _problem(seed=5, n=40, K=23, M=3):
    ds = synth.aniso_dataset(seed, n, 2.0, 3)
    P = synth.omega_from_unit(np.random.default_rng(seed).uniform(size=(K, 5)))
    return ds, P, np.linspace(-0.5, 1.5, M)


def _ref(ds, P, lams):
    import oracle
    return oracle.profile_batch(ds.coords, ds.y, ds.X, P, lams, nthreads=1)


def _same(r, ref):
    for k in ("logL", "sigma2", "beta", "logdet", "status"):
        np.testing.assert_array_equal(r[k], ref[k], err_msg=k)


def test_interleaved_jobs_equal_the_oracle():
    jobs = [_problem(s, n=30 + 7 * s, K=9 + 4 * s) for s in range(4)]
    with nv.Context(64 << 20, n_streams=3, evaluator=oracle_fn()) as ctx:
        ids = [ctx.create_dataset(ds.coords, ds.y, ds.X) for ds, _, _ in jobs]
        sub = [ctx.submit(i, P, lams, batch=4) for i, (ds, P, lams) in zip(ids, jobs)]
        for (ds, P, lams), j in zip(jobs, sub):
            _same(ctx.poll(j, ds.p), _ref(ds, P, lams))
        for i in ids:
            ctx.release_dataset(i)


def test_admission_with_a_small_arena():
    """An arena that holds the job's inputs and outputs but only a few batch
    workspaces at a time: batches wait for space and the job still
    completes; the high-water mark stays within the arena."""
    ds, P, lams = _problem(K=40)
    arena = 1 << 20
    with nv.Context(arena, n_streams=4, evaluator=oracle_fn(delay=0.002)) as ctx:
        d = ctx.create_dataset(ds.coords, ds.y, ds.X)
        _same(ctx.poll(ctx.submit(d, P, lams, batch=8), ds.p), _ref(ds, P, lams))
        used, high = ctx.memory_stats()
        assert high <= arena


def test_cancel_running_and_queued_jobs(tmp_path):
    ds, P, lams = _problem(K=60)
    log = tmp_path / "metrics.jsonl"
    with nv.Context(64 << 20, n_streams=1, evaluator=oracle_fn(delay=0.02)) as ctx:
        ctx.set_metrics_log(str(log))
        d = ctx.create_dataset(ds.coords, ds.y, ds.X)
        running = ctx.submit(d, P, lams, batch=2)     # 30 batches of ~20 ms on one worker
        queued = ctx.submit(d, P[:5], lams, batch=2)  # waits behind it
        time.sleep(0.1)
        ctx.cancel(running)
        ctx.cancel(queued)
        for j in (running, queued):
            with pytest.raises(nv.PlkError) as e:
                ctx.poll(j, ds.p)
            assert e.value.status == nv.PLK_E_CANCELLED
        # the context keeps working after cancellations
        after = ctx.submit(d, P[:6], lams, batch=2)
        _same(ctx.poll(after, ds.p), _ref(ds, P[:6], lams))
        # cancelling a finished job changes nothing: its results stay available
        done = ctx.submit(d, P[:3], lams)
        time.sleep(0.2)
        ctx.cancel(done)
        _same(ctx.poll(done, ds.p), _ref(ds, P[:3], lams))
        with pytest.raises(nv.PlkError):
            ctx.cancel(done)                          # forgotten after its poll
    lines = [json.loads(x) for x in log.read_text().splitlines()]
    outcome = {x["job"]: x["outcome"] for x in lines}
    assert outcome[running["id"]] == "cancelled" and outcome[queued["id"]] == "cancelled"
    assert outcome[after["id"]] == "ok" and outcome[done["id"]] == "ok"
    r = [x for x in lines if x["job"] == running["id"]][0]
    assert 1 <= r["items"] < 30                          # it stopped part-way


def test_fault_arena_allocation_failures_are_absorbed():
    ds, P, lams = _problem(K=17)
    with nv.Context(64 << 20, n_streams=2, evaluator=oracle_fn()) as ctx:
        d = ctx.create_dataset(ds.coords, ds.y, ds.X)
        ctx.inject_fault(nv.FAULT_ARENA_ALLOC, 6)
        _same(ctx.poll(ctx.submit(d, P, lams, batch=8), ds.p), _ref(ds, P, lams))


def test_fault_batch_failure_fails_only_its_job(tmp_path):
    ds, P, lams = _problem(K=12)
    log = tmp_path / "m.jsonl"
    with nv.Context(64 << 20, n_streams=1, evaluator=oracle_fn()) as ctx:
        ctx.set_metrics_log(str(log))
        d = ctx.create_dataset(ds.coords, ds.y, ds.X)
        ctx.inject_fault(nv.FAULT_BATCH, 1)
        bad = ctx.submit(d, P, lams, batch=4)
        with pytest.raises(nv.PlkError) as e:
            ctx.poll(bad, ds.p)
        assert e.value.status == nv.PLK_E_CUDA and "injected batch failure" in str(e.value)
        _same(ctx.poll(ctx.submit(d, P, lams, batch=4), ds.p), _ref(ds, P, lams))
    outs = [json.loads(x)["outcome"] for x in log.read_text().splitlines()]
    assert outs == ["failed", "ok"]


def test_evaluator_failure_fails_the_job():
    ds, P, lams = _problem(K=8)
    with nv.Context(64 << 20, n_streams=2, evaluator=oracle_fn(fail_on=P[5])) as ctx:
        d = ctx.create_dataset(ds.coords, ds.y, ds.X)
        with pytest.raises(nv.PlkError) as e:
            ctx.poll(ctx.submit(d, P, lams, batch=2), ds.p)
        assert e.value.status == nv.PLK_E_CUDA and "evaluator returned" in str(e.value)


def test_fault_dropped_completion_is_still_seen():
    ds, P, lams = _problem(K=4)
    with nv.Context(64 << 20, n_streams=1, evaluator=oracle_fn()) as ctx:
        d = ctx.create_dataset(ds.coords, ds.y, ds.X)
        ctx.inject_fault(nv.FAULT_DROP_COMPLETION, 5)
        for timeout in (-1, 5000):
            t0 = time.perf_counter()
            _same(ctx.poll(ctx.submit(d, P, lams), ds.p, timeout_ms=timeout), _ref(ds, P, lams))
            assert time.perf_counter() - t0 < 2.0


def test_poll_timeout_and_concurrent_pollers():
    ds, P, lams = _problem(K=10)
    with nv.Context(64 << 20, n_streams=2, evaluator=oracle_fn(delay=0.05)) as ctx:
        d = ctx.create_dataset(ds.coords, ds.y, ds.X)
        j = ctx.submit(d, P, lams, batch=1)
        assert ctx.poll(j, ds.p, timeout_ms=0) is None
        assert ctx.poll(j, ds.p, timeout_ms=20) is None
        got = {}
        others = [ctx.submit(d, P[:2], lams) for _ in range(3)]

        def waiter(k, job):
            got[k] = ctx.poll(job, ds.p)
        th = [threading.Thread(target=waiter, args=(k, o)) for k, o in enumerate(others)]
        for t in th:
            t.start()
        _same(ctx.poll(j, ds.p), _ref(ds, P, lams))
        for t in th:
            t.join(timeout=30)
        ref2 = _ref(ds, P[:2], lams)
        for k in range(3):
            _same(got[k], ref2)


def test_metrics_lines(tmp_path):
    ds, P, lams = _problem(K=10)
    log = tmp_path / "m.jsonl"
    with nv.Context(64 << 20, n_streams=2, evaluator=oracle_fn()) as ctx:
        ctx.set_metrics_log(str(log))
        d = ctx.create_dataset(ds.coords, ds.y, ds.X)
        ctx.poll(ctx.submit(d, P, lams, batch=3), ds.p)
        ctx.set_metrics_log(None)
        ctx.poll(ctx.submit(d, P, lams, batch=3), ds.p)    # not logged
    lines = log.read_text().splitlines()
    assert len(lines) == 1
    m = json.loads(lines[0])
    assert m["K"] == 10 and m["items"] == 4 and m["batch"] == 3 and m["outcome"] == "ok"
    assert m["n"] == ds.n and m["p"] == ds.p and m["M"] == len(lams) and m["precision"] == "fp64"
    assert m["queue_wait_s"] >= 0 and m["run_s"] > 0 and m["evals_per_s"] > 0
    assert m["item_ms_p50"] <= m["item_ms_p99"]
    assert 0 < m["arena_high_water"]


def test_host_context_refuses_autotune_and_bad_faults():
    with nv.Context(64 << 20, n_streams=1, evaluator=oracle_fn()) as ctx:
        with pytest.raises(nv.PlkError):
            ctx.autotune(100, 2, 1)
        with pytest.raises(nv.PlkError):
            ctx.inject_fault(99, 1)
        with pytest.raises(nv.PlkError):
            ctx.inject_fault(nv.FAULT_BATCH, -1)


def test_largest_first_policy_orders_jobs_by_dataset_size(tmp_path):
    """With one worker busy on a first job, three jobs queue; FIFO starts them
    in submission order, largest-first by decreasing n; results are the same."""
    small, mid, large = (_problem(s, n=n, K=4) for s, n in ((1, 20), (2, 35), (3, 50)))
    order = {}
    for policy in (nv.SCHED_FIFO, nv.SCHED_LARGEST_FIRST):
        log = tmp_path / f"m{policy}.jsonl"
        with nv.Context(64 << 20, n_streams=1, evaluator=oracle_fn(delay=0.05)) as ctx:
            ctx.set_schedule_policy(policy)
            ctx.set_metrics_log(str(log))
            ids = {name: ctx.create_dataset(ds.coords, ds.y, ds.X) for name, (ds, _, _) in
                   zip(("small", "mid", "large"), (small, mid, large))}
            first = ctx.submit(ids["small"], small[1], small[2], batch=4)
            time.sleep(0.01)
            jobs = {name: ctx.submit(ids[name], prob[1], prob[2], batch=4)
                    for name, prob in (("small", small), ("mid", mid), ("large", large))}
            ctx.poll(first, 3)
            for name, prob in (("small", small), ("mid", mid), ("large", large)):
                _same(ctx.poll(jobs[name], 3), _ref(*prob))
        lines = [json.loads(x) for x in log.read_text().splitlines()][1:]
        order[policy] = [x["n"] for x in sorted(lines, key=lambda x: x["t_start"])]
    assert order[nv.SCHED_FIFO] == [20, 35, 50]
    assert order[nv.SCHED_LARGEST_FIRST] == [50, 35, 20]
    with nv.Context(64 << 20, n_streams=1, evaluator=oracle_fn()) as ctx:
        with pytest.raises(nv.PlkError):
            ctx.set_schedule_policy(7)
