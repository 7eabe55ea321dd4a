"""Serving with continuous batching (fc_submit / fc_poll / fc_cancel).

A served job's results depend only on its own arguments: a job run alone,
run through the synchronous entry point, or admitted between the scans of
other jobs (same lane, different iteration counts, other lanes) gives the
same dchi2, best fits and scan counts bit for bit -- and jobs served in a mix
meet the oracle's bars (tests/_parity.py).  Under a device-memory budget a
job that can never fit is refused at submit, and a job that does not fit
beside the running ones waits for them.
"""
import time

import numpy as np
import pytest

import _parity
import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    import paper_2002_07858_gb300 as m

    m.load()
    return m


@pytest.fixture(scope="module")
def ctx(fc):
    c = fc.fc_create(0)
    yield c
    fc.fc_destroy(c)


@pytest.fixture(scope="module")
def w2():
    return workloads.cfg2()


@pytest.fixture(scope="module")
def g2(fc, ctx, w2):
    gid = fc.fc_load_grid(ctx, w2.S, w2.collapse, w2.n_fit)
    fc.fc_set_frac_cov(ctx, gid, w2.F)
    return gid


def _points(w, n, seed):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(w.G, n, replace=False)).astype(np.int64)


def _wait(fc, ctx, tickets, timeout=600.0):
    """Poll until every ticket is final; returns {ticket: (status, latency_ms)}."""
    out = {}
    t0 = time.time()
    while len(out) < len(tickets) and time.time() - t0 < timeout:
        for t in tickets:
            if t in out:
                continue
            try:
                st, lat = fc.fc_poll(ctx, t)
            except fc.FCError as e:
                out[t] = (e.status, None)
                continue
            if st != fc.FC_PENDING:
                out[t] = (st, lat)
        time.sleep(0.002)
    assert len(out) == len(tickets), "jobs did not complete"
    return out


def _sync(fc, ctx, gid, ps, seed, U, opts):
    return fc.fc_run_points(ctx, gid, ps, seed, U, opts=opts)


# job specs: (points, seed, U, opts) -- same lane with different iteration limits, plus other lanes
def _specs(w2):
    return [
        (_points(w2, 3, 1), 11, 200, dict(max_iter=5)),
        (_points(w2, 2, 2), 12, 150, dict(max_iter=1)),
        (_points(w2, 4, 3), 13, 100, dict(max_iter=3)),
        (_points(w2, 2, 4), 14, 120, dict(max_iter=5, top_k=16)),                  # second lane
        (_points(w2, 2, 5), 15, 64, dict(max_iter=5, precision=0)),                # binary64 lane
        (_points(w2, 2, 6), 16, 90, dict(max_iter=5, cov=1)),                      # fixed covariance
    ]


def test_served_alone_equals_synchronous(fc, ctx, g2, w2):
    ps, seed, U, opts = _specs(w2)[0]
    ref = _sync(fc, ctx, g2, ps, seed, U, opts)
    t, outs = fc.fc_submit(ctx, g2, ps, seed, U, opts=opts, want_bestfit=True, want_nscans=True)
    res = _wait(fc, ctx, [t])
    assert res[t][0] == fc.FC_OK and res[t][1] > 0
    for a, b in zip(outs, ref):
        np.testing.assert_array_equal(a, b)


def test_admitted_mid_iteration_equals_alone(fc, ctx, g2, w2):
    """A large job keeps the lane busy for several scans; the small jobs are
    submitted while it iterates and join its scans.  Every job's outputs
    equal its alone (synchronous) run."""
    big = (_points(w2, 60, 99), 7, 2000, dict(max_iter=5))
    specs = _specs(w2)
    refs = [_sync(fc, ctx, g2, *s) for s in [big] + specs]
    t_big, out_big = fc.fc_submit(ctx, g2, *big[:3], opts=big[3], want_bestfit=True, want_nscans=True)
    tickets = [t_big]
    outs = [out_big]
    for i, s in enumerate(specs):
        time.sleep(0.005 * (i + 1))
        t, o = fc.fc_submit(ctx, g2, *s[:3], opts=s[3], want_bestfit=True, want_nscans=True)
        tickets.append(t)
        outs.append(o)
    res = _wait(fc, ctx, tickets)
    for t, o, r, s in zip(tickets, outs, refs, [big] + specs):
        assert res[t][0] == fc.FC_OK
        np.testing.assert_array_equal(o[0], r[0])
        np.testing.assert_array_equal(o[1], r[1])
        np.testing.assert_array_equal(o[2], r[2])
        lim = s[3]["max_iter"] if s[3].get("cov", 0) == 0 else 1
        assert o[2].min() >= 1 and o[2].max() <= lim


def test_many_small_jobs_interleaved(fc, ctx, g2, w2):
    """A stream of one-point jobs (the serving shape): each equals its own
    synchronous run whatever it was batched with."""
    pts = _points(w2, 24, 123)
    refs = [_sync(fc, ctx, g2, pts[i:i + 1], 1000 + i, 256, None) for i in range(len(pts))]
    tickets, outs = [], []
    for i in range(len(pts)):
        t, o = fc.fc_submit(ctx, g2, pts[i:i + 1], 1000 + i, 256, want_bestfit=True, want_nscans=True)
        tickets.append(t)
        outs.append(o)
        if i % 4 == 3:
            time.sleep(0.003)
    res = _wait(fc, ctx, tickets)
    lats = [res[t][1] for t in tickets]
    assert all(res[t][0] == fc.FC_OK for t in tickets)
    assert all(x > 0 for x in lats)
    for o, r in zip(outs, refs):
        for a, b in zip(o, r):
            np.testing.assert_array_equal(a, b)


def test_cancel_and_continue(fc, ctx, g2, w2):
    big = _points(w2, 200, 5)
    t, _ = fc.fc_submit(ctx, g2, big, 3, 1000)
    fc.fc_cancel(ctx, t)
    res = _wait(fc, ctx, [t])
    assert res[t][0] == fc.FC_ERR_CANCELLED
    with pytest.raises(fc.FCError) as e:
        fc.fc_poll(ctx, t)
    assert e.value.status == fc.FC_ERR_NOT_FOUND
    # the context keeps serving, with exact results
    ps, seed, U, opts = _specs(w2)[2]
    ref = _sync(fc, ctx, g2, ps, seed, U, opts)
    t2, o2 = fc.fc_submit(ctx, g2, ps, seed, U, opts=opts, want_bestfit=True, want_nscans=True)
    res = _wait(fc, ctx, [t2])
    assert res[t2][0] == fc.FC_OK
    for a, b in zip(o2, ref):
        np.testing.assert_array_equal(a, b)


def test_submit_rejects_bad_jobs(fc, ctx, g2, w2):
    with pytest.raises(fc.FCError) as e:
        fc.fc_submit(ctx, g2, np.array([w2.G], np.int64), 1, 10)
    assert e.value.status == fc.FC_ERR_ARG
    with pytest.raises(fc.FCError) as e:
        fc.fc_submit(ctx, g2, np.array([0], np.int64), 1, 10, opts=dict(max_iter=0))
    assert e.value.status == fc.FC_ERR_ARG
    with pytest.raises(fc.FCError) as e:
        fc.fc_submit(ctx, 12345, np.array([0], np.int64), 1, 10)
    assert e.value.status == fc.FC_ERR_NOT_FOUND
    # an empty job completes at once
    t, _ = fc.fc_submit(ctx, g2, np.array([0], np.int64), 1, 0)
    assert _wait(fc, ctx, [t])[t][0] == fc.FC_OK


def test_served_mix_matches_the_oracle(fc, ctx, g2, w2):
    """Jobs submitted together (two mixed lanes with different iteration limits and top-k,
    one binary64 lane) against complete oracle runs of the same points and seeds."""
    specs = [(_points(w2, 2, 31), 41, 96, dict(max_iter=5)),
             (_points(w2, 2, 32), 42, 80, dict(max_iter=3)),
             (_points(w2, 1, 33), 43, 64, dict(max_iter=5, top_k=16)),
             (_points(w2, 1, 34), 44, 48, dict(max_iter=5, precision=0))]
    tickets, outs = [], []
    for ps, seed, U, opts in specs:
        t, o = fc.fc_submit(ctx, g2, ps, seed, U, opts=opts, want_bestfit=True, want_nscans=True)
        tickets.append(t)
        outs.append(o)
    res = _wait(fc, ctx, tickets)
    for t, o, (ps, seed, U, opts) in zip(tickets, outs, specs):
        assert res[t][0] == fc.FC_OK
        od, ob, on = oracle.run_points(w2.S, w2.F, ps, seed, U, collapse=w2.collapse, n_fit=w2.n_fit,
                                       max_iter=opts["max_iter"])
        if opts.get("precision", 1) == 0:
            _parity.check_plain(o[0], o[1], o[2], od, ob, on)
        else:
            _parity.check_grid(fc, ctx, g2, w2, ps, seed, o[0], o[1], o[2], od, ob, on, opts=opts,
                               max_iter=opts["max_iter"], label=f"served {opts}")


def test_budget_refuses_a_job_that_can_never_fit(fc, w2):
    c = fc.fc_create(0, 4 << 30)
    try:
        w1 = workloads.cfg1()
        g = fc.fc_load_grid(c, w1.S)
        fc.fc_set_frac_cov(c, g, w1.F)
        with pytest.raises(fc.FCError) as e:
            fc.fc_submit(c, g, np.array([312], np.int64), 1, 10_000_000)
        assert e.value.status == fc.FC_ERR_BUDGET
        # the context keeps serving jobs that fit
        t, o = fc.fc_submit(c, g, np.array([312], np.int64), 1, 64, want_bestfit=True, want_nscans=True)
        assert _wait(fc, c, [t])[t][0] == fc.FC_OK
    finally:
        fc.fc_destroy(c)


def test_budget_defers_admission_until_memory_frees(fc):
    """Two jobs whose admission estimates together exceed the budget, each fitting alone:
    the second waits until the first has finished, then runs; both give the results of
    their synchronous runs."""
    w1 = workloads.cfg1()
    budget = 8 << 30
    P, U = 24, 262144            # 6.3 M universes: about 0.6 of the budget each
    rng = np.random.default_rng(17)
    jobs = [(np.sort(rng.choice(w1.G, P, replace=False)).astype(np.int64), 51, dict(top_k=8)),
            (np.sort(rng.choice(w1.G, P, replace=False)).astype(np.int64), 52, dict(top_k=16))]
    ref_ctx = fc.fc_create(0)
    try:
        gr = fc.fc_load_grid(ref_ctx, w1.S)
        fc.fc_set_frac_cov(ref_ctx, gr, w1.F)
        refs = [fc.fc_run_points(ref_ctx, gr, ps, seed, U, opts=o) for ps, seed, o in jobs]
    finally:
        fc.fc_destroy(ref_ctx)
    c = fc.fc_create(0, budget)
    try:
        g = fc.fc_load_grid(c, w1.S)
        fc.fc_set_frac_cov(c, g, w1.F)
        tickets, outs = [], []
        for ps, seed, o in jobs:
            t, out = fc.fc_submit(c, g, ps, seed, U, opts=o, want_bestfit=True, want_nscans=True)
            tickets.append(t)
            outs.append(out)
        res = _wait(fc, c, tickets)
        st = fc.fc_get_serve_stats(c)
        assert st["deferred"] > 0
        assert 0 < st["device_bytes"] <= budget
        for t, out, ref in zip(tickets, outs, refs):
            assert res[t][0] == fc.FC_OK
            for a, b in zip(out, ref):
                np.testing.assert_array_equal(a, b)
        # the second job waited for the first: it finished later although it was submitted at once
        assert res[tickets[1]][1] > res[tickets[0]][1]
    finally:
        fc.fc_destroy(c)
