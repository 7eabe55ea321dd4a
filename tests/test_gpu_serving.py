"""Serving with continuous batching (fc_submit / fc_poll / fc_cancel).

A served job's results depend only on its own arguments: a job run alone,
run through the synchronous entry point, or admitted between the scans of
other jobs (same lane, different iteration counts, other lanes) gives the
same dchi2, best fits and scan counts bit for bit.
"""
import time

import numpy as np
import pytest

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
