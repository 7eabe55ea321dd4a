"""Failure detection on the device without a GPU fault.

Every wait of the tensor-core screen on a pipeline barrier is bounded.  The
context's test hook shortens that bound and makes the screen's copy producer
stop issuing after a few pipeline stages, so the consumers' waits run out in
the allowed way: the kernel records a timeout, lets the copies it issued land,
frees its tensor memory and returns.  The call must report FC_ERR_TIMEOUT, no
stale candidate may be read afterwards, and the next call on the same context
must give the oracle's results.
"""
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
def env(fc):
    c = fc.fc_create(0)
    w = workloads.cfg1()
    gid = fc.fc_load_grid(c, w.S)
    fc.fc_set_frac_cov(c, gid, w.F)
    yield c, w, gid
    fc.fc_set_wait_test(c, 0, -1)
    fc.fc_destroy(c)


@pytest.mark.parametrize("stop_after", [0, 1, 2])
def test_screen_wait_runs_out_and_the_context_recovers(fc, env, stop_after):
    ctx, w, gid = env
    U, seed = 256, 3
    fc.fc_set_wait_test(ctx, 150_000_000, stop_after)       # 150 ms bound, producer stops early
    with pytest.raises(fc.FCError) as e:
        fc.fc_run_points(ctx, gid, w.points, seed, U)
    assert e.value.status == fc.FC_ERR_TIMEOUT
    fc.fc_set_wait_test(ctx, 0, -1)
    d, b, n = fc.fc_run_points(ctx, gid, w.points, seed, U)
    od, ob, on = oracle.run_workload(w, U=U, seed=seed)
    _parity.check_grid(fc, ctx, gid, w, w.points, seed, d, b, n, od, ob, on, label="after a timeout")


def test_a_stop_beyond_the_work_changes_nothing(fc, env):
    ctx, w, gid = env
    ref = fc.fc_run_points(ctx, gid, w.points, 5, 200)
    fc.fc_set_wait_test(ctx, 150_000_000, 1 << 40)
    try:
        got = fc.fc_run_points(ctx, gid, w.points, 5, 200)
    finally:
        fc.fc_set_wait_test(ctx, 0, -1)
    for a, r in zip(got, ref):
        np.testing.assert_array_equal(a, r)


def test_wait_test_arguments(fc, env):
    ctx, _, _ = env
    for bad in ((3_000_000_000, -1), (0, -2)):
        with pytest.raises(fc.FCError) as e:
            fc.fc_set_wait_test(ctx, *bad)
        assert e.value.status == fc.FC_ERR_ARG
