"""Large-N paths, kernel choices and the covariance cache.

* N_fit > 61 (K > 64, up to K = 208 at the N_fit = 200 limit): the
  tensor-core screen with 16-column K-slice stages and the tensor-core
  q-vectors (whole S~ tiles, or K slices beside a resident W; binary32
  q-vectors above K = 128), against the oracle (tests/_parity.py's bars).
* Kernel choices (q-vector kernel, screen depth, A-image buffering, top-k
  or list first round) change speed only: the outputs are identical bit for
  bit.
* A covariance cache smaller than the run's distinct covariances reuses
  slots (least recently used first) without changing any output.
* fc_autotune picks a valid choice and reuses its cache file.
"""
import os

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


def _load(fc, ctx, w):
    gid = fc.fc_load_grid(ctx, w.S, w.collapse, w.n_fit)
    fc.fc_set_frac_cov(ctx, gid, w.F)
    return gid


@pytest.fixture(scope="module")
def w3s():
    # the cfg3 shape model (D=3, N=120: K=128) on a 12^3 grid
    return workloads.cfg3(U=100, n_points=4, n_axis=12)


@pytest.fixture(scope="module")
def w70():
    # D=2 grid with N=70 (K=80: K/32 not an integer, partial TMEM chunks)
    S, F, axes = workloads.osc_2d(30, 30, 70, seed=5)
    return workloads.Workload("osc30x30_n70", S, F, None, 70, np.array([100, 465, 777], np.int64), 120, 5, 9, axes)


@pytest.fixture(scope="module")
def w64():
    # N=64: the largest N_fit whose W is staged in shared memory by the binary64-accuracy kernels (K=80)
    S, F, axes = workloads.osc_2d(24, 24, 64, seed=8)
    return workloads.Workload("osc24x24_n64", S, F, None, 64, np.array([50, 300, 571], np.int64), 150, 5, 6, axes)


@pytest.fixture(scope="module")
def w200():
    # the bin limit: N_fit = 200 (K = 208, a 13-step K loop in the screen; binary32 q-vectors; the
    # largest covariance, Cholesky and inverse)
    S, F, axes = workloads.osc_2d(12, 12, 200, seed=9)
    return workloads.Workload("osc12x12_n200", S, F, None, 200, np.array([5, 77, 143], np.int64), 64, 5, 13, axes)


@pytest.fixture(scope="module")
def w150():
    # D=2 grid with N=150 (K=160: q-vectors stream S~ in K slices beside a resident W)
    S, F, axes = workloads.osc_2d(20, 20, 150, seed=6)
    return workloads.Workload("osc20x20_n150", S, F, None, 150, np.array([37, 210, 399], np.int64), 100, 5, 4, axes)


@pytest.mark.parametrize("which", ["w3s", "w64", "w70", "w150", "w200"])
def test_large_n_mixed_vs_oracle(fc, ctx, which, request):
    w = request.getfixturevalue(which)
    gid = _load(fc, ctx, w)
    assert fc.fc_get_tuning(ctx, gid)["qvec"] == fc.FC_QVEC_AUTO
    d, b, n = fc.fc_run_points(ctx, gid, w.points, w.seed, w.U)
    st = fc.fc_get_stats(ctx)
    assert st["screen_launches"] > 0
    od, ob, on = oracle.run_points(w.S, w.F, w.points, w.seed, w.U, collapse=w.collapse, n_fit=w.n_fit)
    _parity.check_grid(fc, ctx, gid, w, w.points, w.seed, d, b, n, od, ob, on, label=w.name)
    fc.fc_unload_grid(ctx, gid)


def test_n_fit_200_plain_and_fake_data(fc, ctx, w200):
    """At the bin limit the plain binary64 path keeps the oracle's indices and scan counts
    and the fake data its bits (systematic factor of 200 bins in global memory)."""
    gid = _load(fc, ctx, w200)
    d, b, n = fc.fc_run_points(ctx, gid, w200.points, w200.seed, w200.U, opts=dict(precision=fc.FC_PREC_FP64))
    od, ob, on = oracle.run_points(w200.S, w200.F, w200.points, w200.seed, w200.U)
    _parity.check_plain(d, b, n, od, ob, on)
    np.testing.assert_array_equal(fc.fc_fake_data(ctx, gid, w200.points, w200.seed, w200.U, 200),
                                  oracle.fake_data(w200.S, w200.F, w200.points, w200.seed, w200.U))
    _, L = fc.fc_covariance(ctx, gid, 77, 200, 200, want_A=False)
    np.testing.assert_array_equal(L, oracle.chol_sys(w200.S[77], w200.F))
    fc.fc_unload_grid(ctx, gid)


def _run_all(fc, ctx, gid, pts, seed, U, **opts):
    return fc.fc_run_points(ctx, gid, pts, seed, U, opts=opts or None)


@pytest.mark.parametrize("which", ["cfg1", "w70", "w3s", "w150"])
def test_kernel_choices_do_not_change_results(fc, ctx, which, request):
    w = workloads.cfg1() if which == "cfg1" else request.getfixturevalue(which)
    gid = _load(fc, ctx, w)
    pts = w.points if len(w.points) > 1 else np.array([w.points[0], 17, 600], np.int64)
    U = 300 if which == "cfg1" else 64
    ref = _run_all(fc, ctx, gid, pts, 3, U)
    choices = [dict(qvec=fc.FC_QVEC_SIMT), dict(qvec=fc.FC_QVEC_TC), dict(qvec=fc.FC_QVEC_TC, screen_stages=2),
               dict(first_round=fc.FC_ROUND_LIST), dict(first_round=fc.FC_ROUND_TOPK, qvec=fc.FC_QVEC_TC)]
    choices.append(dict(slot_rows=128))                           # one covariance per whole tile
    if which == "cfg1":
        choices.append(dict(screen_stages=2, screen_ybuf=2))       # whole-tile stages, double A image
    else:
        choices.append(dict(qvec=fc.FC_QVEC_SIMT, screen_stages=4, screen_ybuf=1))  # shallower K-slice ring
    for ch in choices:
        fc.fc_set_tuning(ctx, gid, **ch)
        got = _run_all(fc, ctx, gid, pts, 3, U)
        for a, r in zip(got, ref):
            np.testing.assert_array_equal(a, r, err_msg=str(ch))
    fc.fc_unload_grid(ctx, gid)


def test_bad_tuning_rejected(fc, ctx):
    w = workloads.cfg1()
    gid = _load(fc, ctx, w)
    for bad in (dict(qvec=7), dict(screen_stages=1), dict(screen_stages=9), dict(screen_ybuf=3), dict(cache_slots=1),
                dict(cache_slots=-4), dict(first_round=3), dict(slot_rows=64)):
        with pytest.raises(fc.FCError) as e:
            fc.fc_set_tuning(ctx, gid, **bad)
        assert e.value.status == fc.FC_ERR_ARG
    fc.fc_unload_grid(ctx, gid)


def test_cache_eviction_keeps_results(fc, ctx):
    """Five runs of 40 points x 4 universes (at most 160 distinct covariances
    per scan) through a 200-slot cache: later runs evict earlier slots."""
    w = workloads.cfg2()
    rng = np.random.default_rng(8)
    runs = [np.sort(rng.choice(w.G, 40, replace=False)).astype(np.int64) for _ in range(5)]
    gid = _load(fc, ctx, w)
    refs = [_run_all(fc, ctx, gid, p, 21, 4) for p in runs]
    fc.fc_set_frac_cov(ctx, gid, w.F)  # forget the cache
    fc.fc_set_tuning(ctx, gid, cache_slots=200)
    evicted = 0
    for p, r in zip(runs + runs[:2], refs + refs[:2]):
        got = _run_all(fc, ctx, gid, p, 21, 4)
        st = fc.fc_get_stats(ctx)
        evicted += st["evicted"]
        for a, b in zip(got, r):
            np.testing.assert_array_equal(a, b)
    assert evicted > 0
    fc.fc_unload_grid(ctx, gid)


def test_autotune(fc, ctx, tmp_path):
    w = workloads.cfg1()
    gid = _load(fc, ctx, w)
    ref = _run_all(fc, ctx, gid, w.points, 0, 200)
    path = str(tmp_path / "tune.txt")
    t = fc.fc_autotune(ctx, gid, path)
    assert t["qvec"] in (fc.FC_QVEC_SIMT, fc.FC_QVEC_TC)
    assert t["screen_stages"] >= 2
    assert t["slot_rows"] in (32, 128)
    assert fc.fc_get_tuning(ctx, gid) == t
    assert os.path.exists(path)
    lines = open(path).read().splitlines()
    assert len(lines) == 1 and "qvec=" in lines[0]
    # a second grid of the same shape is tuned from the file without timing
    gid2 = _load(fc, ctx, w)
    t2 = fc.fc_autotune(ctx, gid2, path)
    assert t2 == t and len(open(path).read().splitlines()) == 1
    got = _run_all(fc, ctx, gid, w.points, 0, 200)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)
    fc.fc_unload_grid(ctx, gid)
    fc.fc_unload_grid(ctx, gid2)


@pytest.mark.parametrize("prec", [0, 1])
def test_scan_waves_when_cache_is_small(fc, ctx, prec):
    """A 48-slot cache and 640 universes: scans after the first need more
    distinct covariances than the cache holds and run in waves; outputs are
    identical to an unlimited cache."""
    w = workloads.cfg2()
    pts = np.sort(np.random.default_rng(3).choice(w.G, 40, replace=False)).astype(np.int64)
    gid = _load(fc, ctx, w)
    ref = _run_all(fc, ctx, gid, pts, 5, 16, precision=prec)
    assert fc.fc_get_stats(ctx)["scan_waves"] == 0
    fc.fc_set_frac_cov(ctx, gid, w.F)
    fc.fc_set_tuning(ctx, gid, cache_slots=48)
    got = _run_all(fc, ctx, gid, pts, 5, 16, precision=prec)
    st = fc.fc_get_stats(ctx)
    assert st["max_distinct_cov"] > 48 and st["scan_waves"] > 0 and st["evicted"] > 0
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)
    fc.fc_unload_grid(ctx, gid)
