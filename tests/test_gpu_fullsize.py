"""Parity at the full workload sizes, in the launch configuration of bench.py.

The whole job runs on the GPU exactly as benchmarked (every true point, every
universe, mixed precision, up to 5 scans); the oracle recomputes a seeded
sample of (point, universe) pairs one by one (its random numbers depend only on
(seed, point, universe)), and properties that hold for every output are
checked over the whole result.  The sample is drawn at random and, on top,
from the universes whose scans were decided by each of the rarer certified
rounds (fc_get_decided_by: rescoring, list, exact-size list, exact scan), so
every path that decides a universe at full size is compared.  Bars are
tests/_parity.py's: |ddchi2| <= 1e-4 absolute, best fits identical except
near-ties verified by the oracle, per-point 68/90/95 % quantiles within
relative 1e-3.  The fake data of all 10^7 universes of the 100x100 job are
compared with the oracle bit for bit.
"""
import concurrent.futures as cf
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


def _grid(fc, ctx, w):
    gid = fc.fc_load_grid(ctx, w.S, w.collapse, w.n_fit)
    fc.fc_set_frac_cov(ctx, gid, w.F)
    return gid


ROUND_NAMES = {1: "certificate", 2: "rescored", 4: "top-16", 8: "list", 16: "exact-size list", 32: "exact scan"}


def _pick_samples(rounds, n_random, n_per_round, rng):
    """Flat universe indices: n_random at random, plus up to n_per_round from the universes
    that any rarer round decided (every bit above the plain certificate)."""
    flat = rounds.ravel()
    pick = list(rng.integers(0, flat.size, n_random))
    for bit in (2, 4, 8, 16, 32):
        idx = np.nonzero(flat & bit)[0]
        if idx.size:
            pick += list(rng.choice(idx, min(n_per_round, idx.size), replace=False))
    return np.unique(np.array(pick, np.int64))


def _check_samples(fc, ctx, gid, w, pts, d, b, n, seed, rounds, n_random, n_per_round, rng_seed, max_iter=5):
    P, U = d.shape
    flat = _pick_samples(rounds, n_random, n_per_round, np.random.default_rng(rng_seed))
    ip, iu = flat // U, (flat % U).astype(np.int32)
    od, ob, on = oracle.run_samples(w.S, w.F, pts[ip], iu, seed, collapse=w.collapse, n_fit=w.n_fit,
                                    max_iter=max_iter)
    seen = {name: int(np.count_nonzero(rounds.ravel()[flat] & bit)) for bit, name in ROUND_NAMES.items()}
    whole = {name: int(np.count_nonzero(rounds & bit)) for bit, name in ROUND_NAMES.items()}
    print(f"{w.name}: {flat.size} samples; samples per deciding round {seen}; whole job {whole}")
    _parity.check_mixed(fc, ctx, gid, w, pts[ip], iu, seed, d[ip, iu], b[ip, iu], n[ip, iu], od, ob, on,
                        max_iter=max_iter, label=w.name)


def _check_properties(w, d, b, n, max_iter=5):
    assert np.all(np.isfinite(d))
    assert d.min() >= -1e-9 * max(1.0, np.abs(d).max())
    assert b.min() >= 0 and b.max() < w.G
    assert n.min() >= 1 and n.max() <= max_iter


def test_cfg2_full_job(fc, ctx):
    """10^4 true points x 1000 universes (10^7 fits), N 90 -> 45."""
    w = workloads.cfg2()
    gid = _grid(fc, ctx, w)
    pts = np.arange(w.G, dtype=np.int64)
    seed = 20261
    d, b, n = fc.fc_run_points(ctx, gid, pts, seed, w.U, opts=dict(precision=fc.FC_PREC_MIXED, top_k=8))
    st = fc.fc_get_stats(ctx)
    rounds = fc.fc_get_decided_by(ctx, d.size).reshape(d.shape)
    assert st["universes"] == w.G * w.U
    _check_properties(w, d, b, n)
    assert np.all(rounds != 0)
    _check_samples(fc, ctx, gid, w, pts, d, b, n, seed, rounds, 64, 24, 7)
    # per-point quantiles (and every universe) against complete oracle runs of two points
    for p in (2550, 7337):
        od, ob, on = oracle.run_points(w.S, w.F, np.array([p]), seed, w.U, collapse=w.collapse, n_fit=w.n_fit)
        _parity.check_grid(fc, ctx, gid, w, [p], seed, d[p:p + 1], b[p:p + 1], n[p:p + 1], od, ob, on,
                           label=f"cfg2 point {p}")
    fc.fc_unload_grid(ctx, gid)


def test_cfg2_fake_data_all_universes(fc, ctx):
    """The fake data of every one of the 10^7 universes of the 100x100 job (10^4 true points x
    1000), bit for bit against the oracle (threads over point chunks: ctypes drops the GIL)."""
    w = workloads.cfg2()
    gid = _grid(fc, ctx, w)
    seed = 20261
    chunk = 250
    nthreads = max(1, len(os.sched_getaffinity(0)))

    def ref(ps):
        return oracle.fake_data(w.S, w.F, ps, seed, w.U, collapse=w.collapse, n_fit=w.n_fit)

    with cf.ThreadPoolExecutor(nthreads) as ex:
        for p0 in range(0, w.G, chunk * nthreads):
            blocks = [np.arange(a, min(a + chunk, w.G), dtype=np.int64)
                      for a in range(p0, min(p0 + chunk * nthreads, w.G), chunk)]
            futs = [ex.submit(ref, ps) for ps in blocks]
            for ps, fu in zip(blocks, futs):
                got = fc.fc_fake_data(ctx, gid, ps, seed, w.U, w.n_fit)
                np.testing.assert_array_equal(got, fu.result(), err_msg=f"points {ps[0]}..{ps[-1]}")
    fc.fc_unload_grid(ctx, gid)


def test_cfg3_full_job(fc, ctx):
    """D=3 64^3 grid, N=120: 2048 seeded true points x 500 universes."""
    w = workloads.cfg3()
    gid = _grid(fc, ctx, w)
    seed = 4099
    d, b, n = fc.fc_run_points(ctx, gid, w.points, seed, w.U)
    rounds = fc.fc_get_decided_by(ctx, d.size).reshape(d.shape)
    _check_properties(w, d, b, n)
    _check_samples(fc, ctx, gid, w, w.points, d, b, n, seed, rounds, 16, 4, 11)
    fc.fc_unload_grid(ctx, gid)


def test_cfg5_batch(fc, ctx):
    """D=6 16^6 grid (16.7 M spectra, N=64, exact ties at zero amplitude): 256 points x 16 universes."""
    import torch

    free, _ = torch.cuda.mem_get_info()
    if free < 120 << 30:
        pytest.skip("needs about 120 GB of free device memory")
    w = workloads.cfg5()
    gid = _grid(fc, ctx, w)
    seed = 77
    d, b, n = fc.fc_run_points(ctx, gid, w.points, seed, w.U)
    _check_properties(w, d, b, n)
    # the oracle scans 16.7 M points per universe-scan: two single-scan samples (fixed covariance)
    d1, b1, n1 = fc.fc_run_points(ctx, gid, w.points[:2], seed, 2, opts=dict(cov=fc.FC_COV_FIXED))
    od, ob, on = oracle.run_samples(w.S, w.F, w.points[:2], np.array([0, 1], np.int32), seed, max_iter=1,
                                    cov=oracle.COV_FIXED)
    gd = np.array([d1[0, 0], d1[1, 1]])
    gb = np.array([b1[0, 0], b1[1, 1]])
    gn = np.array([n1[0, 0], n1[1, 1]])
    _parity.check_mixed(fc, ctx, gid, w, w.points[:2], np.array([0, 1]), seed, gd, gb, gn, od, ob, on,
                        opts=dict(cov=fc.FC_COV_FIXED), max_iter=1, cov=oracle.COV_FIXED, label="cfg5 fixed cov")
    fc.fc_unload_grid(ctx, gid)
