"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Bars (per step of §2 / Algorithm 1):
  fake data and the systematic Cholesky factor ....... bit for bit
  plain binary64 path .................................. |ddchi2| <= 1e-9 max(|dchi2|, 1), same best
                                                         fits and scan counts
  tensor-core screen + double-float rescoring ......... |ddchi2| <= 1e-4 absolute; best fits identical
                                                         except near-ties verified by the oracle
                                                         (|chi2 gap| < 1e-4 at the first differing
                                                         scan); 68/90/95% quantiles within rel 1e-3
(the mixed-path bars are tests/_parity.py's)
"""
import numpy as np
import pytest
from scipy import spatial

import _parity
import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL_PLAIN = 1e-9
TOL_MIXED = 1e-4


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


_grids = {}


def grid(fc, ctx, w):
    key = (w.name, id(ctx))
    if key not in _grids:
        gid = fc.fc_load_grid(ctx, w.S, w.collapse, w.n_fit)
        fc.fc_set_frac_cov(ctx, gid, w.F)
        _grids[key] = gid
    return _grids[key]


@pytest.fixture(scope="module")
def w1():
    return workloads.cfg1()


@pytest.fixture(scope="module")
def w2():
    return workloads.cfg2()


def _cfg2_points(w2, n):
    rng = np.random.default_rng(42)
    return np.sort(rng.choice(w2.G, n, replace=False)).astype(np.int64)


# ------------------------------------------------------------------ a2 / a3 --

@pytest.mark.parametrize("which,p", [("cfg1", 312), ("cfg1", 0), ("cfg2", 1234), ("cfg2", 9999)])
def test_systematic_cholesky_bit_exact(fc, ctx, w1, w2, which, p):
    w = w1 if which == "cfg1" else w2
    gid = grid(fc, ctx, w)
    _, L = fc.fc_covariance(ctx, gid, p, w.n_fit, w.n_full, want_A=False)
    np.testing.assert_array_equal(L, oracle.chol_sys(w.S[p], w.F))


@pytest.mark.parametrize("which,q", [("cfg1", 312), ("cfg1", 624), ("cfg2", 5000), ("cfg2", 17)])
def test_inverse_covariance(fc, ctx, w1, w2, which, q):
    w = w1 if which == "cfg1" else w2
    gid = grid(fc, ctx, w)
    A, _ = fc.fc_covariance(ctx, gid, q, w.n_fit, w.n_full, want_L=False)
    ref = oracle.inv_cov(w.S[q], w.F, w.collapse, w.n_fit)
    assert np.max(np.abs(A - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_fake_data_bit_exact_cfg1(fc, ctx, w1):
    gid = grid(fc, ctx, w1)
    got = fc.fc_fake_data(ctx, gid, w1.points, w1.seed, 1000, w1.n_fit)
    ref = oracle.fake_data(w1.S, w1.F, w1.points, w1.seed, 1000)
    np.testing.assert_array_equal(got, ref)


def test_fake_data_bit_exact_cfg2(fc, ctx, w2):
    """Every 10th grid point of the 100x100 grid x 100 universes (the full 10^7 are in
    test_gpu_fullsize): the sampler's branches (PTRS, inversion, lam = 0) are taken at
    different rates at different points, so the sample spans the grid."""
    gid = grid(fc, ctx, w2)
    pts = np.arange(0, w2.G, 10, dtype=np.int64)
    got = fc.fc_fake_data(ctx, gid, pts, 7, 100, w2.n_fit)
    ref = oracle.fake_data(w2.S, w2.F, pts, 7, 100, collapse=w2.collapse, n_fit=w2.n_fit)
    np.testing.assert_array_equal(got, ref)


def test_fake_data_bit_exact_gauss_and_seed(fc, ctx, w1):
    gid = grid(fc, ctx, w1)
    for seed in (0, 1, 0xDEADBEEFCAFE):
        got = fc.fc_fake_data(ctx, gid, np.array([3, 312, 600]), seed, 300, w1.n_fit, fluct=fc.FC_FLUCT_GAUSS)
        ref = oracle.fake_data(w1.S, w1.F, [3, 312, 600], seed, 300, fluct=oracle.FLUCT_GAUSS)
        np.testing.assert_array_equal(got, ref)


# -------------------------------------------------------------- full path ---

def _compare(fc, ctx, gid, w, pts, seed, d, b, n, od, ob, on, prec, label, **kw):
    """The plain path's bars (prec 0) or the mixed path's (prec 1, tests/_parity.py)."""
    if prec == fc.FC_PREC_FP64:
        _parity.check_plain(d, b, n, od, ob, on)
        return 0
    opts = dict(precision=prec)
    if "cov" in kw:
        opts["cov"] = kw["cov"]
    return _parity.check_grid(fc, ctx, gid, w, pts, seed, d, b, n, od, ob, on, opts=opts, label=label, **kw)[0]


def test_plain_fp64_cfg1(fc, ctx, w1):
    gid = grid(fc, ctx, w1)
    d, b, n = fc.fc_run_points(ctx, gid, w1.points, w1.seed, w1.U, opts=dict(precision=fc.FC_PREC_FP64))
    od, ob, on = oracle.run_workload(w1)
    _parity.check_plain(d, b, n, od, ob, on)
    assert np.all(fc.fc_get_decided_by(ctx, d.size) == fc.FC_DECIDED_PLAIN)


def test_mixed_cfg1(fc, ctx, w1):
    gid = grid(fc, ctx, w1)
    d, b, n = fc.fc_run_points(ctx, gid, w1.points, w1.seed, w1.U, opts=dict(precision=fc.FC_PREC_MIXED))
    st = fc.fc_get_stats(ctx)
    rounds = fc.fc_get_decided_by(ctx, d.size)
    od, ob, on = oracle.run_workload(w1)
    _compare(fc, ctx, gid, w1, w1.points, w1.seed, d, b, n, od, ob, on, 1, "cfg1 mixed")
    assert st["screened"] + st["rescored"] + st["fallback"] == st["scans"]
    # every universe's scans were decided by some round, never by the plain scan
    assert np.all(rounds != 0) and not np.any(rounds & fc.FC_DECIDED_PLAIN)


@pytest.mark.parametrize("topk", [4, 8, 16])
def test_mixed_cfg2_subset(fc, ctx, w2, topk):
    gid = grid(fc, ctx, w2)
    pts = _cfg2_points(w2, 8)
    U = 250
    opts = dict(precision=fc.FC_PREC_MIXED, top_k=topk)
    d, b, n = fc.fc_run_points(ctx, gid, pts, 11, U, opts=opts)
    st = fc.fc_get_stats(ctx)
    od, ob, on = oracle.run_points(w2.S, w2.F, pts, 11, U, collapse=w2.collapse, n_fit=w2.n_fit)
    _parity.check_grid(fc, ctx, gid, w2, pts, 11, d, b, n, od, ob, on, opts=opts, label=f"cfg2 subset top-{topk}")
    print("cfg2 subset stats", st)


def test_plain_fp64_cfg2_subset(fc, ctx, w2):
    gid = grid(fc, ctx, w2)
    pts = _cfg2_points(w2, 3)
    d, b, n = fc.fc_run_points(ctx, gid, pts, 5, 100, opts=dict(precision=fc.FC_PREC_FP64))
    od, ob, on = oracle.run_points(w2.S, w2.F, pts, 5, 100, collapse=w2.collapse, n_fit=w2.n_fit)
    _parity.check_plain(d, b, n, od, ob, on)


@pytest.mark.parametrize("prec", [0, 1])
def test_identity_covariance_nearest_neighbour(fc, ctx, w1, prec):
    gid = grid(fc, ctx, w1)
    d, b, n = fc.fc_run_points(ctx, gid, w1.points, 3, 400, opts=dict(precision=prec, cov=fc.FC_COV_IDENTITY))
    od, ob, on, fk = oracle.run_workload(w1, U=400, seed=3, cov=oracle.COV_IDENTITY, want_fake=True)
    _compare(fc, ctx, gid, w1, w1.points, 3, d, b, n, od, ob, on, prec, "A = I", cov=oracle.COV_IDENTITY)
    dist, idx = spatial.cKDTree(w1.S).query(fk[0].astype(np.float64), k=2)
    clear = dist[:, 1] ** 2 - dist[:, 0] ** 2 > 1e-3
    np.testing.assert_array_equal(b[0][clear], idx[clear, 0])


@pytest.mark.parametrize("prec", [0, 1])
def test_fixed_covariance(fc, ctx, w1, prec):
    gid = grid(fc, ctx, w1)
    d, b, n = fc.fc_run_points(ctx, gid, w1.points, 9, 500, opts=dict(precision=prec, cov=fc.FC_COV_FIXED))
    od, ob, on = oracle.run_workload(w1, U=500, seed=9, cov=oracle.COV_FIXED)
    _compare(fc, ctx, gid, w1, w1.points, 9, d, b, n, od, ob, on, prec, "fixed covariance", cov=oracle.COV_FIXED)
    assert np.all(n == 1)


@pytest.mark.parametrize("prec", [0, 1])
def test_single_scan_entry(fc, ctx, w1, prec):
    gid = grid(fc, ctx, w1)
    rng = np.random.default_rng(5)
    fk = oracle.fake_data(w1.S, w1.F, [312], 21, 300)[0]
    qcov = rng.integers(0, w1.G, 300)
    best, chi2 = fc.fc_scan(ctx, gid, fk, qcov, precision=prec)
    for u in range(0, 300, 7):
        A = oracle.inv_cov(w1.S[qcov[u]], w1.F)
        c = oracle.scan(w1.S, A, fk[u].astype(np.float64))
        assert abs(chi2[u] - c.min()) <= 1e-9 * max(1.0, c.min())
        if prec == 0:
            assert best[u] == int(np.argmin(c))
        else:
            assert c[best[u]] - c.min() < TOL_MIXED


def test_batch_composition_invariance(fc, ctx, w2):
    gid = grid(fc, ctx, w2)
    pts = _cfg2_points(w2, 5)
    d_all, b_all, _ = fc.fc_run_points(ctx, gid, pts, 17, 200)
    d_one, b_one, _ = fc.fc_run_points(ctx, gid, pts[3:4], 17, 200)
    d_rev, _, _ = fc.fc_run_points(ctx, gid, pts[::-1].copy(), 17, 200)
    np.testing.assert_array_equal(d_all[3], d_one[0])
    np.testing.assert_array_equal(b_all[3], b_one[0])
    np.testing.assert_array_equal(d_all[::-1], d_rev)


def test_ragged_universe_count(fc, ctx, w1):
    gid = grid(fc, ctx, w1)
    pts = np.array([312, 5])
    d, b, n = fc.fc_run_points(ctx, gid, pts, 1, 77)
    od, ob, on = oracle.run_points(w1.S, w1.F, pts, 1, 77)
    _compare(fc, ctx, gid, w1, pts, 1, d, b, n, od, ob, on, 1, "ragged U = 77")


def test_quantiles(fc, ctx):
    rng = np.random.default_rng(0)
    x = rng.chisquare(2, (7, 1000))
    p = np.array([0.0, 0.5, 0.68, 0.9, 0.95, 1.0])
    np.testing.assert_allclose(fc.fc_quantiles(ctx, x, p), np.quantile(x, p, axis=1).T, rtol=1e-14)


def test_empty_and_errors(fc, ctx, w1):
    gid = grid(fc, ctx, w1)
    d, b, n = fc.fc_run_points(ctx, gid, np.array([312]), 0, 0)
    assert d.size == 0
    with pytest.raises(fc.FCError) as e:
        fc.fc_run_points(ctx, 12345, np.array([1]), 0, 10)
    assert e.value.status == fc.FC_ERR_NOT_FOUND
    with pytest.raises(fc.FCError) as e:
        fc.fc_run_points(ctx, gid, np.array([w1.G]), 0, 10)
    assert e.value.status == fc.FC_ERR_ARG
    g2 = fc.fc_load_grid(ctx, w1.S)
    with pytest.raises(fc.FCError) as e:
        fc.fc_run_points(ctx, g2, np.array([1]), 0, 10)
    assert e.value.status == fc.FC_ERR_STATE
    fc.fc_unload_grid(ctx, g2)
    bad = w1.S.copy()
    bad[3, 4] = np.nan
    with pytest.raises(fc.FCError) as e:
        fc.fc_load_grid(ctx, bad)
    assert e.value.status == fc.FC_ERR_ARG
    with pytest.raises(fc.FCError) as e:
        fc.fc_run_points(ctx, gid, np.array([1]), 0, 10, opts=dict(max_iter=0))
    assert e.value.status == fc.FC_ERR_ARG


def test_serving_matches_synchronous(fc, ctx, w1, w2):
    g1, g2 = grid(fc, ctx, w1), grid(fc, ctx, w2)
    pts2 = _cfg2_points(w2, 3)
    ref1 = fc.fc_run_points(ctx, g1, w1.points, 4, 300)[0]
    ref2 = fc.fc_run_points(ctx, g2, pts2, 4, 150)[0]
    jobs = []
    for _ in range(3):
        jobs.append((fc.fc_submit(ctx, g1, w1.points, 4, 300), ref1))
        jobs.append((fc.fc_submit(ctx, g2, pts2, 4, 150), ref2))
    import time
    pending = list(jobs)
    t0 = time.time()
    while pending and time.time() - t0 < 120:
        keep = []
        for (t, outs), ref in pending:
            st, lat = fc.fc_poll(ctx, t)
            if st == fc.FC_PENDING:
                keep.append(((t, outs), ref))
            else:
                np.testing.assert_array_equal(outs[0], ref)
                assert lat > 0
        pending = keep
        time.sleep(0.01)
    assert not pending


# ------------------------------------------------ FC region (critical values) --

def test_data_dchi2_and_region(fc, ctx, w1, w2):
    """The observed data's dchi2 at every grid point against the oracle, and the
    accepted region at 68/90 % CL from the points' own universes."""
    g2 = grid(fc, ctx, w2)
    # an "observed" spectrum: one fluctuation of a true point (its fake data)
    obs = oracle.fake_data(w2.S, w2.F, [5555], 3, 1, collapse=w2.collapse, n_fit=w2.n_fit)[0, 0]
    pts = _cfg2_points(w2, 40)
    od, ob, on = oracle.run_data(w2.S, w2.F, pts, obs, collapse=w2.collapse, n_fit=w2.n_fit)
    d, b, n = fc.fc_data_dchi2(ctx, g2, obs, pts, opts=dict(precision=fc.FC_PREC_FP64))
    _parity.check_plain(d, b, n, od, ob, on)
    d, b, n = fc.fc_data_dchi2(ctx, g2, obs, pts, opts=dict(precision=fc.FC_PREC_MIXED))
    assert np.abs(d - od).max() <= _parity.TOL_DCHI2
    for i in np.nonzero((b != ob) | (n != on))[0]:
        traj = [int(fc.fc_data_dchi2(ctx, g2, obs, pts[i:i + 1], opts=dict(max_iter=t))[1][0]) for t in range(1, 6)]
        _parity.check_near_tie(fc, ctx, g2, w2, int(pts[i]), 0, 0, data=obs, gpu=traj)
    # region: universes of each point, then the acceptance at two confidence levels
    U = 400
    du = fc.fc_run_points(ctx, g2, pts, 17, U)[0]
    ddat = fc.fc_data_dchi2(ctx, g2, obs, pts)[0]
    for cl in (0.68, 0.90):
        crit, acc = fc.fc_fc_region(ctx, du, ddat, cl)
        ref = np.quantile(du, cl, axis=1)
        np.testing.assert_allclose(crit, ref, rtol=1e-12, atol=0)
        np.testing.assert_array_equal(acc, (ddat <= ref).astype(np.uint8))
    with pytest.raises(fc.FCError) as e:
        fc.fc_fc_region(ctx, du, ddat, 1.5)
    assert e.value.status == fc.FC_ERR_ARG


def test_device_generated_grid(fc, ctx, w2):
    """Spectra generated on the device from the shape model behind the 100x100 grid give the
    same fit as the host-generated spectra (plain path to 1e-9, mixed path to 1e-4)."""
    m = workloads.osc_2d_model(100, 100, 90, seed=0)
    gd = fc.fc_load_grid_osc(ctx, [m["dm2"], m["s2t"]], [(1, 0)], m["b"], m["f"][None, :], m["L"], m["E"],
                             w2.collapse, w2.n_fit)
    fc.fc_set_frac_cov(ctx, gd, w2.F)
    gh = grid(fc, ctx, w2)
    pts = _cfg2_points(w2, 24)
    # both grids against the oracle on the host spectra (the device's model evaluation differs from
    # numpy's only in the last bits of a spectrum)
    od, ob, on = oracle.run_points(w2.S, w2.F, pts, 9, 64, collapse=w2.collapse, n_fit=w2.n_fit)
    for g in (gd, gh):
        d, b, n = fc.fc_run_points(ctx, g, pts, 9, 64, dict(precision=fc.FC_PREC_FP64))
        _parity.check_plain(d, b, n, od, ob, on)
        d, b, n = fc.fc_run_points(ctx, g, pts, 9, 64, dict(precision=fc.FC_PREC_MIXED))
        _parity.check_grid(fc, ctx, g, w2, pts, 9, d, b, n, od, ob, on, label="device-generated grid")
    # both grids' fake data are the oracle's bit for bit
    fd = fc.fc_fake_data(ctx, gd, pts[:4], 3, 16, w2.n_fit)
    np.testing.assert_array_equal(fd, oracle.fake_data(w2.S, w2.F, pts[:4], 3, 16, collapse=w2.collapse,
                                                       n_fit=w2.n_fit))
    fc.fc_unload_grid(ctx, gd)
    for bad in (dict(E=-m["E"]), dict(terms=[(2, 0)])):
        kw = dict(axes=[m["dm2"], m["s2t"]], terms=[(1, 0)], b=m["b"], f=m["f"][None, :], L=m["L"], E=m["E"],
                  collapse=w2.collapse, n_fit=w2.n_fit)
        kw.update(bad)
        with pytest.raises(fc.FCError) as e:
            fc.fc_load_grid_osc(ctx, **kw)
        assert e.value.status == fc.FC_ERR_ARG


def _osc_case(case):
    """(model arrays, collapse, N_fit, host spectra [G][N_full], true points) of a recompute case."""
    if case == "d2_pairs":
        # the 100 x 100 grid behind cfg2: one term, N 90 -> 45 pairwise (fit bins sum two model bins)
        m2 = workloads.osc_2d_model(100, 100, 90, seed=0)
        m = dict(axes=[m2["dm2"], m2["s2t"]], terms=[(1, 0)], b=m2["b"], f=m2["f"][None, :], L=m2["L"], E=m2["E"],
                 F=m2["F"])
        S = workloads.osc_2d(100, 100, 90, seed=0)[0]
        return m, workloads.pair_collapse(90), 45, S, np.array([0, 1234, 5050, 7777, 9999], np.int64)
    if case == "d6_3terms":
        # the shape of cfg5 at 8 points per axis: D = 6, three terms, N = 64 (K = 80), 262 144 points
        m = workloads.osc_terms_model(8, 3, 64, seed=5)
        return m, None, 64, None, np.array([11, 99_999, 262_143], np.int64)
    # D = 4, two terms, N = 70 (K = 80: the residuals of the flat path, q-vectors in K slices)
    m = workloads.osc_terms_model(6, 2, 70, seed=21)
    S = m["rows"](np.arange(m["G"]))
    return m, None, 70, S, np.array([7, 300, 777, 1295], np.int64)


def _load_osc(fc, ctx, m, coll, n_fit, recompute):
    g = fc.fc_load_grid_osc(ctx, m["axes"], m["terms"], m["b"], m["f"], m["L"], m["E"], coll, n_fit,
                            recompute=recompute)
    fc.fc_set_frac_cov(ctx, g, m["F"])
    return g


@pytest.mark.parametrize("case", ["d2_pairs", "d4_n70", "d6_3terms"])
def test_recomputed_grid(fc, ctx, case):
    """A grid kept as its shape model (FC_GRID_RECOMPUTE: no spectra stored, every row evaluated
    from the model where a kernel reads it, the paper's no-caching choice) gives the stored
    grid's outputs bit for bit on the mixed, plain, list-first, fixed-covariance and fake-data
    paths; both agree with the oracle run on the host's spectra; and it holds a fraction of the
    stored grid's device memory."""
    m, coll, n_fit, S, pts = _osc_case(case)
    b0 = fc.fc_get_stats(ctx)["device_bytes"]
    gs = _load_osc(fc, ctx, m, coll, n_fit, False)
    b1 = fc.fc_get_stats(ctx)["device_bytes"]
    gr = _load_osc(fc, ctx, m, coll, n_fit, True)
    b2 = fc.fc_get_stats(ctx)["device_bytes"]
    stored, kept = b1 - b0, b2 - b1
    nf, G = len(m["b"]), int(m["G"]) if "G" in m else S.shape[0]
    K = ((n_fit + 3 + 15) // 16) * 16
    # stored: S_full, S_fit, Sc (f64), Sdf (2 x f32), Sc32 per point; both: the bf16 image and norms
    assert stored >= G * (8 * nf + 28 * n_fit), (stored, kept)
    assert kept <= G * (4 * K + 16) + (1 << 20), (stored, kept)
    U, seed = (96, 5) if S is not None else (16, 5)
    runs = [("mixed", None, {}), ("plain", dict(precision=fc.FC_PREC_FP64), {}),
            ("list first", None, dict(first_round=fc.FC_ROUND_LIST)), ("fixed covariance", dict(cov=fc.FC_COV_FIXED), {})]
    for label, opts, tuning in runs:
        for g in (gs, gr):
            fc.fc_set_tuning(ctx, g, **tuning)
        a = fc.fc_run_points(ctx, gs, pts, seed, U, opts)
        r = fc.fc_run_points(ctx, gr, pts, seed, U, opts)
        for x, y in zip(a, r):
            np.testing.assert_array_equal(x, y, err_msg=f"{case}: {label}")
    for g in (gs, gr):
        fc.fc_set_tuning(ctx, g)
    np.testing.assert_array_equal(fc.fc_fake_data(ctx, gs, pts, 3, 32, n_fit),
                                  fc.fc_fake_data(ctx, gr, pts, 3, 32, n_fit))
    # the recomputed grid against the oracle on the host's spectra (numpy's sine may differ from the
    # device's in the last bits, hence the contract's tolerances rather than bit equality); the
    # 262 144-point case is held to the stored grid only (the oracle's full scans take minutes there)
    if S is not None:
        d, b, n = fc.fc_run_points(ctx, gr, pts, seed, U)
        od, ob, on = oracle.run_points(S, m["F"], pts, seed, U, collapse=coll, n_fit=n_fit)
        w = workloads.Workload(f"osc_{case}", S, m["F"], coll, n_fit, pts, U, 5, seed)
        _parity.check_grid(fc, ctx, gr, w, pts, seed, d, b, n, od, ob, on, label=f"recomputed {case}")
    fc.fc_unload_grid(ctx, gs)
    fc.fc_unload_grid(ctx, gr)
    with pytest.raises(fc.FCError) as e:
        fc.fc_load_grid_osc(ctx, m["axes"], m["terms"], m["b"], m["f"], m["L"], m["E"], coll, n_fit, flags=2)
    assert e.value.status == fc.FC_ERR_ARG


def _adaptive_reference(w, pts, data_dchi2, cl, U0, U_max, z, seed):
    """The adaptive acceptance rule restated on the oracle's universes: round r draws
    U0, then as many universes as a still-open point has (key seed + r), counts those
    below the data's dchi2, and closes a point once |F - cl| > z sqrt(cl (1 - cl) / U)
    or U reaches U_max; accepted when F <= cl."""
    P = len(pts)
    cnt = np.zeros(P, np.int64)
    used = np.zeros(P, np.int64)
    open_ = list(range(P))
    r = 0
    while open_:
        have = int(used[open_[0]])
        Ur = U0 if r == 0 else min(have, U_max - have)
        du, _, _ = oracle.run_points(w.S, w.F, pts[open_], seed + r, Ur, collapse=w.collapse, n_fit=w.n_fit)
        still = []
        for k, i in enumerate(open_):
            cnt[i] += int((du[k] < data_dchi2[i]).sum())
            used[i] += Ur
            F = cnt[i] / used[i]
            if used[i] < U_max and abs(F - cl) <= z * np.sqrt(cl * (1 - cl) / used[i]):
                still.append(i)
        open_ = still
        r += 1
    F = cnt / used
    return (F <= cl).astype(np.uint8), used.astype(np.int32), F


def test_fc_region_adaptive(fc, ctx, w1):
    """Adaptive universes per point: the plain binary64 path's decisions, universe
    counts and empirical fractions equal the rule run on the oracle's universes."""
    g1 = grid(fc, ctx, w1)
    obs = oracle.fake_data(w1.S, w1.F, [312], 5, 1)[0, 0]
    # the dm2 row and the sin^2 2theta column through the true point: the contour crosses both
    pts = np.unique(np.concatenate([np.arange(300, 325), np.arange(12, 625, 25)])).astype(np.int64)
    od, _, _ = oracle.run_data(w1.S, w1.F, pts, obs)
    cl, U0, U_max, z, seed = 0.9, 32, 256, 2.0, 23
    acc, used, frac = fc.fc_fc_region_adaptive(ctx, g1, pts, od, cl, U0, U_max, z, seed,
                                               opts=dict(precision=fc.FC_PREC_FP64))
    racc, rused, rfrac = _adaptive_reference(w1, pts, od, cl, U0, U_max, z, seed)
    np.testing.assert_array_equal(used, rused)
    np.testing.assert_array_equal(acc, racc)
    np.testing.assert_array_equal(frac, rfrac)
    assert len(np.unique(used)) >= 2          # some points stop at U0, some take more universes
    assert used.min() >= U0 and used.max() <= U_max
    # a point that stopped early is z standard errors from cl
    early = used < U_max
    se = np.sqrt(cl * (1 - cl) / used[early])
    assert np.all(np.abs(frac[early] - cl) > z * se)
    # the tensor-core path takes the same decisions with the same universe counts: its dchi2 agree
    # with the binary64 fit far inside 1e-4 and none of these universes lies that close to the data's
    acc_m, used_m, frac_m = fc.fc_fc_region_adaptive(ctx, g1, pts, od, cl, U0, U_max, z, seed)
    np.testing.assert_array_equal(acc_m, acc)
    np.testing.assert_array_equal(used_m, used)
    np.testing.assert_array_equal(frac_m, frac)
    with pytest.raises(fc.FCError) as e:
        fc.fc_fc_region_adaptive(ctx, g1, pts, od, cl, 64, 32, z, seed)
    assert e.value.status == fc.FC_ERR_ARG
