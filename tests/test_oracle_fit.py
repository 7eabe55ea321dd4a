"""Pins for the oracle's fit (Eq. 1, Algorithms 1-2, the refit loop of §2).

The oracle is compared with: numpy.linalg (Cholesky, inverse), an independent
vectorised numpy brute force of the whole per-universe procedure, a k-d tree
nearest neighbour (A = I), Wilks' chi2_D law for a linear-Gaussian model, the
fake data's first two moments, and the invariant dchi2 >= 0.
"""
import numpy as np
import pytest
from scipy import spatial, stats

import oracle
import workloads


# --------------------------------------------------------------------------
# independent numpy restatement (shares nothing with fc_oracle.c)
# --------------------------------------------------------------------------

def np_collapse_matrix(nf, collapse, nfit):
    C = np.zeros((nfit, nf))
    idx = np.arange(nf) if collapse is None else np.asarray(collapse)
    C[idx, np.arange(nf)] = 1.0
    return C


def np_fit_cov(s_full, F, C):
    Mfull = np.diag(s_full) @ F @ np.diag(s_full) + np.diag(s_full)
    return C @ Mfull @ C.T


def np_fit_universe(S, F, C, d, p, max_iter, cov="iterate"):
    Sfit = S @ C.T
    q = p
    nscan = 0
    for t in range(max_iter if cov == "iterate" else 1):
        A = np.eye(C.shape[0]) if cov == "identity" else np.linalg.inv(np_fit_cov(S[q], F, C))
        R = Sfit - d[None, :]
        chi2 = np.einsum("gi,ij,gj->g", R, A, R)
        g = int(np.argmin(chi2))           # first minimum = strict "<" in index order
        nscan = t + 1
        if g == q:
            break
        q = g
    return chi2[p] - chi2[g], g, nscan


# --------------------------------------------------------------------------

def test_cholesky_matches_numpy():
    rng = np.random.default_rng(0)
    for n in (1, 2, 5, 40, 90, 200):
        X = rng.standard_normal((n, n))
        M = X @ X.T + n * np.eye(n)
        L = oracle.cholesky(M)
        np.testing.assert_allclose(L, np.linalg.cholesky(M), rtol=1e-12, atol=1e-12 * np.abs(L).max())
        assert np.all(np.triu(L, 1) == 0)


def test_cholesky_rejects_non_spd():
    with pytest.raises(np.linalg.LinAlgError):
        oracle.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))


@pytest.mark.parametrize("wl", ["cfg1", "tiny_collapse", "cfg2"])
def test_inverse_covariance_matches_numpy(wl):
    w = {"cfg1": workloads.cfg1, "tiny_collapse": lambda: workloads.tiny(collapse=True, n_full=6),
         "cfg2": workloads.cfg2}[wl]()
    C = np_collapse_matrix(w.n_full, w.collapse, w.n_fit)
    for q in (0, w.G // 2, w.G - 1):
        A = oracle.inv_cov(w.S[q], w.F, w.collapse, w.n_fit)
        ref = np.linalg.inv(np_fit_cov(w.S[q], w.F, C))
        np.testing.assert_allclose(A, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())


def test_chol_sys_matches_numpy():
    w = workloads.cfg2()
    s = w.S[1234]
    Msys = np.diag(s) @ w.F @ np.diag(s)
    np.testing.assert_allclose(oracle.chol_sys(s, w.F), np.linalg.cholesky(Msys), rtol=1e-11, atol=1e-9)
    np.testing.assert_allclose(oracle.chol_sys(s, w.F, gauss=True), np.linalg.cholesky(Msys + np.diag(s)),
                               rtol=1e-11, atol=1e-9)


def test_collapse_spectra_are_pair_sums():
    w = workloads.cfg2()
    Sfit = oracle.collapse_spectra(w.S[:50], w.collapse, w.n_fit)
    np.testing.assert_array_equal(Sfit, w.S[:50, 0::2] + w.S[:50, 1::2])


def test_scan_matches_einsum():
    w = workloads.cfg1()
    rng = np.random.default_rng(4)
    d = w.S[312] + rng.normal(0, 10, w.n_fit)
    A = oracle.inv_cov(w.S[100], w.F)
    got = oracle.scan(w.S, A, d)
    R = w.S - d
    np.testing.assert_allclose(got, np.einsum("gi,ij,gj->g", R, A, R), rtol=1e-11)


@pytest.mark.parametrize("collapse", [False, True])
@pytest.mark.parametrize("cov", [oracle.COV_ITERATE, oracle.COV_FIXED])
def test_brute_force_tiny_grid(collapse, cov):
    """Whole procedure on a 3x3 grid vs the independent numpy restatement."""
    w = workloads.tiny(3, 3, 6 if collapse else 5, U=50, collapse=collapse)
    dchi2, best, ns, fk = oracle.run_workload(w, cov=cov, want_fake=True)
    C = np_collapse_matrix(w.n_full, w.collapse, w.n_fit)
    p = int(w.points[0])
    for u in range(w.U):
        ref = np_fit_universe(w.S, w.F, C, fk[0, u].astype(np.float64), p, w.max_iter,
                              "iterate" if cov == oracle.COV_ITERATE else "fixed")
        assert best[0, u] == ref[1]
        assert ns[0, u] == ref[2]
        assert abs(dchi2[0, u] - ref[0]) <= 1e-12 * max(1.0, abs(ref[0]))


def test_brute_force_exercises_refit():
    """A 5x5 grid where several universes move away from p and refit (q1 != q0)."""
    w = workloads.tiny(5, 5, 8, U=200, seed=11)
    dchi2, best, ns, fk = oracle.run_workload(w, want_fake=True)
    assert (ns >= 2).sum() > 20
    C = np_collapse_matrix(w.n_full, None, w.n_fit)
    p = int(w.points[0])
    for u in np.where(ns[0] >= 2)[0][:40]:
        ref = np_fit_universe(w.S, w.F, C, fk[0, u].astype(np.float64), p, w.max_iter)
        assert (best[0, u], ns[0, u]) == (ref[1], ref[2])
        assert abs(dchi2[0, u] - ref[0]) <= 1e-12 * max(1.0, abs(ref[0]))


def test_dchi2_nonnegative_and_bestfit_in_grid():
    w = workloads.cfg1()
    dchi2, best, ns = oracle.run_workload(w, U=300)
    assert np.all(dchi2 >= 0.0)
    assert np.all((best >= 0) & (best < w.G))
    assert np.all((ns >= 1) & (ns <= w.max_iter))


def test_identity_covariance_is_nearest_neighbour():
    """A = I: chi2 is a squared Euclidean distance, so the best fit is a k-d tree nearest neighbour."""
    w = workloads.cfg1()
    dchi2, best, ns, fk = oracle.run_workload(w, U=300, cov=oracle.COV_IDENTITY, want_fake=True)
    tree = spatial.cKDTree(w.S)
    d = fk[0].astype(np.float64)
    dist, idx = tree.query(d, k=2)
    p = int(w.points[0])
    chi2p = np.sum((w.S[p] - d) ** 2, axis=1)
    np.testing.assert_allclose(chi2p - dchi2[0], dist[:, 0] ** 2, rtol=1e-10)
    clear = dist[:, 1] ** 2 - dist[:, 0] ** 2 > 1e-6
    assert clear.mean() > 0.9
    np.testing.assert_array_equal(best[0][clear], idx[clear, 0])
    assert np.all(ns == 1)


def test_fake_data_moments():
    """Poisson(max(0, s + L z)): mean ~ s and covariance ~ diag(s) F diag(s) + diag(s)."""
    w = workloads.tiny(3, 3, 6, U=20000, seed=5)
    fk = oracle.fake_data(w.S, w.F, w.points, 17, w.U).astype(np.float64)[0]
    s = w.S[int(w.points[0])]
    Mfull = np.diag(s) @ w.F @ np.diag(s) + np.diag(s)
    n = w.U
    assert np.all(np.abs(fk.mean(0) - s) < 5 * np.sqrt(np.diag(Mfull) / n))
    cov = np.cov(fk.T)
    se = np.sqrt((Mfull ** 2 + np.outer(np.diag(Mfull), np.diag(Mfull))) / n)
    assert np.all(np.abs(cov - Mfull) < 6 * se)


def test_fake_data_collapse_is_integer_pair_sum():
    w = workloads.tiny(3, 3, 6, U=40, seed=5)
    full = oracle.fake_data(w.S, w.F, w.points, 3, w.U)
    fit = oracle.fake_data(w.S, w.F, w.points, 3, w.U, collapse=workloads.pair_collapse(6), n_fit=3)
    np.testing.assert_array_equal(fit, full[..., 0::2] + full[..., 1::2])
    assert np.all(full == np.round(full)) and np.all(full >= 0)


def test_wilks_linear_gaussian():
    """Linear model + Gaussian fluctuation + fixed covariance: dchi2 ~ chi2_2, and the grid
    minimum exceeds the continuous minimum by at most the half-cell quadratic bound."""
    w = workloads.linear_gauss(n_axis=121, U=6000)
    dchi2, best, ns, fk = oracle.run_workload(w, cov=oracle.COV_FIXED, fluct=oracle.FLUCT_GAUSS, want_fake=True)
    x = dchi2[0]
    assert np.all(x >= 0)
    assert stats.kstest(x, stats.chi2(2).cdf).pvalue > 1e-3
    s0, J, TH = w.meta["s0"], w.meta["J"], w.meta["theta"]
    p = int(w.points[0])
    A = np.linalg.inv(np.diag(w.S[p]) @ w.F @ np.diag(w.S[p]) + np.diag(w.S[p]))
    H = J.T @ A @ J
    h = np.array([w.axes[0][1] - w.axes[0][0], w.axes[1][1] - w.axes[1][0]])
    bound = 0.25 * np.abs(H) @ h @ h
    d = fk[0].astype(np.float64)
    R = d - s0
    th_star = np.linalg.solve(H, J.T @ A @ R.T).T
    res_c = R - th_star @ J.T
    chi2_cont = np.einsum("ui,ij,uj->u", res_c, A, res_c)
    res_g = d - w.S[best[0]]
    chi2_grid = np.einsum("ui,ij,uj->u", res_g, A, res_g)
    inside = np.all(np.abs(th_star) < np.array([w.axes[0][-1], w.axes[1][-1]]), axis=1)
    gap = chi2_grid - chi2_cont
    assert np.all(gap[inside] >= -1e-9)
    assert np.all(gap[inside] <= bound + 1e-9)


def test_samples_equal_full_pass_entries():
    """A sampled universe is the same computation as that entry of a full pass."""
    w = workloads.tiny(n_a=4, n_b=4, n_full=6, U=12, collapse=True)
    pts = np.array([0, 5, 9, 15], np.int64)
    d, b, n = oracle.run_points(w.S, w.F, pts, 3, 12, collapse=w.collapse, n_fit=w.n_fit)
    rng = np.random.default_rng(1)
    ip = rng.integers(0, len(pts), 20)
    u = rng.integers(0, 12, 20).astype(np.int32)
    ds, bs, ns = oracle.run_samples(w.S, w.F, pts[ip], u, 3, collapse=w.collapse, n_fit=w.n_fit)
    np.testing.assert_array_equal(ds, d[ip, u])
    np.testing.assert_array_equal(bs, b[ip, u])
    np.testing.assert_array_equal(ns, n[ip, u])


def test_data_mode_is_the_universe_procedure():
    """The observed-data statistic is the universe procedure on given data: with a
    universe's own fake data it reproduces that universe, and data equal to a
    grid spectrum gives dchi2 = 0 at that point."""
    w = workloads.tiny(n_a=4, n_b=4, n_full=6, U=6, collapse=True)
    pts = np.array([2, 7, 13], np.int64)
    d, b, n, fk = oracle.run_points(w.S, w.F, pts, 9, 6, collapse=w.collapse, n_fit=w.n_fit, want_fake=True)
    for ip in range(len(pts)):
        for u in (0, 5):
            dd, bb, nn = oracle.run_data(w.S, w.F, pts[ip:ip + 1], fk[ip, u], collapse=w.collapse, n_fit=w.n_fit)
            assert dd[0] == d[ip, u] and bb[0] == b[ip, u] and nn[0] == n[ip, u]
    sfit = oracle.collapse_spectra(w.S, w.collapse, w.n_fit)
    dd, bb, _ = oracle.run_data(w.S, w.F, np.array([7]), sfit[7].astype(np.float32), collapse=w.collapse,
                                n_fit=w.n_fit)
    assert bb[0] == 7 and dd[0] == 0.0
