"""Pins for the oracle's random-number pieces (fake data, §2 step 2).

Each check compares the oracle with something other than itself: published
known-answer vectors, closed forms, numpy's float64 functions, or the exact
normal / Poisson laws (scipy.stats).
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _kat():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,want", _kat())
def test_philox_known_answers(ctr, key, want):
    assert [int(x) for x in oracle.philox4x32_10(ctr, key)] == want


def test_u01_closed_form():
    # u = ((x >> 9) + 1/2) 2^-23 exactly
    assert oracle.u01(0) == 2.0 ** -24
    assert oracle.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert oracle.u01(0x80000000) == 0.5 + 2.0 ** -24
    assert oracle.u01(511) == 2.0 ** -24          # low 9 bits dropped
    assert oracle.u01(512) == 3 * 2.0 ** -24


def test_philox_uniform_statistics():
    # 2^16 blocks -> 2^18 words; KS against U(0,1) and per-bit frequencies
    words = np.array([oracle.philox4x32_10([j, 7, 11, 0], [123, 456]) for j in range(1 << 14)],
                     dtype=np.uint64).ravel()
    u = (((words >> 9).astype(np.float64)) + 0.5) * 2.0 ** -23
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    bits = ((words[:, None] >> np.arange(32, dtype=np.uint64)) & 1).mean(axis=0)
    n = len(words)
    assert np.all(np.abs(bits - 0.5) < 5 * 0.5 / np.sqrt(n))


def _ulp32(x):
    x = np.abs(np.asarray(x, np.float64))
    e = np.floor(np.log2(np.maximum(x, 2.0 ** -126)))
    return 2.0 ** (e - 23)


def test_logf_against_float64():
    rng = np.random.default_rng(1)
    x = np.concatenate([
        rng.uniform(2.0 ** -24, 1.0, 4000),
        np.exp(rng.uniform(-80, 80, 4000)),
        np.float32([2.0 ** -24, 0.5, 1.0, 1.5, 2.0, 10.0, 1e4, 1.41421353816986083984375, 1.4142136573791504]),
    ]).astype(np.float32)
    got = oracle.logf(x).astype(np.float64)
    ref = np.log(x.astype(np.float64))
    err = np.abs(got - ref)
    # absolute error within 2 ulp of the result, or 2^-24 near ln x = 0
    assert np.all(err <= 2 * np.maximum(_ulp32(ref), 2.0 ** -25) + 1e-12)
    assert got[np.where(x == 1.0)[0][0]] == 0.0


def test_expf_against_float64():
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.uniform(-10.0, 0.0, 5000), rng.uniform(-80, 80, 2000),
                        np.float32([0.0, -1e-7, -0.34657359, -10.0])]).astype(np.float32)
    got = oracle.expf(x).astype(np.float64)
    ref = np.exp(x.astype(np.float64))
    rel = np.abs(got - ref) / ref
    assert np.all(rel <= 3 * 2.0 ** -24)
    assert oracle.expf(0.0)[0] == 1.0


def test_sincos_turns_against_float64():
    rng = np.random.default_rng(3)
    u = np.concatenate([rng.uniform(0, 1, 5000), [2.0 ** -24, 0.125, 0.25, 0.375, 0.5, 0.75, 1 - 2.0 ** -24]])
    u = u.astype(np.float32)
    s, c = oracle.sincos_turns(u)
    th = 2 * np.pi * u.astype(np.float64)
    assert np.max(np.abs(s - np.sin(th))) < 4e-7
    assert np.max(np.abs(c - np.cos(th))) < 4e-7
    # quadrant bookkeeping: exact signs at the quarter turns
    q = oracle.sincos_turns(np.float32([0.25, 0.5, 0.75]))
    assert q[0][0] == 1.0 and q[1][1] == -1.0 and q[0][2] == -1.0


def test_normals_ks_and_moments():
    z = np.concatenate([oracle.normals(seed=99, p=5, u=u, n=200) for u in range(1000)]).astype(np.float64)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    n = len(z)
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    # the two members of a Box-Muller pair are uncorrelated
    zz = z.reshape(-1, 2)
    assert abs(np.corrcoef(zz[:, 0], zz[:, 1])[0, 1]) < 5 / np.sqrt(len(zz))


def test_normals_prefix_stable():
    # z[0..n) does not depend on how many normals are requested
    a = oracle.normals(1, 2, 3, 90)
    b = oracle.normals(1, 2, 3, 41)
    np.testing.assert_array_equal(a[:41], b)


@pytest.mark.parametrize("lam", [0.0, 0.3, 5.0, 9.99, 10.0, 47.0, 500.0, 1200.0])
def test_poisson_goodness_of_fit(lam):
    n = 200_000
    x = oracle.poisson_indep(lam, n, seed=2024, p=3, bin=1)
    if lam == 0.0:
        assert np.all(x == 0)
        return
    mean, var = x.mean(), x.var()
    assert abs(mean - lam) < 5 * np.sqrt(lam / n)
    assert abs(var - lam) < 5 * lam * np.sqrt(2.0 / n) + 5 * np.sqrt(lam / n)
    # chi-square goodness of fit on bins with expected count >= 20
    lo, hi = int(stats.poisson.ppf(1e-6, lam)), int(stats.poisson.isf(1e-6, lam)) + 1
    ks = np.arange(lo, hi + 1)
    pmf = stats.poisson.pmf(ks, lam)
    exp_counts = n * pmf
    obs = np.bincount(np.clip(x - lo, 0, hi - lo), minlength=hi - lo + 1)[: hi - lo + 1]
    keep = exp_counts >= 20
    o = np.append(obs[keep], n - obs[keep].sum())
    e = np.append(exp_counts[keep], n - exp_counts[keep].sum())
    chi2 = np.sum((o - e) ** 2 / np.maximum(e, 1e-9))
    dof = len(o) - 1
    assert stats.chi2.sf(chi2, dof) > 1e-4, (lam, chi2, dof)


def test_poisson_stream_consumption_is_per_bin():
    # a bin's draws do not depend on other bins: same (seed, p, u, bin) -> same value
    a = oracle.poisson_draws(47.0, 10, seed=5, p=1, u=2, bin=3)
    b = oracle.poisson_draws(47.0, 10, seed=5, p=1, u=2, bin=3)
    c = oracle.poisson_draws(47.0, 10, seed=5, p=1, u=2, bin=4)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)
