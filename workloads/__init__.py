"""Seeded synthetic inputs for the Feldman-Cousins grid fit.

This module only builds inputs: grid spectra S (G x N_full, float64, row-major,
grid index = row-major linear index of the D-dimensional grid, §2), the
fractional systematic covariance F (N_full x N_full), an optional bin-collapse
map and the true-point list.  It holds none of the method's arithmetic (no
covariance build, no fluctuation, no chi2), so both the CPU oracle and the CUDA
library can be fed from it without sharing any of the method.

The paper's inputs are SBN Monte-Carlo histograms that are not available; the
shape model below stands in for them (an oscillation-like signal on top of a
flat-ish background, with a correlated rank-5 systematic on top of a diagonal
part).  Every draw comes from ``numpy.random.default_rng(seed)`` in a fixed
order so the arrays are reproducible on any machine.
"""
from __future__ import annotations

import dataclasses
import hashlib

import numpy as np

__all__ = [
    "Workload",
    "osc_2d",
    "cfg1",
    "cfg2",
    "cfg3",
    "cfg4_grid",
    "cfg4_pool",
    "cfg4_jobs",
    "cfg5",
    "linear_gauss",
    "tiny",
    "digest",
]


@dataclasses.dataclass
class Workload:
    name: str
    S: np.ndarray            # [G, N_full] float64
    F: np.ndarray            # [N_full, N_full] float64, symmetric PD
    collapse: np.ndarray | None   # [N_full] int32 full-bin -> fit-bin, None = identity
    n_fit: int
    points: np.ndarray       # [P] int64 true grid points
    U: int                   # universes per true point
    max_iter: int
    seed: int
    axes: tuple = ()
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def G(self) -> int:
        return int(self.S.shape[0]) if self.S is not None else int(self.meta["model"]["G"])

    @property
    def n_full(self) -> int:
        return int(self.S.shape[1]) if self.S is not None else int(len(self.meta["model"]["b"]))


def digest(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        a = np.ascontiguousarray(a)
        h.update(str(a.dtype).encode())
        h.update(str(a.shape).encode())
        h.update(a.tobytes())
    return h.hexdigest()[:16]


def _frac_cov(rng, n, rank=5, diag=0.2, sig_lo=0.05, sig_hi=0.2):
    """F = diag(sig) C diag(sig), C = W_hat W_hat^T + diag*I, rows of W unit norm."""
    sig = rng.uniform(sig_lo, sig_hi, n)
    W = rng.standard_normal((n, rank))
    W /= np.linalg.norm(W, axis=1, keepdims=True)
    C = W @ W.T + diag * np.eye(n)
    F = sig[:, None] * C * sig[None, :]
    F = 0.5 * (F + F.T)
    return F, sig


def osc_2d_model(n_dm2: int, n_th: int, n_full: int, seed: int = 0) -> dict:
    """The shape model behind osc_2d: axes dm2 (log-spaced over [1e-2, 1e2] eV^2)
    and sin^2 2theta (log-spaced over [1e-4, 1]), E_i linear over [0.2, 3] GeV.
    Draw order from default_rng(seed): b ~ U(50,500), f ~ U(5,50),
    sig ~ U(0.05,0.2), W ~ N(0,1)[N x 5], L ~ choice{110,470,600}; F from sig, W."""
    rng = np.random.default_rng(seed)
    n = n_full
    b = rng.uniform(50.0, 500.0, n)
    f = rng.uniform(5.0, 50.0, n)
    sig = rng.uniform(0.05, 0.2, n)
    W = rng.standard_normal((n, 5))
    L = rng.choice(np.array([110.0, 470.0, 600.0]), n)
    E = np.linspace(0.2, 3.0, n)
    W = W / np.linalg.norm(W, axis=1, keepdims=True)
    C = W @ W.T + 0.2 * np.eye(n)
    F = sig[:, None] * C * sig[None, :]
    F = 0.5 * (F + F.T)
    return {"b": b, "f": f, "L": L, "E": E, "F": F, "dm2": np.logspace(-2, 2, n_dm2),
            "s2t": np.logspace(-4, 0, n_th)}


def osc_2d(n_dm2: int, n_th: int, n_full: int, seed: int = 0):
    """Two-parameter grid (dm2 slow axis, sin^2 2theta fast axis) of osc_2d_model:
    s_i(p) = b_i + sin^2(2theta) * sin^2(1.27 dm2 L_i / E_i) * f_i."""
    m = osc_2d_model(n_dm2, n_th, n_full, seed)
    b, f, L, E, dm2, s2t = m["b"], m["f"], m["L"], m["E"], m["dm2"], m["s2t"]
    n = n_full
    osc = np.sin(1.27 * dm2[:, None] * L[None, :] / E[None, :]) ** 2   # [n_dm2, n]
    S = b[None, None, :] + s2t[None, :, None] * osc[:, None, :] * f[None, None, :]
    S = np.ascontiguousarray(S.reshape(n_dm2 * n_th, n))
    return S, m["F"], (dm2, s2t)


def cfg1(U: int = 1000) -> Workload:
    """D=2, 25x25 grid, N=40, one true point (dm2=1, sin^2 2theta=0.01), U=1000, <=5 scans, FP64."""
    S, F, axes = osc_2d(25, 25, 40, seed=0)
    p = 12 * 25 + 12
    return Workload("cfg1_d2_25x25_n40", S, F, None, 40, np.array([p], np.int64), U, 5, 0, axes)


def pair_collapse(n_full: int) -> np.ndarray:
    return (np.arange(n_full) // 2).astype(np.int32)


def cfg2(U: int = 1000, points: np.ndarray | None = None) -> Workload:
    """D=2, 100x100 grid, N_full=90 collapsed pairwise to 45; every grid point is a true point."""
    S, F, axes = osc_2d(100, 100, 90, seed=0)
    pts = np.arange(S.shape[0], dtype=np.int64) if points is None else np.asarray(points, np.int64)
    return Workload("cfg2_d2_100x100_n90to45", S, F, pair_collapse(90), 45, pts, U, 5, 0, axes)


def cfg3(U: int = 500, n_points: int = 2048, n_axis: int = 64) -> Workload:
    """D=3 (dm2, |Ue4|^2, |Umu4|^2), 64 log-spaced points per axis, N=120 (60 appearance + 60 disappearance)."""
    rng = np.random.default_rng(0)
    h = 60
    b = rng.uniform(50.0, 500.0, h)
    f = rng.uniform(5.0, 50.0, h)
    bp = rng.uniform(50.0, 500.0, h)
    F, _ = _frac_cov(rng, 2 * h)
    L = rng.choice(np.array([110.0, 470.0, 600.0]), h)
    E = np.linspace(0.2, 3.0, h)
    dm2 = np.logspace(-2, 2, n_axis)
    ue = np.logspace(-4, np.log10(0.5), n_axis)
    um = np.logspace(-4, np.log10(0.5), n_axis)
    osc = np.sin(1.27 * dm2[:, None] * L[None, :] / E[None, :]) ** 2      # [n_axis, h]
    app = b[None, None, None, :] + 4.0 * ue[None, :, None, None] * um[None, None, :, None] \
        * osc[:, None, None, :] * f[None, None, None, :]
    dis = bp[None, None, None, :] * (1.0 - 4.0 * um[None, None, :, None] * (1.0 - um[None, None, :, None])
                                     * osc[:, None, None, :])
    dis = np.broadcast_to(dis, app.shape)
    S = np.ascontiguousarray(np.concatenate([app, dis], axis=-1).reshape(-1, 2 * h))
    pts = np.sort(rng.choice(S.shape[0], n_points, replace=False)).astype(np.int64)
    return Workload("cfg3_d3_64cubed_n120", S, F, None, 2 * h, pts, U, 5, 0, (dm2, ue, um))


def cfg4_grid(D: int, G_target: int, n_full: int, seed: int) -> Workload:
    """One grid of the serving pool: D = 2, 3 or 4 parameters, about G_target
    points (n = round(G_target^(1/D)) per axis), N = n_full bins.

    D=2: the osc_2d model.  D=3: the cfg3 model (appearance bins
    b + 4 Ue Um sin^2(1.27 dm2 L/E) f, then disappearance bins
    b'(1 - 4 Um (1 - Um) sin^2(.))), split N//2 + N - N//2, Um <= 0.45.  D=4: two
    (amplitude, dm2) terms, s = b + sum_j A_j sin^2(1.27 dm2_j L/E) f_j with
    A_j log-spaced over [1e-3, 0.1].  Draw order from default_rng(seed):
    b, f (or f_j), b' (D=3 only), then the fractional covariance, then L.
    """
    n_ax = max(2, int(round(G_target ** (1.0 / D))))
    rng = np.random.default_rng(seed)
    n = n_full
    if D == 2:
        S, F, axes = osc_2d(n_ax, n_ax, n, seed=seed)
    elif D == 3:
        h1, h2 = n // 2, n - n // 2
        b = rng.uniform(50.0, 500.0, h1)
        f = rng.uniform(5.0, 50.0, h1)
        bp = rng.uniform(50.0, 500.0, h2)
        F, _ = _frac_cov(rng, n)
        L = rng.choice(np.array([110.0, 470.0, 600.0]), n)
        E = np.concatenate([np.linspace(0.2, 3.0, h1), np.linspace(0.2, 3.0, h2)])
        dm2 = np.logspace(-2, 2, n_ax)
        ue = np.logspace(-4, np.log10(0.5), n_ax)
        # |Umu4|^2 stops at 0.45 so the disappearance factor 1 - 4 U (1 - U) >= 0.01 keeps M positive definite
        um = np.logspace(-4, np.log10(0.45), n_ax)
        osc = np.sin(1.27 * dm2[:, None] * L[None, :] / E[None, :]) ** 2      # [n_ax, n]
        app = b + 4.0 * ue[None, :, None, None] * um[None, None, :, None] * osc[:, None, None, :h1] * f
        dis = bp * (1.0 - 4.0 * um[None, None, :, None] * (1.0 - um[None, None, :, None]) * osc[:, None, None, h1:])
        dis = np.broadcast_to(dis, (n_ax, n_ax, n_ax, h2))
        S = np.ascontiguousarray(np.concatenate([app, dis], axis=-1).reshape(-1, n))
        axes = (dm2, ue, um)
    elif D == 4:
        b = rng.uniform(50.0, 500.0, n)
        fj = rng.uniform(5.0, 50.0, (2, n))
        F, _ = _frac_cov(rng, n)
        L = rng.choice(np.array([110.0, 470.0, 600.0]), n)
        E = np.linspace(0.2, 3.0, n)
        amp = np.logspace(-3, -1, n_ax)
        dm2 = np.logspace(-2, 2, n_ax)
        osc = np.sin(1.27 * dm2[:, None] * L[None, :] / E[None, :]) ** 2      # [n_ax, n]
        t1 = (amp[:, None, None] * osc[None, :, :] * fj[0]).reshape(n_ax * n_ax, n)
        t2 = (amp[:, None, None] * osc[None, :, :] * fj[1]).reshape(n_ax * n_ax, n)
        S = np.ascontiguousarray((b + t1[:, None, :] + t2[None, :, :]).reshape(-1, n))
        axes = (amp, dm2, amp, dm2)
    else:
        raise ValueError("D must be 2, 3 or 4")
    return Workload(f"cfg4_d{D}_g{S.shape[0]}_n{n}", S, F, None, n, np.zeros(0, np.int64), 0, 5, seed, axes)


def cfg4_pool(n_grids: int = 8, seed: int = 0, G_lo: float = 1e3, G_hi: float = 1e6, N_lo: int = 40,
              N_hi: int = 200) -> list:
    """Resident grids of the serving stream: D ~ U{2,3,4}, G log-uniform in
    [G_lo, G_hi], N ~ U{N_lo..N_hi}; grid k is built from seed 1000 + k."""
    rng = np.random.default_rng(seed)
    D = rng.integers(2, 5, n_grids)
    G = np.exp(rng.uniform(np.log(G_lo), np.log(G_hi), n_grids))
    N = rng.integers(N_lo, N_hi + 1, n_grids)
    return [cfg4_grid(int(D[k]), int(G[k]), int(N[k]), 1000 + k) for k in range(n_grids)]


def cfg4_jobs(pool_sizes: list, rate: float, duration: float, seed: int = 0, U_lo: int = 100,
              U_hi: int = 10000) -> list:
    """Poisson arrivals at `rate` jobs/s over `duration` s.  Job = (arrival s,
    grid k uniform over the pool, one true point uniform over that grid's G,
    job seed, U log-uniform in [U_lo, U_hi])."""
    rng = np.random.default_rng(seed)
    jobs, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        k = int(rng.integers(0, len(pool_sizes)))
        p = int(rng.integers(0, pool_sizes[k]))
        U = int(round(np.exp(rng.uniform(np.log(U_lo), np.log(U_hi)))))
        jobs.append((t, k, p, int(rng.integers(0, 2 ** 62)), U))
    return jobs


def cfg5(n_axis: int = 16, n_points: int = 256, U: int = 16) -> Workload:
    """D=6: three (amplitude, dm2) pairs, 16 points per axis, N=64.

    s = b + sum_j A_j sin^2(1.27 dm2_j L/E) f_j with A_j in linspace(0, 0.1) and
    dm2_j log-spaced over [1e-2, 1e2].  Zero amplitudes give exactly tied spectra.
    """
    rng = np.random.default_rng(0)
    n = 64
    b = rng.uniform(50.0, 500.0, n)
    fj = rng.uniform(5.0, 50.0, (3, n))
    F, _ = _frac_cov(rng, n)
    L = rng.choice(np.array([110.0, 470.0, 600.0]), n)
    E = np.linspace(0.2, 3.0, n)
    amp = np.linspace(0.0, 0.1, n_axis)
    dm2 = np.logspace(-2, 2, n_axis)
    osc = np.sin(1.27 * dm2[:, None] * L[None, :] / E[None, :]) ** 2      # [n_axis, n]
    term = amp[:, None, None] * osc[None, :, :]                          # [amp, dm2, n]
    G = n_axis ** 6
    S = np.empty((G, n), np.float64)
    block = n_axis ** 4
    # axes order: (A1, dm1, A2, dm2, A3, dm3), row-major
    t23 = (term[:, :, None, None, :] * fj[1] + term[None, None, :, :, :] * fj[2]).reshape(block, n)
    t1 = (term * fj[0]).reshape(n_axis * n_axis, n)
    for i in range(n_axis * n_axis):
        S[i * block:(i + 1) * block] = b + t1[i] + t23
    pts = np.sort(rng.choice(G, n_points, replace=False)).astype(np.int64)
    return Workload("cfg5_d6_16pow6_n64", S, F, None, n, pts, U, 5, 0, (amp, dm2))


def osc_terms_model(n_axis: int, n_terms: int, n_full: int, seed: int, amp_hi: float = 0.1) -> dict:
    """A 2 n_terms-axis shape model: axes (A_1, dm2_1, ..., A_T, dm2_T), each with
    n_axis points (A_t linear over [0, amp_hi], dm2_t log-spaced over [1e-2, 1e2]),
    s_i = b_i + sum_t A_t sin^2(1.27 dm2_t L_i / E_i) f_ti, the terms added in
    order t = 0, 1, ....  Draw order from default_rng(seed): b, f [T][N], then
    the fractional covariance, then L.  Returns the model arrays (the form
    fc_load_grid_osc takes) and a function that evaluates the rows of a list of
    grid points on the host."""
    rng = np.random.default_rng(seed)
    n = n_full
    b = rng.uniform(50.0, 500.0, n)
    f = rng.uniform(5.0, 50.0, (n_terms, n))
    F, _ = _frac_cov(rng, n)
    L = rng.choice(np.array([110.0, 470.0, 600.0]), n)
    E = np.linspace(0.2, 3.0, n)
    amp = np.linspace(0.0, amp_hi, n_axis)
    dm2 = np.logspace(-2, 2, n_axis)
    axes = [amp, dm2] * n_terms
    terms = [(2 * t, 2 * t + 1) for t in range(n_terms)]
    osc = np.sin(1.27 * dm2[:, None] * L[None, :] / E[None, :]) ** 2      # [n_axis, n]

    def rows(g):
        g = np.asarray(g, np.int64)
        idx = np.stack(np.unravel_index(g, (n_axis,) * (2 * n_terms)), -1)
        s = np.repeat(b[None, :], len(g), 0)
        for t in range(n_terms):
            s = s + (amp[idx[:, 2 * t]][:, None] * osc[idx[:, 2 * t + 1]]) * f[t]
        return s

    return {"axes": axes, "terms": terms, "b": b, "f": f, "L": L, "E": E, "F": F, "G": n_axis ** (2 * n_terms),
            "rows": rows}


def cfg5_model(n_axis: int = 16, n_points: int = 256, U: int = 16) -> Workload:
    """cfg5 as its shape model (no host spectra): the same draws as cfg5 (b, f, F, L
    from default_rng(0), then the true points), so its grid is cfg5's up to the
    summation order of the three terms.  S is None; meta["model"] holds the
    arrays fc_load_grid_osc takes."""
    m = osc_terms_model(n_axis, 3, 64, seed=0)
    rng = np.random.default_rng(0)
    rng.uniform(50.0, 500.0, 64)
    rng.uniform(5.0, 50.0, (3, 64))
    _frac_cov(rng, 64)
    rng.choice(np.array([110.0, 470.0, 600.0]), 64)
    pts = np.sort(rng.choice(m["G"], n_points, replace=False)).astype(np.int64)
    return Workload("cfg5_d6_16pow6_n64_model", None, m["F"], None, 64, pts, U, 5, 0, (), meta={"model": m})


def linear_gauss(n_axis: int = 121, n: int = 12, half_width: float = 6.0, seed: int = 3, U: int = 10000):
    """Linear signal model s(theta) = s0 + J theta (D=2) on a grid of +-half_width sigma.

    Used with Gaussian fluctuation and a fixed covariance: then dchi2 follows a
    chi-square law with D degrees of freedom (Wilks), up to grid discretisation.
    Returns the workload plus (s0, J, theta grid) for the continuous-minimum check.
    """
    rng = np.random.default_rng(seed)
    s0 = rng.uniform(200.0, 400.0, n)
    J = rng.standard_normal((n, 2)) * 8.0
    F, _ = _frac_cov(rng, n)
    M = np.diag(s0) @ F @ np.diag(s0) + np.diag(s0)
    # grid in units of the parameter standard deviation at the centre
    Fisher = J.T @ np.linalg.solve(M, J)
    cov = np.linalg.inv(Fisher)
    sd = np.sqrt(np.diag(cov))
    t = np.linspace(-half_width, half_width, n_axis)
    th1 = t * sd[0]
    th2 = t * sd[1]
    TH = np.stack(np.meshgrid(th1, th2, indexing="ij"), -1).reshape(-1, 2)
    S = np.ascontiguousarray(s0[None, :] + TH @ J.T)
    p = (n_axis // 2) * n_axis + n_axis // 2
    w = Workload("linear_gauss_d2", S, F, None, n, np.array([p], np.int64), U, 1, seed,
                 (th1, th2), meta=dict(s0=s0, J=J, theta=TH))
    return w


def tiny(n_a: int = 3, n_b: int = 3, n_full: int = 5, seed: int = 7, U: int = 50,
         collapse: bool = False) -> Workload:
    """Tiny oscillation grid for brute-force cross-checks (G <= 9, N <= 5)."""
    S, F, axes = osc_2d(n_a, n_b, n_full, seed=seed)
    coll = pair_collapse(n_full) if collapse else None
    n_fit = (n_full + 1) // 2 if collapse else n_full
    p = (n_a // 2) * n_b + n_b // 2
    return Workload(f"tiny_{n_a}x{n_b}_n{n_full}", S, F, coll, n_fit, np.array([p], np.int64), U, 5, seed, axes)
