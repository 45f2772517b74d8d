"""Pins for the oracle's sampler distribution, Darcy solve, QoIs and MLMC sums."""
import math

import numpy as np
import pytest

from oracle import covariance as cv
from oracle import darcy
from oracle import embedding as em
from oracle import field
from oracle import mlmc


def _R(kind, nu, lam, sigma2, m):
    j, i = np.meshgrid(np.arange(m + 1), np.arange(m + 1), indexing="ij")
    X = np.stack([i.ravel() / m, j.ravel() / m], axis=1)
    d = X[:, None, :] - X[None, :, :]
    return cv.cov(kind, d[..., 0], d[..., 1], nu, lam, sigma2)


@pytest.mark.parametrize("prec", [64, 32])
def test_sample_covariance_matches_R_and_cholesky(prec):
    """Sample covariance of the CE field (Philox normals) against R entrywise
    (§2.1, E[Z Z^T] = R), and a two-sample KS test of a linear functional
    against the dense Cholesky sampler Z = L xi of §2.1 (Eq. (2.4))."""
    m, n_s = 3, 12000
    e = em.setup_embedding(cv.MATERN, 0.5, 0.5, 1.0, m, em.PAD_DOUBLING)
    Z = np.array([np.log(field.sample_k(e, np.ones(e.Lam.shape, bool), None, 9, 0, i, prec)[0]).ravel()
                  for i in range(n_s)])
    R = _R(cv.MATERN, 0.5, 0.5, 1.0, m)
    C = Z.T @ Z / n_s
    sd = np.sqrt((R * R + np.outer(np.diag(R), np.diag(R))) / n_s)
    assert np.max(np.abs(C - R) / sd) < 5.0
    from scipy import stats
    L = np.linalg.cholesky(R)
    Zc = (L @ np.random.default_rng(4).standard_normal((R.shape[0], n_s))).T
    w = np.linspace(-1, 1, R.shape[0])
    assert stats.ks_2samp(Z @ w, Zc @ w).pvalue > 1e-4


def test_plain_coarse_field_is_fine_field_at_even_vertices():
    e = em.setup_embedding(cv.MATERN, 0.5, 0.3, 1.0, 16, em.PAD_DOUBLING)
    full = np.ones(e.Lam.shape, bool)
    kf, kc = field.sample_k(e, full, full, 0, 1, 5)
    assert np.array_equal(kc, kf[::2, ::2])
    mk_c = em.smoothing_mask(e.Lam, e.s // 4 - e.P // 2)
    kf2, kc2 = field.sample_k(e, full, mk_c, 0, 1, 5)
    assert np.array_equal(kf2, kf)
    assert not np.allclose(kc2, kc)


# ------------------------------------------------------------------ Darcy
@pytest.mark.parametrize("m", [4, 8, 32])
def test_constant_k_closed_forms(m):
    """k = 1, f = 0: u = 1 - x nodally, Q_out = 1, u(7/15,7/15) = 8/15,
    ||u||_L2 = 1/sqrt(3).  k = 1, f = 1: u = 1 - x/2 - x^2/2 nodally (the
    three-point stencil is exact on quadratics), Q_out = 3/2, Q_in = 1/2."""
    x = np.arange(m + 1) / m
    k = np.ones((m + 1, m + 1))
    u, (A, F, M) = darcy.solve(k, 0.0)
    assert np.max(np.abs(u - (1 - x)[None, :])) < 1e-13
    q = darcy.qois(u, A, F, M)
    assert np.max(np.abs(q - [1.0, 8.0 / 15.0, 1.0 / math.sqrt(3.0)])) < 1e-13
    u, (A, F, M) = darcy.solve(k, 1.0)
    assert np.max(np.abs(u - (1 - x / 2 - x * x / 2)[None, :])) < 1e-13
    assert abs(darcy.qois(u, A, F, M)[0] - 1.5) < 1e-13
    assert abs(darcy.inflow(u, A, F) - 0.5) < 1e-13


def test_layered_k_parallel_conductors():
    """k = k(x2) only: u = 1 - x1 exactly and Q_out = trapezoid rule of k in x2."""
    m = 16
    ky = np.exp(np.sin(np.arange(m + 1) * 1.3))
    k = np.repeat(ky[:, None], m + 1, axis=1)
    u, (A, F, M) = darcy.solve(k, 0.0)
    x = np.arange(m + 1) / m
    assert np.max(np.abs(u - (1 - x)[None, :])) < 1e-12
    want = (1.0 / m) * (ky.sum() - 0.5 * ky[0] - 0.5 * ky[-1])
    assert abs(darcy.qois(u, A, F, M)[0] - want) < 1e-12


def test_random_k_conservation_symmetry_and_solvers():
    m = 16
    k = np.exp(np.random.default_rng(3).standard_normal((m + 1, m + 1)))
    A, F, M = darcy.assemble(k, 1.0)
    Ad = A.toarray()
    assert np.max(np.abs(Ad - Ad.T)) < 1e-14
    assert np.max(np.abs(Ad.sum(axis=1))) < 1e-13               # constants in the kernel
    assert np.linalg.eigvalsh(Ad).min() > -1e-12
    assert abs(F.sum() - 1.0) < 1e-14                           # integral of f = 1
    assert abs(M.toarray().sum() - 1.0) < 1e-14                 # area of D
    u, (A, F, M) = darcy.solve(k, 1.0, dense=True)
    u2, _ = darcy.solve(k, 1.0, dense=False)
    assert np.max(np.abs(u - u2)) < 1e-12
    q = darcy.qois(u, A, F, M)
    assert abs(q[0] - darcy.inflow(u, A, F) - 1.0) < 1e-12     # Q_out - Q_in = int f
    u0, (A0, F0, _) = darcy.solve(k, 0.0)
    assert abs(darcy.qois(u0, A0, F0, M)[0] - darcy.inflow(u0, A0, F0)) < 1e-12
    assert np.all(u0 <= 1 + 1e-12) and np.all(u0 >= -1e-12)   # maximum principle


def test_point_value_and_mass_exact_on_linear_functions():
    m = 8
    j, i = np.meshgrid(np.arange(m + 1), np.arange(m + 1), indexing="ij")
    x, y = i / m, j / m
    u = 0.3 + 1.7 * x - 0.9 * y
    assert abs(darcy.point_value(u, 7 / 15, 7 / 15) - (0.3 + 0.8 * 7 / 15)) < 1e-14
    assert abs(darcy.point_value(u, 0.61, 0.13) - (0.3 + 1.7 * 0.61 - 0.9 * 0.13)) < 1e-14
    _, _, M = darcy.assemble(np.ones((m + 1, m + 1)))
    v = x.ravel()
    assert abs(v @ (M @ v) - 1.0 / 3.0) < 1e-14


# ------------------------------------------------------------------ MLMC
def test_level_sums_and_estimator():
    Qf = np.array([1.0, 2.0, 4.0])
    Qc = np.array([0.5, 1.0, 1.0])
    N, s1, s2, f1, f2 = mlmc.level_sums(Qf, Qc)
    assert (N, s1, s2, f1, f2) == (3, 4.5, 0.25 + 1 + 9, 7.0, 21.0)
    # telescoping: deterministic Q_l gives the estimator Q_L exactly
    Q = [1.0, 1.5, 1.75]
    sums = [mlmc.level_sums([Q[0]] * 4)] + [mlmc.level_sums([Q[l]] * 3, [Q[l - 1]] * 3)
                                            for l in (1, 2)]
    assert mlmc.estimator(sums) == 1.75


def test_optimal_samples_formula():
    """Eq. (3.6) by hand: V = (4, 1), C = (1, 4): sum sqrt(CV) = 4,
    N_0 = ceil(2/eps^2 * 4 * 2), N_1 = ceil(2/eps^2 * 4 * 0.5)."""
    N = mlmc.optimal_samples([4.0, 1.0], [1.0, 4.0], 0.1)
    assert list(N) == [1600, 400]


def test_richardson_bias_recovers_exact_bias():
    alpha, Ca, h = 1.3, 0.7, 1 / 64
    bias_h = Ca * h ** alpha
    diff = Ca * h ** alpha - Ca * (2 * h) ** alpha        # E[Q_h - Q_2h]
    assert abs(mlmc.richardson_bias(diff, alpha) - bias_h) < 1e-15


def test_level_estimate_end_to_end_small():
    e = em.setup_embedding(cv.MATERN, 0.5, 0.3, 1.0, 8, em.PAD_DOUBLING)
    mf, mc = mlmc.default_masks(e, smoothing=False, finest=True)
    sums, Y = mlmc.level_estimate(e, mf, mc, 0, 1, 0, 4, qoi_index=0)
    assert sums[0] == 4 and abs(sums[1] - Y.sum()) < 1e-15
    for i in range(4):
        kf, kc = field.sample_k(e, mf, mc, 0, 1, i)
        assert abs(Y[i] - (darcy.solve_qois(kf)[0] - darcy.solve_qois(kc)[0])) < 1e-14


def test_tau_rules_solve_their_equations():
    """The numerical solve satisfies the stated equation (the pins against the
    error bounds the rules come from are in test_oracle_tau.py)."""
    assert mlmc.tau_sqrt_s(64 * 64) == 64
    t = mlmc.tau_matern(1 / 32, 32, 1.5, 1.0, 1.0)
    s = 4.0 * (32 + 32) ** 2
    lhs = (s - t + 1) ** (-1.25) * t
    assert abs(lhs - 2 * (1 / 32) ** 2 * 64) < 1e-9 * lhs
    te = mlmc.tau_exponential(4096.0, 1.0, 1.0)
    assert 1 <= te <= 4096


def _coarsest_examples(golden_dir):
    import os
    rows = []
    with open(os.path.join(golden_dir, "coarsest_mesh_examples.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                kind, nu, lam, k = line.split()[:4]
                rows.append((kind, float(nu), float(lam), int(k)))
    return rows


def test_coarsest_mesh_matches_the_paper_examples(golden_dir):
    """Eq. (3.7)-(3.8) against the h0 the paper states for its experiments."""
    rows = _coarsest_examples(golden_dir)
    assert len(rows) == 6
    for kind, nu, lam, k in rows:
        c = cv.SEP_EXP if kind == "sep_exp" else cv.MATERN
        assert mlmc.coarsest_mesh_exponent(c, nu, lam) == k, (kind, nu, lam)
    # the bound itself is admissible (h0 <= bound) and exact powers of two stay
    assert mlmc.coarsest_mesh_exponent(cv.SEP_EXP, 0.5, 0.25) == 2
    assert mlmc.coarsest_mesh_exponent(cv.MATERN, 0.5, 0.125) == 2
    assert mlmc.coarsest_mesh_exponent(cv.SEP_EXP, 0.5, 3.0) == 0


def test_sample_variance_is_the_unbiased_one():
    """V_l in Eq. (3.6) is the unbiased sample variance: for 1, 2, 3, 6 the
    mean is 3 and the variance (4 + 1 + 0 + 9) / 3 = 14/3."""
    y = [1.0, 2.0, 3.0, 6.0]
    mean, var = mlmc.mean_var(len(y), sum(y), sum(v * v for v in y))
    assert mean == 3.0 and abs(var - 14.0 / 3.0) < 1e-15
    assert mlmc.mean_var(1, 2.0, 4.0) == (2.0, 0.0)


def test_default_masks_follow_the_smoothing_reading():
    """MLMC-CES masks (§3.6, with tau_l = sqrt(s_l) as in the numerics of §4):
    plain CE keeps everything; on a level below the finest one smoothed mask,
    dropping the tau smallest eigenvalues (a few more when a tie group
    straddles the cut), drives both grids; on the finest level the fine field
    is unsmoothed and the coarse field keeps the smoothed mask."""
    e = em.setup_embedding(cv.MATERN, 0.5, 0.1, 1.0, 16, em.PAD_SMOOTH)
    s = e.s
    tau = math.isqrt(s)
    assert tau * tau == s                     # s = P^2: tau = P
    f0, c0 = mlmc.default_masks(e, smoothing=False, finest=False)
    assert f0.all() and c0.all()
    f1, c1 = mlmc.default_masks(e, smoothing=True, finest=False)
    dropped = s - int(c1.sum())
    assert np.array_equal(f1, c1)
    assert tau <= dropped <= tau + 8          # symmetric groups of at most 8 on a square grid
    kept, gone = e.Lam[c1], e.Lam[~c1]
    assert kept.min() >= gone.max() * (1 - 1e-10)   # the smallest ones are dropped
    f2, c2 = mlmc.default_masks(e, smoothing=True, finest=True)
    assert f2.all() and np.array_equal(c2, c1)


@pytest.mark.parametrize("m,seed", [(8, 0), (16, 1), (32, 2)])
def test_k_of_x_outflow_between_rayleigh_bounds(m, seed):
    """k varying along the flow only, f = 0.  With the diagonal split the
    five-point conductance of the horizontal edge (a, b)-(a+1, b) is, from the
    legs of the right triangles (each contributes kbar_T / 2),
      (k_a + k_a+1) / 2 on interior rows, (k_a + 2 k_a+1) / 6 on the bottom row
      and (2 k_a + k_a+1) / 6 on the top row,
    so the solution is not y-independent and the series formula is not exact.
    Rayleigh's monotonicity law bounds the outflow (the conductance between
    the Dirichlet sides): cutting every vertical edge gives the independent row
    chains (lower bound); shorting them merges each column into conductance
    m (k_a + k_a+1) / 2, the series formula 1 / sum_a h / ((k_a + k_a+1) / 2)
    (upper bound).  Both coincide at k = 1 (outflow 1)."""
    kx = np.exp(np.random.default_rng(seed).standard_normal(m + 1))
    k = np.tile(kx[None, :], (m + 1, 1))
    q = darcy.solve_qois(k, 0.0)[0]
    ka, kb = kx[:-1], kx[1:]
    rows = [(ka + kb) / 2.0] * (m - 1) + [(ka + 2.0 * kb) / 6.0, (2.0 * ka + kb) / 6.0]
    lower = sum(1.0 / np.sum(1.0 / g) for g in rows)
    upper = 1.0 / np.sum((1.0 / m) / ((ka + kb) / 2.0))
    assert lower * (1 - 1e-12) <= q <= upper * (1 + 1e-12)
    assert upper - lower > 1e-6 * upper            # a genuine interval for random k
    ones = np.ones((m + 1, m + 1))
    assert abs(darcy.solve_qois(ones, 0.0)[0] - 1.0) < 1e-12
