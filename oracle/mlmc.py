"""Monte Carlo / multilevel Monte Carlo combination (§3.3-3.6, §4).

* Y_l = Q_{h_l} - Q_{h_(l-1)} for l >= 1 with the same sample k(., w_i) on
  both grids, Y_0 = Q_{h_0} (§3.4); level sums N, sum Y, sum Y^2, sum Q_f,
  sum Q_f^2.
* MLMC estimator Eq. (3.5): Q_hat = sum_l mean(Y_l); with smoothing (§3.6,
  MLMC-CES) the same sum with the smoothed differences of Algorithm 2.
* Optimal sample sizes Eq. (3.6):
  N_l = ceil(2 eps^-2 (sum_k sqrt(C_k V_k)) sqrt(V_l / C_l)).
* Richardson bias estimate of §4: |E[Q_h - Q]| = |E[Q_h - Q_2h] / (1 - 2^alpha)|,
  and the smoothed variant with the ratio C~_alpha / C_alpha.
* the coarsest mesh of plain MLMC, Eq. (3.7)-(3.8) (§3.6), pinned by the
  examples the paper states in §4.2-4.3 (tests/golden/coarsest_mesh_examples.txt);
* tau rules of §3.6 (the closed form for the separable exponential
  covariance, the equation for the Matern covariance solved numerically); the
  ratio C_s / C_alpha is not given by the paper and is an input here. Pinned
  for every value of it: each rule balances the two terms of its corollary's
  bound, and at nu = 1, J = 0 the Matern rule equals the exponential one with
  the ratio halved.
"""
import math

import numpy as np

from . import darcy
from . import embedding as em
from . import field


def level_sums(Qf, Qc=None):
    """(N, sum Y, sum Y^2, sum Q_f, sum Q_f^2) for one level."""
    Qf = np.asarray(Qf, dtype=np.float64)
    Y = Qf if Qc is None else Qf - np.asarray(Qc, dtype=np.float64)
    return (len(Qf), float(Y.sum()), float((Y * Y).sum()), float(Qf.sum()),
            float((Qf * Qf).sum()))


def mean_var(N, s1, s2):
    mean = s1 / N
    var = (s2 - N * mean * mean) / (N - 1) if N > 1 else 0.0
    return mean, var


def estimator(level_sum_list):
    """Eq. (3.5): sum over levels of the sample mean of Y_l."""
    return sum(s[1] / s[0] for s in level_sum_list)


def optimal_samples(V, C, eps):
    """Eq. (3.6)."""
    V = np.asarray(V, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    total = np.sum(np.sqrt(C * V))
    return np.ceil(2.0 * eps ** -2 * total * np.sqrt(V / C)).astype(np.int64)


def richardson_bias(mean_Y_L, alpha, ratio=1.0):
    """§4: |E[Q_h - Q]| from E[Q_h - Q_2h] (ratio = C~_alpha / C_alpha with smoothing)."""
    return abs(mean_Y_L / (1.0 - ratio * 2.0 ** alpha))


def mse(level_sum_list, bias):
    """Estimated MSE = sum_l V_l / N_l + bias^2."""
    var = 0.0
    for N, s1, s2, *_ in level_sum_list:
        var += mean_var(N, s1, s2)[1] / N
    return var + bias * bias


def coarsest_mesh_exponent(kind, nu, lam):
    """Eq. (3.7) / (3.8): the coarsest mesh of plain MLMC, h0 = 2^-k with the
    largest h0 not above lambda (separable exponential covariance) or
    sqrt(8 nu) lambda (Matern, via the correlation length of Lindgren et al.);
    returns k >= 0."""
    from . import covariance as cv
    bound = lam if kind == cv.SEP_EXP else math.sqrt(8.0 * nu) * lam
    return max(0, math.ceil(-math.log2(bound)))


def tau_sqrt_s(s):
    """tau_l = sqrt(s_l), the rule used in the paper's numerics (§4.1-4.2)."""
    return int(math.isqrt(int(s)))


def tau_exponential(s, alpha, cs_over_calpha=1.0):
    """§3.6, separable exponential covariance: tau = (s+1)/(C_s/(2^a C_a) s^(a/2) + 1).

    C_s / C_alpha is an input (the paper does not give it).
    """
    return (s + 1.0) / (cs_over_calpha / 2.0 ** alpha * s ** (alpha / 2.0) + 1.0)


def tau_matern(h, J, nu, alpha, cs_over_calpha=1.0):
    """§3.6, Matern covariance: solve
    (4(1/h + J)^2 - tau + 1)^(-(1+nu)/2) tau = 2 (C_a/C_s) h^(a+1) (1/h + J)
    for tau in [1, s] by bisection (the left side increases with tau).
    C_s / C_alpha is an input (the paper does not give it).
    """
    s = 4.0 * (1.0 / h + J) ** 2
    rhs = 2.0 / cs_over_calpha * h ** (alpha + 1.0) * (1.0 / h + J)

    def g(t):
        return (s - t + 1.0) ** (-0.5 * (1.0 + nu)) * t - rhs

    lo, hi = 1.0, s
    if g(lo) >= 0:
        return lo
    if g(hi) <= 0:
        return hi
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(mid) > 0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def level_qois(emb, mask_f, mask_c, seed, level, samples, f=0.0, precision=64,
               coarse=True):
    """Algorithm 1/2 step 4 for a list of samples: (Q_f, Q_c) arrays (n_s, 3)."""
    Qf, Qc = [], []
    for i in samples:
        kf, kc = field.sample_k(emb, mask_f, mask_c if coarse else None, seed,
                                level, i, precision)
        Qf.append(darcy.solve_qois(kf, f))
        if coarse:
            Qc.append(darcy.solve_qois(kc, f))
    Qf = np.array(Qf)
    return Qf, (np.array(Qc) if coarse else None)


def level_estimate(emb, mask_f, mask_c, seed, level, first_sample, count,
                   qoi_index=0, f=0.0, precision=64):
    """Algorithm 1 (Algorithm 2 with masks): the level-l sums and per-sample Y."""
    coarse = level > 0
    Qf, Qc = level_qois(emb, mask_f, mask_c, seed, level,
                        range(first_sample, first_sample + count), f, precision,
                        coarse)
    qf = Qf[:, qoi_index]
    qc = Qc[:, qoi_index] if coarse else None
    Y = qf if qc is None else qf - qc
    return level_sums(qf, qc), Y


def default_masks(emb, smoothing, finest):
    """Masks (fine, coarse) for one level.  Plain CE: both full.  MLMC-CES
    (§3.6 estimator; §4: the coarse QoI is computed with the smoothed sample
    used for the fine QoI): the smoothed sample keeps s - tau_l eigenvalues,
    tau_l = sqrt(s_l), and drives both grids; on the finest level the fine
    field is unsmoothed (§3.6) while the coarse field keeps the smoothed one."""
    s = emb.s
    if not smoothing:
        full = np.ones(emb.Lam.shape, dtype=bool)
        return full, full
    smooth = em.smoothing_mask(emb.Lam, s - tau_sqrt_s(s))
    fine = np.ones(emb.Lam.shape, dtype=bool) if finest else smooth
    return fine, smooth
