"""Multilevel Monte Carlo driver on top of the C ABI (host orchestration only).

Every sample -- field, fine and coarse Darcy solves, level differences, level
sums -- is computed by ``mlmc_level_estimate`` on the GPU; this module keeps
the per-level running sums, the measured cost per sample, and applies the
formulas of the paper's §3.3-3.6 and §4:

* estimator, Eq. (3.5): Q_hat = sum_l mean(Y_l) (the MLMC-CES estimator of
  §3.6 when the levels were set up with the smoothing masks);
* optimal sample sizes, Eq. (3.6) (``mlmc_optimal_samples`` of the C ABI);
* Richardson bias estimate of §4: |E[Q_h - Q]| ~ |E[Y_L] / (1 - 2^alpha)|,
  and with smoothing (extrapolant the smoothed coarse QoI)
  |E[Y_L] / (1 - (C~_alpha / C_alpha) 2^alpha)|;
* the coarsest level of plain MLMC from the correlation length,
  Eq. (3.7)-(3.8) (``coarsest_cells``);
* predicted cost versus eps of MLMC / MLMC-CES and of plain MC on the finest
  grid from measured level statistics (``cost_versus_eps``, §4.2-4.3);
* levels added until that bias is within the bias share eps / sqrt(2) of the
  mean-square error (``run_adaptive``; the weak-error test of the adaptive MLMC
  algorithm of Giles, which §3.4 builds on);
* rates alpha, beta, gamma by least squares on log2 |E Y_l|, log2 V[Y_l],
  log2 C_l against l (§4);
* checkpoint / resume of the level state (``save_checkpoint``,
  ``load_checkpoint``, ``resume_runners``; ``run_to_rmse(checkpoint=...)``);
* the smoothing rules of §3.6 (``mlmc_tau_exponential`` and
  ``mlmc_tau_matern`` of the C ABI) give a real tau_l; ``keep_for_tau`` turns
  it into the keep count ce_setup_embedding takes (s = P^2 is known once the
  embedding has been set up, so a rule that depends on s is applied by a
  second set-up with that count).

The cost of a sample on level l is the GPU time of its level estimate
divided by its sample count (CUDA events on the launching stream).
"""
import json
import math
import os
from dataclasses import asdict, dataclass, field
from typing import Callable, List, Optional

import numpy as np

from . import sce


@dataclass
class LevelStats:
    level: int
    n: int
    N: int = 0
    sumY: float = 0.0
    sumY2: float = 0.0
    sumQ: float = 0.0
    sumQ2: float = 0.0
    seconds: float = 0.0
    iters: int = 0
    next_sample: int = 0

    @property
    def mean(self):
        return self.sumY / self.N if self.N else 0.0

    @property
    def var(self):
        if self.N < 2:
            return 0.0
        m = self.mean
        return max((self.sumY2 - self.N * m * m) / (self.N - 1), 0.0)

    @property
    def var_q(self):
        if self.N < 2:
            return 0.0
        m = self.sumQ / self.N
        return max((self.sumQ2 - self.N * m * m) / (self.N - 1), 0.0)

    @property
    def cost(self):
        return self.seconds / self.N if self.N else 0.0


@dataclass
class MLMCResult:
    estimate: float
    rmse: float
    stat_error: float
    bias: float
    seconds: float
    levels: List[LevelStats] = field(default_factory=list)
    N_opt: Optional[List[int]] = None
    alpha: float = float("nan")
    var_share: float = 0.5      # variance target / eps^2 used for the sample sizes


class LevelRunner:
    """Runs batches of one MLMC level through mlmc_level_estimate and accumulates sums."""

    def __init__(self, emb, level, seed, qoi=sce.QOI_POINT, f=1.0, rtol=1e-10, precision=32,
                 maxit=2000, max_batch=65535, stream=None):
        import torch
        self.torch = torch
        self.emb = emb
        self.stats = LevelStats(level=level, n=emb.n)
        self.seed, self.qoi, self.f, self.rtol = seed, qoi, f, rtol
        self.precision, self.maxit, self.max_batch = precision, maxit, max_batch
        self.stream = stream if stream is not None else torch.cuda.current_stream()

    def run(self, count):
        torch = self.torch
        st = self.stats
        while count > 0:
            c = min(count, self.max_batch)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            out, _ = sce.mlmc_level_estimate(self.emb, self.seed, st.level, st.next_sample, c,
                                             qoi_index=self.qoi, f=self.f, rtol=self.rtol,
                                             maxit=self.maxit, precision=self.precision,
                                             stream=self.stream.cuda_stream,
                                             allow_not_converged=True)
            e1.record(self.stream)
            e1.synchronize()
            st.seconds += e0.elapsed_time(e1) / 1000.0
            st.N += out.N
            st.sumY += out.sumY
            st.sumY2 += out.sumY2
            st.sumQ += out.sumQf
            st.sumQ2 += out.sumQf2
            st.iters += out.total_iters
            st.next_sample += c
            count -= c
        return st


class ServedLevelRunner:
    """One MLMC level served by a request server (sce.Server): run(count)
    submits a request for the level's next `count` samples and folds its
    level sums in; submit/collect split the two so that several levels can
    be in flight at once.  The cost of a sample is the request's time on the
    server after admission and set-up, divided by its sample count."""

    def __init__(self, server, tenant, level, n, finest, seed, qoi=sce.QOI_POINT, f=1.0):
        self.server, self.tenant = server, dict(tenant)
        self.stats = LevelStats(level=level, n=n)
        self.finest, self.seed, self.qoi, self.f = finest, seed, qoi, f

    def submit(self, count):
        st = self.stats
        t = self.server.submit({**self.tenant, "n": st.n, "level": st.level, "count": count,
                                "finest": int(self.finest), "seed": self.seed,
                                "first_sample": st.next_sample, "qoi_index": self.qoi,
                                "f": self.f})
        st.next_sample += count
        return t

    def collect(self, ticket):
        r = self.server.wait(ticket)
        if r.status not in (sce.CE_OK, sce.CE_ERR_NOT_CONVERGED):
            raise sce.SceError(r.status, "served level estimate")
        st, o = self.stats, r.sums
        st.N += o.N
        st.sumY += o.sumY
        st.sumY2 += o.sumY2
        st.sumQ += o.sumQf
        st.sumQ2 += o.sumQf2
        st.iters += o.total_iters
        st.seconds += r.t_done - r.t_setup_done
        return st

    def run(self, count):
        return self.collect(self.submit(count))


def _run_levels(runners, counts):
    """Runs counts[l] more samples on every level; levels whose runner can
    submit ahead are all in flight at once."""
    pending = []
    for r, c in zip(runners, counts):
        if c <= 0:
            continue
        if hasattr(r, "submit"):
            pending.append((r, r.submit(c)))
        else:
            r.run(c)
    for r, t in pending:
        r.collect(t)


# ---- checkpoint / resume of the level state.  The state of an MLMC run is
# its per-level sums, counts, next sample indices and measured seconds; the
# normals of sample i of level l depend only on (seed, l, i) (counter-based
# Philox), so a run resumed from a checkpoint draws exactly the samples the
# interrupted run would have drawn next.

CHECKPOINT_VERSION = 1


def save_checkpoint(path, runners, meta=None):
    """Writes the level state of `runners` to `path` (JSON; floats round-trip
    exactly), atomically: a crash while writing leaves the previous file."""
    doc = {"version": CHECKPOINT_VERSION, "meta": meta or {},
           "levels": [asdict(r.stats) for r in runners]}
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(doc, fh)
        fh.flush()
        os.fsync(fh.fileno())
    os.replace(tmp, path)


def load_checkpoint(path):
    """(list of LevelStats, meta) from a file written by save_checkpoint."""
    with open(path) as fh:
        doc = json.load(fh)
    if doc.get("version") != CHECKPOINT_VERSION:
        raise ValueError("unsupported checkpoint version %r" % doc.get("version"))
    return [LevelStats(**d) for d in doc["levels"]], doc.get("meta", {})


def resume_runners(runners, stats):
    """Puts checkpointed level state into fresh runners (same levels and
    grids, in order); raises if they do not match."""
    if len(stats) > len(runners):
        raise ValueError("checkpoint has more levels than runners")
    for r, st in zip(runners, stats):
        if (r.stats.level, r.stats.n) != (st.level, st.n):
            raise ValueError("checkpoint level %d (n = %d) does not match runner level %d "
                             "(n = %d)" % (st.level, st.n, r.stats.level, r.stats.n))
        r.stats = LevelStats(**asdict(st))
    return runners


def coarsest_cells(kind, nu, lam):
    """Cells per side n0 = 1/h0 of the coarsest level of plain MLMC: the
    smallest power of two with 1/n0 <= lambda (separable exponential
    covariance, Eq. (3.7)) or 1/n0 <= sqrt(8 nu) lambda (Matern, Eq. (3.8)).
    MLMC-CES may start coarser (§3.6)."""
    bound = lam if kind == sce.CE_COV_SEP_EXP else math.sqrt(8.0 * nu) * lam
    if not bound > 0:
        raise ValueError("lambda and nu must be positive")
    n0 = 1
    while 1.0 / n0 > bound:
        n0 *= 2
    return n0


def keep_for_tau(s, tau):
    """Eigenvalues to keep when tau (real) are to be dropped: s - round(tau),
    at least one kept (the tie rule of the set-up may drop a few more)."""
    s = int(s)
    drop = int(round(float(tau)))
    return max(1, min(s, s - max(drop, 0)))


def fit_rate(levels, values):
    """Least-squares slope of -log2(values) against the level index (a rate)."""
    lv = np.asarray(levels, dtype=float)
    y = np.log2(np.maximum(np.asarray(values, dtype=float), 1e-300))
    if len(lv) < 2:
        return float("nan")
    A = np.vstack([lv, np.ones_like(lv)]).T
    slope = np.linalg.lstsq(A, y, rcond=None)[0][0]
    return float(-slope)


def rates(stats: List[LevelStats]):
    """(alpha, beta, gamma) of §4 from levels l >= 1: |E Y_l| ~ 2^(-alpha l),
    V[Y_l] ~ 2^(-beta l), C_l ~ 2^(gamma l)."""
    s = [x for x in stats if x.level >= 1 and x.N > 1]
    lv = [x.level for x in s]
    alpha = fit_rate(lv, [abs(x.mean) for x in s])
    beta = fit_rate(lv, [x.var for x in s])
    gamma = -fit_rate(lv, [x.cost for x in s])
    return alpha, beta, gamma


def richardson_bias(stats: List[LevelStats], alpha, ratio=1.0, levels=1):
    """§4: |E[Q_h - Q]| from the finest level's mean E[Y_L] = E[Q_h - Q_2h] by
    Richardson extrapolation, |E[Y_L] / (1 - 2^alpha)|.  With smoothing the
    extrapolant is the smoothed coarse QoI and the denominator becomes
    1 - ratio 2^alpha, ratio = C~_alpha / C_alpha (the constants of the
    smoothed and plain bias, |E[Q~_h - Q]| = C~_alpha h^alpha); infinite when
    that denominator vanishes.

    levels > 1: the robust form of Giles' adaptive algorithm -- the largest of
    |E[Y_(L-j)]| 2^(-j alpha), j < levels (levels l >= 1 only), in the
    numerator, so that one finest level whose mean happens to be small (a
    sign change of E[Y_l] in the pre-asymptotic range) does not end the
    level loop."""
    if not math.isfinite(alpha) or alpha <= 0:
        alpha = 1.0
    d = 1.0 - ratio * 2.0 ** alpha
    if d == 0.0:
        return math.inf
    top = abs(stats[-1].mean)
    for j in range(1, levels):
        if len(stats) - 1 - j < 1:
            break
        top = max(top, abs(stats[-1 - j].mean) * 2.0 ** (-j * alpha))
    return abs(top / d)


def cost_versus_eps(stats: List[LevelStats], eps_list, mc_cost_per_sample=None,
                    choose_levels=False, alpha=None, ratio=1.0, bias_levels=1,
                    alpha_levels=3, alpha_max=None, L_min=1):
    """Predicted cost to a root-mean-square error eps from measured level
    statistics, for the cost-versus-accuracy comparisons of §4.2-4.3 (the
    variance share eps^2/2 in both):

    * multilevel (MLMC, or MLMC-CES when the levels were smoothed):
      sum_l N_l C_l with N_l of Eq. (3.6) from the measured V_l and C_l;
    * plain MC on the finest grid used: N = ceil(2 eps^-2 V[Q_L]) samples,
      V[Q_L] the variance of that level's fine QoI, at mc_cost_per_sample each
      (default: that level's cost per sample, which also solves the coarse
      grid, so an upper bound).

    choose_levels: the finest level L(eps) is the coarsest one whose
    Richardson bias (alpha fitted on the `alpha_levels` finest of the measured
    levels, at most alpha_max; ``richardson_bias`` with `bias_levels`) is at
    most eps/sqrt(2), as the adaptive algorithm would pick it (the last
    measured level if none is), and at least L_min (as in ``run_adaptive``);
    otherwise every measured level is used.  The
    statistics of a level that is not the finest stand in for it as the
    finest (under smoothing its fine field would then be unsmoothed).

    Returns one dict per eps: eps, L, N (per level), mlmc_seconds, mc_N,
    mc_seconds."""
    V = [max(s.var, 1e-300) for s in stats]
    C = [max(s.cost, 1e-12) for s in stats]
    a = alpha
    if choose_levels and a is None:
        a = fit_alpha(stats, alpha_levels, alpha_max)
    out = []
    for eps in eps_list:
        L = len(stats) - 1
        if choose_levels:
            for l in range(max(1, L_min), len(stats)):
                if richardson_bias(stats[:l + 1], a, ratio, bias_levels) <= eps / math.sqrt(2.0):
                    L = l
                    break
        N = [int(n) for n in sce.mlmc_optimal_samples(V[:L + 1], C[:L + 1], eps)]
        vq = stats[L].var_q
        c_mc = C[L] if mc_cost_per_sample is None else float(mc_cost_per_sample)
        mc_N = int(math.ceil(2.0 * vq / (eps * eps)))
        out.append({"eps": eps, "L": L, "N": N,
                    "mlmc_seconds": sum(n * c for n, c in zip(N, C[:L + 1])),
                    "mc_N": mc_N, "mc_seconds": mc_N * c_mc})
    return out


def fit_alpha(stats: List[LevelStats], finest=None, alpha_max=None):
    """alpha of §4 from |E Y_l| of levels l >= 1; with `finest`, from the
    `finest` finest levels only (the coarse levels of a rough field are not
    yet in the asymptotic regime, and the Richardson estimate extrapolates
    from the finest one); at most alpha_max when given (a fit through a
    pre-asymptotic dip of |E Y_l| can return rates no discretisation has)."""
    s = [x for x in stats if x.level >= 1 and x.N > 1]
    if finest is not None:
        s = s[-finest:]
    a = fit_rate([x.level for x in s], [abs(x.mean) for x in s])
    if alpha_max is not None and math.isfinite(a):
        a = min(a, alpha_max)
    return a


def run_to_rmse(runners: List[LevelRunner], eps, pilot=None, alpha=None, max_rounds=10,
                ratio=1.0, var_share=0.5, alpha_levels=None, alpha_max=None, bias_levels=1,
                checkpoint=None):
    """MLMC with the fixed level set of `runners` to a root-mean-square error eps:
    pilot samples, then the optimal N_l from the measured V_l and C_l for the
    variance target var_share * eps^2 (Eq. (3.6) as printed: var_share = 1/2),
    topped up until no level needs more than 1 % extra samples.  alpha (given,
    or fitted on the `alpha_levels` finest levels, all levels l >= 1 if None)
    enters the Richardson bias.  Returns the estimate, the estimated RMSE
    (statistical error and bias) and the GPU seconds spent.

    checkpoint: a file path; if it exists, the runners resume from the level
    state in it (``resume_runners``), and the state is saved there after the
    pilot and after every round, so that an interrupted run can be restarted
    with the same arguments and continues where it stopped."""
    if not 0.0 < var_share <= 1.0:
        raise ValueError("var_share must be in (0, 1]")
    if checkpoint and os.path.exists(checkpoint):
        resume_runners(runners, load_checkpoint(checkpoint)[0])
    pilot = pilot or [100] * len(runners)
    _run_levels(runners, [p - r.stats.N for r, p in zip(runners, pilot)])
    if checkpoint:
        save_checkpoint(checkpoint, runners, {"eps": eps})
    N_opt = None
    # Eq. (3.6) sizes for the variance target eps_v^2 / 2 = var_share eps^2
    eps_v = eps * math.sqrt(2.0 * var_share)
    for _ in range(max_rounds):
        V = [max(r.stats.var, 1e-300) for r in runners]
        C = [max(r.stats.cost, 1e-12) for r in runners]
        N_opt = sce.mlmc_optimal_samples(V, C, eps_v)
        extra = [max(0, int(n) - r.stats.N) for n, r in zip(N_opt, runners)]
        if all(e <= 0.01 * r.stats.N for e, r in zip(extra, runners)):
            break
        _run_levels(runners, extra)
        if checkpoint:
            save_checkpoint(checkpoint, runners, {"eps": eps})
    stats = [r.stats for r in runners]
    est = sum(s.mean for s in stats)
    stat_err = math.sqrt(sum(s.var / s.N for s in stats))
    a = alpha if alpha is not None else fit_alpha(stats, alpha_levels, alpha_max)
    bias = richardson_bias(stats, a, ratio, bias_levels)
    return MLMCResult(estimate=est, rmse=math.sqrt(stat_err ** 2 + bias ** 2), stat_error=stat_err,
                      bias=bias, seconds=sum(s.seconds for s in stats), levels=stats,
                      N_opt=[int(n) for n in N_opt], alpha=a, var_share=var_share)


def run_adaptive(make_runner: Callable[[int, bool], LevelRunner], eps, L0=2, L_max=8,
                 pilot=100, alpha=None, ratio=1.0, max_rounds=10, restart_previous_finest=True,
                 alpha_levels=None, fill_variance=False, pilot_new=None, alpha_max=None,
                 bias_levels=1, L_min=0):
    """MLMC to a root-mean-square error eps with the number of levels chosen as
    it runs: start on levels 0..L0, run ``run_to_rmse`` (variance share
    eps^2/2), and while the Richardson bias of the finest level exceeds the
    bias share eps/sqrt(2) and fewer than L_max + 1 levels are in use, add the
    next level (pilot samples, then the sample sizes of Eq. (3.6) again).

    fill_variance: when L_max is reached with a bias b between eps/sqrt(2) and
    eps, the mean-square error eps^2 = b^2 + variance can still be met by a
    smaller variance share: the sample sizes are recomputed for the variance
    target eps^2 - b^2 (var_share = 1 - (b/eps)^2, the general split of the
    MSE between bias and variance of the adaptive MLMC algorithm of Giles, of
    which Eq. (3.6)'s ratio 1/2 is one choice) and topped up; the bias is then
    re-estimated from the larger samples and the share recomputed, up to three
    times.  The result's var_share records the share used.

    make_runner(level, finest) builds the runner of a level.  Under MLMC-CES
    the finest level's fine field is not smoothed (§3.6), so a level that stops
    being the finest is rebuilt with make_runner(level, False) and sampled
    afresh (restart_previous_finest; the time of its discarded samples is kept
    in the cost).  Plain MLMC, whose levels do not depend on which is finest,
    passes restart_previous_finest=False.  Returns the MLMCResult of the final
    level set; its `seconds` include every discarded sample.

    pilot_new: pilot samples of a level added (or rebuilt) after the first
    L0 + 1 (default `pilot`): on fine levels Eq. (3.6) asks for few samples,
    and a large pilot there dominates the cost.  alpha_levels, alpha_max and
    bias_levels go to the bias estimate (``fit_alpha``, ``richardson_bias``).
    L_min: the bias test may end the level loop only once the finest level is
    at least L_min (the Richardson estimate assumes the asymptotic regime,
    which the coarse meshes MLMC-CES allows do not reach: below the coarsest
    mesh of plain MLMC, Eq. (3.7)-(3.8), E[Y_l] can be small by accident)."""
    if L0 < 0 or L_max < L0:
        raise ValueError("need 0 <= L0 <= L_max")
    runners = [make_runner(l, l == L0) for l in range(L0 + 1)]
    pilots = [pilot] * (L0 + 1)
    pnew = pilot if pilot_new is None else pilot_new
    discarded = 0.0
    kw = dict(alpha=alpha, max_rounds=max_rounds, ratio=ratio, alpha_levels=alpha_levels,
              alpha_max=alpha_max, bias_levels=bias_levels)
    while True:
        res = run_to_rmse(runners, eps, pilot=pilots, **kw)
        L = len(runners) - 1
        if (res.bias <= eps / math.sqrt(2.0) and L >= L_min) or L >= L_max:
            break
        if restart_previous_finest:
            discarded += runners[L].stats.seconds
            runners[L] = make_runner(L, False)
            pilots[L] = pnew
        runners.append(make_runner(L + 1, True))
        pilots.append(pnew)
    if fill_variance:
        for _ in range(3):
            if not eps / math.sqrt(2.0) < res.bias < eps:
                break
            share = 1.0 - (res.bias / eps) ** 2
            if share >= res.var_share * 0.999 and res.rmse <= eps:
                break
            res = run_to_rmse(runners, eps, pilot=pilots, var_share=share, **kw)
    res.seconds += discarded
    return res
