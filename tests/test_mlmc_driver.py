"""Host logic of the MLMC driver (Eq. (3.5), (3.6) and the §4 bias and rate
estimates) with a synthetic level sampler standing in for the GPU."""
import math

import numpy as np
import pytest

from oracle import mlmc as omlmc


class FakeRunner:
    """Level l draws Y ~ N(mu_l, V_l) at cost C_l seconds per sample."""

    def __init__(self, level, mu, V, C, rng):
        from paper_2306_13493_gb300.mlmc import LevelStats
        self.stats = LevelStats(level=level, n=16 << level)
        self.mu, self.V, self.C, self.rng = mu, V, C, rng

    def run(self, count):
        y = self.rng.normal(self.mu, math.sqrt(self.V), count)
        st = self.stats
        st.N += count
        st.sumY += float(y.sum())
        st.sumY2 += float((y * y).sum())
        st.seconds += self.C * count
        st.next_sample += count
        return st


@pytest.fixture(scope="module")
def drv():
    from paper_2306_13493_gb300 import build, sce
    build.build_library()
    sce.load()
    from paper_2306_13493_gb300 import mlmc
    return mlmc


def test_rate_fits_recover_power_laws(drv):
    lv = np.arange(1, 6)
    assert abs(drv.fit_rate(lv, 3.0 * 2.0 ** (-1.3 * lv)) - 1.3) < 1e-12
    stats = []
    for l in range(0, 6):
        s = drv.LevelStats(level=l, n=16 << l, N=10)
        mean, var, cost = 0.5 * 2.0 ** (-1.0 * l), 0.1 * 2.0 ** (-1.9 * l), 1e-6 * 2.0 ** (1.87 * l)
        s.sumY = mean * s.N
        s.sumY2 = var * (s.N - 1) + s.N * mean * mean
        s.seconds = cost * s.N
        stats.append(s)
    a, b, g = drv.rates(stats)
    assert abs(a - 1.0) < 1e-9 and abs(b - 1.9) < 1e-9 and abs(g - 1.87) < 1e-9
    # §4 Richardson: |E Y_L| / (2^alpha - 1)
    assert abs(drv.richardson_bias(stats, a) - 0.5 * 2.0 ** -5 / (2.0 - 1.0)) < 1e-15


def test_run_to_rmse_meets_variance_target(drv):
    rng = np.random.default_rng(7)
    V = [1e-3, 2e-4, 5e-5, 1.2e-5]
    C = [1e-6, 4e-6, 1.6e-5, 6.4e-5]
    runners = [FakeRunner(l, 0.0, V[l], C[l], rng) for l in range(4)]
    eps = 2e-3
    res = drv.run_to_rmse(runners, eps, pilot=[200] * 4, alpha=1.0)
    # Eq. (3.6) with the true V, C: the sampled N must be close to it
    want = omlmc.optimal_samples(V, C, eps)
    got = np.array([r.stats.N for r in runners])
    assert np.all(got >= 0.7 * want) and np.all(got <= 1.5 * want + 200)
    assert res.stat_error <= eps / math.sqrt(2.0) * 1.15
    assert abs(res.estimate - sum(r.stats.mean for r in runners)) < 1e-15


class FakeSubmitRunner(FakeRunner):
    """FakeRunner with the submit/collect split of a served level."""

    def __init__(self, *a):
        super().__init__(*a)
        self.in_flight = 0

    def submit(self, count):
        self.in_flight += 1
        return count

    def collect(self, count):
        self.in_flight -= 1
        return FakeRunner.run(self, count)


def test_levels_in_flight_give_the_same_run(drv):
    """run_to_rmse with runners that submit ahead (all levels in flight, then
    collected in level order) reproduces the level-by-level run exactly."""
    V = [1e-3, 2e-4, 5e-5, 1.2e-5]
    C = [1e-6, 4e-6, 1.6e-5, 6.4e-5]
    out = []
    for cls in (FakeRunner, FakeSubmitRunner):
        rng = np.random.default_rng(11)
        runners = [cls(l, 0.0, V[l], C[l], rng) for l in range(4)]
        res = drv.run_to_rmse(runners, 2e-3, pilot=[200] * 4, alpha=1.0)
        out.append((res.estimate, res.stat_error, [r.stats.N for r in runners]))
        if cls is FakeSubmitRunner:
            assert all(r.in_flight == 0 for r in runners)
    assert out[0] == out[1]


def test_richardson_bias_with_smoothing(drv):
    """§4: with |E[Q_h - Q]| = C h^a and |E[Q~_2h - Q]| = C~ (2h)^a (same sign),
    E[Q_h - Q~_2h] = h^a (C - C~ 2^a), and the smoothed Richardson estimate
    with ratio C~/C recovers C h^a exactly; ratio 1 is the plain estimate.
    The oracle's form agrees."""
    for a in (0.7, 1.0, 1.9):
        for C, Ct in ((0.3, 0.3), (0.3, 0.25), (0.2, 0.05), (0.1, 0.4)):
            h = 2.0 ** -5
            s = drv.LevelStats(level=5, n=512, N=4)
            s.sumY = s.N * h ** a * (C - Ct * 2.0 ** a)
            got = drv.richardson_bias([s], a, Ct / C)
            assert got == pytest.approx(C * h ** a, rel=1e-12)
            assert got == pytest.approx(omlmc.richardson_bias(s.mean, a, Ct / C), rel=1e-15)
    s = drv.LevelStats(level=1, n=32, N=1, sumY=1.0)
    assert drv.richardson_bias([s], 1.0, 0.5) == math.inf


def test_run_adaptive_adds_levels_until_the_bias_test_passes(drv):
    """Level l has E[Y_l] = 0.08 2^-l, so the Richardson bias of a finest level
    L is 0.08 2^-L; with eps = 0.006 the test (bias <= eps/sqrt(2)) first
    passes at L = 5.  Every level that stops being the finest is rebuilt and
    its discarded samples' time is kept in the cost."""
    rng = np.random.default_rng(3)
    made, all_runners = [], []

    def make_runner(level, finest):
        made.append((level, finest))
        r = FakeRunner(level, 0.08 * 2.0 ** -level, 1e-6 * 4.0 ** -level, 1e-6 * 4.0 ** level, rng)
        r.finest = finest
        all_runners.append(r)
        return r

    eps = 0.006
    res = drv.run_adaptive(make_runner, eps, L0=2, L_max=8, pilot=100)
    assert len(res.levels) == 6 and [s.level for s in res.levels] == list(range(6))
    assert made == [(0, False), (1, False), (2, True), (2, False), (3, True), (3, False),
                    (4, True), (4, False), (5, True)]
    assert res.bias <= eps / math.sqrt(2.0) and res.bias == pytest.approx(0.08 / 32, rel=0.02)
    assert res.seconds == pytest.approx(sum(r.stats.seconds for r in all_runners), rel=1e-12)
    # stopping at L_max even when the test fails
    res2 = drv.run_adaptive(make_runner, eps, L0=1, L_max=3, pilot=100)
    assert len(res2.levels) == 4 and res2.bias > eps / math.sqrt(2.0)
    # plain MLMC: no rebuilds
    made.clear()
    drv.run_adaptive(make_runner, eps, L0=2, L_max=8, pilot=100, restart_previous_finest=False)
    assert [l for l, _ in made] == [0, 1, 2, 3, 4, 5]
    with pytest.raises(ValueError):
        drv.run_adaptive(make_runner, eps, L0=3, L_max=2)


def test_cost_versus_eps(drv):
    """Multilevel cost = sum N_l C_l with N_l of Eq. (3.6) (the oracle's rule);
    plain MC = ceil(2 eps^-2 V[Q_L]) samples at the finest level's cost; with
    V_l falling faster than C_l grows, the multilevel cost scales as eps^-2
    and MC's ratio to it grows as the finest level's variance share does."""
    V = [1e-3, 2e-4, 5e-5, 1.2e-5]
    C = [1e-6, 4e-6, 1.6e-5, 6.4e-5]
    vq = 2.5e-3
    stats = []
    for l in range(4):
        s = drv.LevelStats(level=l, n=16 << l, N=1000)
        s.sumY, s.sumY2 = 0.0, V[l] * (s.N - 1)
        s.sumQ, s.sumQ2 = 0.0, vq * (s.N - 1)
        s.seconds = C[l] * s.N
        stats.append(s)
    eps_list = [1e-2, 1e-3]
    out = drv.cost_versus_eps(stats, eps_list)
    for e, c in zip(eps_list, out):
        N = omlmc.optimal_samples(V, C, e)
        assert c["N"] == list(N)
        assert c["mlmc_seconds"] == pytest.approx(float(np.dot(N, C)), rel=1e-12)
        assert c["mc_N"] == math.ceil(2.0 * vq / e ** 2)
        assert c["mc_seconds"] == pytest.approx(c["mc_N"] * C[-1], rel=1e-12)
    # eps^-2 scaling once the ceilings of Eq. (3.6) no longer matter
    far = drv.cost_versus_eps(stats, [1e-3, 1e-4])
    assert far[1]["mlmc_seconds"] / far[0]["mlmc_seconds"] == pytest.approx(100.0, rel=5e-3)
    assert out[0]["mc_seconds"] > out[0]["mlmc_seconds"]
    assert drv.cost_versus_eps(stats, [1e-3], mc_cost_per_sample=1.0)[0]["mc_seconds"] == \
        math.ceil(2.0 * vq / 1e-6)


def test_coarsest_cells_matches_the_paper_examples(golden_dir):
    from paper_2306_13493_gb300 import mlmc, sce
    import os
    with open(os.path.join(golden_dir, "coarsest_mesh_examples.txt")) as fh:
        rows = [l.split()[:4] for l in fh if l.strip() and not l.startswith("#")]
    for kind, nu, lam, k in rows:
        c = sce.CE_COV_SEP_EXP if kind == "sep_exp" else sce.CE_COV_MATERN
        assert mlmc.coarsest_cells(c, float(nu), float(lam)) == 2 ** int(k)
    assert mlmc.coarsest_cells(sce.CE_COV_SEP_EXP, 0.5, 0.25) == 4
    with pytest.raises(ValueError):
        mlmc.coarsest_cells(sce.CE_COV_MATERN, 0.0, 0.1)


def test_workloads_keep_the_stated_configurations():
    """The synthetic workloads keep the parameters their JSON `config` quotes
    (the paper-shaped oscillatory MLMC-CES step and the plain 33 x 33 case),
    and the CES keep counts drop tau = sqrt(s) = P except on the finest level's
    fine field."""
    import workloads as w
    o = w.OSCILLATORY
    assert (o.nu, o.lam, o.sigma2, o.n0) == (0.5, 0.02, 1.0, 16)
    assert o.N == [20000, 8000, 3000, 1000, 300, 100]
    assert [n for _, n, _ in o.levels] == [16, 32, 64, 128, 256, 512]
    assert o.pad_mode == 2 and o.smoothing and o.rtol == 1e-10
    p = w.PLAIN_SMALL
    assert (p.nu, p.lam, p.sigma2, p.n0, p.N, p.pad_mode, p.smoothing, p.qoi, p.f, p.seed) == \
        (0.5, 0.3, 1.0, 32, [256], 1, False, 0, 0.0, 0)
    assert w.keep_counts(64, finest=False, smoothing=True) == (64 * 64 - 64, 64 * 64 - 64)
    assert w.keep_counts(64, finest=True, smoothing=True) == (-1, 64 * 64 - 64)
    assert w.keep_counts(64, finest=True, smoothing=False) == (-1, -1)


def test_run_adaptive_fills_the_variance_share_when_the_levels_run_out(drv):
    """E[Y_l] = 0.08 2^-l and L_max = 4: the bias 0.005 exceeds eps/sqrt(2)
    for eps = 0.006, but is below eps, so the variance target becomes
    eps^2 - bias^2 (a smaller share than Eq. (3.6)'s 1/2) and the estimated
    total RMSE meets eps; without fill_variance it does not."""
    rng = np.random.default_rng(11)

    def make_runner(level, finest):
        return FakeRunner(level, 0.08 * 2.0 ** -level, 1e-2 * 16.0 ** -level,
                          1e-6 * 4.0 ** level, rng)

    eps = 0.006
    plain = drv.run_adaptive(make_runner, eps, L0=2, L_max=4, pilot=100, alpha=1.0)
    assert plain.var_share == 0.5 and plain.rmse > eps
    res = drv.run_adaptive(make_runner, eps, L0=2, L_max=4, pilot=100, alpha=1.0,
                           fill_variance=True)
    assert len(res.levels) == 5
    assert res.bias == pytest.approx(0.005, rel=0.05)
    assert res.var_share == pytest.approx(1.0 - (res.bias / eps) ** 2, rel=0.05)
    assert res.var_share < 0.5
    assert res.stat_error <= eps * math.sqrt(res.var_share) * 1.1
    assert res.rmse <= eps * 1.02
    assert sum(s.N for s in res.levels) > sum(s.N for s in plain.levels)


def test_alpha_from_the_finest_levels(drv):
    """Pre-asymptotic coarse levels (E[Y_1] small) spoil a fit over all
    levels; the fit over the three finest recovers the rate."""
    stats = []
    for l, m in zip(range(6), [0.6, 0.003, 0.016, 0.008, 0.004, 0.002]):
        s = drv.LevelStats(level=l, n=16 << l, N=10)
        s.sumY = m * s.N
        stats.append(s)
    assert abs(drv.fit_alpha(stats, 3) - 1.0) < 1e-12
    assert abs(drv.fit_alpha(stats) - 1.0) > 0.2


def test_robust_bias_and_alpha_cap(drv):
    """A finest level whose mean is accidentally small does not end the level
    loop under the three-level test: the bias is the largest of
    |E Y_(L-j)| 2^(-j alpha); alpha_max caps a fit through such a dip."""
    stats = []
    for l, m in zip(range(4), [0.6, 0.02, 0.012, 1e-6]):
        s = drv.LevelStats(level=l, n=4 << l, N=10)
        s.sumY = m * s.N
        stats.append(s)
    assert drv.richardson_bias(stats, 1.0) == pytest.approx(1e-6)
    assert drv.richardson_bias(stats, 1.0, levels=3) == pytest.approx(0.012 / 2)
    # level 0 (Q itself) never enters: levels 3, 2, 1 give 1e-6, 0.006, 0.005
    assert drv.richardson_bias(stats, 1.0, levels=5) == pytest.approx(0.006)
    assert drv.fit_alpha(stats, 3) > 5
    assert drv.fit_alpha(stats, 3, alpha_max=2.0) == 2.0


def test_cost_versus_eps_chooses_the_finest_level(drv):
    """With E[Y_l] = 0.08 2^-l (alpha = 1), eps = 0.01 needs the bias
    0.08 2^-L <= eps/sqrt(2), i.e. L = 4; eps = 0.004 needs L = 5 = the last
    level; a smaller eps falls back to the last level.  Plain MC runs on the
    chosen level's grid."""
    stats = []
    for l in range(6):
        s = drv.LevelStats(level=l, n=16 << l, N=100)
        mean, var, cost = 0.08 * 2.0 ** -l, 1e-3 * 4.0 ** -l, 1e-6 * 4.0 ** l
        s.sumY = mean * s.N
        s.sumY2 = var * (s.N - 1) + s.N * mean * mean
        s.sumQ2 = (1e-3 + 0.4) * s.N
        s.sumQ = math.sqrt(0.4) * s.N
        s.seconds = cost * s.N
        stats.append(s)
    out = drv.cost_versus_eps(stats, [0.01, 0.004, 1e-4], choose_levels=True, alpha=1.0)
    assert [o["L"] for o in out] == [4, 5, 5]
    assert len(out[0]["N"]) == 5 and len(out[1]["N"]) == 6
    assert out[0]["mc_seconds"] == pytest.approx(out[0]["mc_N"] * 1e-6 * 4.0 ** 4)
    assert [o["L"] for o in drv.cost_versus_eps(stats, [0.01])] == [5]


def test_run_adaptive_respects_the_minimum_finest_level(drv):
    """Levels whose means vanish by accident (pre-asymptotic) would end the
    loop at once; with L_min the loop goes on to at least L_min and the bias
    is then estimated in the asymptotic range."""
    rng = np.random.default_rng(2)
    means = [0.6, 1e-7, 1e-7, 0.004, 0.002, 0.001, 0.0005]

    def make_runner(level, finest):
        return FakeRunner(level, means[level], 1e-12, 1e-6 * 4.0 ** level, rng)

    eps = 2e-3
    early = drv.run_adaptive(make_runner, eps, L0=2, L_max=6, pilot=50, alpha=1.0,
                             bias_levels=1, restart_previous_finest=False)
    assert len(early.levels) == 3
    res = drv.run_adaptive(make_runner, eps, L0=2, L_max=6, pilot=50, alpha=1.0, bias_levels=1,
                           restart_previous_finest=False, L_min=5)
    assert len(res.levels) == 6 and res.bias == pytest.approx(0.001, rel=1e-3)


class CounterRunner:
    """Level l's sample i is a fixed function of (l, i) -- like the
    counter-based normals -- at cost C_l per sample; raises once `fail_at`
    run() calls have been made (an interruption)."""

    calls = 0
    fail_at = None

    def __init__(self, level):
        from paper_2306_13493_gb300.mlmc import LevelStats
        self.stats = LevelStats(level=level, n=16 << level)

    def run(self, count):
        if CounterRunner.fail_at is not None and CounterRunner.calls >= CounterRunner.fail_at:
            raise RuntimeError("interrupted")
        CounterRunner.calls += 1
        st = self.stats
        i = np.arange(st.next_sample, st.next_sample + count, dtype=np.float64)
        y = 0.05 * 2.0 ** -st.level + 0.02 * 2.0 ** (-st.level) * np.sin(1.7 * i + st.level)
        st.N += count
        st.sumY += float(y.sum())
        st.sumY2 += float((y * y).sum())
        st.sumQ += float(y.sum())
        st.sumQ2 += float((y * y).sum())
        st.seconds += 1e-6 * 4.0 ** st.level * count
        st.next_sample += count
        return st


def test_checkpoint_resume_continues_the_same_run(drv, tmp_path):
    """A run to an RMSE interrupted after its pilot and resumed from its
    checkpoint ends with exactly the level sums, sample counts and estimate
    of the uninterrupted run; the checkpoint file round-trips the state."""
    eps = 2e-3
    CounterRunner.calls, CounterRunner.fail_at = 0, None
    full = drv.run_to_rmse([CounterRunner(l) for l in range(4)], eps, pilot=[50] * 4, alpha=1.0)
    ck = str(tmp_path / "state.json")
    CounterRunner.calls, CounterRunner.fail_at = 0, 4       # dies in the first top-up round
    with pytest.raises(RuntimeError):
        drv.run_to_rmse([CounterRunner(l) for l in range(4)], eps, pilot=[50] * 4, alpha=1.0,
                        checkpoint=ck)
    stats, meta = drv.load_checkpoint(ck)
    assert [s.N for s in stats] == [50] * 4 and meta["eps"] == eps
    CounterRunner.calls, CounterRunner.fail_at = 0, None
    res = drv.run_to_rmse([CounterRunner(l) for l in range(4)], eps, pilot=[50] * 4, alpha=1.0,
                          checkpoint=ck)
    assert [s.N for s in res.levels] == [s.N for s in full.levels]
    assert [(s.sumY, s.sumY2, s.next_sample) for s in res.levels] == \
        [(s.sumY, s.sumY2, s.next_sample) for s in full.levels]
    assert res.estimate == full.estimate
    again, _ = drv.load_checkpoint(ck)
    assert [s.N for s in again] == [s.N for s in res.levels]
    with pytest.raises(ValueError):
        drv.resume_runners([CounterRunner(1)], again)
