"""GPU parity of one MLMC level (Algorithm 1 / 2 end to end) against the oracle."""
import numpy as np
import pytest

from oracle import covariance as ocv
from oracle import embedding as oem
from oracle import mlmc as omlmc
from tests.gpu_common import lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sce():
    return lib()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("level,smooth,finest,qi", [(0, False, True, 0), (1, False, True, 0),
                                                   (2, True, False, 1), (1, True, True, 2),
                                                   (3, "quarter", False, 1)])
def test_level_estimate_matches_oracle(sce, level, smooth, finest, qi, precision):
    """smooth = "quarter": a coarse field that keeps only s/4 - sqrt(s/4) of
    the level's eigenvalues (distinct fine and coarse masks on a non-finest
    level)."""
    import torch
    import workloads
    n = 16
    oe = oem.setup_embedding(ocv.MATERN, 0.5, 0.02, 1.0, n, oem.PAD_SMOOTH)
    s, P = oe.s, oe.P
    if smooth == "quarter":
        keep_f, keep_c = s - P, s // 4 - P // 2
        mf, mc = oem.smoothing_mask(oe.Lam, keep_f), oem.smoothing_mask(oe.Lam, keep_c)
    else:
        mf, mc = omlmc.default_masks(oe, smooth, finest)
        keep_f, keep_c = workloads.keep_counts(P, finest, smooth)
    emb = sce.ce_setup_embedding(ocv.MATERN, 0.5, 0.02, 1.0, n, pad_mode=oem.PAD_SMOOTH,
                                 keep_fine=keep_f, keep_coarse=keep_c)
    count, seed, first = 9, 2, 5
    Y = torch.empty(count, dtype=torch.float64, device="cuda")
    qf = torch.empty(count, 3, dtype=torch.float64, device="cuda")
    qc = torch.empty(count, 3, dtype=torch.float64, device="cuda")
    out, st = sce.mlmc_level_estimate(emb, seed, level, first, count, qoi_index=qi, f=1.0,
                                      rtol=1e-12, precision=precision, Y=Y, qoi_f=qf, qoi_c=qc)
    assert st == 0 and out.N == count and out.n_failed == 0
    (N, s1, s2, f1, f2), oY = omlmc.level_estimate(oe, mf, mc, seed, level, first, count,
                                                   qoi_index=qi, f=1.0, precision=precision)
    tol = 1e-9 if precision == 64 else 1e-5
    Yg = Y.cpu().numpy()
    scale = max(np.max(np.abs(oY)), 1e-3)
    assert np.max(np.abs(Yg - oY)) < tol * max(scale, 1.0)
    assert abs(out.sumQf - f1) < tol * abs(f1) * 1.0 + 1e-12
    assert abs(out.sumY - Yg.sum()) < 1e-12 * max(1.0, abs(out.sumY))
    assert abs(out.sumY2 - (Yg * Yg).sum()) < 1e-12 * max(1.0, out.sumY2)


def _level_setup(sce, levels, n0=8):
    import workloads
    embs = []
    L = max(levels)
    for l in levels:
        n = n0 << l
        e0 = sce.ce_setup_embedding(ocv.MATERN, 0.5, 0.05, 1.0, n, pad_mode=oem.PAD_SMOOTH)
        kf, kc = workloads.keep_counts(e0.P, l == L, True)
        e0.close()
        embs.append(sce.ce_setup_embedding(ocv.MATERN, 0.5, 0.05, 1.0, n,
                                           pad_mode=oem.PAD_SMOOTH, keep_fine=kf, keep_coarse=kc))
    return embs


@pytest.mark.parametrize("conc,chunk_vertices", [(4, None), (8, 700), (1, None)])
def test_estimate_levels_equals_level_by_level(sce, conc, chunk_vertices, monkeypatch):
    """All levels in one call (concurrent streams, coarse solves on their own
    stream, several chunks per level when chunk_vertices is small) give
    bit-identical Y and level sums to one mlmc_level_estimate per level."""
    import torch
    levels = [0, 1, 2, 3, 4]
    counts = [70, 40, 23, 9, 5]
    embs = _level_setup(sce, levels)
    if chunk_vertices is not None:
        monkeypatch.setenv("SCE_MLMC_CHUNK_VERTICES", str(chunk_vertices))
    ref, Yref = [], []
    for l, e, c in zip(levels, embs, counts):
        Y = torch.empty(c, dtype=torch.float64, device="cuda")
        qf = torch.empty(c, 3, dtype=torch.float64, device="cuda")
        out, st = sce.mlmc_level_estimate(e, 7, l, 100 + l, c, qoi_index=1, f=1.0, rtol=1e-10,
                                          precision=32, Y=Y, qoi_f=qf)
        assert st == 0
        ref.append(out)
        Yref.append((Y.clone(), qf.clone()))
    tasks = []
    for l, e, c in zip(levels, embs, counts):
        tasks.append({"emb": e, "level": l, "first_sample": 100 + l, "count": c,
                      "Y": torch.full((c,), float("nan"), dtype=torch.float64, device="cuda"),
                      "qoi_f": torch.full((c, 3), float("nan"), dtype=torch.float64,
                                          device="cuda")})
    sums, stats, st = sce.mlmc_estimate_levels(tasks, 7, qoi_index=1, f=1.0, rtol=1e-10,
                                               precision=32, max_concurrency=conc)
    torch.cuda.synchronize()
    assert st == 0 and stats == [0] * len(levels)
    for r, o, t, (Y, qf) in zip(ref, sums, tasks, Yref):
        assert (o.N, o.sumY, o.sumY2, o.sumQf, o.sumQf2) == (r.N, r.sumY, r.sumY2, r.sumQf, r.sumQf2)
        assert (o.n_failed, o.max_iters, o.total_iters) == (r.n_failed, r.max_iters, r.total_iters)
        assert torch.equal(t["Y"], Y) and torch.equal(t["qoi_f"], qf)
    for e in embs:
        e.close()


def test_estimate_levels_waits_for_the_callers_stream(sce):
    """Work queued on the caller's stream before the call (here: the writes
    of the first samples' index range into Y) is ordered before the levels'
    streams, and the caller's stream is ordered after them."""
    import torch
    embs = _level_setup(sce, [0, 1])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        Y0 = torch.zeros(30, dtype=torch.float64, device="cuda")
        Y1 = torch.zeros(20, dtype=torch.float64, device="cuda")
        torch.cuda._sleep(20_000_000)          # keep the stream busy before the call
        Y0.fill_(float("nan"))
        tasks = [{"emb": embs[0], "level": 0, "first_sample": 0, "count": 30, "Y": Y0},
                 {"emb": embs[1], "level": 1, "first_sample": 0, "count": 20, "Y": Y1}]
        sums, stats, st = sce.mlmc_estimate_levels(tasks, 3, qoi_index=1, f=1.0,
                                                   max_concurrency=2, stream=s.cuda_stream)
        tot = Y0.sum() + Y1.sum()               # queued after the call on the same stream
    s.synchronize()
    assert st == 0
    assert torch.isfinite(Y0).all() and torch.isfinite(Y1).all()
    assert abs(float(tot) - (sums[0].sumY + sums[1].sumY)) < 1e-9
    for e in embs:
        e.close()


# Levels of the oscillatory workload (Matern nu = 0.5, lambda = 0.02, smooth
# periodisation J = n, n_l = 16 * 2^l) whose fine solve is the batched
# multigrid-CG solver: levels 2 (n = 64) and 3 (n = 128).  By default the
# coarse solve runs first and the fine solve starts from its prolonged
# solution (nested iteration); SCE_NESTED=0 starts both from the lifting.
# The chunk bound splits the level into several chunks (2 samples each).
@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("nested", [True, False])
@pytest.mark.parametrize("level,finest", [(2, False), (3, True)])
def test_batched_level_estimate_matches_oracle(sce, level, finest, nested, precision,
                                               monkeypatch):
    """Algorithm 2 step 4 and Eq. (3.5) on the path the oscillatory MLMC step
    runs for n >= 64: per-sample Y against the oracle's direct solves, 1e-9
    (FP64) / 1e-5 (FP32 normals and field), and the level sums."""
    import torch
    import workloads
    w = workloads.OSCILLATORY
    n = w.n0 << level
    monkeypatch.setenv("SCE_MLMC_CHUNK_VERTICES", str(2 * (n + 1) * (n + 1)))
    monkeypatch.setenv("SCE_NESTED", "1" if nested else "0")
    oe = oem.setup_embedding(ocv.MATERN, w.nu, w.lam, w.sigma2, n, oem.PAD_SMOOTH)
    mf, mc = omlmc.default_masks(oe, True, finest)
    keep_f, keep_c = workloads.keep_counts(oe.P, finest, True)
    emb = sce.ce_setup_embedding(ocv.MATERN, w.nu, w.lam, w.sigma2, n, pad_mode=oem.PAD_SMOOTH,
                                 keep_fine=keep_f, keep_coarse=keep_c)
    assert emb.P == oe.P
    count, first = 5, 1 << 33
    Y = torch.full((count,), float("nan"), dtype=torch.float64, device="cuda")
    out, st = sce.mlmc_level_estimate(emb, w.seed, level, first, count, qoi_index=w.qoi,
                                      f=w.f, rtol=1e-12, precision=precision, Y=Y)
    torch.cuda.synchronize()
    emb.close()
    assert st == 0 and out.N == count and out.n_failed == 0
    (N, s1, s2, f1, f2), oY = omlmc.level_estimate(oe, mf, mc, w.seed, level, first, count,
                                                   qoi_index=w.qoi, f=w.f, precision=precision)
    tol = 1e-9 if precision == 64 else 1e-5
    Yg = Y.cpu().numpy()
    assert np.max(np.abs(Yg - oY)) < tol
    assert abs(out.sumY - s1) < tol * count
    assert abs(out.sumQf - f1) < tol * abs(f1)
    assert abs(out.sumQf2 - f2) < 2 * tol * abs(f2)
    assert abs(out.sumY - Yg.sum()) < 1e-12 * max(1.0, abs(out.sumY))
    assert abs(out.sumY2 - (Yg * Yg).sum()) < 1e-12 * max(1.0, out.sumY2)


# Level 1 of the oscillatory workload (n = 32 fine, 16 coarse): both solves
# run in the one-block solver; by default the fine one starts from the
# prolonged coarse solution (SCE_NESTED_SMALL=0: from the lifting).
def test_small_grid_level_estimate_nested_matches_oracle(sce, monkeypatch):
    """Algorithm 2 step 4 and Eq. (3.5) on the one-block path of the small
    levels: per-sample Y against the oracle at 1e-5, and the nested start never
    needs more CG iterations in total than the start from the lifting."""
    import torch
    import workloads
    w = workloads.OSCILLATORY
    level = 1
    n = w.n0 << level
    oe = oem.setup_embedding(ocv.MATERN, w.nu, w.lam, w.sigma2, n, oem.PAD_SMOOTH)
    mf, mc = omlmc.default_masks(oe, True, False)
    keep_f, keep_c = workloads.keep_counts(oe.P, False, True)
    emb = sce.ce_setup_embedding(ocv.MATERN, w.nu, w.lam, w.sigma2, n, pad_mode=oem.PAD_SMOOTH,
                                 keep_fine=keep_f, keep_coarse=keep_c)
    count, first = 23, 7
    outs = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("SCE_NESTED_SMALL", flag)
        Y = torch.full((count,), float("nan"), dtype=torch.float64, device="cuda")
        out, st = sce.mlmc_level_estimate(emb, w.seed, level, first, count, qoi_index=w.qoi,
                                          f=w.f, rtol=1e-12, precision=32, Y=Y)
        torch.cuda.synchronize()
        assert st == 0 and out.N == count and out.n_failed == 0
        outs[flag] = (out, Y.cpu().numpy())
    emb.close()
    (N, s1, s2, f1, f2), oY = omlmc.level_estimate(oe, mf, mc, w.seed, level, first, count,
                                                   qoi_index=w.qoi, f=w.f, precision=32)
    for out, Yg in outs.values():
        assert np.max(np.abs(Yg - oY)) < 1e-5
        assert abs(out.sumQf - f1) < 1e-5 * abs(f1)
    assert outs["1"][0].total_iters <= outs["0"][0].total_iters


@pytest.mark.parametrize("nested", [True, False])
def test_estimate_levels_batched_levels_match_oracle(sce, nested, monkeypatch):
    """The all-levels call on levels 2 and 3 of the oscillatory workload
    (concurrent streams, chunked, FP32 path): per-sample Y equals the
    oracle's to 1e-5."""
    import torch
    import workloads
    w = workloads.OSCILLATORY
    monkeypatch.setenv("SCE_NESTED", "1" if nested else "0")
    monkeypatch.setenv("SCE_MLMC_CHUNK_VERTICES", str(3 * 129 * 129))
    tasks, oracle_Y = [], []
    embs = []
    for level, count in ((2, 7), (3, 4)):
        n = w.n0 << level
        finest = level == 3
        oe = oem.setup_embedding(ocv.MATERN, w.nu, w.lam, w.sigma2, n, oem.PAD_SMOOTH)
        mf, mc = omlmc.default_masks(oe, True, finest)
        kf, kc = workloads.keep_counts(oe.P, finest, True)
        e = sce.ce_setup_embedding(ocv.MATERN, w.nu, w.lam, w.sigma2, n,
                                   pad_mode=oem.PAD_SMOOTH, keep_fine=kf, keep_coarse=kc)
        embs.append(e)
        first = 11 * level
        tasks.append({"emb": e, "level": level, "first_sample": first, "count": count,
                      "Y": torch.full((count,), float("nan"), dtype=torch.float64,
                                      device="cuda")})
        oracle_Y.append(omlmc.level_estimate(oe, mf, mc, w.seed, level, first, count,
                                             qoi_index=w.qoi, f=w.f, precision=32)[1])
    sums, stats, st = sce.mlmc_estimate_levels(tasks, w.seed, qoi_index=w.qoi, f=w.f,
                                               rtol=1e-12, precision=32, max_concurrency=2)
    torch.cuda.synchronize()
    assert st == 0 and stats == [0, 0]
    for t, oY, s in zip(tasks, oracle_Y, sums):
        Yg = t["Y"].cpu().numpy()
        assert np.max(np.abs(Yg - oY)) < 1e-5
        assert s.N == t["count"] and s.n_failed == 0
    for e in embs:
        e.close()


def test_level_runner_resumes_from_a_checkpoint(sce, tmp_path):
    """A LevelRunner that ran 40 then 25 samples, and one that ran 40, was
    checkpointed, and whose state a fresh runner took over for the other 25,
    hold the same level sums bit for bit (counter-based normals: the resumed
    runner draws samples 40..64)."""
    from paper_2306_13493_gb300 import mlmc as gm
    embs = _level_setup(sce, [0, 1])
    a = [gm.LevelRunner(embs[l], l, 9, qoi=1, f=1.0) for l in (0, 1)]
    for r in a:
        r.run(40)
        r.run(25)
    b = [gm.LevelRunner(embs[l], l, 9, qoi=1, f=1.0) for l in (0, 1)]
    for r in b:
        r.run(40)
    ck = str(tmp_path / "levels.json")
    gm.save_checkpoint(ck, b)
    c = gm.resume_runners([gm.LevelRunner(embs[l], l, 9, qoi=1, f=1.0) for l in (0, 1)],
                          gm.load_checkpoint(ck)[0])
    for r in c:
        r.run(25)
    for ra, rc in zip(a, c):
        assert (ra.stats.N, ra.stats.sumY, ra.stats.sumY2, ra.stats.sumQ, ra.stats.next_sample) == \
            (rc.stats.N, rc.stats.sumY, rc.stats.sumY2, rc.stats.sumQ, rc.stats.next_sample)
    for e in embs:
        e.close()
