"""GPU parity of the batched Darcy solve (operator, multigrid-CG, QoIs) against the oracle."""
import math

import numpy as np
import pytest

from oracle import covariance as ocv
from oracle import darcy as odarcy
from oracle import embedding as oem
from oracle import field as ofield
from tests.gpu_common import lib, torch_dtype

pytestmark = pytest.mark.gpu

# QoI parity: the FP64 residual target rtol = 1e-12 makes the GPU solution the
# discrete solution to ~1e-11; both precisions solve the same discrete system
# for the k they are given (FP32 k is promoted exactly), so both compare at 1e-9.
QOI_TOL = 1e-9


@pytest.fixture(scope="module")
def sce():
    return lib()


def _solve(sce, k_np, precision, f=0.0, rtol=1e-12, maxit=1000, allow=False):
    import torch
    count, n = k_np.shape[0], k_np.shape[1] - 1
    k = torch.tensor(k_np, dtype=torch_dtype(precision), device="cuda")
    qoi = torch.empty(count, 3, dtype=torch.float64, device="cuda")
    iters = torch.empty(count, dtype=torch.int32, device="cuda")
    status = torch.empty(count, dtype=torch.int32, device="cuda")
    u = torch.empty(count, n + 1, n + 1, dtype=torch.float64, device="cuda")
    rc = sce.darcy_solve_batch(n, k, count, qoi, f=f, rtol=rtol, maxit=maxit, precision=precision,
                               iters=iters, status=status, u_out=u, allow_not_converged=allow)
    torch.cuda.synchronize()
    return rc, qoi.cpu().numpy(), iters.cpu().numpy(), status.cpu().numpy(), u.cpu().numpy()


def _oracle_k(n, count, nu=0.5, lam=0.1, sigma2=1.0, seed=0, precision=64):
    oe = oem.setup_embedding(ocv.MATERN, nu, lam, sigma2, n, oem.PAD_DOUBLING)
    full = np.ones(oe.Lam.shape, dtype=bool)
    ks = [ofield.sample_k(oe, full, None, seed, 0, i, precision)[0] for i in range(count)]
    ks = np.array(ks)
    return ks.astype(np.float32) if precision == 32 else ks


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("n", [4, 8, 32, 128])
def test_constant_k_closed_forms(sce, n, precision):
    k = np.ones((3, n + 1, n + 1))
    x = np.arange(n + 1) / n
    rc, q, it, stt, u = _solve(sce, k, precision, f=0.0)
    assert rc == 0 and np.all(stt == 0)
    assert np.max(np.abs(u - (1 - x)[None, None, :])) < 1e-11
    assert np.max(np.abs(q - [1.0, 8.0 / 15.0, 1 / math.sqrt(3)])) < 1e-11
    rc, q, it, stt, u = _solve(sce, k, precision, f=1.0)
    assert np.max(np.abs(u - (1 - x / 2 - x * x / 2)[None, None, :])) < 1e-11
    assert np.max(np.abs(q[:, 0] - 1.5)) < 1e-11


@pytest.mark.parametrize("precision", [64, 32])
def test_layered_k(sce, precision):
    n = 64
    ky = np.exp(np.sin(np.arange(n + 1) * 1.3))
    k = np.repeat(ky[:, None], n + 1, axis=1)[None].repeat(2, axis=0)
    if precision == 32:
        k = k.astype(np.float32)
        ky = k[0, :, 0].astype(np.float64)
    rc, q, it, stt, u = _solve(sce, k, precision)
    want = (1.0 / n) * (ky.sum() - 0.5 * ky[0] - 0.5 * ky[-1])
    assert np.max(np.abs(q[:, 0] - want)) < 1e-10 * want


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("n,count,lam,sigma2,f", [(16, 7, 0.1, 1.0, 0.0), (32, 3, 0.05, 1.0, 1.0),
                                                  (64, 2, 0.02, 3.0, 0.0), (8, 5, 0.3, 1.0, 1.0)])
def test_random_fields_against_oracle(sce, n, count, lam, sigma2, f, precision):
    k = _oracle_k(n, count, lam=lam, sigma2=sigma2, seed=n, precision=precision)
    rc, q, it, stt, u = _solve(sce, k, precision, f=f)
    assert rc == 0 and np.all(stt == 0), (it, stt)
    for c in range(count):
        ou, (A, F, M) = odarcy.solve(k[c].astype(np.float64), f)
        oq = odarcy.qois(ou, A, F, M)
        assert np.max(np.abs(u[c] - ou)) < QOI_TOL
        assert np.max(np.abs(q[c] - oq) / np.maximum(np.abs(oq), 1e-3)) < QOI_TOL, (q[c], oq)


def test_full_size_sampled_solve(sce):
    """n = 512 (263169 vertices), sigma^2 = 3 field: two samples, mixed precision."""
    k = _oracle_k(512, 2, nu=0.5, lam=0.02, sigma2=1.0, seed=1, precision=32)
    rc, q, it, stt, u = _solve(sce, k, 32, rtol=1e-11)
    assert rc == 0
    for c in range(2):
        oq = odarcy.solve_qois(k[c].astype(np.float64))
        assert np.max(np.abs(q[c] - oq) / np.abs(oq)) < 1e-8


def test_not_converged_status(sce):
    k = _oracle_k(32, 3, lam=0.05, seed=9)
    rc, q, it, stt, u = _solve(sce, k, 64, maxit=1, allow=True)
    assert rc == sce.CE_ERR_NOT_CONVERGED
    assert np.all(stt == sce.CE_ERR_NOT_CONVERGED)
    assert np.all(it <= 1)


@pytest.mark.parametrize("n", [4, 8, 16, 32, 64])
def test_block_per_sample_solver_matches_batched_and_oracle(sce, n, monkeypatch):
    """The one-block-per-sample solver (small grids) and the grid-wide batched
    solver solve the same discrete problem: both match the oracle."""
    k = _oracle_k(n, 5, lam=0.05, sigma2=2.0, seed=100 + n, precision=32)
    monkeypatch.setenv("SCE_SMALL_MAX_N", "64")
    rc1, q1, it1, st1, u1 = _solve(sce, k, 32, f=1.0)
    monkeypatch.setenv("SCE_SMALL_MAX_N", "0")
    rc2, q2, it2, st2, u2 = _solve(sce, k, 32, f=1.0)
    assert rc1 == 0 and rc2 == 0 and np.all(st1 == 0) and np.all(st2 == 0)
    for c in range(5):
        ou, (A, F, M) = odarcy.solve(k[c].astype(np.float64), 1.0)
        oq = odarcy.qois(ou, A, F, M)
        for q, u in ((q1, u1), (q2, u2)):
            assert np.max(np.abs(u[c] - ou)) < QOI_TOL
            assert np.max(np.abs(q[c] - oq) / np.maximum(np.abs(oq), 1e-3)) < QOI_TOL


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("n", [16, 64, 128, 256])
def test_fused_cycle_matches_level_by_level_cycle(sce, n, precision, monkeypatch):
    """The tiled down/up kernels + one-block tail apply the same V(1,1) cycle as
    the level-by-level kernels: same iteration counts (up to one, from rounding
    order) and QoIs equal to solver accuracy; both match the oracle."""
    k = _oracle_k(n, 3, lam=0.03, sigma2=2.0, seed=200 + n, precision=precision)
    monkeypatch.setenv("SCE_SMALL_MAX_N", "0")
    monkeypatch.setenv("SCE_MG_FUSED", "1")
    rc1, q1, it1, st1, u1 = _solve(sce, k, precision, f=1.0)
    monkeypatch.setenv("SCE_MG_FUSED", "0")
    rc2, q2, it2, st2, u2 = _solve(sce, k, precision, f=1.0)
    assert rc1 == 0 and rc2 == 0
    assert np.max(np.abs(it1.astype(int) - it2.astype(int))) <= 1, (it1, it2)
    assert np.max(np.abs(q1 - q2)) < 1e-10
    oq = odarcy.solve_qois(k[0].astype(np.float64), 1.0)
    assert np.max(np.abs(q1[0] - oq) / np.maximum(np.abs(oq), 1e-3)) < QOI_TOL


def test_results_independent_of_batch_composition(sce):
    """A sample's result is bit-identical alone and inside a larger batch."""
    k = _oracle_k(32, 6, lam=0.05, seed=4, precision=32)
    _, q_all, _, _, _ = _solve(sce, k, 32)
    _, q_one, _, _, _ = _solve(sce, k[3:4], 32)
    assert np.array_equal(q_all[3], q_one[0])


@pytest.mark.parametrize("precision,maxit", [(32, 1000), (64, 1000), (32, 6)])
def test_graph_replay_matches_stream_launches(sce, precision, maxit, monkeypatch):
    """On a created stream the inner CG iterations are replayed from a captured
    CUDA graph four at a time; per-sample results, iteration counts and
    statuses equal those of plain stream launches (SCE_GRAPHS=0), also when
    the iteration budget is not a multiple of four."""
    import torch
    n, count = 128, 5
    k_np = _oracle_k(n, count, lam=0.05, seed=4, precision=precision)
    out = []
    # the second graph solve takes over the first one's cached solver and graph
    for graphs in ("1", "1", "0"):
        monkeypatch.setenv("SCE_GRAPHS", graphs)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            k = torch.tensor(k_np, dtype=torch_dtype(precision), device="cuda")
            qoi = torch.empty(count, 3, dtype=torch.float64, device="cuda")
            iters = torch.empty(count, dtype=torch.int32, device="cuda")
            status = torch.empty(count, dtype=torch.int32, device="cuda")
            rc = sce.darcy_solve_batch(n, k, count, qoi, f=1.0, rtol=1e-12, maxit=maxit,
                                       precision=precision, iters=iters, status=status,
                                       stream=s.cuda_stream, allow_not_converged=True)
        s.synchronize()
        out.append((rc, qoi.cpu().numpy(), iters.cpu().numpy(), status.cpu().numpy()))
    sce.darcy_solver_cache_clear()
    (rc0, q0, i0, s0) = out[-1]
    for rc1, q1, i1, s1 in out[:-1]:
        assert rc1 == rc0
        assert np.array_equal(q1, q0) and np.array_equal(i1, i0) and np.array_equal(s1, s0)
        if maxit == 6:
            assert rc1 == sce.CE_ERR_NOT_CONVERGED and np.all(i1 <= 6)


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("graphs", ["0", "1"])
def test_folded_cg_scalars_match_reduction_launches(sce, precision, graphs, monkeypatch):
    """CG's alpha (SCE_CG_FOLD=1, the default) or alpha and beta (2) formed
    inside the CG kernels (every block sums the partials in the fixed order)
    against the separate reduction launches (0), on the tiled (n = 256) and
    the fused n = 64 V-cycle.  FP64: all three sum in FP64 in the same order,
    so QoIs, iteration counts and statuses agree bit for bit.  FP32: the
    folded scalars are formed in float-float and FP32 (the launches in FP64),
    so the solves take slightly different rounding paths to the same
    tolerance: QoIs within 10 rtol |Q|, iteration counts within one."""
    import torch
    for n in (256, 64):
        count = 3
        k_np = _oracle_k(n, count, lam=0.05, seed=9, precision=precision)
        out = []
        for fold in ("0", "1", "2"):
            monkeypatch.setenv("SCE_CG_FOLD", fold)
            monkeypatch.setenv("SCE_GRAPHS", graphs)
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                k = torch.tensor(k_np, dtype=torch_dtype(precision), device="cuda")
                qoi = torch.empty(count, 3, dtype=torch.float64, device="cuda")
                iters = torch.empty(count, dtype=torch.int32, device="cuda")
                status = torch.empty(count, dtype=torch.int32, device="cuda")
                rc = sce.darcy_solve_batch(n, k, count, qoi, f=1.0, rtol=1e-12,
                                           precision=precision, iters=iters, status=status,
                                           stream=s.cuda_stream)
            s.synchronize()
            sce.darcy_solver_cache_clear()
            out.append((rc, qoi.cpu().numpy(), iters.cpu().numpy(), status.cpu().numpy()))
        rc0, q0, i0, s0 = out[0]
        assert rc0 == 0 and np.all(s0 == 0)
        for rc1, q1, i1, s1 in out[1:]:
            assert rc1 == 0 and np.all(s1 == 0)
            if precision == 64:
                assert np.array_equal(q0, q1) and np.array_equal(i0, i1)
            else:
                assert np.max(np.abs(q0 - q1)) < 10 * 1e-12 * max(1.0, np.max(np.abs(q0)))
                assert np.max(np.abs(i0 - i1)) <= 1


def test_cached_graphs_give_the_same_mlmc_step(sce, monkeypatch):
    """Two all-levels MLMC calls with SCE_GRAPHS=1 (the second reusing every
    level's cached solver and graph) give the per-sample Y and level sums of
    plain stream launches bit for bit."""
    import torch
    import workloads
    w = workloads.OSCILLATORY
    embs = []
    for l, n in ((2, 64), (3, 128), (4, 256)):
        e0 = sce.ce_setup_embedding(0, w.nu, w.lam, w.sigma2, n, pad_mode=w.pad_mode)
        kf, kc = workloads.keep_counts(e0.P, l == 4, True)
        e0.close()
        embs.append((l, sce.ce_setup_embedding(0, w.nu, w.lam, w.sigma2, n, pad_mode=w.pad_mode,
                                               keep_fine=kf, keep_coarse=kc)))
    runs = []
    for graphs in ("1", "1", "0"):
        monkeypatch.setenv("SCE_GRAPHS", graphs)
        s = torch.cuda.Stream()
        tasks = [{"emb": e, "level": l, "first_sample": 4, "count": c,
                  "Y": torch.full((c,), float("nan"), dtype=torch.float64, device="cuda")}
                 for (l, e), c in zip(embs, (9, 5, 3))]
        sums, stats, st = sce.mlmc_estimate_levels(tasks, 3, qoi_index=1, f=1.0, rtol=1e-10,
                                                   precision=32, max_concurrency=3,
                                                   stream=s.cuda_stream)
        s.synchronize()
        assert st == 0
        runs.append(([t["Y"].clone() for t in tasks],
                     [(o.N, o.sumY, o.sumY2, o.sumQf, o.sumQf2, o.total_iters) for o in sums]))
    sce.darcy_solver_cache_clear()
    for Ys, sm in runs[:-1]:
        assert sm == runs[-1][1]
        assert all(torch.equal(a, b) for a, b in zip(Ys, runs[-1][0]))
    for _, e in embs:
        e.close()


@pytest.mark.parametrize("precision", [32, 64])
def test_tile_heights_give_the_same_solves(sce, precision, monkeypatch):
    """Every window height of the tiled multigrid kernels (16, 24, 32, 48
    rows) computes each vertex of a V-cycle identically; only the order in
    which the per-tile partial sums of r . z are added follows the tiling.
    The solutions and QoIs of a random field on n = 256 (tiled levels 256
    and 128, ragged tiles at the grid's edges) match the oracle's direct
    solve, and agree across heights to the accuracy of two solves stopped at
    rtol = 1e-12 on different rounding paths: QoIs within 10 rtol |Q|, u
    within 1e-10, iteration counts within one."""
    n, count = 256, 3
    k = _oracle_k(n, count, lam=0.05, seed=4, precision=precision)
    ref = None
    for h in (32, 16, 24, 48):
        monkeypatch.setenv("SCE_TILE_SH", str(h))
        rc, q, it, stt, u = _solve(sce, k, precision, f=1.0)
        assert rc == 0 and np.all(stt == 0)
        if ref is None:
            ref = (q, it, u)
            Q = np.array([odarcy.solve_qois(k[i].astype(np.float64), 1.0) for i in range(count)])
            assert np.max(np.abs(q - Q)) < QOI_TOL
        else:
            assert np.max(np.abs(q - ref[0])) < 10 * 1e-12 * max(1.0, np.max(np.abs(ref[0]))), h
            assert np.max(np.abs(it - ref[1])) <= 1, h
            assert np.max(np.abs(u - ref[2])) < 1e-10, h


def test_tile_autotuner_picks_a_height(sce, monkeypatch):
    monkeypatch.delenv("SCE_TILE_SH", raising=False)
    n, count = 128, 4
    k = _oracle_k(n, count, lam=0.05, seed=5, precision=32)
    before = _solve(sce, k, 32, f=1.0)
    h = sce.darcy_autotune_tiles(n, 32, count=64, reps=1)
    assert h in (16, 24, 32, 48, 64)
    after = _solve(sce, k, 32, f=1.0)
    # another window height: the same solve up to the stopping tolerance (rtol 1e-12)
    assert np.max(np.abs(before[1] - after[1])) < 10 * 1e-12 * max(1.0, np.max(np.abs(before[1])))
    assert np.max(np.abs(before[4] - after[4])) < 1e-10
    with pytest.raises(sce.SceError):
        sce.darcy_autotune_tiles(64, 32)


def test_small16_solver_sweeps(sce, monkeypatch):
    """The n = 16 one-block solver with V(2,2) (SCE_SMALL16_NU=2) against its
    V(1,1) default: both match the oracle's direct solves and agree to the
    stopping tolerance; V(2,2) takes fewer CG iterations in total."""
    n, count = 16, 24
    k = _oracle_k(n, count, lam=0.02, seed=12, precision=32)
    out = {}
    for nu in ("1", "2"):
        monkeypatch.setenv("SCE_SMALL16_NU", nu)
        out[nu] = _solve(sce, k, 32, f=1.0)
    monkeypatch.delenv("SCE_SMALL16_NU", raising=False)
    for nu in ("1", "2"):
        assert out[nu][0] == 0 and np.all(out[nu][3] == 0)
        for i in range(0, count, 5):
            u, _ = odarcy.solve(k[i].astype(np.float64), f=1.0)[:2]
            assert np.max(np.abs(out[nu][4][i] - u)) < 1e-8
    assert np.max(np.abs(out["1"][1] - out["2"][1])) < 10 * 1e-12 * max(1.0, np.max(np.abs(out["1"][1])))
    assert out["2"][2].sum() < out["1"][2].sum(), (out["1"][2], out["2"][2])


@pytest.mark.parametrize("n", [64, 128, 256, 512])
def test_coarse_level_sweeps_same_solution_fewer_iterations(sce, n, monkeypatch):
    """Three sweeps per side on the coarse levels of at most 128 cells of a
    grid of 128 cells or more (the default, SCE_MG_NU_COARSE) against two
    everywhere: both cycles are symmetric preconditioners, so the solves agree
    to the stopping tolerance and match the oracle; on the oscillatory field
    the stronger coarse cycle takes no more CG iterations in total.  n = 64:
    both settings give the same V(2,2) cycle; 128: the fused n = 64 cycle is a
    coarse level; 256, 512: tiled coarse levels with three sweeps too."""
    count = 4 if n <= 256 else 2
    k = _oracle_k(n, count, lam=0.02, seed=9, precision=32)
    out = {}
    for nu in ("2", "3"):
        monkeypatch.setenv("SCE_MG_NU_COARSE", nu)
        out[nu] = _solve(sce, k, 32, f=1.0)
    monkeypatch.delenv("SCE_MG_NU_COARSE", raising=False)
    for nu in ("2", "3"):
        assert out[nu][0] == 0 and np.all(out[nu][3] == 0)
    scale = max(1.0, np.max(np.abs(out["2"][1])))
    assert np.max(np.abs(out["2"][1] - out["3"][1])) < 10 * 1e-12 * scale
    assert np.max(np.abs(out["2"][4] - out["3"][4])) < 1e-10
    assert out["3"][2].sum() <= out["2"][2].sum(), (out["3"][2], out["2"][2])
    if n <= 128:
        for i in range(count):
            u, _ = odarcy.solve(k[i].astype(np.float64), f=1.0)[:2]
            assert np.max(np.abs(out["3"][4][i] - u)) < 1e-8


@pytest.mark.parametrize("n,small", [(32, "32"), (64, "64"), (64, "0"), (128, "0")])
def test_padded_shared_memory_rows_are_bit_identical(sce, n, small, monkeypatch):
    """Rows of n + 2 values for the shared-memory levels of at least 32 cells
    change addresses only: the fused n = 64 cycle (padded by default, against
    SCE_SMEM_PAD=0; as the finest level at n = 64, as a coarse level at
    n = 128) and the one-block solvers (n = 32, 64; padded with
    SCE_SMALL_PAD=1) give bit-identical solutions, QoIs and iteration counts."""
    monkeypatch.setenv("SCE_SMALL_MAX_N", small)
    k = _oracle_k(n, 5, lam=0.03, seed=21, precision=32)
    out = {}
    for pad in ("0", "1"):
        monkeypatch.setenv("SCE_SMEM_PAD", pad)
        monkeypatch.setenv("SCE_SMALL_PAD", pad)
        out[pad] = _solve(sce, k, 32, f=1.0)
    monkeypatch.delenv("SCE_SMALL_PAD", raising=False)
    assert out["1"][0] == 0 and np.all(out["1"][3] == 0)
    for i in (1, 2, 4):
        assert np.array_equal(out["0"][i], out["1"][i]), i
