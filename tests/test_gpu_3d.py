"""GPU parity of the three-dimensional path (embedding, field, Darcy solve,
level estimate) against the oracle's d = 3 instance of the method."""
import math

import numpy as np
import pytest

from oracle import covariance as ocv
from oracle import darcy3d as od3
from oracle import embedding as oem
from oracle import field3d as of3
from tests.gpu_common import TOL32, lib, rel_err

pytestmark = pytest.mark.gpu

# QoI parity at the FP64 residual target rtol = 1e-12 (the GPU solution is the
# discrete solution to ~1e-11; both sides solve the same system for the same
# FP32 k, promoted exactly)
QOI_TOL = 1e-9

CASES3 = [
    # kind, nu, lam, sigma2, n, pad mode
    (ocv.MATERN, 0.5, 0.3, 1.0, 4, oem.PAD_DOUBLING),
    (ocv.MATERN, 0.5, 0.05, 1.0, 8, oem.PAD_SMOOTH),
    (ocv.MATERN, 1.5, 0.1, 1.0, 8, oem.PAD_DOUBLING),
    (ocv.SEP_EXP, 0.0, 0.1, 2.0, 8, oem.PAD_NONE),
    (ocv.MATERN, 2.5, 0.2, 1.0, 2, oem.PAD_DOUBLING),      # smallest grid
    (ocv.MATERN, 0.5, 0.1, 1.0, 16, oem.PAD_SMOOTH),       # 64^3 embedding
]


@pytest.fixture(scope="module")
def sce():
    return lib()


def _setup_both(sce, case, keep_f=-1, keep_c=-1):
    kind, nu, lam, s2, n, mode = case
    emb = sce.ce3_setup_embedding(kind, nu, lam, s2, n, pad_mode=mode, keep_fine=keep_f,
                                  keep_coarse=keep_c)
    oe = of3.setup_embedding3(kind, nu, lam, s2, n, mode)
    return emb, oe


def _fields(sce, emb, seed, level, first, count, coarse=True):
    import torch
    n = emb.n
    kf = torch.empty(count, n + 1, n + 1, n + 1, dtype=torch.float32, device="cuda")
    kc = (torch.empty(count, n // 2 + 1, n // 2 + 1, n // 2 + 1, dtype=torch.float32,
                      device="cuda") if coarse else None)
    sce.ce3_sample_batch(emb, seed, level, first, count, kf, kc)
    torch.cuda.synchronize()
    return kf.cpu().numpy(), (kc.cpu().numpy() if coarse else None)


# ------------------------------------------------------------------ embedding
@pytest.mark.parametrize("case", CASES3)
def test_embedding3_eigenvalues(sce, case):
    import torch
    emb, oe = _setup_both(sce, case)
    assert (emb.info.P, emb.info.J, emb.info.s) == (oe.P, oe.J, oe.P ** 3)
    lam = torch.empty(oe.P ** 3, dtype=torch.float64)
    sce.ce3_get_eigenvalues(emb, lam)
    got = lam.numpy().reshape(oe.P, oe.P, oe.P)
    assert np.max(np.abs(got - oe.Lam)) <= 1e-12 * oe.lambda_max
    assert abs(emb.info.lambda_min - oe.lambda_min) <= 1e-12 * oe.lambda_max
    assert emb.info.max_imag <= 1e-11 * oe.lambda_max


def test_embedding3_not_psd_reported(sce):
    with pytest.raises(sce.SceError) as ex:
        sce.ce3_setup_embedding(ocv.MATERN, 0.5, 0.5, 1.0, 8, pad_mode=oem.PAD_NONE)
    assert ex.value.status == sce.CE_ERR_NOT_PSD


@pytest.mark.parametrize("case", [CASES3[1], CASES3[3]])
def test_masks3_match(sce, case):
    """Masks equal the oracle's rule applied to the same eigenvalues (the
    device's, so that near-ties are decided on identical numbers)."""
    import torch
    emb0, oe = _setup_both(sce, case)
    s = oe.P ** 3
    lam = torch.empty(s, dtype=torch.float64)
    sce.ce3_get_eigenvalues(emb0, lam)
    L = lam.numpy().reshape(oe.P, oe.P, oe.P)
    r = math.isqrt(s)
    for keep_f, keep_c in [(s - r, s // 8 - r), (1000, 37), (sce.CE_KEEP_TAU_SQRT_S, -1)]:
        emb, _ = _setup_both(sce, case, keep_f, keep_c)
        for which, keep in ((0, keep_f), (1, keep_c)):
            k = s - r if keep == sce.CE_KEEP_TAU_SQRT_S else keep
            got = np.zeros(s, dtype=np.uint8)
            sce.ce3_get_mask(emb, which, got)
            assert np.array_equal(got.astype(bool), oem.smoothing_mask(L, k).ravel()), (which, k)


# ------------------------------------------------------------------ fields
@pytest.mark.parametrize("case", CASES3)
def test_fields3_plain(sce, case):
    emb, oe = _setup_both(sce, case)
    full = np.ones(oe.Lam.shape, dtype=bool)
    count, seed, level, first = 3, 11, 1, 5
    kf, kc = _fields(sce, emb, seed, level, first, count)
    for c in range(count):
        okf, okc = of3.sample_k3(oe, full, full, seed, level, first + c, 32)
        assert rel_err(kf[c], okf) < TOL32
        assert np.array_equal(kc[c], kf[c][::2, ::2, ::2])
        assert rel_err(kc[c], okc) < TOL32


@pytest.mark.parametrize("case", [CASES3[1], CASES3[3], CASES3[5]])
def test_fields3_smoothed(sce, case):
    emb0, oe = _setup_both(sce, case)
    s = oe.P ** 3
    r = math.isqrt(s)
    keep_f, keep_c = s - r, s // 8 - r
    emb, _ = _setup_both(sce, case, keep_f, keep_c)
    mf = np.zeros(s, dtype=np.uint8)
    mc = np.zeros(s, dtype=np.uint8)
    sce.ce3_get_mask(emb, 0, mf)
    sce.ce3_get_mask(emb, 1, mc)
    mf = mf.astype(bool).reshape(oe.Lam.shape)
    mc = mc.astype(bool).reshape(oe.Lam.shape)
    count, seed, level, first = 2, 2, 4, 0
    kf, kc = _fields(sce, emb, seed, level, first, count)
    for c in range(count):
        okf, okc = of3.sample_k3(oe, mf, mc, seed, level, first + c, 32)
        assert rel_err(kf[c], okf) < TOL32
        assert rel_err(kc[c], okc) < TOL32


def test_fields3_full_size_sampled(sce):
    """n = 64 with a 256^3 smooth-periodisation embedding (the finest level
    of the three-dimensional MLMC workload): one sample, all vertices."""
    case = (ocv.MATERN, 0.5, 0.1, 1.0, 64, oem.PAD_SMOOTH)
    emb, oe = _setup_both(sce, case)
    assert oe.P == 256
    full = np.ones(oe.Lam.shape, dtype=bool)
    kf, _ = _fields(sce, emb, 3, 3, 7, 1, coarse=False)
    okf, _ = of3.sample_k3(oe, full, None, 3, 3, 7, 32)
    assert rel_err(kf[0], okf) < TOL32


# ------------------------------------------------------------------ Darcy
def _solve3(sce, k_np, f=0.0, rtol=1e-12, maxit=1000, allow=False):
    import torch
    count, n = k_np.shape[0], k_np.shape[1] - 1
    k = torch.tensor(k_np, dtype=torch.float32, device="cuda")
    qoi = torch.empty(count, 3, dtype=torch.float64, device="cuda")
    iters = torch.empty(count, dtype=torch.int32, device="cuda")
    status = torch.empty(count, dtype=torch.int32, device="cuda")
    u = torch.empty(count, n + 1, n + 1, n + 1, dtype=torch.float64, device="cuda")
    rc = sce.darcy3_solve_batch(n, k, count, qoi, f=f, rtol=rtol, maxit=maxit, iters=iters,
                                status=status, u_out=u, allow_not_converged=allow)
    torch.cuda.synchronize()
    return rc, qoi.cpu().numpy(), iters.cpu().numpy(), status.cpu().numpy(), u.cpu().numpy()


def _oracle_k3(n, count, lam=0.2, sigma2=1.0, seed=0):
    oe = of3.setup_embedding3(ocv.MATERN, 0.5, lam, sigma2, n, oem.PAD_SMOOTH)
    full = np.ones(oe.Lam.shape, dtype=bool)
    ks = [of3.sample_k3(oe, full, None, seed, 0, i, 32)[0] for i in range(count)]
    return np.array(ks).astype(np.float32)


@pytest.mark.parametrize("n", [2, 4, 8, 16])
def test_darcy3_constant_k_closed_forms(sce, n):
    k = np.full((2, n + 1, n + 1, n + 1), 2.0, dtype=np.float32)
    x = np.arange(n + 1) / n
    rc, q, it, stt, u = _solve3(sce, k, f=0.0)
    assert rc == 0 and np.all(stt == 0)
    assert np.max(np.abs(u - (1 - x)[None, None, None, :])) < 1e-11
    assert np.max(np.abs(q - [2.0, 8.0 / 15.0, 1 / math.sqrt(3)])) < 1e-11
    rc, q, it, stt, u = _solve3(sce, k, f=1.0)
    exact = 1 - x + x * (1 - x) / 4.0
    assert np.max(np.abs(u - exact[None, None, None, :])) < 1e-11
    assert np.max(np.abs(q[:, 0] - 2.5)) < 1e-11


@pytest.mark.parametrize("n,count,f", [(4, 3, 0.0), (8, 2, 1.0), (16, 2, 1.0)])
def test_darcy3_random_fields_against_oracle(sce, n, count, f):
    k = _oracle_k3(n, count, seed=n)
    rc, q, it, stt, u = _solve3(sce, k, f=f)
    assert rc == 0 and np.all(stt == 0), (it, stt)
    for c in range(count):
        ou, (A, F, M) = od3.solve3(k[c].astype(np.float64), f)
        oq = od3.qois3(ou, A, F, M)
        assert np.max(np.abs(u[c] - ou)) < QOI_TOL
        assert np.max(np.abs(q[c] - oq) / np.maximum(np.abs(oq), 1e-3)) < QOI_TOL, (q[c], oq)


def test_darcy3_full_size_residual(sce):
    """n = 64 (274625 vertices): the returned u satisfies the oracle's
    assembled equations to the requested relative residual, and the QoIs are
    the oracle's functionals of that u."""
    n = 64
    k = _oracle_k3(n, 1, lam=0.1, seed=4)
    rc, q, it, stt, u = _solve3(sce, k, f=1.0, rtol=1e-10)
    assert rc == 0
    A, F, M = od3.assemble3(k[0].astype(np.float64), 1.0)
    left, right = od3.dirichlet_nodes3(n)
    free = np.ones(A.shape[0], dtype=bool)
    free[left] = False
    free[right] = False
    uf = u[0].ravel()
    u0 = np.zeros_like(uf)
    u0[left] = 1.0
    r = (F - A @ uf)[free]
    r0 = (F - A @ u0)[free]
    assert np.linalg.norm(r) <= 2e-10 * np.linalg.norm(r0)
    assert np.array_equal(uf[left], np.ones(left.size)) and not uf[right].any()
    oq = od3.qois3(u[0], A, F, M)
    assert np.max(np.abs(q[0] - oq) / np.abs(oq)) < 1e-12


def test_darcy3_results_independent_of_batch(sce):
    k = _oracle_k3(8, 4, seed=21)
    _, qa, ita, _, _ = _solve3(sce, k, f=1.0, rtol=1e-10)
    for c in range(4):
        _, qc, itc, _, _ = _solve3(sce, k[c:c + 1], f=1.0, rtol=1e-10)
        assert np.array_equal(qc[0], qa[c]) and itc[0] == ita[c]


def test_darcy3_not_converged_status(sce):
    k = _oracle_k3(16, 2, seed=9)
    rc, q, it, stt, u = _solve3(sce, k, f=1.0, rtol=1e-12, maxit=2, allow=True)
    assert rc == sce.CE_ERR_NOT_CONVERGED
    assert np.all(stt == sce.CE_ERR_NOT_CONVERGED)


# ------------------------------------------------------------------ level estimate
@pytest.mark.parametrize("level,smooth", [(0, False), (1, False), (2, True)])
def test_mlmc3_level_estimate_against_oracle(sce, level, smooth):
    import torch
    n, count, seed, first = 8, 5, 7, 3
    case = (ocv.MATERN, 0.5, 0.1, 1.0, n, oem.PAD_SMOOTH)
    emb0, oe = _setup_both(sce, case)
    s = oe.P ** 3
    r = math.isqrt(s)
    kf_keep, kc_keep = (s - r, s // 8 - r) if smooth else (-1, -1)
    emb, _ = _setup_both(sce, case, kf_keep, kc_keep)
    Y = torch.empty(count, dtype=torch.float64, device="cuda")
    out, st = sce.mlmc3_level_estimate(emb, seed, level, first, count, qoi_index=0, f=1.0,
                                       rtol=1e-12, Y=Y)
    assert st == 0 and out.N == count and out.n_failed == 0
    mf = np.zeros(s, dtype=np.uint8)
    mc = np.zeros(s, dtype=np.uint8)
    sce.ce3_get_mask(emb, 0, mf)
    sce.ce3_get_mask(emb, 1, mc)
    mf = mf.astype(bool).reshape(oe.Lam.shape)
    mc = mc.astype(bool).reshape(oe.Lam.shape)
    kfs, kcs = _fields(sce, emb, seed, level, first, count, coarse=level > 0)
    want = []
    for c in range(count):
        okf, okc = of3.sample_k3(oe, mf, mc if level > 0 else None, seed, level, first + c, 32)
        assert rel_err(kfs[c], okf) < TOL32
        # the QoIs of the device's own FP32 fields, solved by the oracle
        qf = od3.solve_qois3(kfs[c].astype(np.float64), 1.0)[0]
        qc = od3.solve_qois3(kcs[c].astype(np.float64), 1.0)[0] if level > 0 else 0.0
        want.append(qf - qc)
    got = Y.cpu().numpy()
    assert np.max(np.abs(got - np.array(want))) < QOI_TOL
    assert abs(out.sumY - got.sum()) < 1e-12 * max(1.0, abs(got).sum())


def test_mlmc3_estimate_levels_concurrent_matches_serial(sce):
    """All levels in one call, levels in flight together on their own streams,
    give the level sums and Y of one level-by-level call each, bit for bit."""
    import torch
    ns, counts, seed = (4, 8, 16), (9, 5, 3), 13
    embs = [sce.ce3_setup_embedding(ocv.MATERN, 0.5, 0.1, 1.0, n, pad_mode=oem.PAD_SMOOTH,
                                    keep_fine=-1 if l == len(ns) - 1 else sce.CE_KEEP_TAU_SQRT_S,
                                    keep_coarse=sce.CE_KEEP_TAU_SQRT_S)
            for l, n in enumerate(ns)]
    ser = []
    for l, (e, c) in enumerate(zip(embs, counts)):
        Y = torch.empty(c, dtype=torch.float64, device="cuda")
        o, _ = sce.mlmc3_level_estimate(e, seed, l, 2 * c, c, qoi_index=1, f=1.0, rtol=1e-10, Y=Y)
        ser.append((o, Y.cpu().numpy()))
    Ys = [torch.empty(c, dtype=torch.float64, device="cuda") for c in counts]
    tasks = [{"emb": e, "level": l, "first_sample": 2 * c, "count": c, "Y": Y}
             for l, (e, c, Y) in enumerate(zip(embs, counts, Ys))]
    sums, stats, st = sce.mlmc3_estimate_levels(tasks, seed, qoi_index=1, f=1.0, rtol=1e-10,
                                                max_concurrency=3)
    torch.cuda.synchronize()
    assert st == 0 and all(s == 0 for s in stats)
    for (o, y), s, Y in zip(ser, sums, Ys):
        assert np.array_equal(Y.cpu().numpy(), y)
        assert (s.N, s.sumY, s.sumY2, s.sumQf, s.sumQf2) == (o.N, o.sumY, o.sumY2, o.sumQf, o.sumQf2)
        assert (s.max_iters, s.total_iters) == (o.max_iters, o.total_iters)


def test_three_dimensional_empty_batches_and_bad_sizes(sce):
    """count = 0 is a no-op for every 3D entry point; a problem whose n does
    not match the handle is refused."""
    import ctypes
    import torch
    emb = sce.ce3_setup_embedding(ocv.MATERN, 0.5, 0.2, 1.0, 4, pad_mode=oem.PAD_DOUBLING)
    k = torch.empty(1, dtype=torch.float32, device="cuda")
    q = torch.empty(3, dtype=torch.float64, device="cuda")
    sce.ce3_sample_batch(emb, 1, 0, 0, 0, k, None)
    assert sce.darcy3_solve_batch(4, k, 0, q) == 0
    out, st = sce.mlmc3_level_estimate(emb, 1, 1, 0, 0)
    assert st == 0 and out.N == 0
    sums, stats, st = sce.mlmc3_estimate_levels([], 1)
    assert st == 0 and sums == []
    bad = sce.darcy_problem(8, 1.0, 1e-10, 100, 32)          # handle has n = 4
    o = sce.mlmc_level_sums()
    assert sce.load().mlmc3_level_estimate(emb.handle, ctypes.byref(bad), 1, 0, 0, 2, 0,
                                           ctypes.byref(o), None, None) == sce.CE_ERR_INVALID_ARG
