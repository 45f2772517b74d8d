"""GPU parity of the field path (Algorithm 1 steps 1-3 and 4(a)-(f)) against the oracle."""
import numpy as np
import pytest

from oracle import covariance as ocv
from oracle import embedding as oem
from oracle import field as ofield
from oracle import rng as orng
from tests.gpu_common import TOL32, TOL64, lib, rel_err, torch_dtype

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sce():
    return lib()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("seed,level,first", [(0, 0, 0), (3, 5, 17), ((1 << 40) + 7, 2, (1 << 33) + 5)])
def test_normals_bit_exact(sce, precision, seed, level, first):
    import torch
    count, length = 3, 4 * 1000 + 4
    out = torch.empty(count * length, dtype=torch_dtype(precision), device="cuda")
    sce.ce_normals(seed, level, first, count, length, precision, out)
    got = out.cpu().numpy().reshape(count, length)
    for c in range(count):
        want = orng.normals(seed, level, first + c, length, precision)
        assert got[c].dtype == want.dtype
        bad = np.nonzero(got[c].view(np.uint64 if precision == 64 else np.uint32)
                         != want.view(np.uint64 if precision == 64 else np.uint32))[0]
        assert bad.size == 0, (c, bad[:5], got[c][bad[:5]], want[bad[:5]])


CASES = [
    # kind, nu, lam, sigma2, n, pad mode
    (ocv.MATERN, 0.5, 0.3, 1.0, 32, oem.PAD_DOUBLING),     # 33x33 grid, doubled to 128
    (ocv.MATERN, 0.5, 0.02, 1.0, 16, oem.PAD_SMOOTH),      # oscillatory, smooth periodisation
    (ocv.MATERN, 1.5, 0.05, 1.0, 64, oem.PAD_DOUBLING),
    (ocv.MATERN, 2.5, 0.1, 3.0, 8, oem.PAD_DOUBLING),
    (ocv.SEP_EXP, 0.0, 0.1, 1.0, 16, oem.PAD_NONE),
    (ocv.MATERN, 0.5, 0.3, 1.0, 4, oem.PAD_DOUBLING),      # smallest grid
]


def _setup_both(sce, case, keep_f=-1, keep_c=-1):
    kind, nu, lam, s2, n, mode = case
    emb = sce.ce_setup_embedding(kind, nu, lam, s2, n, pad_mode=mode, keep_fine=keep_f,
                                 keep_coarse=keep_c)
    oe = oem.setup_embedding(kind, nu, lam, s2, n, mode)
    return emb, oe


@pytest.mark.parametrize("case", CASES)
def test_embedding_eigenvalues(sce, case):
    import torch
    emb, oe = _setup_both(sce, case)
    assert (emb.info.P, emb.info.J) == (oe.P, oe.J)
    lam = torch.empty(oe.P * oe.P, dtype=torch.float64)
    sce.ce_get_eigenvalues(emb, lam)
    got = lam.numpy().reshape(oe.P, oe.P)
    assert np.max(np.abs(got - oe.Lam)) <= 1e-12 * oe.lambda_max
    assert abs(emb.info.lambda_max - oe.lambda_max) <= 1e-12 * oe.lambda_max
    assert abs(emb.info.lambda_min - oe.lambda_min) <= 1e-12 * oe.lambda_max
    assert emb.info.max_imag <= 1e-11 * oe.lambda_max


def test_not_psd_is_reported(sce):
    with pytest.raises(sce.SceError) as ex:
        sce.ce_setup_embedding(ocv.MATERN, 0.5, 0.3, 1.0, 32, pad_mode=oem.PAD_NONE)
    assert ex.value.status == sce.CE_ERR_NOT_PSD


def test_invalid_arguments(sce):
    for args in [(ocv.MATERN, 0.7, 0.3, 1.0, 32), (ocv.MATERN, 0.5, 0.3, 1.0, 24),
                 (ocv.MATERN, 0.5, -1.0, 1.0, 32)]:
        with pytest.raises(sce.SceError) as ex:
            sce.ce_setup_embedding(*args)
        assert ex.value.status == sce.CE_ERR_INVALID_ARG


@pytest.mark.parametrize("case", [CASES[0], CASES[1]])
def test_smoothing_masks_match(sce, case):
    emb0, oe = _setup_both(sce, case)
    s, P = oe.s, oe.P
    for keep_f, keep_c in [(s - P, s // 4 - P // 2), (1000, 37), (s // 2, -1)]:
        emb, _ = _setup_both(sce, case, keep_f, keep_c)
        for which, keep in ((0, keep_f), (1, keep_c)):
            got = np.zeros(s, dtype=np.uint8)
            sce.ce_get_mask(emb, which, got)
            want = oem.smoothing_mask(oe.Lam, keep).ravel()
            assert np.array_equal(got.astype(bool), want), (which, keep)
        assert emb.info.keep_eff_fine == oem.smoothing_mask(oe.Lam, keep_f).sum()


def _fields(sce, emb, precision, seed, level, first, count, coarse=True):
    import torch
    n = emb.n
    dt = torch_dtype(precision)
    kf = torch.empty(count, n + 1, n + 1, dtype=dt, device="cuda")
    kc = torch.empty(count, n // 2 + 1, n // 2 + 1, dtype=dt, device="cuda") if coarse else None
    sce.ce_sample_batch(emb, seed, level, first, count, precision, kf, kc)
    torch.cuda.synchronize()
    return kf.cpu().numpy(), (kc.cpu().numpy() if coarse else None)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("case", CASES)
def test_fields_plain(sce, case, precision):
    emb, oe = _setup_both(sce, case)
    full = np.ones(oe.Lam.shape, dtype=bool)
    count, seed, level, first = 5, 11, 1, 3        # ragged count, offset samples
    kf, kc = _fields(sce, emb, precision, seed, level, first, count)
    tol = TOL64 if precision == 64 else TOL32
    for c in range(count):
        okf, okc = ofield.sample_k(oe, full, full, seed, level, first + c, precision)
        assert rel_err(kf[c], okf) < tol
        assert rel_err(kc[c], okc) < tol
        assert np.array_equal(kc[c], kf[c][::2, ::2])


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[4]])
def test_fields_smoothed(sce, case, precision):
    emb0, oe = _setup_both(sce, case)
    s, P = oe.s, oe.P
    keep_f, keep_c = s - P, s // 4 - P // 2
    emb, _ = _setup_both(sce, case, keep_f, keep_c)
    mf = oem.smoothing_mask(oe.Lam, keep_f)
    mc = oem.smoothing_mask(oe.Lam, keep_c)
    count, seed, level, first = 3, 2, 4, 0
    kf, kc = _fields(sce, emb, precision, seed, level, first, count)
    tol = TOL64 if precision == 64 else TOL32
    for c in range(count):
        okf, okc = ofield.sample_k(oe, mf, mc, seed, level, first + c, precision)
        assert rel_err(kf[c], okf) < tol
        assert rel_err(kc[c], okc) < tol


@pytest.mark.parametrize("precision", [64, 32])
def test_fields_full_size_sampled(sce, precision):
    """n = 512 with a 2048 x 2048 smooth-periodisation embedding (the finest
    level of the oscillatory MLMC workload): two samples, all vertices."""
    case = (ocv.MATERN, 0.5, 0.02, 1.0, 512, oem.PAD_SMOOTH)
    emb, oe = _setup_both(sce, case)
    assert oe.P == 2048
    full = np.ones(oe.Lam.shape, dtype=bool)
    kf, _ = _fields(sce, emb, precision, 2, 5, 40, 2, coarse=False)
    tol = TOL64 if precision == 64 else TOL32
    for c in range(2):
        okf, _ = ofield.sample_k(oe, full, None, 2, 5, 40 + c, precision)
        assert rel_err(kf[c], okf) < tol


def test_concurrent_sampling_of_different_sizes():
    """Host threads sampling fields of very different embedding sizes at the
    same time (the situation of levels in flight together) all succeed and
    give the fields a single thread gives: the FFT kernels' shared-memory
    limit is only ever raised, so one thread cannot shrink it under another's
    launch."""
    import threading
    import torch
    from tests.gpu_common import lib
    sce = lib()
    sizes = [(16, 16), (64, 2), (256, 1)]
    embs = [sce.ce_setup_embedding(ocv.MATERN, 0.5, 0.05, 1.0, n, pad_mode=oem.PAD_SMOOTH)
            for n, _ in sizes]
    ref = []
    for e, (n, c) in zip(embs, sizes):
        k = torch.empty(c, n + 1, n + 1, dtype=torch.float32, device="cuda")
        sce.ce_sample_batch(e, 5, 0, 0, c, 32, k_fine=k)
        torch.cuda.synchronize()
        ref.append(k.clone())
    errors, bad = [], []

    def worker(i):
        e, (n, c) = embs[i], sizes[i]
        s = torch.cuda.Stream()
        k = torch.empty(c, n + 1, n + 1, dtype=torch.float32, device="cuda")
        try:
            for _ in range(40):
                sce.ce_sample_batch(e, 5, 0, 0, c, 32, k_fine=k, stream=s.cuda_stream)
            s.synchronize()
            if not torch.equal(k, ref[i]):
                bad.append(i)
        except Exception as exc:   # reported below
            errors.append(repr(exc))

    ts = [threading.Thread(target=worker, args=(i,)) for i in range(len(sizes))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    for e in embs:
        e.close()
    assert not errors, errors
    assert not bad


def test_fft_autotune_changes_time_not_fields():
    """ce_autotune_fft picks launch shapes for the row and column passes; the
    fields sampled before and after are bit-identical (plain and masked)."""
    import torch
    from tests.gpu_common import lib
    sce = lib()
    for n, kf, kc in ((32, -1, -1), (64, None, None)):
        emb = sce.ce_setup_embedding(ocv.MATERN, 0.5, 0.05, 1.0, n, pad_mode=oem.PAD_SMOOTH)
        if kf is None:   # distinct coarse mask: the masked row pass
            s, P = emb.info.s, emb.P
            emb.close()
            emb = sce.ce_setup_embedding(ocv.MATERN, 0.5, 0.05, 1.0, n, pad_mode=oem.PAD_SMOOTH,
                                         keep_fine=s - P, keep_coarse=s // 4)
        out = []
        for tune in (False, True):
            if tune:
                shapes = sce.ce_autotune_fft(emb, 32, count=8, reps=2)
                assert shapes["row"][0] >= 1 and shapes["col"][0] >= 1
            k = torch.empty(6, n + 1, n + 1, dtype=torch.float32, device="cuda")
            kc_t = torch.empty(6, n // 2 + 1, n // 2 + 1, dtype=torch.float32, device="cuda")
            sce.ce_sample_batch(emb, 3, 1, 10, 6, 32, k_fine=k, k_coarse=kc_t)
            torch.cuda.synchronize()
            out.append((k.clone(), kc_t.clone()))
        assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
        emb.close()


@pytest.mark.parametrize("n,pad,masked,count", [
    (4, oem.PAD_DOUBLING, False, 5),     # short lines: 64 or more lines per staged chunk
    (16, oem.PAD_SMOOTH, True, 37),      # ragged last chunk, coarse-masked pass
    (32, oem.PAD_DOUBLING, False, 3),    # plain coarse field taken from the fine pass
    (64, oem.PAD_SMOOTH, True, 9),
    (512, oem.PAD_SMOOTH, True, 2),      # P = 2048: one line per chunk
])
def test_staged_column_pass_bit_identical(monkeypatch, n, pad, masked, count):
    """The column pass with its lines staged by bulk copies (the default in
    FP32) gives the same bits as the per-block column kernel
    (SCE_COL_BULK=0), for every register budget it can be built for."""
    import torch
    from tests.gpu_common import lib
    sce = lib()
    emb = sce.ce_setup_embedding(ocv.MATERN, 0.5, 0.05, 1.0, n, pad_mode=pad)
    if masked:
        s, P = emb.info.s, emb.P
        emb.close()
        emb = sce.ce_setup_embedding(ocv.MATERN, 0.5, 0.05, 1.0, n, pad_mode=pad,
                                     keep_fine=s - P, keep_coarse=s // 4)
    out = {}
    for mode in ("0", "4", "5", "6"):
        if mode == "0":
            monkeypatch.setenv("SCE_COL_BULK", "0")
        else:
            monkeypatch.delenv("SCE_COL_BULK", raising=False)
            monkeypatch.setenv("SCE_COLB_MINB", mode)
        k = torch.full((count, n + 1, n + 1), -1.0, dtype=torch.float32, device="cuda")
        kc = torch.full((count, n // 2 + 1, n // 2 + 1), -1.0, dtype=torch.float32, device="cuda")
        sce.ce_sample_batch(emb, 11, 3, 1000, count, 32, k_fine=k, k_coarse=kc)
        torch.cuda.synchronize()
        out[mode] = (k.clone(), kc.clone())
    monkeypatch.delenv("SCE_COLB_MINB", raising=False)
    emb.close()
    k0, kc0 = out["0"]
    assert bool(torch.isfinite(k0).all()) and float(k0.min()) > 0.0
    assert bool(torch.isfinite(kc0).all()) and float(kc0.min()) > 0.0
    for mode in ("4", "5", "6"):
        assert torch.equal(out[mode][0], k0), mode
        assert torch.equal(out[mode][1], kc0), mode
