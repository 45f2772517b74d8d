"""GPU parity of the quasi-Monte Carlo sampler (randomly shifted rank-1
lattice normals) against the oracle."""
import numpy as np
import pytest

from oracle import covariance as ocv
from oracle import embedding as oem
from oracle import mlmc as omlmc
from oracle import qmc as oqmc
from tests.gpu_common import TOL32, TOL64, lib, rel_err, torch_dtype

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sce():
    return lib()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("n,pad,keep", [(8, oem.PAD_DOUBLING, None), (16, oem.PAD_SMOOTH, "quarter")])
def test_lattice_fields_match_oracle(sce, n, pad, keep, precision):
    import torch
    N, a, seed, level = 64, 21, 9, 2
    oe = oem.setup_embedding(ocv.MATERN, 1.5, 0.1, 1.0, n, pad)
    s, P = oe.s, oe.P
    if keep is None:
        kf = kc = -1
        mf = mc = np.ones(oe.Lam.shape, dtype=bool)
    else:
        kf, kc = s - P, s // 4
        mf, mc = oem.smoothing_mask(oe.Lam, kf), oem.smoothing_mask(oe.Lam, kc)
    emb = sce.ce_setup_embedding(ocv.MATERN, 1.5, 0.1, 1.0, n, pad_mode=pad, keep_fine=kf,
                                 keep_coarse=kc)
    q = sce.QmcLattice(emb, N, a)
    dt = torch_dtype(precision)
    first, count, shift = 5, 7, 3
    k = torch.empty(count, n + 1, n + 1, dtype=dt, device="cuda")
    kcg = torch.empty(count, n // 2 + 1, n // 2 + 1, dtype=dt, device="cuda")
    sce.ce_sample_batch_qmc(q, seed, level, shift, first, count, precision, k_fine=k, k_coarse=kcg)
    torch.cuda.synchronize()
    tol = TOL64 if precision == 64 else TOL32
    for c in range(count):
        of, oc = oqmc.sample_k_qmc(oe, mf, mc, N, a, seed, level, shift, first + c)
        assert rel_err(np.log(k[c].double().cpu().numpy()), np.log(of)) < tol
        assert rel_err(np.log(kcg[c].double().cpu().numpy()), np.log(oc)) < tol
    q.close()
    emb.close()


def test_lattice_level_estimate_matches_oracle(sce):
    import torch
    n, N, a, seed, level, shift = 16, 32, 13, 4, 1, 6
    oe = oem.setup_embedding(ocv.MATERN, 0.5, 0.1, 1.0, n, oem.PAD_SMOOTH)
    full = np.ones(oe.Lam.shape, dtype=bool)
    emb = sce.ce_setup_embedding(ocv.MATERN, 0.5, 0.1, 1.0, n, pad_mode=oem.PAD_SMOOTH)
    q = sce.QmcLattice(emb, N, a)
    count, first = 9, 11
    Y = torch.empty(count, dtype=torch.float64, device="cuda")
    out, st = sce.mlmc_level_estimate_qmc(q, seed, level, shift, first, count, qoi_index=1, f=1.0,
                                          rtol=1e-12, precision=64, Y=Y)
    assert st == 0 and out.N == count
    from oracle import darcy as odarcy
    oY = []
    for i in range(first, first + count):
        kf, kc = oqmc.sample_k_qmc(oe, full, full, N, a, seed, level, shift, i)
        oY.append(odarcy.solve_qois(kf, 1.0)[1] - odarcy.solve_qois(kc, 1.0)[1])
    oY = np.array(oY)
    assert np.max(np.abs(Y.cpu().numpy() - oY)) < 1e-9
    q.close()
    emb.close()


def test_lattice_arguments_are_checked(sce):
    emb = sce.ce_setup_embedding(ocv.MATERN, 0.5, 0.1, 1.0, 8, pad_mode=oem.PAD_DOUBLING)
    for N, a in ((48, 5), (64, 6), (0, 5)):
        with pytest.raises(sce.SceError):
            sce.QmcLattice(emb, N, a)
    q = sce.QmcLattice(emb, 16, 5)
    import torch
    k = torch.empty(2, 9, 9, dtype=torch.float32, device="cuda")
    with pytest.raises(sce.SceError):        # points 15, 16: beyond N
        sce.ce_sample_batch_qmc(q, 1, 0, 0, 15, 2, 32, k_fine=k)
    q.close()
    emb.close()
