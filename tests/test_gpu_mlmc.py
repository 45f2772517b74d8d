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
