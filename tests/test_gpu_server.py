"""The request server (continuous batching of MLMC level requests): each
result is the same alone and in the mix, admission keeps the reserved
footprint within the budget, the embedding cache is reused."""
import numpy as np
import pytest

from tests.gpu_common import lib

pytestmark = pytest.mark.gpu

# a mix of grid sizes, levels, covariances and sample counts
MIX = [
    dict(nu=0.5, lam=0.05, sigma2=1.0, n=16, level=0, count=40),
    dict(nu=1.5, lam=0.05, sigma2=1.0, n=64, level=2, count=9),
    dict(nu=0.5, lam=0.03, sigma2=2.0, n=32, level=1, count=25, finest=1),
    dict(nu=0.5, lam=0.05, sigma2=1.0, n=128, level=3, count=4),
    dict(nu=1.5, lam=0.08, sigma2=0.5, n=16, level=0, count=70, qoi_index=0, f=0.0),
    dict(nu=0.5, lam=0.05, sigma2=1.0, n=64, level=2, count=12, first_sample=9),
    dict(nu=0.5, lam=0.02, sigma2=1.0, n=256, level=4, count=3, smoothing=0),
    dict(nu=1.5, lam=0.05, sigma2=1.0, n=32, level=1, count=17, qoi_index=2),
]


@pytest.fixture(scope="module")
def sce():
    return lib()


def _alone(sce, r):
    """mlmc_level_estimate on its own, with an embedding set up for this request."""
    import torch
    smooth = r.get("smoothing", 1)
    kf = (sce.CE_KEEP_ALL if r.get("finest", 0) else sce.CE_KEEP_TAU_SQRT_S) if smooth else -1
    kc = sce.CE_KEEP_TAU_SQRT_S if smooth else -1
    emb = sce.ce_setup_embedding(sce.CE_COV_MATERN, r["nu"], r["lam"], r["sigma2"], r["n"],
                                 pad_mode=sce.CE_PAD_SMOOTH, keep_fine=kf, keep_coarse=kc)
    Y = torch.empty(r["count"], dtype=torch.float64, device="cuda")
    out, st = sce.mlmc_level_estimate(emb, r.get("seed", 0), r["level"], r.get("first_sample", 0),
                                      r["count"], qoi_index=r.get("qoi_index", 1),
                                      f=r.get("f", 1.0), rtol=1e-10, maxit=2000, precision=32,
                                      Y=Y)
    emb.close()
    return out, st, Y


def test_each_result_is_the_same_alone_and_in_the_mix(sce):
    import torch
    alone = [_alone(sce, r) for r in MIX]
    with sce.Server(slots=4, precision=32, rtol=1e-10, maxit=2000) as srv:
        Ys = [torch.full((r["count"],), float("nan"), dtype=torch.float64, device="cuda")
              for r in MIX]
        tickets = [srv.submit({**r, "Y": Y}) for r, Y in zip(MIX, Ys)]
        res = [srv.wait(t) for t in tickets]
        stats = srv.stats()
    torch.cuda.synchronize()
    for (out, st, Y), r, Yg in zip(alone, res, Ys):
        assert r.status == st == 0
        s = r.sums
        assert (s.N, s.sumY, s.sumY2, s.sumQf, s.sumQf2) == (out.N, out.sumY, out.sumY2,
                                                            out.sumQf, out.sumQf2)
        assert s.total_iters == out.total_iters
        assert torch.equal(Yg, Y)
    # several requests were on the device at once
    assert stats["peak_in_flight"] >= 2
    assert stats["completed"] == len(MIX) and stats["queued"] == 0 and stats["reserved"] == 0
    # distinct (covariance, n, smoothing rule) keys
    keys = {(r["nu"], r["lam"], r["sigma2"], r["n"], r.get("smoothing", 1), r.get("finest", 0))
            for r in MIX}
    assert stats["cache_misses"] == len(keys)
    assert stats["cache_hits"] == len(MIX) - len(keys)


def test_admission_keeps_the_reserved_footprint_within_the_budget(sce):
    """With a budget below one request's footprint every request reserves the
    whole budget, so the requests run one at a time although 4 slots are free."""
    reqs = [dict(nu=0.5, lam=0.05, sigma2=1.0, n=64, level=1, count=20, first_sample=20 * i)
            for i in range(5)]
    with sce.Server(slots=4, hbm_budget=1 << 20) as srv:
        tickets = [srv.submit(r) for r in reqs]
        res = [srv.wait(t) for t in tickets]
        stats = srv.stats()
    assert all(r.status == 0 and r.footprint == 1 << 20 for r in res)
    iv = sorted((r.t_admit, r.t_done) for r in res)
    for (a0, d0), (a1, d1) in zip(iv, iv[1:]):
        assert a1 >= d0
    assert stats["peak_in_flight"] == 1 and stats["peak_reserved"] == 1 << 20
    # admitted in arrival order (the queue's head always fits)
    order = sorted(range(len(res)), key=lambda i: res[i].t_admit)
    assert order == list(range(len(res)))


def test_generous_budget_overlaps_and_footprints_are_bounded(sce):
    reqs = [dict(nu=0.5, lam=0.05, sigma2=1.0, n=128, level=2, count=8, first_sample=8 * i)
            for i in range(6)]
    with sce.Server(slots=3) as srv:
        tickets = [srv.submit(r) for r in reqs]
        res = [srv.wait(t) for t in tickets]
        stats = srv.stats()
    assert all(r.status == 0 for r in res)
    assert stats["peak_in_flight"] >= 2
    assert stats["peak_reserved"] <= stats["budget"]
    # the footprint bound covers at least the fields and the FP64 solution of the batch
    assert all(r.footprint >= 8 * 129 * 129 * (4 + 8) for r in res)


def test_wait_timeout_and_unknown_ticket(sce):
    with sce.Server(slots=1) as srv:
        t = srv.submit(dict(nu=0.5, lam=0.02, sigma2=1.0, n=512, level=5, count=20))
        assert srv.wait(t, timeout=0.0) is None        # still running
        r = srv.wait(t)
        assert r.status == 0 and r.sums.N == 20
        with pytest.raises(sce.SceError):
            srv.wait(t)                                  # retired
    with pytest.raises(sce.SceError):
        sce.Server(slots=0)


def test_tau_rule_equals_explicit_keep_counts(sce):
    """CE_KEEP_TAU_SQRT_S resolves to keep = s - P once the padding fixed P."""
    a = sce.ce_setup_embedding(sce.CE_COV_MATERN, 0.5, 0.05, 1.0, 32, pad_mode=sce.CE_PAD_SMOOTH,
                               keep_fine=sce.CE_KEEP_TAU_SQRT_S,
                               keep_coarse=sce.CE_KEEP_TAU_SQRT_S)
    P, s = a.info.P, a.info.s
    b = sce.ce_setup_embedding(sce.CE_COV_MATERN, 0.5, 0.05, 1.0, 32, pad_mode=sce.CE_PAD_SMOOTH,
                               keep_fine=s - P, keep_coarse=s - P)
    for which in (0, 1):
        ma, mb = np.zeros(s, np.uint8), np.zeros(s, np.uint8)
        sce.ce_get_mask(a, which, ma)
        sce.ce_get_mask(b, which, mb)
        assert np.array_equal(ma, mb)
    assert a.info.keep_eff_fine == b.info.keep_eff_fine <= s - P
    a.close()
    b.close()


def test_sliced_request_is_the_same_alone_and_in_the_mix(sce):
    """A request above slice_vertices runs as sample slices (at most two in
    flight, each finished slice queueing the next behind newer requests):
    its per-sample Y equals mlmc_level_estimate's, its sums equal the
    slice-order sum of the slices' own level estimates, and both are the
    same alone and among other requests."""
    import torch
    big = dict(nu=0.5, lam=0.05, sigma2=1.0, n=64, level=2, count=23, first_sample=5)
    per = (3 * 65 * 65) // (65 * 65)          # slice_vertices = 3 (n+1)^2: 3 samples a slice
    _, _, Y_ref = _alone(sce, big)
    want = np.zeros(5)
    for k0 in range(0, big["count"], per):
        out, st, _ = _alone(sce, {**big, "first_sample": big["first_sample"] + k0,
                                  "count": min(per, big["count"] - k0)})
        assert st == 0
        want += [out.N, out.sumY, out.sumY2, out.sumQf, out.sumQf2]
    got = []
    for mix in ([], MIX[:5]):
        with sce.Server(slots=3, precision=32, rtol=1e-10, maxit=2000,
                        slice_vertices=3 * 65 * 65) as srv:
            Y = torch.full((big["count"],), float("nan"), dtype=torch.float64, device="cuda")
            t = srv.submit({**big, "Y": Y})
            others = [srv.submit(r) for r in mix]
            r = srv.wait(t)
            for o in others:
                assert srv.wait(o).status == 0
            stats = srv.stats()
        torch.cuda.synchronize()
        assert r.status == 0 and stats["reserved"] == 0 and stats["queued"] == 0
        s = r.sums
        got.append(((s.N, s.sumY, s.sumY2, s.sumQf, s.sumQf2), Y.clone()))
        assert torch.equal(Y, Y_ref)
    assert got[0][0] == got[1][0] == tuple(want)


def test_injected_oom_fails_one_request_and_the_server_recovers(sce):
    """Host-side fault injection: the library's next allocation fails with
    CE_ERR_OOM inside a request's level estimate.  That request reports it,
    its reservation is released, and the following request (same embedding,
    now cached) is served and equals the result alone."""
    import torch
    r = dict(nu=0.5, lam=0.05, sigma2=1.0, n=64, level=2, count=6)
    out, st, Y_ref = _alone(sce, r)
    with sce.Server(slots=1, precision=32, rtol=1e-10, maxit=2000) as srv:
        assert srv.wait(srv.submit(r)).status == 0          # embedding now resident
        sce.sce_test_fail_allocs(1)
        try:
            bad = srv.wait(srv.submit(r))
        finally:
            sce.sce_test_fail_allocs(0)
        assert bad.status == sce.CE_ERR_OOM
        assert srv.stats()["reserved"] == 0
        Y = torch.full((r["count"],), float("nan"), dtype=torch.float64, device="cuda")
        good = srv.wait(srv.submit({**r, "Y": Y}))
        stats = srv.stats()
    torch.cuda.synchronize()
    assert good.status == 0 and torch.equal(Y, Y_ref)
    assert good.sums.sumY == out.sumY
    assert stats["completed"] == 3 and stats["reserved"] == 0
