"""ce_sample_levels: the fields of several levels in one persistent launch.

Its fields must equal those of one ce_sample_batch call per level bit for bit
(plain and smoothed embeddings, distinct coarse masks, ragged sample counts),
and a column block whose wait for its sample's row blocks cannot end must give
up after its bound and make the call return CE_ERR_TIMEOUT, leaving the device
usable."""
import pytest

from tests.gpu_common import lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sce():
    return lib()


def _levels(sce):
    import workloads
    w = workloads.OSCILLATORY
    out = []
    for level, n, count, smooth, finest in ((0, 16, 37, False, False), (1, 32, 21, True, False),
                                            (2, 64, 9, True, False), (3, 128, 5, True, True),
                                            (4, 256, 3, False, False)):
        e0 = sce.ce_setup_embedding(0, w.nu, w.lam, w.sigma2, n, pad_mode=w.pad_mode)
        kf, kc = workloads.keep_counts(e0.P, finest, smooth)
        e0.close()
        e = sce.ce_setup_embedding(0, w.nu, w.lam, w.sigma2, n, pad_mode=w.pad_mode,
                                   keep_fine=kf, keep_coarse=kc)
        out.append((e, level, n, count))
    return out


def _tensors(n, count, fill=float("nan")):
    import torch
    return (torch.full((count, n + 1, n + 1), fill, dtype=torch.float32, device="cuda"),
            torch.full((count, n // 2 + 1, n // 2 + 1), fill, dtype=torch.float32, device="cuda"))


def test_levels_in_one_launch_equal_per_level_calls(sce):
    import torch
    levels = _levels(sce)
    tasks, refs = [], []
    for i, (e, level, n, count) in enumerate(levels):
        kf, kc = _tensors(n, count)
        first = 1000 * i + 7
        coarse = kc if i != 4 else None        # one task without a coarse field
        tasks.append({"emb": e, "level": level, "first_sample": first, "count": count,
                      "k_fine": kf, "k_coarse": coarse})
        rf, rc = _tensors(n, count)
        sce.ce_sample_batch(e, 9, level, first, count, 32, rf, rc if coarse is not None else None)
        refs.append((rf, rc if coarse is not None else None))
    sce.ce_sample_levels(tasks, 9)
    torch.cuda.synchronize()
    for t, (rf, rc) in zip(tasks, refs):
        assert torch.equal(t["k_fine"], rf)
        if rc is not None:
            assert torch.equal(t["k_coarse"], rc)
    for e, *_ in levels:
        e.close()


def test_starved_wait_times_out_and_the_device_stays_usable(sce):
    import torch
    levels = _levels(sce)[:2]
    tasks = []
    for e, level, n, count in levels:
        kf, kc = _tensors(n, count)
        tasks.append({"emb": e, "level": level, "first_sample": 0, "count": count,
                      "k_fine": kf, "k_coarse": kc})
    with pytest.raises(sce.SceError) as ex:
        sce.ce_sample_levels(tasks, 9, wait_cycles=2_000_000, starve_task=1)
    assert ex.value.status == sce.CE_ERR_TIMEOUT
    assert "gave up" in sce.last_error()
    # the context is intact: the same call without starvation succeeds
    sce.ce_sample_levels(tasks, 9)
    torch.cuda.synchronize()
    e, level, n, count = levels[1]
    rf, rc = _tensors(n, count)
    sce.ce_sample_batch(e, 9, level, 0, count, 32, rf, rc)
    torch.cuda.synchronize()
    assert torch.equal(tasks[1]["k_fine"], rf) and torch.equal(tasks[1]["k_coarse"], rc)
    for e, *_ in levels:
        e.close()


def test_persistent_estimate_equals_the_streams_path(sce):
    """mlmc_estimate_levels_persistent (all fields in one persistent launch,
    then the solves) gives bit-identical per-sample Y and level sums to
    mlmc_estimate_levels (each level samples its own fields)."""
    import torch
    levels = _levels(sce)[:4]
    runs = []
    for persistent in (False, True):
        tasks = [{"emb": e, "level": level, "first_sample": 3 + level, "count": count,
                  "Y": torch.full((count,), float("nan"), dtype=torch.float64, device="cuda")}
                 for e, level, n, count in levels]
        sums, stats, st = sce.mlmc_estimate_levels(tasks, 5, qoi_index=1, f=1.0, rtol=1e-10,
                                                   precision=32, max_concurrency=4,
                                                   persistent=persistent)
        torch.cuda.synchronize()
        assert st == 0 and stats == [0] * len(levels)
        runs.append((tasks, sums))
    for (ta, sa), (tb, sb) in zip(zip(*runs[0]), zip(*runs[1])):
        assert torch.equal(ta["Y"], tb["Y"])
        assert (sa.N, sa.sumY, sa.sumY2, sa.sumQf, sa.sumQf2) == \
            (sb.N, sb.sumY, sb.sumY2, sb.sumQf, sb.sumQf2)
    for e, *_ in levels:
        e.close()
