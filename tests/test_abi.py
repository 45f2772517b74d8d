"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point include/sce.h declares; host-only entry points agree with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import mlmc as omlmc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "sce.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2306_13493_gb300 import build, sce
    build.build_library()
    return sce.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ce_setup_embedding", "ce_sample_batch", "darcy_solve_batch", "mlmc_level_estimate",
              "ce_destroy", "ce_status_string", "ce_normals", "mlmc_optimal_samples"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2306_13493_gb300 import sce
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in sce.EXPORTED, name


def test_status_strings(lib):
    from paper_2306_13493_gb300 import sce
    assert sce.status_string(0) == "ok"
    assert "converge" in sce.status_string(sce.CE_ERR_NOT_CONVERGED)


def test_optimal_samples_matches_oracle(lib):
    from paper_2306_13493_gb300 import sce
    V = np.array([3.1e-2, 4.0e-3, 9.0e-4, 1.7e-4])
    C = np.array([1.0, 4.2, 17.0, 70.0])
    for eps in (1e-2, 2.5e-3, 1e-3):
        assert list(sce.mlmc_optimal_samples(V, C, eps)) == list(omlmc.optimal_samples(V, C, eps))
    with pytest.raises(sce.SceError):
        sce.mlmc_optimal_samples([1.0], [0.0], 1e-2)


def test_tau_rules_match_oracle(lib):
    """§3.6: the library's closed form and Newton solve against the oracle's
    closed form and bisection, for any C_s / C_alpha (the oracle's rules are
    pinned against the error bounds in test_oracle_tau.py)."""
    from paper_2306_13493_gb300 import sce
    for alpha in (0.5, 1.0, 1.5, 2.0):
        for ratio in (0.05, 1.0, 20.0):
            for h in (1 / 4, 1 / 16, 1 / 64, 1 / 512):
                s = 4.0 / (h * h)
                got = sce.mlmc_tau_exponential(s, alpha, ratio)
                assert got == pytest.approx(omlmc.tau_exponential(s, alpha, ratio), rel=1e-12)
                for J in (0, 3, 16, 64):
                    for nu in (0.5, 1.5, 2.5):
                        got = sce.mlmc_tau_matern(h, J, nu, alpha, ratio)
                        want = omlmc.tau_matern(h, J, nu, alpha, ratio)
                        assert got == pytest.approx(want, rel=1e-10), (alpha, ratio, h, J, nu)
    for bad in ((0.5, 1.0, 1.0), (16.0, 0.0, 1.0), (16.0, 1.0, -1.0), (float("inf"), 1.0, 1.0)):
        with pytest.raises(sce.SceError):
            sce.mlmc_tau_exponential(*bad)
    for bad in ((0.0, 0, 1.5, 1.0, 1.0), (0.1, -1, 1.5, 1.0, 1.0), (0.1, 0, 0.0, 1.0, 1.0),
                (0.1, 0, 1.5, 0.0, 1.0), (0.1, 0, 1.5, 1.0, 0.0)):
        with pytest.raises(sce.SceError):
            sce.mlmc_tau_matern(*bad)


def test_keep_counts_from_tau():
    from paper_2306_13493_gb300 import mlmc
    assert mlmc.keep_for_tau(4096, 64.0) == 4032
    assert mlmc.keep_for_tau(4096, 63.5) == 4032      # rounds half to even: 64 dropped
    assert mlmc.keep_for_tau(4096, 0.4) == 4096
    assert mlmc.keep_for_tau(4096, 5000.0) == 1       # at least one eigenvalue kept


def test_struct_layouts_match_header():
    from paper_2306_13493_gb300 import sce
    assert ctypes.sizeof(sce.ce_cov) == 32
    assert ctypes.sizeof(sce.ce_embedding_info) == 4 * 3 + 4 + 8 * 3 + 8 * 3
    assert ctypes.sizeof(sce.mlmc_level_sums) == 8 * 5 + 8 + 8
    # mlmc_level_task: pointer, u32 (+pad), u64, int (+pad), 3 pointers, sums, int (+pad)
    assert sce.mlmc_level_task.sums.offset == 56
    assert sce.mlmc_level_task.status.offset == 112
    assert ctypes.sizeof(sce.mlmc_level_task) == 120
    # mlmc3_level_task: pointer, u32 (+pad), u64, int (+pad), pointer, sums, int (+pad)
    assert sce.mlmc3_level_task.sums.offset == 40
    assert sce.mlmc3_level_task.status.offset == 96
    assert ctypes.sizeof(sce.mlmc3_level_task) == 104
    # server structs: config int, (pad), i64, int, int, double, int (+pad), i64
    assert ctypes.sizeof(sce.sce_server_config) == 48
    assert sce.sce_server_config.slice_vertices.offset == 40
    # persistent field task: pointer, u32 (+pad), u64, int (+pad), 2 pointers
    assert ctypes.sizeof(sce.ce_field_task) == 48 and sce.ce_field_task.k_fine.offset == 32
    assert ctypes.sizeof(sce.ce_levels_opts) == 16
    # request: ce_cov 32, ce_pad 12, n 4, level 4, smoothing 4, finest 4, (pad 4),
    # seed 8, first_sample 8, count 4, qoi 4, f 8, Y 8
    assert sce.sce_request.seed.offset == 64 and ctypes.sizeof(sce.sce_request) == 104
    assert sce.sce_result.footprint.offset == 64 and ctypes.sizeof(sce.sce_result) == 104
    assert ctypes.sizeof(sce.sce_server_stats_t) == 96


def test_server_rejects_bad_configs_on_the_host(lib):
    """sce_server_create checks its config before any CUDA call."""
    from paper_2306_13493_gb300 import sce
    h = ctypes.c_void_p()
    for cfg in (sce.sce_server_config(0, 0, 8, 32, 1e-10, 100),      # no slots
                sce.sce_server_config(4, 0, 0, 32, 1e-10, 100),      # no cache
                sce.sce_server_config(4, 0, 8, 16, 1e-10, 100),      # precision
                sce.sce_server_config(4, 0, 8, 32, 0.0, 100)):       # rtol
        assert lib.sce_server_create(ctypes.byref(cfg), ctypes.byref(h)) == sce.CE_ERR_INVALID_ARG
    assert lib.sce_server_submit(None, None, None) == sce.CE_ERR_INVALID_ARG
    lib.sce_server_destroy(None)


def test_estimate_levels_rejects_bad_arguments_on_the_host():
    """Argument checks return before any CUDA call (safe without a GPU)."""
    from paper_2306_13493_gb300 import sce
    lib = sce.load()
    prob = sce.darcy_problem(16, 1.0, 1e-10, 100, 32)
    tasks = (sce.mlmc_level_task * 2)()
    tasks[0].emb, tasks[0].count = 1, 4           # fake handle, never dereferenced
    tasks[1].emb, tasks[1].count = None, 4        # missing handle
    assert lib.mlmc_estimate_levels(ctypes.byref(prob), 1, 0, tasks, 2, 4, None) == \
        sce.CE_ERR_INVALID_ARG
    tasks[1].emb, tasks[1].count = 1, -1          # negative count
    assert lib.mlmc_estimate_levels(ctypes.byref(prob), 1, 0, tasks, 2, 4, None) == \
        sce.CE_ERR_INVALID_ARG
    assert lib.mlmc_estimate_levels(ctypes.byref(prob), 1, 3, tasks, 0, 4, None) == \
        sce.CE_ERR_INVALID_ARG                    # qoi_index out of range
    assert lib.mlmc_estimate_levels(None, 1, 0, tasks, 0, 4, None) == sce.CE_ERR_INVALID_ARG
    bad = sce.darcy_problem(16, 1.0, 1e-10, 100, 16)   # precision neither 32 nor 64
    assert lib.mlmc_estimate_levels(ctypes.byref(bad), 1, 0, tasks, 0, 4, None) == \
        sce.CE_ERR_INVALID_ARG
    assert lib.mlmc_estimate_levels(ctypes.byref(prob), 1, 0, tasks, 0, 4, None) == sce.CE_OK


def test_three_dimensional_entry_points_reject_bad_arguments_on_the_host():
    """Argument checks of the d = 3 entry points return before any CUDA call."""
    from paper_2306_13493_gb300 import sce
    lib = sce.load()
    cov = sce.ce_cov(0, 0.5, 0.1, 1.0)
    pad = sce.ce_pad(sce.CE_PAD_DOUBLING, -1, 512)
    h = ctypes.c_void_p()
    for n in (3, 1, 512):                                  # not a power of two / out of range
        assert lib.ce3_setup_embedding(ctypes.byref(cov), n, ctypes.byref(pad), None, None,
                                       ctypes.byref(h), None) == sce.CE_ERR_INVALID_ARG
    bad_nu = sce.ce_cov(0, 0.7, 0.1, 1.0)
    assert lib.ce3_setup_embedding(ctypes.byref(bad_nu), 8, ctypes.byref(pad), None, None,
                                   ctypes.byref(h), None) == sce.CE_ERR_INVALID_ARG
    fake = ctypes.c_void_p(16)                             # never dereferenced
    for prob in (sce.darcy_problem(8, 1.0, 1e-10, 100, 64),     # FP32 fields only
                 sce.darcy_problem(6, 1.0, 1e-10, 100, 32),
                 sce.darcy_problem(8, 1.0, 0.0, 100, 32)):
        assert lib.darcy3_solve_batch(ctypes.byref(prob), fake, 1, fake, None, None, None,
                                      None) == sce.CE_ERR_INVALID_ARG
    out = sce.mlmc_level_sums()
    prob = sce.darcy_problem(8, 1.0, 1e-10, 100, 32)
    assert lib.mlmc3_level_estimate(None, ctypes.byref(prob), 1, 0, 0, 4, 0, ctypes.byref(out),
                                    None, None) == sce.CE_ERR_INVALID_ARG
    assert lib.ce3_sample_batch(None, 1, 0, 0, 4, None, None, None) == sce.CE_ERR_INVALID_ARG
    tasks = (sce.mlmc3_level_task * 2)()
    tasks[0].emb, tasks[0].count = 16, 4
    tasks[1].emb, tasks[1].count = None, 4                 # missing handle
    assert lib.mlmc3_estimate_levels(ctypes.byref(prob), 1, 0, tasks, 2, 4, None) == \
        sce.CE_ERR_INVALID_ARG
    assert lib.mlmc3_estimate_levels(ctypes.byref(prob), 1, 3, tasks, 0, 4, None) == \
        sce.CE_ERR_INVALID_ARG                             # qoi_index out of range
    assert lib.mlmc3_estimate_levels(ctypes.byref(prob), 1, 0, tasks, 0, 4, None) == sce.CE_OK


def test_missing_library_is_an_error(tmp_path):
    """No fallback: a library that is not there makes load() raise."""
    from paper_2306_13493_gb300 import sce
    with pytest.raises(RuntimeError, match="not built"):
        sce.load(str(tmp_path / "libsce.so"))
