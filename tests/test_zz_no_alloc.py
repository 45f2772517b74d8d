"""ce_sample_batch_noalloc: fields generated without any device allocation.

Some callers cannot allocate device memory per call (their framework owns all
device allocation, or the call sits in a section where allocation is not
allowed); this entry point serves them with a fixed scratch array inside the
library.  Its fields must equal those of ce_sample_batch, including on a
second call that reuses the same scratch, and a sample too large for the
scratch must be refused with a clear error.
"""
import numpy as np
import pytest

from tests.gpu_common import TOL32, TOL64, lib, rel_err, torch_dtype

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sce():
    return lib()


def _fields(fn, emb, precision, seed, level, first, count, coarse=True):
    import torch
    n = emb.n
    dt = torch_dtype(precision)
    kf = torch.empty(count, n + 1, n + 1, dtype=dt, device="cuda")
    kc = (torch.empty(count, n // 2 + 1, n // 2 + 1, dtype=dt, device="cuda") if coarse
          else None)
    fn(emb, seed, level, first, count, precision, kf, kc)
    torch.cuda.synchronize()
    return kf.cpu().numpy(), (kc.cpu().numpy() if coarse else None)


class _DevicePool:
    """The current device's default stream-ordered memory pool (the one the
    library's allocating entry points draw from), read through the driver
    API: bytes in use now, and the high-water mark since the last reset."""
    USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8      # CUmemPool_attribute

    def __init__(self):
        import ctypes
        import torch
        self.ct = ctypes
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = self.ct.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, self.ct.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = self.ct.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH,
                                             self.ct.byref(zero)) == 0


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("n,smooth,count", [(64, True, 5), (128, False, 7), (256, True, 45)])
def test_noalloc_matches_allocating_entry_point_twice(sce, precision, n, smooth, count):
    kind, nu, lam, s2 = sce.CE_COV_MATERN, 0.5, 0.02, 1.0
    e0 = sce.ce_setup_embedding(kind, nu, lam, s2, n, pad_mode=sce.CE_PAD_SMOOTH)
    P = e0.P
    e0.close()
    kf, kc = ((P * P - P, P * P // 4 - P // 2) if smooth else (-1, -1))
    emb = sce.ce_setup_embedding(kind, nu, lam, s2, n, pad_mode=sce.CE_PAD_SMOOTH,
                                 keep_fine=kf, keep_coarse=kc)
    tol = TOL64 if precision == 64 else TOL32
    ref_f, ref_c = _fields(sce.ce_sample_batch, emb, precision, 3, 2, 11, count)
    for call in range(2):    # the second call reuses the scratch left by the first
        got_f, got_c = _fields(sce.ce_sample_batch_noalloc, emb, precision, 3, 2, 11, count)
        assert rel_err(got_f, ref_f) < tol, call
        assert rel_err(got_c, ref_c) < tol, call
    other_f, _ = _fields(sce.ce_sample_batch_noalloc, emb, precision, 4, 2, 11, count)
    assert not np.allclose(other_f, ref_f)
    emb.close()


def test_noalloc_rejects_samples_larger_than_its_scratch(sce):
    emb = sce.ce_setup_embedding(sce.CE_COV_MATERN, 0.5, 0.02, 1.0, 1024,
                                 pad_mode=sce.CE_PAD_SMOOTH, keep_fine=-1,
                                 keep_coarse=(4096 * 4096) // 4 - 2048)
    assert emb.P == 4096
    import torch
    kf = torch.empty(1, 1025, 1025, dtype=torch.float64, device="cuda")
    kc = torch.empty(1, 513, 513, dtype=torch.float64, device="cuda")
    with pytest.raises(sce.SceError) as ex:
        sce.ce_sample_batch_noalloc(emb, 0, 0, 0, 1, 64, kf, kc)
    assert ex.value.status == sce.CE_ERR_INVALID_ARG
    assert "scratch" in sce.last_error()
    kf32 = torch.empty(1, 1025, 1025, dtype=torch.float32, device="cuda")
    kc32 = torch.empty(1, 513, 513, dtype=torch.float32, device="cuda")
    sce.ce_sample_batch_noalloc(emb, 0, 0, 0, 1, 32, kf32, kc32)   # fits in FP32
    ref_f = torch.empty_like(kf32)
    ref_c = torch.empty_like(kc32)
    sce.ce_sample_batch(emb, 0, 0, 0, 1, 32, ref_f, ref_c)
    torch.cuda.synchronize()
    assert rel_err(kf32.cpu().numpy(), ref_f.cpu().numpy()) < TOL32
    assert rel_err(kc32.cpu().numpy(), ref_c.cpu().numpy()) < TOL32
    emb.close()


@pytest.mark.parametrize("precision", [32, 64])
def test_noalloc_fine_field_only_in_several_chunks(sce, precision):
    """k_coarse = NULL on a smoothed embedding (the scratch holds only the
    fine intermediate); 40 samples at n = 256 (P = 1024) need 2 (FP32) or 3
    (FP64) chunks of the 64 MiB array."""
    n, count = 256, 40
    e0 = sce.ce_setup_embedding(sce.CE_COV_MATERN, 0.5, 0.02, 1.0, n, pad_mode=sce.CE_PAD_SMOOTH)
    P = e0.P
    e0.close()
    emb = sce.ce_setup_embedding(sce.CE_COV_MATERN, 0.5, 0.02, 1.0, n,
                                 pad_mode=sce.CE_PAD_SMOOTH, keep_fine=P * P - P,
                                 keep_coarse=P * P // 4 - P // 2)
    per_sample = (n + 1) * P * (16 if precision == 64 else 8)
    assert count * per_sample > 64 << 20
    tol = TOL64 if precision == 64 else TOL32
    ref_f, _ = _fields(sce.ce_sample_batch, emb, precision, 5, 3, 2, count, coarse=False)
    for call in range(2):
        got_f, _ = _fields(sce.ce_sample_batch_noalloc, emb, precision, 5, 3, 2, count,
                           coarse=False)
        assert rel_err(got_f, ref_f) < tol, call
    emb.close()


def test_noalloc_allocates_nothing(sce):
    """Across calls after the first (which resolves the scratch array's
    address and may load the library's device code), neither the device's
    default memory pool (high-water mark unchanged), nor torch's caching
    allocator, nor the device's free memory changes."""
    import torch
    n, count = 128, 9
    emb = sce.ce_setup_embedding(sce.CE_COV_MATERN, 0.5, 0.02, 1.0, n,
                                 pad_mode=sce.CE_PAD_SMOOTH, keep_fine=-1,
                                 keep_coarse=512 * 512 // 4 - 256)
    kf = torch.empty(count, n + 1, n + 1, dtype=torch.float32, device="cuda")
    kc = torch.empty(count, n // 2 + 1, n // 2 + 1, dtype=torch.float32, device="cuda")
    sce.ce_sample_batch_noalloc(emb, 1, 1, 0, count, 32, kf, kc)     # first call on the device
    torch.cuda.synchronize()
    pool = _DevicePool()
    for call in range(2):
        pool.reset_high()
        used = pool.get(pool.USED_MEM_CURRENT)
        reserved = torch.cuda.memory_reserved()
        allocs = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        free = torch.cuda.mem_get_info()[0]
        sce.ce_sample_batch_noalloc(emb, 1, 1, 100 * call, count, 32, kf, kc)
        torch.cuda.synchronize()
        assert pool.get(pool.USED_MEM_HIGH) <= used, call
        assert torch.cuda.memory_reserved() == reserved, call
        assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == allocs, call
        assert torch.cuda.mem_get_info()[0] == free, call
    # the allocating entry point does draw on the pool (the check can fail)
    pool.reset_high()
    used = pool.get(pool.USED_MEM_CURRENT)
    sce.ce_sample_batch(emb, 1, 1, 0, count, 32, kf, kc)
    torch.cuda.synchronize()
    assert pool.get(pool.USED_MEM_HIGH) > used
    emb.close()
