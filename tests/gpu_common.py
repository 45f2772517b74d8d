"""Shared helpers of the GPU parity tests (they call the CUDA path through the
C ABI binding and compare with the oracle)."""
import numpy as np

# Tolerances (relative, max over elements) of the parity tests:
#   FP64 path: 1e-10; FP32 path (FP32 normals, FFT, exp): 1e-5.
TOL64 = 1e-10
TOL32 = 1e-5


def lib():
    from paper_2306_13493_gb300 import build, sce
    build.build_library()
    sce.load()
    return sce


def rel_err(got, want):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    return float(np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-300))


def torch_dtype(precision):
    import torch
    return torch.float64 if precision == 64 else torch.float32
