"""Synthetic workload definitions shared by the benchmark, the tests and the
CPU baseline.  Parameters only -- no arithmetic of the method lives here.

The paper (§4) samples its random fields synthetically (no dataset); the
workloads below follow its experiments: unit square, Matern covariance,
levels h_l = 2^-l h_0 with the field sampled on the solve's grid.
"""
from dataclasses import dataclass, field
from typing import List


@dataclass
class MLMCWorkload:
    name: str
    nu: float
    lam: float
    sigma2: float
    n0: int                      # coarsest grid (cells per side)
    N: List[int]                 # samples per level
    pad_mode: int                # 1 = classical doubling, 2 = smooth periodisation
    smoothing: bool              # MLMC-CES (tau_l = sqrt(s_l), finest level unsmoothed)
    qoi: int                     # 0 outflow, 1 u(7/15, 7/15), 2 L2 norm
    f: float
    seed: int
    rtol: float = 1e-10
    kind: int = 0                # 0 Matern

    @property
    def levels(self):
        return [(l, self.n0 << l, self.N[l]) for l in range(len(self.N))]

    def describe(self):
        ns = [self.n0 << l for l in range(len(self.N))]
        return (f"{'MLMC-CES' if self.smoothing else 'MLMC'} Matern nu={self.nu} "
                f"lambda={self.lam} sigma2={self.sigma2}; n={ns[0]}..{ns[-1]} "
                f"(L={len(ns) - 1}); N_l={'/'.join(map(str, self.N))}; "
                f"{'smooth periodisation J=n' if self.pad_mode == 2 else 'doubling'}; "
                f"{'tau_l=sqrt(s_l), finest unsmoothed; ' if self.smoothing else ''}"
                f"Q={['outflow', 'u(7/15,7/15)', 'L2 norm'][self.qoi]}, f={self.f}, "
                f"rtol={self.rtol}")


# Oscillatory field, smoothed vs plain CE MLMC (the headline workload).
OSCILLATORY = MLMCWorkload(
    name="mlmc_oscillatory", nu=0.5, lam=0.02, sigma2=1.0, n0=16,
    N=[20000, 8000, 3000, 1000, 300, 100], pad_mode=2, smoothing=True, qoi=1, f=1.0, seed=2)

# Plain method, small: 33 x 33 vertices, doubled embedding, outflow, f = 0.
PLAIN_SMALL = MLMCWorkload(
    name="plain_33x33", nu=0.5, lam=0.3, sigma2=1.0, n0=32, N=[256], pad_mode=1,
    smoothing=False, qoi=0, f=0.0, seed=0)


def shard_first_sample(step, rank, world, N):
    """First sample index of `rank`'s block of N samples in step `step`: the
    sample ranges of all (step, rank) pairs tile [0, inf) without overlap, so
    a sharded run draws exactly the samples of a single-rank run."""
    return (step * world + rank) * N


def keep_counts(P, finest, smoothing):
    """(keep_fine, keep_coarse) for one level of MLMC-CES: the smoothed sample
    drops tau = sqrt(s) = P eigenvalues and drives both grids, except that the
    finest level's fine field is unsmoothed; -1 = no truncation."""
    if not smoothing:
        return -1, -1
    s = P * P
    return (-1 if finest else s - P), s - P


@dataclass
class ServedWorkload:
    """Requests of the served MLMC loop: each request is one MLMC level
    (fine grid n0 * 2^level, coarse grid half of it) of one covariance
    ("tenant"), with a log-uniform sample count.  Tenants are drawn once:
    nu from nu_choices, lambda log-uniform in lam_range, sigma^2 uniform in
    sigma2_range; requests draw a tenant and a level uniformly."""
    n0: int = 16
    levels: int = 7                      # levels 0..6: n = 16..1024
    count_range: tuple = (1, 4096)
    nu_choices: tuple = (0.5, 1.5)
    lam_range: tuple = (0.01, 0.1)
    sigma2_range: tuple = (0.5, 3.0)
    tenants: int = 6
    load: float = 0.75                   # arrival rate / measured service capacity
    arrival_seed: int = 5
    mlmc_seed: int = 6
    mlmc_eps: float = 5e-4
    mlmc_levels: int = 5                 # the adaptive client's levels 0..4

    def draw_tenants(self):
        import numpy as np
        rng = np.random.default_rng(self.arrival_seed)
        out = []
        for _ in range(self.tenants):
            out.append({"nu": float(rng.choice(self.nu_choices)),
                        "lam": float(np.exp(rng.uniform(*np.log(self.lam_range)))),
                        "sigma2": float(rng.uniform(*self.sigma2_range))})
        return out

    def draw_request(self, rng, tenants):
        import numpy as np
        t = int(rng.integers(len(tenants)))
        level = int(rng.integers(self.levels))
        lo, hi = self.count_range
        count = int(min(hi, max(lo, round(float(np.exp(rng.uniform(np.log(lo), np.log(hi))))))))
        return {**tenants[t], "tenant": t, "level": level, "n": self.n0 << level, "count": count}


SERVED = ServedWorkload()


@dataclass
class PrecisionStudy:
    """Precision study at scale: the mixed path (FP32 normals, FFT, exp and
    multigrid, FP64 eigenvalues and refinement) against the all-FP64 path and
    the FP64 oracle, on one fine grid without padding beyond P = 2n."""
    nus: tuple = (0.5, 2.5)
    lam: float = 0.01
    sigma2: float = 3.0
    n: int = 1024                        # 1025^2 vertices
    pad_mode: int = 1                    # classical embedding, doubled only if not PSD
    J: int = 0                           # P = 2n = 2048
    count: int = 512
    oracle_samples: int = 16
    f: float = 1.0
    seed: int = 4
    rtol: float = 1e-10


PRECISION_STUDY = PrecisionStudy()


@dataclass
class MixedLaunch:
    """One launch holding samples of several levels of uneven size: each
    sample is a level pair (fine grid n, coarse grid n/2), FP32 field with
    float-float refinement; classical embedding P = 2n (doubled if needed),
    no smoothing."""
    nu: float = 1.5
    lam: float = 0.05
    sigma2: float = 1.0
    buckets: tuple = ((64, 4096), (128, 1024), (256, 256), (512, 64), (1024, 16))
    pad_mode: int = 1
    qoi: int = 1
    f: float = 1.0
    seed: int = 3
    rtol: float = 1e-10

    def describe(self):
        return (f"Matern nu={self.nu} lambda={self.lam} sigma2={self.sigma2}; level pairs "
                + ", ".join(f"{c}@{n}^2" for n, c in self.buckets)
                + "; classical embedding P=2n; Q=u(7/15,7/15), f=1, rtol=1e-10")


MIXED_LAUNCH = MixedLaunch()


@dataclass
class SmoothingStudy:
    """Smoothing error on one grid (§4.1): Q_h with the full spectrum against
    Q~_h with tau = sqrt(s) eigenvalues dropped, from the same normals, for
    the separable exponential covariance (no padding needed, Lemma 3) and
    Matern nu = 1.5 (smooth periodisation); QoI ||u||_L2, f = 1."""
    covs: tuple = ((1, 0.0, 0.3), (1, 0.0, 0.1), (0, 1.5, 0.1), (0, 1.5, 0.03))   # (kind, nu, lam)
    sigma2: float = 1.0
    ns: tuple = (16, 32, 64, 128, 256)
    samples: tuple = (1024, 1024, 512, 256, 128)
    seed: int = 7
    f: float = 1.0
    qoi: int = 2


SMOOTHING_STUDY = SmoothingStudy()


@dataclass
class QmcStudy:
    """MLQMC against MLMC at equal sample counts: per level, R random shifts
    of an N-point Korobov lattice against R N Philox samples."""
    nu: float = 1.5
    lam: float = 0.1
    sigma2: float = 1.0
    n0: int = 16
    levels: int = 4
    N: int = 256
    R: int = 16
    a: int = 1597
    qoi: int = 2
    f: float = 1.0
    seed: int = 8


QMC_STUDY = QmcStudy()


@dataclass
class ThreeD:
    """Three-dimensional MLMC-CES (the d = 3 instance of the method): unit
    cube, Matern covariance, smooth periodisation (J = n, P = 4n), levels
    n = n0 * 2^l, tau = floor(sqrt(s)) eigenvalues dropped from every field
    except the finest level's fine field; Q = u(7/15, 7/15, 7/15), f = 1.
    The CPU baseline runs the oracle on levels 0..2 only: one direct solve on
    the 65^3 grid of level 3 takes minutes."""
    nu: float = 0.5
    lam: float = 0.1
    sigma2: float = 1.0
    n0: int = 8
    N: tuple = (4000, 1000, 250, 60)
    qoi: int = 1
    f: float = 1.0
    seed: int = 9
    rtol: float = 1e-10
    cpu_samples: tuple = (32, 16, 1)

    @property
    def levels(self):
        return [(l, self.n0 << l, self.N[l]) for l in range(len(self.N))]

    def describe(self):
        ns = [self.n0 << l for l in range(len(self.N))]
        return (f"3D MLMC-CES Matern nu={self.nu} lambda={self.lam} sigma2={self.sigma2}; "
                f"n={ns[0]}..{ns[-1]} per side (L={len(ns) - 1}); "
                f"N_l={'/'.join(map(str, self.N))}; smooth periodisation J=n (P=4n); "
                f"tau_l=floor(sqrt(s_l)), finest unsmoothed; Q=u(7/15,7/15,7/15), f={self.f}, "
                f"rtol={self.rtol}")


THREE_D = ThreeD()
