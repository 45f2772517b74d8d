"""The capture-derived constants of bench.py still describe the current kernels.

bench.py reports a kernel family's DRAM traffic and instruction-issue fraction
from ratios measured in one ncu capture of the kernel, and only while the
kernel's source text hashes to the captured one.  These host checks fail when
a kernel named there has changed since its capture (the ratio must then be
measured again), and check that every such family has a declared bound.
"""
import bench


def test_capture_digests_match_the_current_sources():
    stale = []
    for table in (bench.TRAFFIC_PER_ALG, bench.INSTR_PER_ALG):
        for family, (ratio, path, kernel, digest) in table.items():
            assert ratio > 0.0, family
            if bench.kernel_source_digest(path, kernel) != digest:
                stale.append((family, path, kernel))
    assert not stale, stale


def test_issue_bound_families_are_declared():
    for family in bench.INSTR_PER_ALG:
        assert bench.KERNEL_BOUND.get(family) == "issue", family
