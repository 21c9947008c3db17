"""Host arithmetic of the bench line's roofline entries (no GPU): the enforcer's algorithmic
bytes over its non-zero tile pairs, and the committed ncu summaries' traffic figures."""
import numpy as np
import torch

import bench


def _pairs(n):
    t = 32 if n <= 2048 else 64
    nt = (n + t - 1) // t
    return t, nt, nt * (nt + 1) // 2


def test_nonzero_pair_fraction_counts_tile_pairs():
    n = 300  # 32-wide tiles: 10 x 10, 55 pairs on and above the diagonal
    t, nt, pairs = _pairs(n)
    F = torch.zeros((n, n + 1), dtype=torch.float64)
    assert bench.nonzero_pair_fraction(F) == 0.0
    F[:, n] = 1.0  # the environment column does not count
    assert bench.nonzero_pair_fraction(F) == 0.0
    F[5, 200] = 0.1  # tile (0, 6): one pair
    assert bench.nonzero_pair_fraction(F) == 1 / pairs
    F[200, 5] = 0.1  # its transpose: the same pair
    assert bench.nonzero_pair_fraction(F) == 1 / pairs
    F[299, 299] = 0.2  # the ragged last diagonal tile
    assert bench.nonzero_pair_fraction(F) == 2 / pairs


def test_nonzero_pair_fraction_uses_the_enforcers_tile_width():
    for n in (2048, 2049):
        t, nt, pairs = _pairs(n)
        F = torch.zeros((n, n + 1), dtype=torch.float64)
        F[t, t] = 1.0  # tile (1, 1)
        F[t - 1, t - 1] = 1.0  # tile (0, 0)
        assert bench.nonzero_pair_fraction(F) == 2 / pairs


def test_enforce_bytes():
    n = 1000
    assert bench.enforce_bytes(n, 0) == 0.0
    first = 16.0 * n * (n + 1)
    assert bench.enforce_bytes(n, 1) == first
    later = 16.0 * (n * (n + 1) / 2 + n)
    assert np.isclose(bench.enforce_bytes(n, 5), first + 4 * later)
    # zero tile pairs skipped after the first iteration: only the upper triangle shrinks
    sparse = 16.0 * (0.25 * n * (n + 1) / 2 + n)
    assert np.isclose(bench.enforce_bytes(n, 5, 0.25), first + 4 * sparse)


def test_profiled_traffic_reads_the_committed_summaries():
    # each figure is per unit, applies only while the kernel source has the captured hash
    for summary, source in (("exact_gemm_spacecraft.md", "tc_gemm.cuh"), ("gemm_pair_n4096.md", "tc_gemm.cuh"),
                            ("enforce_persistent_n6144.md", "enforce.cu"), ("trace_kernel_spacecraft.md", "trace.cu")):
        v = bench.profiled_traffic(summary, source, 1.0)
        assert v is None or v > 0.0
    assert bench.profiled_traffic("no_such_summary.md", "trace.cu", 1.0) is None
