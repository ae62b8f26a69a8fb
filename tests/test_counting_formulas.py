"""The paper's counting formulas against the benchmark's byte and flop accounting (CPU only).

Eq. 11: flops of A_L per point, 12(N+1) + 15 (111 at N = 7); with the 8 FP64 words a point of
the stored-factor operator moves (u, w, 6 factors) that is 13.875 flop/word, the paper's 13.8
(Section 5.1). The rematerialised count 30(N+1) + 96 over 3 words per point gives 112 (Section
5.1). Eq. 9: n_gs = E((N+1)^3 - (N-1)^3) boundary copies, 2 n_gs / n = 1.15625 at N = 7, and
Eq. 10's per-iteration words 20 n + 2 n_gs."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_eq11_and_intensity():
    assert bench.flops_eq11(7) == 111
    assert [bench.flops_eq11(N) for N in (3, 5, 9, 11)] == [63, 87, 135, 159]
    words = bench.ax_bytes_per_point("stored", "f64", 7) / 8
    assert words == 8
    assert bench.flops_eq11(7) / words == pytest.approx(13.875)
    # remat: the paper's 30(N+1)+96 flops over u, w and one per-point word
    assert (30 * 8 + 96) / 3 == 112
    assert bench.ax_bytes_per_point("otfscale", "f64", 7) == pytest.approx(8 * 3 + 8 * 21 / 512)


def test_eq9_and_eq10_words():
    N, E = 7, 32 ** 3
    Np = N + 1
    n = E * Np ** 3
    n_gs = E * (Np ** 3 - (N - 1) ** 3)
    assert n_gs == 9_699_328
    assert 2 * n_gs / n == pytest.approx(1.15625)
    assert (20 * n + 2 * n_gs) / n == pytest.approx(21.15625)
    # the fused, preconditioned iteration the benchmark counts: operator 10 words, update 8,
    # gather-scatter 2 n_gs / n, plus one multiplicity byte
    assert bench.cg_bytes_per_point(N) == pytest.approx(8 * (18 + 1.15625) + 1)
