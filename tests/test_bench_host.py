"""Host-side arithmetic of bench.py (no GPU): the algorithmic counts it divides by, checked
against closed forms of the ladder's work (packed pairs a<b, i<j, e<f)."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_ladder_counts_at_o32_v240():
    a = bench.algorithmic(32, 240, 1200)
    Pv, Po = 240 * 239 // 2, 32 * 31 // 2
    assert a["form_cmac"] == 1200 * Pv * 240 ** 2          # naux P_v v^2 = 1.98e12
    assert a["ladder_cmac"] - a["form_cmac"] == Po * Pv ** 2  # P_o P_v^2 = 4.08e11
    assert abs(a["form_cmac"] / 1.98e12 - 1) < 0.01
    assert abs((a["ladder_cmac"] - a["form_cmac"]) / 4.08e11 - 1) < 0.01
    assert a["ring_cmac"] == 32 ** 3 * 240 ** 3


def test_formation_flops_executed_bounds():
    v, naux = 240, 1200
    alg = bench.algorithmic(32, v, naux)["form_cmac"] * 8
    # one group of all a: every (b, f) row against every (a, e) column
    assert bench.formation_flops_executed(v, naux, v) == 8 * v ** 4 * naux
    prev = None
    for ga in (1, 16, 32, 64):
        f = bench.formation_flops_executed(v, naux, ga)
        assert f >= alg            # rows b >= a0 cover every pair a < b at least once
        if prev is not None:
            assert f >= prev       # coarser groups form more of the b < a half
        prev = f
    # single a per group: rows b >= a form the pairs a <= b, i.e. P_v + v diagonal blocks
    assert bench.formation_flops_executed(v, naux, 1) == 8 * naux * v ** 2 * (v * (v + 1) // 2 - 1)


def test_replica_throughput_and_reduce_without_process_group():
    assert bench.replica_throughput(4, 10, 1000.0) == 40.0
    assert bench.reduce_max(3.5) == 3.5
