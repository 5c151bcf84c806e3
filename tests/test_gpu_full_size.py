"""Parity at the benchmark's full size: the two-round card game of
264,306,001 nodes in the bench's layout (member order, tiles at depths 4-7)
and launch form (per-level kernels replayed from a graph, autotuned lanes).
Two FP64 iterations must equal the oracle's regrets and average sums
bitwise (the oracle walks the whole tree twice, a few seconds in C)."""
import numpy as np
import pytest

import gamegen as gg
import oracle
from paper_2609_11923_gb300 import cfr

pytestmark = pytest.mark.gpu


def test_full_size_card_game_two_fp64_iterations_match_oracle_bitwise():
    g = gg.large_card()
    s = cfr.Solver(g, precision=cfr.P64, exec_form=cfr.EXEC_GRAPH)
    assert list(cfr.cfr_export_array(s.h, "level_tiled")[4:]) == [1, 1, 1, 1]
    s.autotune()
    s.iterate(2)
    s.synchronize()
    R, avg, t = s.get_state()
    assert t == 2
    o = oracle.Oracle(g)
    o.iterate(2)
    np.testing.assert_array_equal(R, o.R)
    np.testing.assert_array_equal(avg, o.sbar)
