"""The streaming FP32 backward (lanes_per_set = 512) against the oracle.

Its chunks and staged index arithmetic are checked on the CPU first
(tests/test_stream_layout.py, tests/test_layout_emulation.py); here the
kernel itself runs: FP32 exploitability within 1e-4 of the pot of the
oracle's at T = 1,000 in every launch form that uses it, deterministic runs,
split calls equal to one call, both update orders and every update rule.
"""
import numpy as np
import pytest
import torch

import gamegen as gg
import oracle
from paper_2609_11923_gb300 import cfr
from tests.fp32_band import fp32_band, fp32_bar

pytestmark = pytest.mark.gpu

GAMES = {
    "tiny": lambda: gg.tiny_card(),
    "card_4x4": lambda: gg.large_card(4, 4, 1, 1),
    "card_4x2_cap2": lambda: gg.large_card(4, 2, 2, 2),
    "rt10": lambda: gg.random_tree(4, depth=10),
    "endgame": lambda: gg.endgame(7, 200000),
    "wide_root": lambda: gg.endgame(2, 100000),
}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield
    torch.cuda.synchronize()


def streaming(g, form=cfr.EXEC_GRAPH, tiles=cfr.TILES_AUTO, **kw):
    s = cfr.Solver(g, precision=cfr.P32, exec_form=form, lanes_per_set=cfr.STREAM_LANES, member_tiles=tiles, **kw)
    lanes = cfr.cfr_export_array(s.h, "level_lanes")
    ok = cfr.cfr_export_array(s.h, "stream_ok")
    assert (lanes[ok.astype(bool)] == cfr.STREAM_LANES).all() and ok.any()
    return s


@pytest.mark.parametrize("tiles", [cfr.TILES_AUTO, cfr.TILES_ON])
@pytest.mark.parametrize("name", list(GAMES))
def test_streaming_fp32_within_1e4_pot(name, tiles):
    g = GAMES[name]()
    s = streaming(g, tiles=tiles)
    s.iterate(1000)
    s.synchronize()
    e_or = oracle.solve(g, 1000).exploitability()
    assert abs(s.exploitability() - e_or) <= 1e-4 * g.pot, (s.exploitability(), e_or)


def test_streaming_forms_agree_bitwise_runs_repeat_and_split_calls_equal_one_call():
    g = gg.large_card(4, 4, 1, 1)
    outs = []
    for form, parts in ((cfr.EXEC_LEVELS, (60,)), (cfr.EXEC_GRAPH, (60,)), (cfr.EXEC_GRAPH, (7, 50, 0, 3))):
        s = streaming(g, form=form, tiles=cfr.TILES_ON)
        for n in parts:
            s.iterate(n)
        s.synchronize()
        outs.append(s.get_state())
    for R, avg, t in outs[1:]:
        assert t == 60
        np.testing.assert_array_equal(R, outs[0][0])
        np.testing.assert_array_equal(avg, outs[0][1])


@pytest.mark.parametrize("rule,orule", [(cfr.RULE_CFR_PLUS, oracle.CFR_PLUS), (cfr.RULE_CFR, oracle.CFR),
                                        (cfr.RULE_PCFR_PLUS, oracle.PCFR_PLUS)])
@pytest.mark.parametrize("order", [cfr.ORDER_SIMULTANEOUS, cfr.ORDER_ALTERNATING])
def test_streaming_every_rule_and_order_within_tolerance(rule, orule, order):
    # vanilla CFR with alternating updates is ill-conditioned on this game:
    # FP32-sized payoff perturbations alone move the oracle by about 1e-3
    # at T = 300, so the bar there is the oracle's own band (fp32_band)
    g = gg.large_card(3, 2, 1, 1)
    s = streaming(g, rule=rule, order=order, tiles=cfr.TILES_ON)
    s.iterate(300)
    s.synchronize()
    e_or, delta = fp32_band(lambda: gg.large_card(3, 2, 1, 1), 300, rule=orule, order=order)
    assert abs(s.exploitability() - e_or) <= fp32_bar(g.pot, delta), (s.exploitability(), e_or, delta)


def test_streaming_matches_the_lane_group_kernel_closely_after_one_iteration():
    # one iteration from the uniform strategy: the two FP32 kernels sum the
    # same terms in different fixed orders, so R agrees to FP32 rounding
    g = gg.large_card(4, 4, 1, 1)
    a = streaming(g, tiles=cfr.TILES_ON)
    b = cfr.Solver(g, precision=cfr.P32, exec_form=cfr.EXEC_GRAPH, lanes_per_set=8, member_tiles=cfr.TILES_ON)
    o = oracle.solve(g, 1)
    for s in (a, b):
        s.iterate(1)
        s.synchronize()
    Ra, Rb = a.get_state()[0], b.get_state()[0]
    scale = np.abs(o.R).max()
    assert np.abs(Ra - o.R).max() <= 1e-5 * scale
    assert np.abs(Ra - Rb).max() <= 1e-5 * scale


def test_autotune_may_pick_streaming_and_keeps_the_tolerance():
    g = gg.large_card(4, 4, 1, 1)
    s = cfr.Solver(g, precision=cfr.P32, exec_form=cfr.EXEC_GRAPH, member_tiles=cfr.TILES_ON)
    lanes = s.autotune(reps=3)
    assert set(lanes) <= {1, 2, 4, 8, 16, 32, 256, cfr.STREAM_LANES}
    s.iterate(1000)
    s.synchronize()
    assert abs(s.exploitability() - oracle.solve(g, 1000).exploitability()) <= 1e-4 * g.pot


def test_stalled_copies_time_out_and_the_context_survives():
    # the copy warp stops issuing after each CTA's first chunks: the compute
    # threads' and the update warp's bounded waits for the next chunk run
    # out, the launch ends, cfr_synchronize reports the timeout, and after a
    # reset the same handle solves bitwise like a fresh one
    g = gg.large_card(6, 4, 1, 2)  # 14.6M nodes: up to 1,518 chunks per depth
    s = streaming(g, tiles=cfr.TILES_ON)
    chunks = cfr.cfr_export_array(s.h, "stream_c0")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert (chunks[1:] - chunks[:-1]).max() > 2 * (2 * sms)  # some CTA has more chunks than its two stages
    cfr.cfr_debug_set(s.h, cfr.DEBUG_STREAM_STALL, 1)
    s.iterate(1)
    with pytest.raises(cfr.CfrError) as ei:
        s.synchronize()
    assert ei.value.code == cfr.CFR_ERR_TIMEOUT
    cfr.cfr_debug_set(s.h, cfr.DEBUG_STREAM_STALL, 0)
    s.reset()
    s.iterate(40)
    s.synchronize()
    ref = streaming(g, tiles=cfr.TILES_ON)
    ref.iterate(40)
    ref.synchronize()
    np.testing.assert_array_equal(s.get_state()[0], ref.get_state()[0])
    np.testing.assert_array_equal(s.get_state()[1], ref.get_state()[1])
