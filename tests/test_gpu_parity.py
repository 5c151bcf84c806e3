"""GPU parity of the sm_103a path (through the C ABI) against the FP64 oracle.

Bars (from the method's target): the FP64 mode matches the oracle's average
strategy within 1e-12 (entries are probabilities; we also expect bitwise
equality where the summation order is the oracle's), and the FP32 mode
reaches the oracle's exploitability within 1e-4 of the pot at equal
iteration counts.
"""
import numpy as np
import pytest
import torch

import gamegen as gg
import oracle
from paper_2609_11923_gb300 import cfr

pytestmark = pytest.mark.gpu

FORMS = {"levels": cfr.EXEC_LEVELS, "graph": cfr.EXEC_GRAPH, "persistent": cfr.EXEC_PERSISTENT}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield
    torch.cuda.synchronize()


def solve_gpu(spec, iters, precision=cfr.P64, form=cfr.EXEC_GRAPH, **kw):
    s = cfr.Solver(spec, precision=precision, exec_form=form, **kw)
    if iters:
        s.iterate(iters)
    s.synchronize()
    return s


def assert_strategy_close(a, b, tol=1e-12):
    d = np.abs(a - b)
    assert d.max(initial=0.0) <= tol, "max |diff| %.3e at slot %d" % (d.max(), int(d.argmax()))


# ------------------------------------------------------------- P64 parity
@pytest.mark.parametrize("form", list(FORMS))
def test_p64_tiny_card_10k_iterations_match_oracle_bitwise(form):
    g = gg.tiny_card()
    o = oracle.solve(g, 10000)
    s = solve_gpu(g, 10000, form=FORMS[form])
    np.testing.assert_array_equal(s.avg_strategy(), o.avg_strategy())
    R, avg, t = s.get_state()
    np.testing.assert_array_equal(R, o.R)
    np.testing.assert_array_equal(avg, o.sbar)
    assert t == 10000


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_p64_random_tree_1000_iterations_match_oracle(seed, form):
    g = gg.random_tree(seed, depth=9)
    o = oracle.solve(g, 1000)
    s = solve_gpu(g, 1000, form=FORMS[form])
    a = s.avg_strategy()
    assert_strategy_close(a, o.avg_strategy())
    np.testing.assert_array_equal(a, o.avg_strategy())


@pytest.mark.parametrize("name,make", [
    ("kuhn", lambda: gg.kuhn()),
    ("card_3x2", lambda: gg.large_card(3, 2, 1, 1)),
    ("card_4x2", lambda: gg.large_card(4, 2, 2, 2)),
    ("endgame_narrow_root", lambda: gg.endgame(5, 4000)),
    ("single_member_sets", lambda: gg.random_tree(9, depth=8, max_group=1)),
])
def test_p64_other_games_match_oracle(name, make):
    g = make()
    o = oracle.solve(g, 1000)
    s = solve_gpu(g, 1000)
    assert_strategy_close(s.avg_strategy(), o.avg_strategy())


def test_p64_wide_chance_root_matches_oracle():
    g = gg.endgame(2, 100000)  # deal root with more than 1024 outcomes
    assert np.diff(g.child_begin)[0] > 1024
    o = oracle.solve(g, 300)
    for form in FORMS.values():
        s = solve_gpu(g, 300, form=form)
        assert_strategy_close(s.avg_strategy(), o.avg_strategy())


# ------------------------------------------------------------- P32 parity
@pytest.mark.parametrize("name,make", [
    ("random_tree", lambda: gg.random_tree(4, depth=10)),
    ("card_4x2", lambda: gg.large_card(4, 2, 2, 2)),
    ("endgame", lambda: gg.endgame(7, 200000)),
    ("tiny", lambda: gg.tiny_card()),
])
def test_p32_exploitability_within_1e4_pot(name, make):
    g = make()
    o = oracle.solve(g, 1000)
    e_or = o.exploitability()
    s = solve_gpu(g, 1000, precision=cfr.P32)
    e_gpu = s.exploitability()
    assert abs(e_gpu - e_or) <= 1e-4 * g.pot, (e_gpu, e_or)


# ------------------------------------------------------- exploitability
@pytest.mark.parametrize("name,make", [
    ("tiny", lambda: gg.tiny_card()),
    ("random_tree", lambda: gg.random_tree(3, depth=9)),
    ("card_4x2", lambda: gg.large_card(4, 2, 2, 2)),
    ("wide_root", lambda: gg.endgame(2, 100000)),
])
def test_gpu_best_response_matches_oracle(name, make):
    g = make()
    s = solve_gpu(g, 200)
    sigma = s.avg_strategy()
    e, b1, b2, u = cfr.cfr_exploitability(s.h, s._s())
    ob1, ob2, ou = oracle.Oracle(g).best_response(sigma)
    assert b1 == pytest.approx(ob1, abs=1e-10)
    assert b2 == pytest.approx(ob2, abs=1e-10)
    assert u == pytest.approx(ou, abs=1e-10)
    assert e == pytest.approx(0.5 * (ob1 - ob2), abs=1e-10)


# ---------------------------------------------------- execution semantics
def test_p32_forms_agree_bitwise_and_runs_repeat():
    g = gg.random_tree(6, depth=10)
    outs = []
    for form in (cfr.EXEC_LEVELS, cfr.EXEC_GRAPH, cfr.EXEC_PERSISTENT, cfr.EXEC_GRAPH):
        s = solve_gpu(g, 100, precision=cfr.P32, form=form, lanes_per_set=8)
        outs.append(s.get_state())
    for R, avg, t in outs[1:]:
        np.testing.assert_array_equal(R, outs[0][0])
        np.testing.assert_array_equal(avg, outs[0][1])


@pytest.mark.parametrize("form", list(FORMS))
def test_split_calls_equal_one_call(form):
    g = gg.random_tree(8, depth=9)
    a = cfr.Solver(g, precision=cfr.P32, exec_form=FORMS[form])
    for n in (2, 8, 0, 3):
        a.iterate(n)
    b = solve_gpu(g, 13, precision=cfr.P32, form=FORMS[form])
    ra, sa, ta = a.get_state()
    rb, sb, tb = b.get_state()
    assert ta == tb == 13
    np.testing.assert_array_equal(ra, rb)
    np.testing.assert_array_equal(sa, sb)


def test_reset_replays_from_iteration_one():
    g = gg.tiny_card()
    s = solve_gpu(g, 57, precision=cfr.P32)
    s.reset()
    s.iterate(40)
    ref = solve_gpu(g, 40, precision=cfr.P32)
    np.testing.assert_array_equal(s.get_state()[0], ref.get_state()[0])
    np.testing.assert_array_equal(s.avg_strategy(), ref.avg_strategy())


def test_state_roundtrip_resumes_bitwise():
    g = gg.random_tree(10, depth=9)
    a = solve_gpu(g, 300)
    R, avg, t = a.get_state()
    b = cfr.Solver(g, precision=cfr.P64)
    b.set_state(R, avg, t)
    b.iterate(700)
    ref = oracle.solve(g, 1000)
    np.testing.assert_array_equal(b.avg_strategy(), ref.avg_strategy())


def test_set_payoffs_equals_solving_the_new_game():
    g = gg.tiny_card()
    g2 = gg.tiny_card()
    rng = np.random.default_rng(1)
    new_pay = np.where(g.kind == gg.TERMINAL, rng.uniform(-2, 2, g.n_nodes), 0.0)
    g2.payoff[:] = new_pay
    s = cfr.Solver(g, precision=cfr.P64)
    s.set_payoffs(new_pay)
    s.iterate(500)
    o = oracle.solve(g2, 500)
    np.testing.assert_array_equal(s.avg_strategy(), o.avg_strategy())


def test_barrier_timeout_reports_error_and_context_survives():
    g = gg.random_tree(12, depth=10)
    s = cfr.Solver(g, precision=cfr.P32, exec_form=cfr.EXEC_PERSISTENT, persistent_ctas=4,
                   barrier_spin_limit=2000)
    cfr.cfr_debug_set(s.h, cfr.DEBUG_BARRIER_MISSING_ARRIVALS, 1)
    s.iterate(3)
    with pytest.raises(cfr.CfrError) as ei:
        s.synchronize()
    assert ei.value.code == cfr.CFR_ERR_TIMEOUT
    cfr.cfr_debug_set(s.h, cfr.DEBUG_BARRIER_MISSING_ARRIVALS, 0)
    s.reset()
    s.iterate(50)
    s.synchronize()
    ref = solve_gpu(g, 50, precision=cfr.P32, form=cfr.EXEC_PERSISTENT, persistent_ctas=4)
    np.testing.assert_array_equal(s.get_state()[0], ref.get_state()[0])


# ------------------------------------------------------------ edge cases
def test_root_terminal_game():
    g = gg.from_lists([(gg.TERMINAL, -1, [], None, 1.25)], [])
    s = solve_gpu(g, 5)
    assert s.get_state()[2] == 5
    e, b1, b2, u = cfr.cfr_exploitability(s.h, s._s())
    assert (e, b1, b2, u) == (0.0, 1.25, 1.25, 1.25)


def test_all_chance_game():
    g = gg.from_lists(
        [
            (gg.CHANCE, -1, [1, 2], [0.25, 0.75], 0.0),
            (gg.CHANCE, -1, [3, 4], [0.5, 0.5], 0.0),
            (gg.TERMINAL, -1, [], None, 4.0),
            (gg.TERMINAL, -1, [], None, -1.0),
            (gg.TERMINAL, -1, [], None, 2.0),
        ],
        [],
    )
    s = solve_gpu(g, 3)
    e, b1, b2, u = cfr.cfr_exploitability(s.h, s._s())
    assert e == 0.0 and u == pytest.approx(0.25 * 0.5 * 1.0 + 0.75 * 4.0)


def test_sixty_four_action_sets_match_oracle():
    # root P1 set with 64 actions, each leading to a P2 set of 3 actions
    nodes = [(gg.P1, 0, list(range(1, 65)), None, 0.0)]
    rng = np.random.default_rng(0)
    nxt = 65
    for a in range(64):
        nodes.append((gg.P2, 1, [nxt, nxt + 1, nxt + 2], None, 0.0))
        nxt += 3
    for _ in range(64 * 3):
        nodes.append((gg.TERMINAL, -1, [], None, float(rng.uniform(-1, 1))))
    g = gg.from_lists(nodes, [(0, 64), (1, 3)])
    o = oracle.solve(g, 300)
    for form in FORMS.values():
        s = solve_gpu(g, 300, form=form)
        assert_strategy_close(s.avg_strategy(), o.avg_strategy())


def test_vanilla_cfr_rule_matches_oracle():
    g = gg.kuhn()
    o = oracle.solve(g, 1000, rule=oracle.CFR)
    s = solve_gpu(g, 1000, rule=cfr.RULE_CFR)
    np.testing.assert_array_equal(s.avg_strategy(), o.avg_strategy())
    assert abs(s.exploitability() - 1.32e-2) <= 3e-3 * 1.32e-2


def test_current_strategy_matches_regret_matching():
    g = gg.random_tree(13, depth=8)
    o = oracle.solve(g, 77)
    s = solve_gpu(g, 77)
    np.testing.assert_array_equal(s.current_strategy(), o.current_strategy())


def test_device_output_equals_host_output():
    g = gg.tiny_card()
    s = solve_gpu(g, 100, precision=cfr.P32)
    d = s.avg_strategy_device().cpu().numpy()
    np.testing.assert_array_equal(d, s.avg_strategy())


def test_autotune_keeps_fp64_parity_and_picks_valid_lanes():
    g = gg.random_tree(14, depth=9)
    s = cfr.Solver(g, precision=cfr.P64)
    lanes = s.autotune(reps=2)
    assert len(lanes) == s.counts["depth_blocks"]
    assert set(lanes) <= {1, 2, 4, 8, 16, 32, 256}
    assert s.get_state()[2] == 0  # the trials were reset
    s.iterate(300)
    np.testing.assert_array_equal(s.avg_strategy(), oracle.solve(g, 300).avg_strategy())


def test_pull_grids_are_one_wave_and_keep_fp64_parity():
    # the pulling forward's grid: one wave (the blocks all SMs hold at once),
    # never more than the depth's nodes need, unchanged by autotune; the grid
    # does not change any result (each node's reach is computed alone)
    g = gg.large_card(4, 4, 1, 1)
    s = cfr.Solver(g, precision=cfr.P64, exec_form=cfr.EXEC_GRAPH)
    D = s.counts["depth_blocks"]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    li = cfr.cfr_export_array(s.h, "level_int").astype(int)
    nodes = [li[d + 2] - li[d + 1] for d in range(D - 1)]
    need = [min(max(1, -(-n // (4 * 256))), 152 * 16) for n in nodes]  # blocks of 256 threads, 4 nodes each
    grid0 = cfr.cfr_export_array(s.h, "pull_grid").astype(int)
    assert len(grid0) == D and grid0[D - 1] == 0
    for d in range(D - 1):
        assert 1 <= grid0[d] <= need[d]
        if need[d] <= sms:  # a wave holds at least one block per SM
            assert grid0[d] == need[d]
    s.autotune(reps=2)
    np.testing.assert_array_equal(cfr.cfr_export_array(s.h, "pull_grid"), grid0)
    s.iterate(200)
    np.testing.assert_array_equal(s.avg_strategy(), oracle.solve(g, 200).avg_strategy())


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32, 256])
def test_every_lane_count_matches_oracle_in_fp64(lanes):
    g = gg.large_card(3, 2, 1, 1)
    s = solve_gpu(g, 200, lanes_per_set=lanes)
    np.testing.assert_array_equal(s.avg_strategy(), oracle.solve(g, 200).avg_strategy())
    p = solve_gpu(g, 200, precision=cfr.P32, form=cfr.EXEC_PERSISTENT, lanes_per_set=lanes)
    assert abs(p.exploitability() - oracle.solve(g, 200).exploitability()) <= 1e-4 * g.pot


@pytest.mark.parametrize("precision", [cfr.P64, cfr.P32])
def test_one_block_per_set_handles_sets_longer_than_a_block(precision):
    # one information set of 412 members: two member chunks of the block form
    g = gg.random_tree(4, depth=10, p_chance=0.6, max_group=1000)
    o = oracle.solve(g, 300)
    s = solve_gpu(g, 300, precision=precision, form=cfr.EXEC_LEVELS, lanes_per_set=256)
    if precision == cfr.P64:
        np.testing.assert_array_equal(s.avg_strategy(), o.avg_strategy())
    else:
        assert abs(s.exploitability() - o.exploitability()) <= 1e-4 * g.pot


@pytest.mark.parametrize("form", [cfr.EXEC_GRAPH, cfr.EXEC_PERSISTENT])
def test_p64_mid_game_card_deals_match_oracle_bitwise(form):
    # 10,920 chance nodes of 12 internal children each (written warp-wide)
    # under a wide deal root
    g = gg.large_card(4, 4, 1, 1)
    o = oracle.solve(g, 60)
    s = solve_gpu(g, 60, form=form)
    np.testing.assert_array_equal(s.avg_strategy(), o.avg_strategy())
    assert abs(s.exploitability() - o.exploitability()) <= 1e-12


def test_launch_floor_is_positive_and_leaves_the_state_alone():
    g = gg.random_tree(5, depth=9)
    s = solve_gpu(g, 20, precision=cfr.P32)
    before = s.get_state()
    gms, pms = cfr.cfr_launch_floor(s.h, 20, s._s())
    assert 0.0 < gms < 50.0 and 0.0 < pms < 50.0
    after = s.get_state()
    np.testing.assert_array_equal(before[0], after[0])
    np.testing.assert_array_equal(before[1], after[1])
    assert before[2] == after[2]
    s.iterate(10)  # the solver still works after the floor measurement
    s.synchronize()


RULES = [(cfr.RULE_CFR_PLUS, oracle.CFR_PLUS), (cfr.RULE_CFR, oracle.CFR), (cfr.RULE_PCFR_PLUS, oracle.PCFR_PLUS)]


@pytest.mark.parametrize("form", [cfr.EXEC_GRAPH, cfr.EXEC_LEVELS, cfr.EXEC_PERSISTENT])
@pytest.mark.parametrize("rule,orule", RULES)
@pytest.mark.parametrize("order", [cfr.ORDER_SIMULTANEOUS, cfr.ORDER_ALTERNATING])
def test_p64_every_rule_and_order_matches_oracle_bitwise(form, rule, orule, order):
    g = gg.tiny_card()
    o = oracle.solve(g, 400, rule=orule, order=order)
    s = solve_gpu(g, 400, form=form, rule=rule, order=order)
    np.testing.assert_array_equal(s.avg_strategy(), o.avg_strategy())
    R, avg, t = s.get_state()
    np.testing.assert_array_equal(R, o.R)
    np.testing.assert_array_equal(avg, o.sbar)
    assert t == 400
    np.testing.assert_array_equal(s.current_strategy(), o.current_strategy())


@pytest.mark.parametrize("rule,orule", RULES[::2])
def test_p64_alternating_on_a_random_tree_and_split_calls(rule, orule):
    g = gg.random_tree(6, depth=9)
    o = oracle.solve(g, 150, rule=orule, order=oracle.ALTERNATING)
    s = cfr.Solver(g, precision=cfr.P64, exec_form=cfr.EXEC_GRAPH, rule=rule, order=cfr.ORDER_ALTERNATING)
    for n in (7, 100, 43):
        s.iterate(n)
    s.synchronize()
    np.testing.assert_array_equal(s.avg_strategy(), o.avg_strategy())
    assert abs(s.exploitability() - o.exploitability()) <= 1e-12


@pytest.mark.parametrize("order", [cfr.ORDER_SIMULTANEOUS, cfr.ORDER_ALTERNATING])
def test_p32_pcfr_plus_within_tolerance(order):
    g = gg.large_card(3, 2, 1, 1)
    o = oracle.solve(g, 300, rule=oracle.PCFR_PLUS, order=order)
    s = solve_gpu(g, 300, precision=cfr.P32, rule=cfr.RULE_PCFR_PLUS, order=order)
    assert abs(s.exploitability() - o.exploitability()) <= 1e-4 * g.pot


def test_alternating_counts_twice_the_bytes_and_bad_options_are_rejected():
    g = gg.tiny_card()
    a = cfr.cfr_compile(g, cfr.make_options(order=cfr.ORDER_SIMULTANEOUS))
    b = cfr.cfr_compile(g, cfr.make_options(order=cfr.ORDER_ALTERNATING))
    try:
        assert cfr.cfr_get_counts(b)["algo_bytes_per_iter"] == 2 * cfr.cfr_get_counts(a)["algo_bytes_per_iter"]
    finally:
        cfr.cfr_destroy(a)
        cfr.cfr_destroy(b)
    for kw in ({"order": 2}, {"rule": 3}):
        with pytest.raises(cfr.CfrError):
            cfr.cfr_compile(g, cfr.make_options(**kw))


@pytest.mark.parametrize("form", [cfr.EXEC_GRAPH, cfr.EXEC_PERSISTENT])
def test_set_root_chance_then_solve_equals_the_oracle_on_the_new_game(form):
    from tests.test_compiler import with_root_chance
    g = gg.endgame(5, 4000)
    n = int(g.child_begin[1] - g.child_begin[0])
    p = np.random.default_rng(9).dirichlet(np.ones(n))
    s = solve_gpu(g, 50, form=form)  # a solve under the old distribution first
    s.set_root_chance(p)
    s.reset()
    s.iterate(300)
    s.synchronize()
    o = oracle.solve(with_root_chance(g, p), 300)
    np.testing.assert_array_equal(s.avg_strategy(), o.avg_strategy())
    assert abs(s.exploitability() - o.exploitability()) <= 1e-12


@pytest.mark.parametrize("reach_order,tiles", [(cfr.REACH_BFS, cfr.TILES_AUTO), (cfr.REACH_SLOTS, cfr.TILES_AUTO),
                                               (cfr.REACH_MEMBERS, cfr.TILES_ON), (cfr.REACH_MEMBERS, cfr.TILES_OFF)])
@pytest.mark.parametrize("form", [cfr.EXEC_GRAPH, cfr.EXEC_PERSISTENT])
@pytest.mark.parametrize("name,iters", [("tiny", 400), ("rt", 150), ("wide", 60), ("card", 40)])
def test_p64_reach_layouts_match_oracle_bitwise(reach_order, tiles, form, name, iters):
    g = {"tiny": gg.tiny_card, "rt": lambda: gg.random_tree(5, depth=9), "wide": lambda: gg.endgame(2, 100000),
         "card": lambda: gg.large_card(3, 2, 1, 1)}[name]()
    s = solve_gpu(g, iters, form=form, reach_order=reach_order, member_tiles=tiles)
    np.testing.assert_array_equal(s.avg_strategy(), oracle.solve(g, iters).avg_strategy())
    assert abs(s.exploitability() - oracle.solve(g, iters).exploitability()) <= 1e-12


def test_pinned_host_arrays_bind_to_the_same_results():
    # page-locking the compiled arrays changes how cfr_bind copies, not what
    g = gg.large_card(3, 2, 1, 1)
    a = cfr.Solver(g, precision=cfr.P64, exec_form=cfr.EXEC_GRAPH)
    b = cfr.Solver(g, precision=cfr.P64, exec_form=cfr.EXEC_GRAPH)
    b.pin_host()
    b.pin_host()  # idempotent
    cfr.cfr_bind(b.h, b.arena_ptr, b.arena_bytes, b._s())  # upload again from the pinned arrays
    for s in (a, b):
        s.iterate(30)
        s.synchronize()
    np.testing.assert_array_equal(a.avg_strategy(), b.avg_strategy())
    b.pin_host(False)
    b.pin_host(False)


def test_capture_failure_falls_back_warns_once_and_gives_the_same_floats(capfd):
    # Section 4.3: if capture fails the solver warns once and runs the same
    # kernels in the same order eagerly, computing identical floats. The
    # failure is injected on the host (the captured graph is discarded).
    g = gg.random_tree(3, depth=9)
    ref = solve_gpu(g, 30, precision=cfr.P32, form=cfr.EXEC_GRAPH, lanes_per_set=8)
    s = cfr.Solver(g, precision=cfr.P32, exec_form=cfr.EXEC_GRAPH, lanes_per_set=8)
    cfr.cfr_debug_set(s.h, cfr.DEBUG_FAIL_GRAPH_CAPTURE, 1)
    capfd.readouterr()
    for n in (10, 15, 5):
        s.iterate(n)
    s.synchronize()
    err = capfd.readouterr().err
    assert err.count("graph capture failed") == 1, err
    assert s.counts_now()["exec_form"] == cfr.EXEC_LEVELS
    for a, b in zip(s.get_state(), ref.get_state()):
        np.testing.assert_array_equal(a, b)


def test_rebinding_recaptures_instead_of_replaying_a_stale_graph():
    # Section 4.3 refuses to replay a graph whose buffers moved; here binding
    # again drops the graph, so the next call captures against the new arena
    # and the old arena is never written again.
    g = gg.tiny_card()
    s = solve_gpu(g, 20, precision=cfr.P64, form=cfr.EXEC_GRAPH)
    old = s.arena
    new = torch.empty_like(old)
    new_ptr = (new.data_ptr() + 255) & ~255
    cfr.cfr_bind(s.h, new_ptr, s.arena_bytes, s._s())  # fresh state in the new arena
    s.arena, s.arena_ptr = new, new_ptr
    torch.cuda.synchronize()
    snapshot = old.clone()
    s.iterate(30)
    s.synchronize()
    assert torch.equal(old, snapshot), "the old arena was written after rebinding"
    R, avg, t = s.get_state()
    o = oracle.solve(g, 30)
    assert t == 30
    np.testing.assert_array_equal(R, o.R)
    np.testing.assert_array_equal(avg, o.sbar)


@pytest.mark.parametrize("name,make,lanes,order", [
    ("rt", lambda: gg.random_tree(6, depth=10), 8, cfr.ORDER_SIMULTANEOUS),
    ("card", lambda: gg.large_card(4, 4, 1, 1), 8, cfr.ORDER_SIMULTANEOUS),
    # the streaming backward copies its first chunks' inputs other than the
    # children's values before the programmatic-dependent wait
    ("card_stream", lambda: gg.large_card(4, 4, 1, 1), cfr.STREAM_LANES, cfr.ORDER_SIMULTANEOUS),
    ("card_stream_alt", lambda: gg.large_card(4, 2, 2, 2), cfr.STREAM_LANES, cfr.ORDER_ALTERNATING)])
def test_graph_iterations_and_launch_overlap_leave_the_state_bitwise_unchanged(name, make, lanes, order):
    # k iterations per graph (the paper's alternative-execution table) and
    # programmatic dependent launch change how the launches are issued, not
    # what they compute: 37 = 3 x 10 + 7 iterations use both graphs
    g = make()
    outs = []
    for form, k, ov in ((cfr.EXEC_LEVELS, 0, cfr.OVERLAP_OFF), (cfr.EXEC_LEVELS, 0, cfr.OVERLAP_ON),
                        (cfr.EXEC_GRAPH, 0, cfr.OVERLAP_OFF), (cfr.EXEC_GRAPH, 1, cfr.OVERLAP_ON),
                        (cfr.EXEC_GRAPH, 10, cfr.OVERLAP_ON), (cfr.EXEC_GRAPH, 10, cfr.OVERLAP_OFF)):
        s = solve_gpu(g, 0, precision=cfr.P32, form=form, lanes_per_set=lanes, graph_iters=k, launch_overlap=ov,
                      order=order)
        if lanes == cfr.STREAM_LANES:
            assert cfr.cfr_export_array(s.h, "stream_ok").any()
        for n in (20, 17):
            s.iterate(n)
        s.synchronize()
        outs.append(s.get_state())
    for R, avg, t in outs[1:]:
        assert t == 37
        np.testing.assert_array_equal(R, outs[0][0])
        np.testing.assert_array_equal(avg, outs[0][1])


@pytest.mark.parametrize("order,halves", [(cfr.ORDER_SIMULTANEOUS, 1), (cfr.ORDER_ALTERNATING, 2)])
def test_launch_count_gate(order, halves):
    # one iteration is 2D - 1 kernel launches in member order (a forward and
    # a backward per depth, no forward for the deepest), twice that under
    # alternating updates; k iterations per graph are k times that; the
    # persistent form is one launch per call. (The paper's compiled
    # iteration issues 87 kernels per iteration on its turn subgame.)
    g = gg.large_card(4, 4, 1, 1)
    s = solve_gpu(g, 12, precision=cfr.P32, form=cfr.EXEC_GRAPH, order=order, graph_iters=5)
    c = s.counts_now()
    D = c["depth_blocks"]
    assert c["graph_kernels"] == halves * (2 * D - 1)
    assert c["graph_k_kernels"] == 5 * halves * (2 * D - 1)
    p = solve_gpu(g, 3, precision=cfr.P32, form=cfr.EXEC_PERSISTENT, order=order)
    assert p.counts_now()["graph_kernels"] == 0
