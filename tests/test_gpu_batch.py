"""Batched solves: one launch for many independent games (batched serving).

Checks: FP64 batched iterates equal the oracle's; a solve's result is bitwise
the same alone and inside a mix of other solves; batched exploitability
equals the single-solve evaluator; the continuous-batching server admits by
memory, overlaps arrivals with running solves, and returns for every request
exactly what solving it alone returns.
"""
import time

import numpy as np
import pytest
import torch

import gamegen as gg
import oracle
from paper_2609_11923_gb300 import cfr, serve

pytestmark = pytest.mark.gpu


def bound(specs, precision=cfr.P32, reach_order=cfr.REACH_MEMBERS, tiles=cfr.TILES_AUTO):
    opts = cfr.make_options(precision=precision, reach_order=reach_order, member_tiles=tiles)
    hs = [cfr.cfr_compile(sp, opts) for sp in specs]
    pool = serve.DevicePool(sum(cfr.cfr_plan(h) + 512 for h in hs) + 4096)
    s = int(torch.cuda.current_stream().cuda_stream)
    for h in hs:
        n = cfr.cfr_plan(h)
        cfr.cfr_bind(h, pool.ptr(pool.alloc(n)), n, s)
    tb = cfr.cfr_batch_table_bytes(len(hs))
    table = torch.empty(tb + 16, dtype=torch.uint8, device="cuda")
    return pool, hs, table, (table.data_ptr() + 15) & ~15, tb, s


def mixed_specs(n, seed0=100):
    out = []
    for i in range(n):
        out.append(gg.endgame(seed0 + i, 2000 + 3000 * (i % 5)) if i % 3 else gg.random_tree(seed0 + i, depth=7))
    return out


@pytest.mark.parametrize("reach_order,tiles", [(cfr.REACH_BFS, cfr.TILES_AUTO), (cfr.REACH_SLOTS, cfr.TILES_AUTO),
                                               (cfr.REACH_MEMBERS, cfr.TILES_AUTO), (cfr.REACH_MEMBERS, cfr.TILES_ON)])
def test_batched_fp64_matches_oracle(reach_order, tiles):
    specs = [gg.tiny_card(), gg.kuhn(), gg.endgame(5, 4000), gg.endgame(2, 100000), gg.random_tree(3, depth=8),
             gg.large_card(3, 2, 1, 1)]
    pool, hs, table, tp, tb, s = bound(specs, cfr.P64, reach_order, tiles)
    cfr.cfr_batch_iterate(hs, 300, tp, tb, 256, 4, s)
    for sp, h in zip(specs, hs):
        out = np.empty(cfr.cfr_get_counts(h)["n_slots"])
        cfr.cfr_avg_strategy(h, out, False, s)
        np.testing.assert_array_equal(out, oracle.solve(sp, 300).avg_strategy())
        cfr.cfr_destroy(h)


@pytest.mark.parametrize("rule,orule", [(cfr.RULE_PCFR_PLUS, oracle.PCFR_PLUS), (cfr.RULE_CFR, oracle.CFR)])
@pytest.mark.parametrize("order", [cfr.ORDER_SIMULTANEOUS, cfr.ORDER_ALTERNATING])
def test_batched_rules_and_orders_match_oracle(rule, orule, order):
    specs = [gg.tiny_card(), gg.endgame(5, 4000), gg.random_tree(3, depth=8)]
    opts = cfr.make_options(precision=cfr.P64, rule=rule, order=order)
    hs = [cfr.cfr_compile(sp, opts) for sp in specs]
    pool = serve.DevicePool(sum(cfr.cfr_plan(h) + 512 for h in hs) + 4096)
    s = int(torch.cuda.current_stream().cuda_stream)
    for h in hs:
        n = cfr.cfr_plan(h)
        cfr.cfr_bind(h, pool.ptr(pool.alloc(n)), n, s)
    tb = cfr.cfr_batch_table_bytes(len(hs))
    table = torch.empty(tb + 16, dtype=torch.uint8, device="cuda")
    cfr.cfr_batch_iterate(hs, 200, (table.data_ptr() + 15) & ~15, tb, 256, 4, s)
    for sp, h in zip(specs, hs):
        out = np.empty(cfr.cfr_get_counts(h)["n_slots"])
        cfr.cfr_avg_strategy(h, out, False, s)
        np.testing.assert_array_equal(out, oracle.solve(sp, 200, rule=orule, order=order).avg_strategy())
        cfr.cfr_destroy(h)


@pytest.mark.parametrize("threads,lanes", [(256, 4), (1024, 8), (256, 32), (1024, 2)])
def test_solve_alone_equals_solve_in_mix(threads, lanes):
    specs = mixed_specs(12)
    pick = [1, 5, 10]
    pool, hs, table, tp, tb, s = bound(specs)
    iters = [100 + 7 * i for i in range(len(specs))]  # uneven work in the mix
    cfr.cfr_batch_iterate(hs, 0, tp, tb, threads, lanes, s, iters=iters)
    for i in pick:
        p2, h2, t2, tp2, tb2, _ = bound([specs[i]])
        cfr.cfr_batch_iterate(h2, iters[i], tp2, tb2, threads, lanes, s)
        a = cfr.cfr_get_state(hs[i], cfr.cfr_get_counts(hs[i])["n_slots"], s)
        b = cfr.cfr_get_state(h2[0], cfr.cfr_get_counts(h2[0])["n_slots"], s)
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])
        assert a[2] == b[2] == iters[i]
        cfr.cfr_destroy(h2[0])
    for h in hs:
        cfr.cfr_destroy(h)


def test_batched_exploitability_equals_single():
    specs = mixed_specs(8, seed0=300) + [gg.endgame(2, 100000)]
    pool, hs, table, tp, tb, s = bound(specs, cfr.P64)
    cfr.cfr_batch_iterate(hs, 120, tp, tb, 256, 4, s)
    ex = cfr.cfr_batch_exploitability(hs, tp, tb, 256, 4, s)
    for row, h in zip(ex, hs):
        single = cfr.cfr_exploitability(h, s)
        np.testing.assert_allclose(row, single, rtol=0, atol=1e-10)
        cfr.cfr_destroy(h)


def test_batched_fp32_reaches_oracle_exploitability():
    specs = [gg.endgame(11, 20000), gg.endgame(12, 5000), gg.random_tree(13, depth=9)]
    pool, hs, table, tp, tb, s = bound(specs, cfr.P32)
    cfr.cfr_batch_iterate(hs, 1000, tp, tb, 256, 4, s)
    ex = cfr.cfr_batch_exploitability(hs, tp, tb, 256, 4, s)
    for sp, row, h in zip(specs, ex, hs):
        assert abs(row[0] - oracle.solve(sp, 1000).exploitability()) <= 1e-4 * sp.pot
        cfr.cfr_destroy(h)


def test_server_continuous_batching_results_equal_alone():
    rng = np.random.default_rng(0)
    specs = [gg.endgame(400 + i, int(rng.integers(1000, 20000))) for i in range(16)]
    arrivals = np.cumsum(rng.exponential(0.01, size=len(specs)))
    reqs = [serve.Request(i, sp, float(t)) for i, (sp, t) in enumerate(zip(specs, arrivals))]
    # a pool for about four solves at a time: admission is limited by memory
    hs0 = [cfr.cfr_compile(sp) for sp in specs]
    sizes = sorted(cfr.cfr_plan(h) for h in hs0)
    for h in hs0:
        cfr.cfr_destroy(h)
    # requests of 8,000 edges or more run as 4-CTA clusters on the side stream
    srv = serve.Server(pool_bytes=4 * sizes[-1] + 4096, max_active=64, check_every=50, max_iters=600,
                       target=1e-3, keep_strategies=True, big_edges=8000, cluster=4)
    res = srv.serve(reqs)
    srv.close()
    assert sorted(r.rid for r in res) == list(range(len(specs)))
    assert srv.rounds > 1
    assert 0 < sum(srv.is_big(sp) for sp in specs) < len(specs)  # both launch kinds ran
    for r in res:
        assert r.finished >= r.admitted >= r.arrival - 1e-9
        assert r.exploitability <= 1e-3 * r.pot or r.iterations == 600
        # the same solve alone, same iteration count and launch shape
        p2, h2, t2, tp2, tb2, s = bound([specs[r.rid]])
        if srv.is_big(specs[r.rid]):
            cfr.cfr_batch_iterate(h2, r.iterations, tp2, tb2, srv.big_threads, srv.big_lanes, s, cluster=srv.cluster)
        else:
            cfr.cfr_batch_iterate(h2, r.iterations, tp2, tb2, srv.threads, srv.lanes, s)
        alone = np.empty(len(r.strategy))
        cfr.cfr_avg_strategy(h2[0], alone, False, s)
        np.testing.assert_array_equal(r.strategy, alone)
        cfr.cfr_destroy(h2[0])


@pytest.mark.parametrize("cluster", [2, 8])
def test_clustered_fp64_matches_oracle(cluster):
    # a wide deal root (summed by the cluster's first CTA), a deep random tree
    # and card games, each instance shared by `cluster` CTAs
    specs = [gg.endgame(2, 100000), gg.random_tree(3, depth=10), gg.large_card(3, 2, 1, 1), gg.tiny_card()]
    pool, hs, table, tp, tb, s = bound(specs, cfr.P64)
    cfr.cfr_batch_iterate(hs, 120, tp, tb, 1024, 8, s, cluster=cluster)
    for sp, h in zip(specs, hs):
        out = np.empty(cfr.cfr_get_counts(h)["n_slots"])
        cfr.cfr_avg_strategy(h, out, False, s)
        np.testing.assert_array_equal(out, oracle.solve(sp, 120).avg_strategy())
        cfr.cfr_destroy(h)


def test_clustered_fp32_alone_equals_in_mix():
    specs = mixed_specs(9, seed0=300)
    pool, hs, table, tp, tb, s = bound(specs)
    iters = [80 + 11 * i for i in range(len(specs))]
    cfr.cfr_batch_iterate(hs, 0, tp, tb, 256, 8, s, iters=iters, cluster=4)
    for i in (0, 4, 8):
        p2, h2, t2, tp2, tb2, _ = bound([specs[i]])
        cfr.cfr_batch_iterate(h2, iters[i], tp2, tb2, 256, 8, s, cluster=4)
        a = np.empty(cfr.cfr_get_counts(hs[i])["n_slots"])
        b = np.empty_like(a)
        cfr.cfr_avg_strategy(hs[i], a, False, s)
        cfr.cfr_avg_strategy(h2[0], b, False, s)
        np.testing.assert_array_equal(a, b)
        cfr.cfr_destroy(h2[0])
    for h in hs:
        cfr.cfr_destroy(h)


def test_cluster_size_is_checked():
    pool, hs, table, tp, tb, s = bound([gg.tiny_card()])
    with pytest.raises(cfr.CfrError):
        cfr.cfr_batch_iterate(hs, 1, tp, tb, 256, 4, s, cluster=3)
    cfr.cfr_destroy(hs[0])


def test_server_rejects_a_request_larger_than_the_pool_and_serves_the_rest():
    # the admission check answers a request that can never fit at once
    # (it used to wait forever for memory that would never free up)
    small = [gg.endgame(500 + i, 3000) for i in range(4)]
    big = gg.endgame(600, 400000)
    hs0 = [cfr.cfr_compile(sp) for sp in small + [big]]
    sizes = [cfr.cfr_plan(h) for h in hs0]
    for h in hs0:
        cfr.cfr_destroy(h)
    pool = 2 * max(sizes[:4]) + 4096
    assert sizes[4] > pool
    reqs = [serve.Request(i, sp, 0.0) for i, sp in enumerate(small)] + [serve.Request(99, big, 0.0)]
    srv = serve.Server(pool_bytes=pool, max_active=8, check_every=50, max_iters=300, cluster=1)
    res = {r.rid: r for r in srv.serve(reqs)}
    srv.close()
    assert res[99].status == "rejected" and "exceeds" in res[99].message and res[99].iterations == 0
    for i in range(4):
        assert res[i].status in ("solved", "capped") and res[i].iterations > 0


def test_server_cancels_queued_and_active_requests_between_rounds():
    specs = [gg.endgame(700 + i, 4000) for i in range(6)]
    reqs = [serve.Request(i, sp, 0.0) for i, sp in enumerate(specs)]
    reqs.append(serve.Request(50, gg.endgame(750, 4000), 30.0))  # arrives long after: cancelled while queued

    def on_round(srv, active):
        if srv.rounds == 2:
            srv.cancel(1)  # active: retired at this round boundary
            srv.cancel(50)  # not yet arrived

    srv = serve.Server(pool_bytes=1 << 28, max_active=8, check_every=20, max_iters=400, target=1e-9,
                       keep_strategies=True, cluster=1, on_round=on_round)
    t = time.perf_counter()
    res = {r.rid: r for r in srv.serve(reqs)}
    srv.close()
    assert time.perf_counter() - t < 25.0  # did not wait for the cancelled arrival
    assert res[1].status == "cancelled" and res[1].iterations == 40
    assert res[50].status == "cancelled" and res[50].iterations == 0
    for i in (0, 2, 3, 4, 5):
        assert res[i].status == "capped" and res[i].iterations == 400
    # the cancelled solve left the others untouched: each equals its solve alone
    for i in (0, 2):
        p2, h2, t2, tp2, tb2, s = bound([specs[i]])
        cfr.cfr_batch_iterate(h2, 400, tp2, tb2, srv.threads, srv.lanes, s)
        alone = np.empty(len(res[i].strategy))
        cfr.cfr_avg_strategy(h2[0], alone, False, s)
        np.testing.assert_array_equal(res[i].strategy, alone)
        cfr.cfr_destroy(h2[0])


def test_server_answers_an_invalid_spec_with_an_error_result():
    bad = gg.from_lists([(gg.P1, 0, [1, 2], None, 0.0), (gg.TERMINAL, -1, [], None, 1.0),
                         (gg.TERMINAL, -1, [], None, -1.0)], [(0, 3)])  # 2 children, set says 3 actions
    reqs = [serve.Request(0, bad, 0.0), serve.Request(1, gg.endgame(800, 3000), 0.0)]
    srv = serve.Server(pool_bytes=1 << 26, max_active=4, check_every=50, max_iters=100, cluster=1)
    res = {r.rid: r for r in srv.serve(reqs)}
    srv.close()
    assert res[0].status == "error" and "CFR_ERR_INVALID_SPEC" in res[0].message
    assert res[1].status in ("solved", "capped")
