"""Host compiler: bit-exact arrays against an independent flattener, the
compile invariants of the paper (tree coverage, parent depth < child depth,
D = number of parent depths), validation errors, and the C-ABI surface.
CPU only: nothing here launches a kernel."""
import ctypes
import dataclasses
import os
import re

import numpy as np
import pytest

import gamegen as gg
from paper_2609_11923_gb300 import cfr
from tests.flatten_ref import flatten

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

GAMES = {
    "kuhn": lambda: gg.kuhn(),
    "leduc": lambda: gg.leduc(),
    "tiny": lambda: gg.tiny_card(),
    "rt6": lambda: gg.random_tree(1, depth=6),
    "rt8": lambda: gg.random_tree(2, depth=8, max_group=16),
    "endgame": lambda: gg.endgame(3, 3000),
    "card_small": lambda: gg.large_card(3, 2, 1, 1),
    "wide_root": lambda: gg.endgame(2, 100000),
}


@pytest.mark.parametrize("reach_order,tiles", [(cfr.REACH_BFS, cfr.TILES_AUTO), (cfr.REACH_SLOTS, cfr.TILES_AUTO),
                                               (cfr.REACH_MEMBERS, cfr.TILES_AUTO), (cfr.REACH_MEMBERS, cfr.TILES_ON),
                                               (cfr.REACH_MEMBERS, cfr.TILES_OFF)])
@pytest.mark.parametrize("name", list(GAMES))
def test_arrays_bit_exact(name, reach_order, tiles):
    g = GAMES[name]()
    ref = flatten(g, reach_order, tiles)
    h = cfr.cfr_compile(g, cfr.make_options(reach_order=reach_order, member_tiles=tiles))
    try:
        for key in cfr.EXPORT:
            if key in ("level_lanes", "pull_grid"):  # runtime choices, not compiled arrays
                continue
            if key == "set_info" or key.startswith("stream_"):  # derived from these arrays (test_stream_layout)
                continue
            got = cfr.cfr_export_array(h, key)
            np.testing.assert_array_equal(got, ref[key], err_msg=key)
        assert cfr.cfr_get_counts(h)["depth_blocks"] == ref["D"]
    finally:
        cfr.cfr_destroy(h)


def test_relabelled_spec_compiles_to_the_same_arrays():
    g = gg.tiny_card()
    rng = np.random.default_rng(0)
    perm = np.concatenate([[0], 1 + rng.permutation(g.n_nodes - 1)])
    h1, h2 = cfr.cfr_compile(g), cfr.cfr_compile(gg.permute_nodes(g, perm))
    try:
        for key in ("child_begin", "node_slot", "iset_slot", "iset_mem", "mem_node", "tmpl", "spec_slot_of"):
            np.testing.assert_array_equal(cfr.cfr_export_array(h1, key), cfr.cfr_export_array(h2, key))
    finally:
        cfr.cfr_destroy(h1)
        cfr.cfr_destroy(h2)


@pytest.mark.parametrize("name", ["tiny", "rt8", "card_small"])
def test_compile_invariants(name):
    g = GAMES[name]()
    h = cfr.cfr_compile(g)
    try:
        cb = cfr.cfr_export_array(h, "child_begin")
        lb = cfr.cfr_export_array(h, "level_begin")
        N = g.n_nodes
        # every non-root node is written by exactly one forward edge (coverage)
        cover = np.zeros(N, dtype=int)
        for v in range(N):
            cover[cb[v]:cb[v + 1]] += 1
        assert cover[0] == 0 and (cover[1:] == 1).all()
        # parents live one level above their children
        depth = np.searchsorted(lb, np.arange(N), side="right") - 1
        for v in range(N):
            if cb[v + 1] > cb[v]:
                assert (depth[cb[v]:cb[v + 1]] == depth[v] + 1).all()
        # the template carries each terminal's full chance product exactly once
        # (Prop. 1): with payoff 1 everywhere, folding values back up with
        # chance edges as multiplier 1 and any strategy gives root value 1
        ones = np.where(g.kind == gg.TERMINAL, 1.0, 0.0)
        h1 = cfr.cfr_compile(_bad(g, payoff=ones))
        try:
            tm = cfr.cfr_export_array(h1, "tmpl")
            slot = cfr.cfr_export_array(h1, "node_slot")
            v = tm.copy()
            for x in range(N - 1, -1, -1):
                if cb[x + 1] > cb[x]:
                    kids = v[cb[x]:cb[x + 1]]
                    v[x] = kids.sum() if slot[x] < 0 else kids.mean()
            assert v[0] == pytest.approx(1.0, abs=1e-12)
        finally:
            cfr.cfr_destroy(h1)
    finally:
        cfr.cfr_destroy(h)


def test_template_is_chance_times_payoff_on_kuhn():
    g = gg.kuhn()
    h = cfr.cfr_compile(g)
    try:
        tm = cfr.cfr_export_array(h, "tmpl")
        new = cfr.cfr_export_array(h, "new_of_spec")
        term = np.nonzero(g.kind == gg.TERMINAL)[0]
        np.testing.assert_array_equal(tm[new[term]], g.payoff[term] * (1.0 / 6.0))
    finally:
        cfr.cfr_destroy(h)


def _bad(g, **changes):
    kw = dict(kind=g.kind.copy(), infoset=g.infoset.copy(), child_begin=g.child_begin.copy(),
              child=g.child.copy(), chance_prob=g.chance_prob.copy(), payoff=g.payoff.copy(),
              iset_player=g.iset_player.copy(), iset_nact=g.iset_nact.copy(), pot=g.pot)
    kw.update(changes)
    return gg.GameSpec(**kw)


def test_invalid_specs_are_rejected():
    g = gg.kuhn()
    child = g.child.copy()
    child[3] = child[2]  # a node with two parents
    cases = [
        _bad(g, child=child),
        _bad(g, chance_prob=g.chance_prob * 0.5),                # probabilities do not sum to 1
        _bad(g, iset_player=1 - g.iset_player),                  # set owned by the other player
        _bad(g, iset_nact=g.iset_nact + 1),                      # action count mismatch
        _bad(g, payoff=np.where(g.kind == gg.TERMINAL, np.nan, 0.0)),
    ]
    for bad in cases:
        with pytest.raises(cfr.CfrError) as ei:
            cfr.cfr_compile(bad)
        assert ei.value.code == -2


def test_members_at_different_depths_are_rejected():
    # P1 set 0 has members at depths 0 and 2
    spec = gg.from_lists(
        [
            (gg.P1, 0, [1, 2], None, 0.0),
            (gg.TERMINAL, -1, [], None, 1.0),
            (gg.P2, 1, [3, 4], None, 0.0),
            (gg.P1, 0, [5, 6], None, 0.0),
            (gg.TERMINAL, -1, [], None, 0.0),
            (gg.TERMINAL, -1, [], None, 2.0),
            (gg.TERMINAL, -1, [], None, -1.0),
        ],
        [(0, 2), (1, 2)],
    )
    with pytest.raises(cfr.CfrError) as ei:
        cfr.cfr_compile(spec)
    assert "depth" in str(ei.value)


def test_calls_before_bind_report_not_bound():
    # every call that needs device memory refuses before cfr_bind, without
    # touching the device (host-side check)
    g = gg.kuhn()
    h = cfr.cfr_compile(g)
    A = cfr.cfr_get_counts(h)["n_slots"]
    z = np.zeros(A)
    calls = {
        "iterate": lambda: cfr.cfr_iterate(h, 1, 0),
        "iterate_noalloc": lambda: cfr.cfr_iterate_noalloc(h, 1, 0),
        "synchronize": lambda: cfr.cfr_synchronize(h, 0),
        "avg_strategy": lambda: cfr.cfr_avg_strategy(h, np.empty(A), False, 0),
        "current_strategy": lambda: cfr.cfr_current_strategy(h, np.empty(A), False, 0),
        "exploitability": lambda: cfr.cfr_exploitability(h, 0),
        "reset": lambda: cfr.cfr_reset(h, 0),
        "set_payoffs": lambda: cfr.cfr_set_payoffs(h, np.zeros(g.n_nodes), 0),
        "get_state": lambda: cfr.cfr_get_state(h, A, 0),
        "set_state": lambda: cfr.cfr_set_state(h, z, z, 0, 0),
        "autotune": lambda: cfr.cfr_autotune(h, 1, 0),
        "launch_floor": lambda: cfr.cfr_launch_floor(h, 1, 0),
        "profile_iteration": lambda: cfr.cfr_profile_iteration(h, cfr.cfr_get_counts(h)["depth_blocks"], 0),
        "batch_iterate": lambda: cfr.cfr_batch_iterate([h], 1, 4096, 4096),
        "batch_exploitability": lambda: cfr.cfr_batch_exploitability([h], 4096, 4096),
    }
    try:
        for name, call in calls.items():
            with pytest.raises(cfr.CfrError) as ei:
                call()
            assert ei.value.code == cfr.CFR_ERR_NOT_BOUND, name
        assert cfr.cfr_plan(h) > 0
    finally:
        cfr.cfr_destroy(h)


def test_bind_refuses_a_small_or_misaligned_arena_before_touching_it():
    # both checks come before any device access: the pointers below are
    # never dereferenced
    h = cfr.cfr_compile(gg.kuhn())
    try:
        need = cfr.cfr_plan(h)
        with pytest.raises(cfr.CfrError) as ei:
            cfr.cfr_bind(h, 1 << 20, need - 1, 0)
        assert ei.value.code == cfr.CFR_ERR_ARENA_SMALL and str(need) in str(ei.value)
        with pytest.raises(cfr.CfrError) as ei:
            cfr.cfr_bind(h, (1 << 20) + 16, need, 0)
        assert ei.value.code == cfr.CFR_ERR_ARG and "aligned" in str(ei.value)
        with pytest.raises(cfr.CfrError) as ei:  # still unbound afterwards
            cfr.cfr_iterate(h, 1, 0)
        assert ei.value.code == cfr.CFR_ERR_NOT_BOUND
    finally:
        cfr.cfr_destroy(h)


def test_bad_options_are_rejected():
    with pytest.raises(cfr.CfrError):
        cfr.cfr_compile(gg.kuhn(), cfr.make_options(precision=7))
    with pytest.raises(cfr.CfrError):
        cfr.cfr_compile(gg.kuhn(), cfr.make_options(lanes_per_set=3))


def test_library_exports_every_declared_symbol():
    header = open(os.path.join(ROOT, "include", "cfr.h")).read()
    names = set(re.findall(r"^\s*(?:int|void|size_t|const char \*)\s*\**\s*(cfr_\w+)\s*\(", header, re.M))
    assert {"cfr_compile", "cfr_iterate", "cfr_avg_strategy", "cfr_exploitability"} <= names
    lib = ctypes.CDLL(cfr.LIB_PATH)
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert names <= set(cfr.EXPORTED)


def test_library_exports_every_mlp_symbol():
    header = open(os.path.join(ROOT, "include", "mlp.h")).read()
    names = set(re.findall(r"^\s*(?:int|void)\s+(mlp_\w+)\s*\(", header, re.M))
    assert {"mlp_gemm", "mlp_softmax_xent", "mlp_relu_grad", "mlp_colsum", "mlp_adam", "mlp_to_bf16"} <= names
    lib = ctypes.CDLL(cfr.LIB_PATH)
    for n in sorted(names):
        assert hasattr(lib, n), n


def with_root_chance(g, p):
    """The same game with the root's outcome probabilities replaced."""
    cp = np.array(g.chance_prob, dtype=np.float64, copy=True)
    cp[g.child_begin[0]:g.child_begin[1]] = p
    return dataclasses.replace(g, chance_prob=cp, _owner=None,
                               **{f: np.array(getattr(g, f), copy=True) for f in
                                  ("kind", "infoset", "child_begin", "child", "payoff", "iset_player", "iset_nact")})


@pytest.mark.parametrize("name", ["endgame", "card_small", "tiny"])
def test_set_root_chance_gives_the_template_of_a_fresh_compile(name):
    g = GAMES[name]()
    n = int(g.child_begin[1] - g.child_begin[0])
    p = np.random.default_rng(3).dirichlet(np.ones(n))
    h1, h2 = cfr.cfr_compile(g), cfr.cfr_compile(with_root_chance(g, p))
    try:
        cfr.cfr_set_root_chance(h1, p)
        for key in ("tmpl", "tmpl_vs"):
            np.testing.assert_array_equal(cfr.cfr_export_array(h1, key), cfr.cfr_export_array(h2, key))
        with pytest.raises(cfr.CfrError):
            cfr.cfr_set_root_chance(h1, p[:-1])  # wrong count
        q = p.copy()
        q[0] = -0.1
        with pytest.raises(cfr.CfrError):
            cfr.cfr_set_root_chance(h1, q)
    finally:
        cfr.cfr_destroy(h1)
        cfr.cfr_destroy(h2)


def test_set_root_chance_needs_a_chance_root():
    g = gg.random_tree(11, depth=5, p_chance=0.0)  # decision root
    h = cfr.cfr_compile(g)
    try:
        with pytest.raises(cfr.CfrError) as ei:
            cfr.cfr_set_root_chance(h, np.ones(int(g.child_begin[1] - g.child_begin[0])))
        assert "not a chance node" in str(ei.value)
    finally:
        cfr.cfr_destroy(h)


@pytest.mark.parametrize("reach_order", [cfr.REACH_MEMBERS, cfr.REACH_BFS, cfr.REACH_SLOTS])
@pytest.mark.parametrize("precision", [cfr.P32, cfr.P64])
@pytest.mark.parametrize("name", ["tiny", "rt8", "card_small", "wide_root"])
def test_iteration_bytes_are_the_sum_of_the_launches(name, reach_order, precision):
    # the per-iteration algorithmic bytes (roofline numerator of the whole
    # iteration) and the per-depth launch bytes count the same accesses
    h = cfr.cfr_compile(GAMES[name](), cfr.make_options(precision=precision, reach_order=reach_order))
    try:
        c = cfr.cfr_get_counts(h)
        per_launch = [cfr.cfr_level_bytes(h, d) for d in range(c["depth_blocks"])]
        assert c["algo_bytes_per_iter"] == sum(f + b for f, b in per_launch)
        if reach_order == cfr.REACH_MEMBERS:  # the deepest depth has no forward launch
            assert per_launch[-1][0] == 0
            # the pull of depth d: edge records and own reach of depth d + 1's
            # internal nodes, the reach of their distinct parents, the σ of
            # depth d's slots (recounted here from the exported arrays)
            T = 4 if precision == cfr.P32 else 8
            li = cfr.cfr_export_array(h, "level_int").astype(int)
            ie = cfr.cfr_export_array(h, "int_edge").astype(int).reshape(-1, 2)
            isl, lis = cfr.cfr_export_array(h, "iset_slot").astype(int), cfr.cfr_export_array(h, "level_iset").astype(int)
            for d in range(c["depth_blocks"] - 1):
                kids = li[d + 2] - li[d + 1]
                parents = len(set(ie[li[d + 1]:li[d + 2], 0].tolist()) - {-1})
                slots = isl[lis[2 * d + 2]] - isl[lis[2 * d]]
                assert per_launch[d][0] == 8 * kids + 2 * T * parents + 2 * T * kids + T * slots, d
    finally:
        cfr.cfr_destroy(h)


@pytest.mark.parametrize("tiles", [cfr.TILES_AUTO, cfr.TILES_ON])
@pytest.mark.parametrize("name", ["tiny", "rt8", "card_small", "endgame", "wide_root"])
def test_member_order_layout_properties(name, tiles):
    # what the member-order kernels rely on, checked against the tree itself
    # (not against a second flattener): a set's members sit at ranks
    # base + k * stride (stride 4 inside a tile of four consecutive sets with
    # equal member counts, else 1) within their depth's rank
    # range; every internal node's edge names its parent's rank and the
    # parent's slot + action (-1 under chance); ranks are one permutation
    h = cfr.cfr_compile(GAMES[name](), cfr.make_options(member_tiles=tiles))
    try:
        ex = lambda k: cfr.cfr_export_array(h, k).astype(np.int64)
        cb, ns, lb = ex("child_begin"), ex("node_slot"), ex("level_begin")
        im, mn, li, lint = ex("iset_mem"), ex("mem_node"), ex("level_iset"), ex("level_int")
        edge, irk = ex("int_edge").reshape(-1, 2), ex("iset_rank").reshape(-1, 2)
        N, D = len(ns), len(lint) - 1
        internal = np.nonzero(cb[1:] > cb[:-1])[0]
        assert len(edge) == len(internal) == lint[D]
        parent = np.full(N, -1)
        for x in range(N):
            parent[cb[x]:cb[x + 1]] = x
        depth = np.searchsorted(lb, np.arange(N), side="right") - 1
        rank = np.full(N, -1)
        for I in range(len(im) - 1):
            assert irk[I, 1] in (1, 4)
            k = np.arange(im[I], im[I + 1])
            rank[mn[k]] = irk[I, 0] + (k - im[I]) * irk[I, 1]
            d = depth[mn[im[I]]]
            assert np.all((rank[mn[k]] >= lint[d]) & (rank[mn[k]] < lint[d + 1]))
        # chance nodes above a ranked node: their rank is that node's parent rank
        for d in range(D - 1, 0, -1):
            for x in internal[(depth[internal] == d) & (rank[internal] >= 0)]:
                p = parent[x]
                if rank[p] < 0:
                    rank[p] = edge[rank[x], 0]
                assert edge[rank[x], 0] == rank[p]
        known = internal[rank[internal] >= 0]
        assert len(set(rank[known].tolist())) == len(known)  # no two nodes share a rank
        for x in known:
            p = parent[x]
            if p < 0:
                assert tuple(edge[rank[x]]) == (-1, -1)
            else:
                assert edge[rank[x], 0] == rank[p]
                assert edge[rank[x], 1] == (-1 if ns[p] < 0 else ns[p] + (x - cb[p]))
        # the rest (chance nodes with no internal child) fill the free ranks
        # of their depth, and those ranks' edges name their parents
        rest = internal[rank[internal] < 0]
        free = np.setdiff1d(np.arange(len(internal)), rank[known])
        assert len(free) == len(rest)
        assert sorted(depth[rest].tolist()) == sorted((np.searchsorted(lint, free, side="right") - 1).tolist())
        assert sorted(edge[free, 0].tolist()) == sorted(rank[parent[rest]].tolist())
        # tiles: four consecutive sets, consecutive bases, equal member counts
        for I in range(len(im) - 1):
            if irk[I, 1] == 4 and (I == 0 or irk[I - 1, 1] != 4 or irk[I, 0] != irk[I - 1, 0] + 1):
                group = list(range(I, I + 4))
                assert [irk[j, 0] for j in group] == [irk[I, 0] + j for j in range(4)]
                assert len({im[j + 1] - im[j] for j in group}) == 1
    finally:
        cfr.cfr_destroy(h)


def test_binding_constants_mirror_the_header():
    # every enumerator of include/cfr.h has the same value in the Python
    # binding (options, node kinds, status codes), and the options struct has
    # the header's fields in the header's order
    header = open(os.path.join(ROOT, "include", "cfr.h")).read()
    header = re.sub(r"/\*.*?\*/", "", header, flags=re.S)
    values = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", header, re.S):
        for name, val in re.findall(r"(CFR_\w+)\s*=\s*(-?\d+)", body):
            values[name] = int(val)
    py = {"CFR_P64": cfr.P64, "CFR_P32": cfr.P32, "CFR_OK": cfr.CFR_OK,
          "CFR_DEBUG_BARRIER_MISSING_ARRIVALS": cfr.DEBUG_BARRIER_MISSING_ARRIVALS,
          "CFR_DEBUG_FAIL_GRAPH_CAPTURE": cfr.DEBUG_FAIL_GRAPH_CAPTURE,
          "CFR_DEBUG_STREAM_STALL": cfr.DEBUG_STREAM_STALL}
    py.update({"CFR_OVERLAP_AUTO": cfr.OVERLAP_AUTO, "CFR_OVERLAP_ON": cfr.OVERLAP_ON, "CFR_OVERLAP_OFF": cfr.OVERLAP_OFF})
    for prefix in ("EXEC_", "RULE_", "ORDER_", "REACH_", "TILES_"):
        py.update({"CFR_" + n: getattr(cfr, n) for n in dir(cfr) if n.startswith(prefix)})
    py.update({name: code for code, name in cfr.ERRORS.items()})
    kinds = {"CFR_TERMINAL": gg.TERMINAL, "CFR_CHANCE": gg.CHANCE, "CFR_PLAYER1": gg.P1, "CFR_PLAYER2": gg.P2}
    py.update(kinds)
    assert set(values) == set(py), set(values) ^ set(py)
    for name, v in values.items():
        assert py[name] == v, name
    for cname, pyclass in (("cfr_options", cfr.Options), ("cfr_counts", cfr.Counts), ("cfr_game_spec", cfr.GameSpecC)):
        body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (cname, cname), header, re.S).group(1)
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if decl:  # "type a, b" or "const type *a"
                names = decl.split(None, 1)[1] if not decl.startswith("const") else decl.split(None, 2)[2]
                fields += [n.strip(" *") for n in names.split(",")]
        assert fields == [f[0] for f in pyclass._fields_], cname
        assert ctypes.sizeof(pyclass) >= 4 * len(fields)


def test_auto_picks_the_form_by_the_measured_crossover():
    # the persistent form up to 768 nodes in FP32 and 350 in FP64 (where it
    # was measured faster than graph replay), graph replay above
    cases = [(gg.tiny_card(), cfr.P32, cfr.EXEC_PERSISTENT), (gg.tiny_card(), cfr.P64, cfr.EXEC_PERSISTENT),
             (gg.random_tree(3, depth=6), cfr.P32, cfr.EXEC_PERSISTENT),
             (gg.random_tree(3, depth=6), cfr.P64, cfr.EXEC_GRAPH),
             (gg.random_tree(3, depth=7), cfr.P32, cfr.EXEC_GRAPH)]
    for g, prec, form in cases:
        h = cfr.cfr_compile(g, cfr.make_options(precision=prec, exec_form=cfr.EXEC_AUTO))
        try:
            assert cfr.cfr_get_counts(h)["exec_form"] == form, (g.n_nodes, prec)
        finally:
            cfr.cfr_destroy(h)
