"""The compiled layouts compute CFR+ exactly (CPU only).

A plain-Python FP64 run of the kernels' scheme over the exported arrays (in
member order the pulling forward over the internal nodes' edges and the
backward over the sets' rank bases and strides; in breadth-first and
value-slot order the pushing forward over the internal-node records and the
backward over the rank table; value blocks and value slots in all) with the
kernels' summation order must reach the oracle's cumulative regrets and
average sums bitwise. This checks the layouts without a GPU and
independently of the kernels' code.
"""
import numpy as np
import pytest

import gamegen as gg
import oracle
from paper_2609_11923_gb300 import cfr

P2BIT = 1 << 30
MASK = P2BIT - 1

GAMES = {
    "kuhn": lambda: gg.kuhn(),
    "leduc": lambda: gg.leduc(),
    "tiny": lambda: gg.tiny_card(),
    "rt6": lambda: gg.random_tree(1, depth=6),
    "card_small": lambda: gg.large_card(3, 2, 1, 1),
    "endgame": lambda: gg.endgame(3, 3000),
    "wide_root": lambda: gg.endgame(2, 100000),  # a deal root of more than 1,024 outcomes
}


def emulate(h, iters, rule=oracle.CFR_PLUS, order=oracle.SIMULTANEOUS, stream=False):
    """stream: at the depths that can stream, the set passes read everything
    from per-chunk copies of the staged ranges, with the streaming kernel's
    index arithmetic (an index outside a staged range raises)."""
    ex = lambda k: cfr.cfr_export_array(h, k)
    lint, edge = ex("level_int").astype(int), ex("int_edge").astype(int).reshape(-1, 2)
    isl, im, ivb, li = ex("iset_slot").astype(int), ex("iset_mem").astype(int), ex("iset_vb").astype(int), \
        ex("level_iset").astype(int)
    irk, mvs = ex("iset_rank").astype(int).reshape(-1, 2), ex("mem_vs").astype(int)
    chb, chn, chs, lch = ex("ch_vb").astype(int), ex("ch_nch").astype(int), ex("ch_vs").astype(int), \
        ex("level_chance").astype(int)
    wvb, wn, wvs = ex("wide_vb").astype(int), ex("wide_nch").astype(int), ex("wide_vs").astype(int)
    lb, vslot = ex("level_begin").astype(int), ex("vslot").astype(int)
    members = len(ex("int_edge")) > 0
    if not members:
        islot, imask, icr = ex("int_slot").astype(int), ex("int_mask").view(np.uint32).astype(np.int64), \
            ex("int_cirank").astype(int)
        big, mirk = ex("big_irank").astype(int), ex("mem_irank").astype(int)
    v = [float(x) for x in ex("tmpl_vs")]
    D, I, A = len(lint) - 1, len(isl) - 1, int(isl[-1])
    node_of_slot = np.empty(len(vslot), dtype=int)
    node_of_slot[vslot] = np.arange(len(vslot))
    wide_depth = np.searchsorted(lb, node_of_slot[wvs], side="right") - 1 if len(wvs) else []
    if stream:
        sinfo = ex("set_info").astype(int).reshape(-1, 8)
        chunks = ex("stream_chunks").astype(int).reshape(-1, 16)
        sc0, sok = ex("stream_c0").astype(int), ex("stream_ok").astype(int)
    sigma = [0.0] * A
    for s in range(I):
        for a in range(isl[s], isl[s + 1]):
            sigma[a] = 1.0 / (isl[s + 1] - isl[s])
    R, avg = [0.0] * A, [0.0] * A
    reach = [[0.0, 0.0] for _ in range(lint[D])]

    def child_reach(r, s, a):
        r = list(r)
        if s >= 0:
            lane = 1 if s & P2BIT else 0
            r[lane] = r[lane] * sigma[(s & MASK) + a]
        return r

    def forward():
        reach[0] = [1.0, 1.0]
        if members:
            for d in range(D - 1):  # the launch of depth d pulls depth d + 1
                for q in range(lint[d + 1], lint[d + 2]):
                    p, s = edge[q]
                    reach[q] = child_reach(reach[p], s, 0)
            return
        for q in range(lint[D]):  # every parent pushes to its internal children
            s, m, c = islot[q], int(imask[q]), icr[q]
            if m & (1 << 31):  # listed children (-1: terminal)
                for a in range(big[c]):
                    if big[c + 1 + a] >= 0:
                        reach[big[c + 1 + a]] = child_reach(reach[q], s, a)
                continue
            a = 0
            while m:
                if m & 1:
                    reach[c] = child_reach(reach[q], s, a)
                    c += 1
                m >>= 1
                a += 1

    def chance_sums(d):
        if d == 0:  # the root's value is not needed
            return
        if stream and sok[d]:
            # the streaming kernel's chance chunks: each node summed from
            # its chunk's staged copies of the children's values and of the
            # chance arrays, with the kernel's index arithmetic
            for k in chunks[sc0[d]:sc0[d + 1]]:
                if k[10] != 1:
                    continue
                I0, I1, va, nva, ka, nka = k[0], k[1], k[4], k[5], k[6], k[7]
                sv = staged(v, va, nva, float("nan"))
                svb, snc, svs = staged(list(chb), ka, nka, -1), staged(list(chn), ka, nka, -1), \
                    staged(list(chs), ka, nka, -1)
                for i in range(I0, I1):
                    q = i - ka
                    p0 = svb[q] - va
                    assert 0 <= p0 and p0 + snc[q] <= nva
                    acc = 0.0
                    for c in range(p0, p0 + snc[q]):
                        acc = acc + sv[c]
                    v[svs[q]] = acc
        else:
            for i in range(lch[d], lch[d + 1]):
                acc = 0.0
                for c in range(chb[i], chb[i] + chn[i]):
                    acc = acc + v[c]
                v[chs[i]] = acc
        for i in range(len(wvs)):
            if wide_depth[i] == d:
                acc = 0.0
                for c in range(wvb[i], wvb[i] + wn[i]):
                    acc = acc + v[c]
                v[wvs[i]] = acc

    def set_pass(s, d, t, upd):
        p2 = s >= li[2 * d + 1]
        sb, na = isl[s], isl[s + 1] - isl[s]
        sig = sigma[sb:sb + na]
        racc, macc = [0.0] * na, [0.0] * na
        for k in range(im[s], im[s + 1]):
            r = reach[irk[s, 0] + (k - im[s]) * irk[s, 1]] if members else reach[mirk[k]]
            cb, M = ivb[s] + (k - im[s]), im[s + 1] - im[s]  # child a at cb + a * M
            vh = 0.0
            for a in range(na):
                vh = vh + sig[a] * v[cb + a * M]
            v[mvs[k]] = vh
            po, pw = (r[0], r[1]) if p2 else (r[1], r[0])
            f = (-1.0 if p2 else 1.0) * po
            for a in range(na):
                racc[a] = racc[a] + f * (v[cb + a * M] - vh)
                macc[a] = macc[a] + pw * sig[a]
        if (2 if p2 else 1) not in upd:  # the other player's sets only pass values up
            return
        w = float(t) * float(t) if rule == oracle.PCFR_PLUS else float(t)
        pos = []
        for a in range(na):
            rn = R[sb + a] + racc[a]
            if rule != oracle.CFR:
                rn = rn if rn > 0.0 else 0.0
            R[sb + a] = rn
            avg[sb + a] = avg[sb + a] + w * macc[a]
            x = rn + racc[a] if rule == oracle.PCFR_PLUS else rn
            pos.append(x if x > 0.0 else 0.0)
        tot = 0.0
        for a in range(na):
            tot = tot + pos[a]
        for a in range(na):
            sigma[sb + a] = pos[a] / tot if tot > 0.0 else 1.0 / na

    def staged(arr, start, count, pad):
        """A copy of arr[start:start+count], the part past the end filled
        with pad (the padding of the device buffer, never used)."""
        out = list(arr[start:start + count])
        assert start >= 0 and len(out) <= count
        return out + [pad] * (count - len(out))

    def stream_set(k, st, s, t, upd):
        """The set pass of set s from chunk k's staged copies st."""
        I0, I1, ra, nra, va, nva, ka, nka, sa, nsa = k[:10]
        sreach, sval, smem, ssig, sR, sA = st
        get = lambda a, i: a[i] if 0 <= i < len(a) else (_ for _ in ()).throw(IndexError(i))
        sb, na, m0, nm, vb, r0, rs, fl = sinfo[s]
        p2 = (fl >> 8) & 1
        sig = [get(ssig, sb - sa + a) for a in range(na)]
        racc, macc = [0.0] * na, [0.0] * na
        for q in range(nm):
            r = get(sreach, r0 - ra + q * rs)
            hh = get(smem, m0 - ka + q)
            cb = vb - va + q
            vc = [get(sval, cb + a * nm) for a in range(na)]
            vh = 0.0
            for a in range(na):
                vh = vh + sig[a] * vc[a]
            v[hh] = vh
            po, pw = (r[0], r[1]) if p2 else (r[1], r[0])
            f = (-1.0 if p2 else 1.0) * po
            for a in range(na):
                racc[a] = racc[a] + f * (vc[a] - vh)
                macc[a] = macc[a] + pw * sig[a]
        if (2 if p2 else 1) not in upd:
            return
        w = float(t) * float(t) if rule == oracle.PCFR_PLUS else float(t)
        pos = []
        for a in range(na):
            rn = get(sR, sb - sa + a) + racc[a]
            if rule != oracle.CFR:
                rn = rn if rn > 0.0 else 0.0
            R[sb + a] = rn
            avg[sb + a] = get(sA, sb - sa + a) + w * macc[a]
            x = rn + racc[a] if rule == oracle.PCFR_PLUS else rn
            pos.append(x if x > 0.0 else 0.0)
        tot = 0.0
        for a in range(na):
            tot = tot + pos[a]
        for a in range(na):
            sigma[sb + a] = pos[a] / tot if tot > 0.0 else 1.0 / na

    def stream_depth(d, t, upd):
        nan2 = [float("nan"), float("nan")]
        for k in chunks[sc0[d]:sc0[d + 1]]:
            if k[10] != 0:  # chance chunks: chance_sums
                continue
            I0, I1, ra, nra, va, nva, ka, nka, sa, nsa = k[:10]
            st = (staged(reach, ra, nra, nan2), staged(v, va, nva, float("nan")), staged(list(mvs), ka, nka, -1),
                  staged(sigma, sa, nsa, float("nan")), staged(R, sa, nsa, float("nan")),
                  staged(avg, sa, nsa, float("nan")))
            I = I0
            while I < I1:
                G = sinfo[I, 7] & 7
                assert G in (1, 4)
                for s in range(I, I + G):
                    stream_set(k, st, s, t, upd)
                I += G

    halves = [(1, 2)] if order == oracle.SIMULTANEOUS else [(1,), (2,)]  # players whose sets update
    for t in range(1, iters + 1):
        for upd in halves:
            forward()
            for d in range(D - 1, -1, -1):
                chance_sums(d)
                if stream and sok[d]:
                    stream_depth(d, t, upd)
                    continue
                for s in range(li[2 * d], li[2 * d + 2]):
                    set_pass(s, d, t, upd)
    return np.array(R), np.array(avg)


@pytest.mark.parametrize("order,tiles", [(cfr.REACH_MEMBERS, cfr.TILES_AUTO), (cfr.REACH_MEMBERS, cfr.TILES_ON),
                                         (cfr.REACH_BFS, cfr.TILES_AUTO), (cfr.REACH_SLOTS, cfr.TILES_AUTO)])
@pytest.mark.parametrize("name", list(GAMES))
def test_layouts_reach_the_oracles_iterates(name, order, tiles):
    g = GAMES[name]()
    iters = 4
    h = cfr.cfr_compile(g, cfr.make_options(precision=cfr.P64, reach_order=order, member_tiles=tiles))
    try:
        R, avg = emulate(h, iters)
        spec_of = cfr.cfr_export_array(h, "spec_slot_of").astype(int)
    finally:
        cfr.cfr_destroy(h)
    o = oracle.Oracle(g)
    o.iterate(iters)
    np.testing.assert_array_equal(R, o.R[spec_of])
    np.testing.assert_array_equal(avg, o.sbar[spec_of])


@pytest.mark.parametrize("rule", [oracle.CFR, oracle.PCFR_PLUS])
@pytest.mark.parametrize("order", [oracle.SIMULTANEOUS, oracle.ALTERNATING])
@pytest.mark.parametrize("name", ["tiny", "card_small"])
def test_update_rules_and_orders_on_the_member_layout(name, rule, order):
    # the update rules (vanilla CFR without the clamp; PCFR+ matching R + r,
    # quadratic averaging weight) and alternating halves over the tiled
    # member layout reach the oracle's iterates bitwise
    g = GAMES[name]()
    iters = 4
    h = cfr.cfr_compile(g, cfr.make_options(precision=cfr.P64, member_tiles=cfr.TILES_ON))
    try:
        R, avg = emulate(h, iters, rule, order)
        spec_of = cfr.cfr_export_array(h, "spec_slot_of").astype(int)
    finally:
        cfr.cfr_destroy(h)
    o = oracle.Oracle(g, rule=rule, order=order)
    o.iterate(iters)
    np.testing.assert_array_equal(R, o.R[spec_of])
    np.testing.assert_array_equal(avg, o.sbar[spec_of])


@pytest.mark.parametrize("seed,depth,p_chance,max_group", [(7, 7, 0.1, 1), (8, 8, 0.4, 4), (9, 7, 0.6, 40),
                                                           (10, 9, 0.2, 2), (11, 6, 0.0, 8)])
@pytest.mark.parametrize("order,tiles", [(cfr.REACH_MEMBERS, cfr.TILES_ON), (cfr.REACH_MEMBERS, cfr.TILES_OFF),
                                         (cfr.REACH_BFS, cfr.TILES_AUTO)])
def test_random_shapes_reach_the_oracles_iterates(seed, depth, p_chance, max_group, order, tiles):
    # random perfect-recall trees of several shapes (single-member sets tile
    # everywhere; chance-heavy trees put chance nodes between sets)
    g = gg.random_tree(seed, depth=depth, p_chance=p_chance, max_group=max_group)
    iters = 3
    h = cfr.cfr_compile(g, cfr.make_options(precision=cfr.P64, reach_order=order, member_tiles=tiles))
    try:
        R, avg = emulate(h, iters)
        spec_of = cfr.cfr_export_array(h, "spec_slot_of").astype(int)
    finally:
        cfr.cfr_destroy(h)
    o = oracle.Oracle(g)
    o.iterate(iters)
    np.testing.assert_array_equal(R, o.R[spec_of])
    np.testing.assert_array_equal(avg, o.sbar[spec_of])


@pytest.mark.parametrize("tiles", [cfr.TILES_AUTO, cfr.TILES_ON])
@pytest.mark.parametrize("name", ["kuhn", "tiny", "rt6", "card_small", "endgame", "wide_root"])
def test_streaming_chunks_reach_the_oracles_iterates(name, tiles):
    # the streaming backward's data paths: every set pass reads its members'
    # reach, children's values, own value slots and its slots' strategy,
    # regret and average from the chunk's staged copies, with the kernel's
    # index arithmetic; in FP64 and the oracle's member order this must give
    # the oracle's iterates bitwise
    g = GAMES[name]()
    iters = 3
    h = cfr.cfr_compile(g, cfr.make_options(precision=cfr.P32, member_tiles=tiles))
    try:
        assert cfr.cfr_export_array(h, "stream_ok").any()
        R, avg = emulate(h, iters, stream=True)
        spec_of = cfr.cfr_export_array(h, "spec_slot_of").astype(int)
    finally:
        cfr.cfr_destroy(h)
    o = oracle.Oracle(g)
    o.iterate(iters)
    np.testing.assert_array_equal(R, o.R[spec_of])
    np.testing.assert_array_equal(avg, o.sbar[spec_of])
