"""The streaming FP32 backward's chunks, checked on the CPU against the
compiled arrays before any kernel runs them.

For every depth that streams: the chunks cover the depth's sets in order,
in whole groups (a tile of four sets or one untiled set); each chunk's staged
bytes fit one stage; every copy starts on a 16-byte boundary and has a size
that is a multiple of 16 bytes, and stays inside its array's 256-byte padded
buffer; and every shared-memory index the kernel computes (reach of each
member, its children's values, its own value slot, the set's slots) lies in
the staged range. The arithmetic done from the staged copies is emulated in
tests/test_layout_emulation.py.
"""
import numpy as np
import pytest

import gamegen as gg
from paper_2609_11923_gb300 import cfr

STAGE = 48 * 1024  # bytes of a stage (the compute threads' data)
SIDE = 2048  # bytes of a side slot (the control warp's data)

GAMES = {
    "tiny": lambda: gg.tiny_card(),
    "kuhn": lambda: gg.kuhn(),
    "card_3x2": lambda: gg.large_card(3, 2, 1, 1),
    "card_4x4": lambda: gg.large_card(4, 4, 1, 1),
    "card_4x2_cap2": lambda: gg.large_card(4, 2, 2, 2),
    "rt9": lambda: gg.random_tree(5, depth=9),
    "rt_singletons": lambda: gg.random_tree(9, depth=8, max_group=1),
    "endgame": lambda: gg.endgame(7, 200000),
    "wide_root": lambda: gg.endgame(2, 100000),
}


def layout(k):
    """Byte offsets of the staged arrays (the kernel's stream_layout): the
    stage the compute threads read, and the side slot the control warp reads
    (set records, R, average)."""
    I0, I1, ra, nra, va, nva, ka, nka, sa, nsa = k[:10]
    off = {"reach": 0}
    off["val"] = off["reach"] + 8 * nra
    off["mem"] = off["val"] + 4 * nva
    off["info"] = off["mem"] + 4 * nka
    off["sig"] = off["info"] + 32 * (I1 - I0)
    off["total"] = off["sig"] + 4 * nsa
    off["s_R"] = 32 * (I1 - I0)
    off["s_avg"] = off["s_R"] + 8 * nsa
    off["s_total"] = off["s_avg"] + 8 * nsa
    return off


def padded(nbytes):
    return max(256, (max(nbytes, 1) + 255) // 256 * 256)


@pytest.mark.parametrize("tiles", [cfr.TILES_AUTO, cfr.TILES_ON])
@pytest.mark.parametrize("name", list(GAMES))
def test_stream_chunks_cover_the_sets_and_stay_in_bounds(name, tiles):
    g = GAMES[name]()
    h = cfr.cfr_compile(g, cfr.make_options(precision=cfr.P32, member_tiles=tiles))
    try:
        ex = lambda n: cfr.cfr_export_array(h, n).astype(np.int64)
        c = cfr.cfr_get_counts(h)
        info = ex("set_info").reshape(-1, 8)
        chunks = ex("stream_chunks").reshape(-1, 16)
        c0, ok = ex("stream_c0"), ex("stream_ok")
        isl, im, ivb, irk, li = ex("iset_slot"), ex("iset_mem"), ex("iset_vb"), ex("iset_rank").reshape(-1, 2), \
            ex("level_iset")
        D = c["depth_blocks"]
        assert len(c0) == D + 1 and len(ok) == D
        # set descriptors mirror the compiled arrays
        assert len(info) == c["n_infosets"]
        np.testing.assert_array_equal(info[:, 0], isl[:-1])
        np.testing.assert_array_equal(info[:, 1], np.diff(isl))
        np.testing.assert_array_equal(info[:, 2], im[:-1])
        np.testing.assert_array_equal(info[:, 3], np.diff(im))
        np.testing.assert_array_equal(info[:, 4], ivb)
        np.testing.assert_array_equal(info[:, 5:7], irk)
        p2 = np.zeros(len(info), dtype=bool)
        for d in range(D):
            p2[li[2 * d + 1]:li[2 * d + 2]] = True
        np.testing.assert_array_equal((info[:, 7] >> 8) & 1, p2)
        n_int, N, n_dec, A = c["n_internal"], c["n_nodes"], c["n_decision"], c["n_slots"]
        streamed = 0
        for d in range(D):
            if not ok[d]:
                assert c0[d + 1] == c0[d]
                continue
            assert d > 0
            nxt = li[2 * d]
            kinds = chunks[c0[d]:c0[d + 1], 10]
            assert set(kinds) <= {0, 1} and (np.diff(kinds) >= 0).all()  # set chunks, then chance chunks
            for k in chunks[c0[d]:c0[d + 1]]:
                if k[10] != 0:
                    continue
                I0, I1, ra, nra, va, nva, ka, nka, sa, nsa = k[:10]
                assert I0 == nxt and I1 > I0
                nxt = I1
                # whole groups
                I = I0
                while I < I1:
                    G = info[I, 7] & 7
                    assert G in (1, 4)
                    if G == 4:
                        assert (info[I + 1:I + 4, 7] & 7 == 0).all()
                        assert (info[I:I + 4, 6] == 4).all()
                        np.testing.assert_array_equal(info[I:I + 4, 5], info[I, 5] + np.arange(4))
                        assert len(set(info[I:I + 4, 3])) == 1
                    else:
                        assert info[I, 6] == 1
                    I += G
                assert I == I1
                off = layout(k)
                assert off["total"] <= STAGE and off["s_total"] <= SIDE
                for key in ("val", "mem", "info", "sig", "total", "s_R", "s_avg", "s_total"):
                    assert off[key] % 16 == 0
                # copies: 16-byte aligned starts, inside the padded buffers
                assert ra % 2 == 0 and nra % 2 == 0 and va % 4 == 0 and nva % 4 == 0
                assert ka % 4 == 0 and nka % 4 == 0 and sa % 4 == 0 and nsa % 4 == 0
                assert 0 <= ra and 8 * (ra + nra) <= padded(8 * max(n_int, 1))
                assert 0 <= va and 4 * (va + nva) <= padded(4 * N)
                assert 0 <= ka and 4 * (ka + nka) <= padded(4 * n_dec)
                assert 0 <= sa and 4 * (sa + nsa) <= padded(4 * (A + 1)) and 8 * (sa + nsa) <= padded(8 * A)
                # every index the kernel forms lies in the staged ranges
                for I in range(I0, I1):
                    sb, na, m0, nm, vb, r0, rs, _ = info[I]
                    q = np.arange(nm)
                    rr = r0 - ra + q * rs
                    assert rr.min() >= 0 and rr.max() < nra
                    cc = vb - va + q[:, None] + np.arange(na)[None, :] * nm
                    assert cc.min() >= 0 and cc.max() < nva
                    mm = m0 - ka + q
                    assert mm.min() >= 0 and mm.max() < nka
                    assert sb - sa >= 0 and sb - sa + na <= nsa
                    assert 0 <= I - I0 < I1 - I0
                streamed += 1
            assert nxt == li[2 * d + 2]
        if name.startswith("card_4x4") or name == "rt9":
            assert streamed > 0
    finally:
        cfr.cfr_destroy(h)


CHANCE_MAX = 1024  # chance nodes per chance chunk at most


@pytest.mark.parametrize("name", list(GAMES))
def test_stream_chance_chunks_cover_the_chance_nodes_and_stay_in_bounds(name):
    # a streaming depth's narrow chance nodes go in chance chunks, in order;
    # each chunk stages its nodes' children (one run of value slots) and its
    # entries of the three chance arrays: 16-byte aligned copies inside the
    # padded buffers, a stage's bytes at most, and every index the kernel
    # forms (a node's entry, its children in the run) inside what is staged
    g = GAMES[name]()
    h = cfr.cfr_compile(g, cfr.make_options(precision=cfr.P32, lanes_per_set=cfr.STREAM_LANES))
    try:
        ex = lambda n: cfr.cfr_export_array(h, n).astype(np.int64)
        c = cfr.cfr_get_counts(h)
        ok, lch, c0 = ex("stream_ok"), ex("level_chance"), ex("stream_c0")
        chunks = ex("stream_chunks").reshape(-1, 16)
        chb, chn = ex("ch_vb"), ex("ch_nch")
        N, n_narrow = c["n_nodes"], len(chb)
        nodes = 0
        for d in range(c["depth_blocks"]):
            ks = [k for k in chunks[c0[d]:c0[d + 1]] if k[10] == 1]
            if not ok[d]:
                assert not ks
                continue
            nxt = lch[d]
            for k in ks:
                I0, I1, ra, nra, va, nva, ka, nka, sa, nsa = k[:10]
                assert I0 == nxt and I1 > I0 and I1 - I0 <= CHANCE_MAX
                nxt = I1
                assert ra == nra == sa == nsa == 0 and (k[11:] == 0).all()
                assert va % 4 == 0 and nva % 4 == 0 and ka % 4 == 0 and nka % 4 == 0
                assert 4 * nva + 3 * 4 * nka <= STAGE
                assert 0 <= va and 4 * (va + nva) <= padded(4 * N)
                assert 0 <= ka <= I0 and I1 <= ka + nka and 4 * (ka + nka) <= padded(4 * n_narrow)
                cb, n = chb[I0:I1], chn[I0:I1]
                assert (cb >= va).all() and (cb + n <= va + nva).all()
                nodes += I1 - I0
            assert nxt == lch[d + 1]
        if name.startswith("card"):
            assert nodes > 0
    finally:
        cfr.cfr_destroy(h)


def test_streaming_needs_fp32_member_order():
    g = gg.tiny_card()
    for kw in ({"precision": cfr.P64}, {"reach_order": cfr.REACH_BFS}):
        with pytest.raises(cfr.CfrError):
            cfr.cfr_compile(g, cfr.make_options(lanes_per_set=cfr.STREAM_LANES, **kw))
    h = cfr.cfr_compile(g, cfr.make_options(precision=cfr.P64))
    try:
        assert len(cfr.cfr_export_array(h, "stream_chunks")) == 0
    finally:
        cfr.cfr_destroy(h)
