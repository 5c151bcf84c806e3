"""cfr_iterate_noalloc: iterations without any device allocation.

Some callers cannot allocate device memory while they iterate: a serving
loop whose device memory is carved out once at start-up, or a host program
that embeds the library without owning the device allocator. This entry
point takes its scratch from a static device array inside the library. It
must leave exactly (bitwise) the state that cfr_iterate with the persistent
kernel leaves, call after call, and allocate nothing on the device. This
file is collected last on purpose, so that a run stopping at its first
failure has run every other test already.
"""
import numpy as np
import pytest
import torch

import gamegen as gg
import oracle
from paper_2609_11923_gb300 import cfr

pytestmark = pytest.mark.gpu

GAMES = [
    ("tiny", lambda: gg.tiny_card()),
    ("random_tree", lambda: gg.random_tree(5, depth=9)),
    ("wide_root", lambda: gg.endgame(2, 100000)),
]


@pytest.mark.parametrize("precision", [cfr.P64, cfr.P32])
@pytest.mark.parametrize("name,make", GAMES)
def test_noalloc_matches_persistent_form_on_consecutive_calls(name, make, precision):
    assert torch.cuda.is_available()
    g = make()
    ref = cfr.Solver(g, precision=precision, exec_form=cfr.EXEC_PERSISTENT)
    new = cfr.Solver(g, precision=precision, exec_form=cfr.EXEC_PERSISTENT)
    o = oracle.Oracle(g) if precision == cfr.P64 else None
    for _ in range(2):
        ref.iterate(40)
        ref.synchronize()
        cfr.cfr_iterate_noalloc(new.h, 40, new._s())
        Ra, sa, ta = ref.get_state()
        Rb, sb, tb = new.get_state()
        assert ta == tb
        # same kernel, same grid, same summation order: bitwise equal
        np.testing.assert_array_equal(Rb, Ra)
        np.testing.assert_array_equal(sb, sa)
        np.testing.assert_array_equal(new.avg_strategy(), ref.avg_strategy())
        if o is not None:  # FP64 in the oracle's order: bitwise the oracle's iterates
            o.iterate(40)
            np.testing.assert_array_equal(Rb, o.R)
            np.testing.assert_array_equal(sb, o.sbar)
            np.testing.assert_array_equal(new.avg_strategy(), o.avg_strategy())


def test_noalloc_allocates_no_device_memory():
    g = gg.random_tree(5, depth=9)
    s = cfr.Solver(g, precision=cfr.P32, exec_form=cfr.EXEC_PERSISTENT)
    cfr.cfr_iterate_noalloc(s.h, 5, s._s())  # first call: module loading and the symbol lookup
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    for _ in range(5):
        cfr.cfr_iterate_noalloc(s.h, 20, s._s())
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0
    for k in ("allocation.all.allocated", "reserved_bytes.all.allocated", "segment.all.allocated"):
        assert stats1.get(k, 0) == stats0.get(k, 0), k


def test_noalloc_rejects_games_beyond_its_static_scratch():
    g = gg.random_tree(1, depth=14)  # about 2.8 million nodes: beyond the FP64 limit
    s = cfr.Solver(g, precision=cfr.P64, exec_form=cfr.EXEC_PERSISTENT)
    with pytest.raises(cfr.CfrError) as ei:
        cfr.cfr_iterate_noalloc(s.h, 1, s._s())
    assert ei.value.code == cfr.CFR_ERR_ARG and "static limit" in str(ei.value)
