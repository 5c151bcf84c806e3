"""cfr_iterate_noalloc: iterations without any device allocation.

Callers that cannot allocate device memory while they iterate (code running
during a CUDA graph capture, serving loops with a fixed memory budget) use
this entry point; its scratch lives in a static device array inside the
library. It must leave exactly the state that cfr_iterate with the persistent
kernel leaves, call after call. This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import gamegen as gg
from paper_2609_11923_gb300 import cfr

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [cfr.P64, cfr.P32])
@pytest.mark.parametrize("name,make", [
    ("tiny", lambda: gg.tiny_card()),
    ("random_tree", lambda: gg.random_tree(5, depth=9)),
    ("wide_root", lambda: gg.endgame(2, 100000)),
])
def test_noalloc_matches_persistent_form_on_consecutive_calls(name, make, precision):
    assert torch.cuda.is_available()
    g = make()
    ref = cfr.Solver(g, precision=precision, exec_form=cfr.EXEC_PERSISTENT)
    new = cfr.Solver(g, precision=precision, exec_form=cfr.EXEC_PERSISTENT)
    for _ in range(2):
        ref.iterate(40)
        ref.synchronize()
        cfr.cfr_iterate_noalloc(new.h, 40, new._s())
        Ra, sa, ta = ref.get_state()
        Rb, sb, tb = new.get_state()
        assert ta == tb
        np.testing.assert_allclose(Rb, Ra, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(sb, sa, rtol=1e-12, atol=1e-12)
        assert np.abs(new.avg_strategy() - ref.avg_strategy()).max(initial=0.0) <= 1e-12


def test_noalloc_rejects_games_beyond_its_static_scratch():
    g = gg.random_tree(1, depth=14)  # about 2.5 million nodes: beyond the FP64 limit
    s = cfr.Solver(g, precision=cfr.P64, exec_form=cfr.EXEC_PERSISTENT)
    with pytest.raises(cfr.CfrError) as ei:
        cfr.cfr_iterate_noalloc(s.h, 1, s._s())
    assert ei.value.code == -1 and "static limit" in str(ei.value)
