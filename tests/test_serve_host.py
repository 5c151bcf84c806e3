"""Host logic of the serving loop (no GPU): the device-pool allocator."""
from paper_2609_11923_gb300 import serve


def test_device_pool_first_fit_and_coalescing():
    p = serve.DevicePool(1 << 20, device=None)
    a = p.alloc(1000)
    b = p.alloc(5000)
    c = p.alloc(300)
    assert a == 0 and b == 1024 and c == 1024 + 5120
    p.release(b, 5000)
    assert p.alloc(4000) == 1024  # reuses the hole
    p.release(1024, 4000)
    p.release(a, 1000)
    p.release(c, 300)
    assert p.free == [(0, p.size)] and p.used == 0


def test_device_pool_refuses_when_full():
    p = serve.DevicePool(4096, device=None)
    assert p.alloc(4096) == 0
    assert p.alloc(1) is None
    p.release(0, 4096)
    assert p.alloc(2048) == 0 and p.alloc(2048) == 2048 and p.alloc(256) is None


def _q(sizes):
    return [(i, n) for i, n in enumerate(sizes)]  # (rid, footprint)


def test_admission_rejects_requests_larger_than_the_pool():
    p = serve.DevicePool(10 * 1024, device=None)
    adm, rej, head = serve.admit(_q([4096, 20 * 1024, 2048]), 8, p, lambda e: e[1], key=lambda e: e[0])
    assert [e[0] for e, _, _ in adm] == [0, 2]
    assert [e[0] for e, _ in rej] == [1] and "exceeds" in rej[0][1]
    assert head == (None, 0)


def test_admission_backfills_around_a_blocked_head_for_a_bounded_number_of_passes():
    p = serve.DevicePool(8192, device=None)
    held = p.alloc(6144)  # an active solve holds most of the pool
    q = _q([4096, 1024, 512])  # the head needs 4096: does not fit yet
    head = (None, 0)
    for wait in range(1, 4):
        adm, rej, head = serve.admit(q, 8, p, lambda e: e[1], head, hol_rounds=3, key=lambda e: e[0])
        if wait == 1:
            assert [e[0] for e, _, _ in adm] == [1, 2]  # backfilled around the head
            q = q[:1] + [(3, 256)]
        else:
            assert adm == [] or [e[0] for e, _, _ in adm] == [3]
        for e, off, n in adm:
            p.release(off, n)
        assert head == (0, wait)
    # the head has now waited hol_rounds passes: nothing passes it any more
    adm, rej, head = serve.admit(q, 8, p, lambda e: e[1], head, hol_rounds=3, key=lambda e: e[0])
    assert adm == [] and head == (0, 4)
    p.release(held, 6144)  # the active solve retires: the head fits, then the rest
    adm, rej, head = serve.admit(q, 8, p, lambda e: e[1], head, hol_rounds=3, key=lambda e: e[0])
    assert [e[0] for e, _, _ in adm] == [0, 3] and head == (None, 0)


def test_admission_respects_free_slots():
    p = serve.DevicePool(1 << 20, device=None)
    adm, rej, head = serve.admit(_q([256] * 5), 2, p, lambda e: e[1], key=lambda e: e[0])
    assert [e[0] for e, _, _ in adm] == [0, 1] and rej == [] and head == (None, 0)
