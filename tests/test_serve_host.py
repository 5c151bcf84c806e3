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
