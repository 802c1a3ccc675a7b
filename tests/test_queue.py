"""The host side of the diffeomorphic sampler (Sec. 3.3): the bounded
concurrent FIFO bucket, on the CPU with host threads (no GPU)."""
import threading

import numpy as np
import pytest

import paper_2108_11775_gb300 as pdmp


def test_fifo_capacity_and_partial_push():
    q = pdmp.Queue(3, 10)
    a = np.arange(24, dtype=np.float32).reshape(8, 3)
    assert q.push(a) == 8 and q.size() == 8
    assert q.push(a, timeout_ms=0) == 2                 # only two slots left; no wait
    assert q.size() == 10
    out = q.pop(5)
    assert np.array_equal(out, a[:5])
    assert q.push(a[:5]) == 5                            # wraps around the ring
    rest = q.pop(100)
    assert np.array_equal(rest, np.concatenate([a[5:8], a[:2], a[:5]]))
    assert q.size() == 0 and q.pop(3).shape == (0, 3)


def test_push_waits_for_room_until_timeout_or_close():
    q = pdmp.Queue(1, 4)
    assert q.push(np.ones(4)) == 4
    assert q.push(np.ones(2), timeout_ms=30) == 0        # times out, nothing pushed
    res = {}
    t = threading.Thread(target=lambda: res.setdefault("n", q.push(np.full(3, 7.0), timeout_ms=5000)))
    t.start()
    q.pop(2)                                             # room for two: the waiting push takes them
    t.join(timeout=10)
    q2 = pdmp.Queue(1, 1)
    q2.push(np.ones(1))
    t2 = threading.Thread(target=lambda: res.setdefault("closed", q2.push(np.ones(1), timeout_ms=60000)))
    t2.start()
    q2.close()                                           # wakes the waiting push at once
    t2.join(timeout=10)
    assert not t2.is_alive() and res["closed"] == 0
    assert res["n"] == 2 and q.size() == 4


def test_concurrent_producer_consumer_preserves_order():
    q = pdmp.Queue(2, 64)
    n = 20000
    data = np.stack([np.arange(n, dtype=np.float32), -np.arange(n, dtype=np.float32)], axis=1)

    def producer():
        done = 0
        while done < n:
            done += q.push(data[done:done + 97], timeout_ms=100)

    t = threading.Thread(target=producer)
    t.start()
    got = []
    total = 0
    while total < n:
        out = q.pop(50)
        got.append(out)
        total += out.shape[0]
    t.join(timeout=30)
    allv = np.concatenate(got)
    assert np.array_equal(allv, data)


def test_queue_argument_checks():
    L = pdmp.lib()
    import ctypes
    h = ctypes.c_void_p()
    assert L.pdmp_queue_create(0, 10, ctypes.byref(h)) == 1
    assert L.pdmp_queue_create(9, 10, ctypes.byref(h)) == 1
    assert L.pdmp_queue_create(2, 0, ctypes.byref(h)) == 1
    assert L.pdmp_queue_pop(None, None, 1, None) == 1
