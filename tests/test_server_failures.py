"""Failure paths of the continuous-batching server, injected on the host only.

Nothing here faults, traps or hangs a GPU: requests are held back by pausing admission
(ws_server_pause), withdrawn (ws_server_cancel), refused by the queue limit or the memory
budget, or asked for under an unknown id; every wait is a bounded host-side poll.
"""
import ctypes
import time

import numpy as np
import pytest

from paper_2204_14242_gb300 import binding as B
from paper_2204_14242_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    B.load()
    c = B.Context(0, 4 << 30)
    yield c
    c.close()


def small_request(seed=1, k=6):
    return W.request_stream(n_requests=1, seed=seed, kmin=k, kmax=k)[0].configs


def raw_poll(srv, rid, timeout_us=0):
    n = 1024
    res = np.zeros(n, B.RESULT)
    order = np.zeros(n, np.int32)
    return B.load().ws_server_poll(srv.handle, ctypes.c_uint64(rid), res.ctypes.data, order.ctypes.data,
                                   int(timeout_us))


def test_full_queue_refuses_with_eagain(ctx):
    with B.Server(ctx, W.a100(), mem_budget=256 << 20, max_queue=3) as srv:
        srv.pause(True)
        ids = [srv.submit(small_request(s)) for s in range(3)]
        with pytest.raises(B.WsError) as e:
            srv.submit(small_request(9))
        assert e.value.code == B.WS_EAGAIN
        st = srv.stats()
        assert st["queued"] == 3 and st["rejected"] == 1 and st["steps"] == 0
        # after resuming, the queued requests complete and the queue takes new ones
        srv.pause(False)
        for rid in ids:
            rc, res, order = srv.poll(rid, timeout_us=30_000_000)
            assert rc == B.WS_OK and (res["status"] == 0).all()
        rid = srv.submit(small_request(9))
        assert srv.poll(rid, timeout_us=30_000_000)[0] == B.WS_OK


def test_poll_returns_within_its_timeout(ctx):
    with B.Server(ctx, W.a100(), mem_budget=256 << 20) as srv:
        srv.pause(True)
        rid = srv.submit(small_request())
        for timeout_us in (0, 20_000, 200_000):
            t = time.perf_counter()
            rc, _, _ = srv.poll(rid, timeout_us=timeout_us)
            dt = time.perf_counter() - t
            assert rc == B.WS_EAGAIN
            assert timeout_us * 1e-6 * 0.9 <= dt < timeout_us * 1e-6 + 1.0, (timeout_us, dt)
        srv.pause(False)
        assert srv.poll(rid, timeout_us=30_000_000)[0] == B.WS_OK


def test_unknown_and_collected_ids_are_not_found(ctx):
    with B.Server(ctx, W.a100(), mem_budget=256 << 20) as srv:
        assert raw_poll(srv, 987654321) == B.WS_ENOTFOUND
        assert srv.cancel(987654321) == B.WS_ENOTFOUND
        rid = srv.submit(small_request())
        assert srv.poll(rid, timeout_us=30_000_000)[0] == B.WS_OK
        assert raw_poll(srv, rid) == B.WS_ENOTFOUND      # a collected result is forgotten
        assert srv.cancel(rid) == B.WS_ENOTFOUND


def test_cancel_withdraws_a_queued_request(ctx):
    hw = W.a100()
    with B.Server(ctx, hw, mem_budget=256 << 20) as srv:
        srv.pause(True)
        keep, drop = small_request(3), small_request(4)
        r_keep, r_drop = srv.submit(keep), srv.submit(drop)
        assert srv.cancel(r_drop) == B.WS_OK
        assert srv.poll(r_drop, timeout_us=0)[0] == B.WS_ECANCELED
        assert raw_poll(srv, r_drop) == B.WS_ENOTFOUND
        srv.pause(False)
        rc, res, order = srv.poll(r_keep, timeout_us=30_000_000)
        assert rc == B.WS_OK
        alone, alone_order = B.ws_estimate_batch(ctx, keep, hw)
        assert res.tobytes() == alone.tobytes() and order.tobytes() == alone_order.tobytes()
        st = srv.stats()
        assert st["canceled"] == 1 and st["completed"] == 1


def test_a_field_that_never_fits_the_budget_is_refused(ctx):
    """Budget 2 MiB: one field of a 25-point candidate on a 640x512x512 array-of-structs
    layout (x stride of 5 doubles, so its sets are walked address by address into bitmap
    scratch) needs more than that however many scratch passes the server would use."""
    N = (640, 512, 512)
    st = (5, 5 * N[0], 5 * N[0] * N[1])
    src = W.Field(8, [W.Access(*o) for o in W.star_offsets(4)], strides=st)
    dst = W.Field(8, [W.Access(0, 0, 0, 1)], strides=st, const_off=1)
    big = [W.Config(N=N, B=(32, 4, 2), fields=[src, dst], flops_per_lup=25.0)]
    info = B.ws_describe_fields(big[0], W.a100())
    field_bytes = [4 * (2 * int(f["words"][0]) + 4 * int(f["words"][1])) for f in info]
    assert max(field_bytes) > 2 << 20
    with B.Server(ctx, W.a100(), mem_budget=2 << 20) as srv:
        with pytest.raises(B.WsError) as e:
            srv.submit(big)
        assert e.value.code == B.WS_ENOMEM
        assert srv.stats()["rejected"] == 1
        # small requests still run on the same server
        rid = srv.submit([W.stencil_7pt_128()])
        assert srv.poll(rid, timeout_us=30_000_000)[0] == B.WS_OK


def test_destroy_with_queued_requests_returns_promptly(ctx):
    srv = B.Server(ctx, W.a100(), mem_budget=256 << 20)
    srv.pause(True)
    for s in range(5):
        srv.submit(small_request(s))
    st = srv.stats()
    assert st["queued"] == 5 and st["steps"] == 0
    t = time.perf_counter()
    srv.close()                # cancels the queued requests and joins the worker
    assert time.perf_counter() - t < 5.0
