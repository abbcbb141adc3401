"""Host logic of the serving loop (tdvp_server_*) without a GPU: argument checks,
the queue (first in, first out, pause, cancel, timeouts), the error path of a
request that cannot reach a device, the counters, and the footprint estimate.
Device work is covered by tests/test_gpu_serve.py."""
import ctypes as C

import pytest
import torch

from paper_2606_04771_b300._lib import RequestC, TdvpError, lib
from paper_2606_04771_b300.serve import QuenchServer, Request, footprint_bytes

pytestmark = pytest.mark.skipif(torch.cuda.is_available(), reason="checks the path on which no device is reachable")


def _req(**kw):
    d = dict(L=8, U=4.0, t_final=0.1, chi=32)
    d.update(kw)
    return Request(**d)


def test_invalid_arguments_are_rejected():
    h = C.c_void_p()
    assert lib().tdvp_server_create(0.0, 2, None, C.byref(h)) == -1
    assert lib().tdvp_server_create(1e9, 0, None, C.byref(h)) == -1
    with QuenchServer(hbm_budget_gb=1.0, max_active=1) as s:
        for bad in (dict(L=1), dict(chi=0), dict(dt=0.0), dict(dt=-0.1), dict(t_final=-1.0), dict(eps=-1e-9)):
            with pytest.raises(TdvpError, match="EINVAL"):
                s.submit(_req(**bad))
        r, _ = _req().c()
        r.symmetry = 7
        i = C.c_longlong()
        assert lib().tdvp_server_submit(s.h, C.byref(r), C.byref(i)) == -1
        r, _ = _req().c()
        occ = (C.c_int * 8)(1, 2, 1, 5, 1, 2, 1, 2)
        r.occupations = C.cast(occ, C.c_void_p)
        assert lib().tdvp_server_submit(s.h, C.byref(r), C.byref(i)) == -1
        with pytest.raises(TdvpError, match="EINVAL"):
            s.poll(12345)
        with pytest.raises(TdvpError, match="EINVAL"):
            s.info(12345)


def test_queue_pause_cancel_and_timeouts():
    with QuenchServer(hbm_budget_gb=1.0, max_active=1) as s:
        s.pause(True)
        ids = [s.submit(_req(L=8 + 2 * k)) for k in range(4)]
        assert ids == sorted(ids) and len(set(ids)) == 4
        assert all(s.poll(i) == "queued" for i in ids)
        assert s.wait(ids[0], timeout=0.05) is None  # still queued: ETIMEOUT
        with pytest.raises(TdvpError, match="ESTATE"):
            s.result(ids[0])
        s.cancel(ids[1])
        assert s.poll(ids[1]) == "cancelled"
        with pytest.raises(TdvpError, match="ECANCELED"):
            s.result(ids[1])
        st = s.stats()
        assert (st["submitted"], st["queued"], st["cancelled"], st["running"]) == (4, 3, 1, 0)
        s.pause(False)
        # no device here: every admitted request ends FAILED with ECUDA, in submission order
        for i in (ids[0], ids[2], ids[3]):
            assert s.wait(i, timeout=30) == "failed"
            with pytest.raises(TdvpError, match="ECUDA"):
                s.result(i)
        adm = [s.info(i)["t_admit"] for i in (ids[0], ids[2], ids[3])]
        assert adm == sorted(adm)
        assert all(s.info(i)["status"] == -6 for i in (ids[0], ids[2], ids[3]))
        st = s.stats()
        assert (st["failed"], st["done"], st["queued"], st["peak_active"]) == (3, 0, 0, 1)
        s.cancel(ids[0])  # an ended request is left as it is
        assert s.poll(ids[0]) == "failed"


def test_destroy_with_queued_requests_returns():
    s = QuenchServer(hbm_budget_gb=1.0, max_active=2)
    s.pause(True)
    for k in range(5):
        s.submit(_req(L=6 + k))
    s.close()
    s.close()  # idempotent


def test_footprint_estimate():
    a = footprint_bytes(_req(L=20, chi=256))
    assert footprint_bytes(_req(L=40, chi=256)) > a
    big = footprint_bytes(_req(L=20, chi=8192))
    assert big / footprint_bytes(_req(L=20, chi=4096)) == pytest.approx(4.0, rel=0.01)  # chi^2 at large chi
    assert footprint_bytes(_req(L=20, chi=256), krylov_max=30) > a
    r = RequestC()
    b = C.c_double()
    assert lib().tdvp_server_footprint(C.byref(r), 20, C.byref(b)) == -1  # L = 0
