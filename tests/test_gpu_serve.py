"""Serving loop on the device: mixed quench requests run concurrently (worker
threads, one stream each, continuous admission) give the same observables as each
request run alone; admission keeps the HBM footprint estimates within the budget;
the estimate bounds the device bytes a request holds; results match a Chain."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KEYS = ("n", "sz", "docc", "s_ent")


def _reqs():
    from paper_2606_04771_b300.serve import Request

    return [Request(L=8, U=4.0, t_final=0.5, chi=64, precision="bf16x4", mode="two"),
            Request(L=10, U=2.0, t_final=0.3, chi=64, precision="fp64", mode="adaptive"),
            Request(L=12, U=8.0, t_final=0.4, chi=32, precision="bf16x4", mode="adaptive"),
            Request(L=7, U=4.0, t_final=0.3, chi=64, precision="fp64", mode="two", symmetry="u1u1", vacancy=True),
            Request(L=16, U=4.0, t_final=0.25, chi=128, precision="3xtf32", mode="two", symmetry="u1u1")]


def _alone(r):
    from paper_2606_04771_b300.serve import QuenchServer

    with QuenchServer(max_active=1) as s:
        i = s.submit(r)
        assert s.wait(i, timeout=600) == "done"
        return s.result(i)


@pytest.mark.parametrize("merge", [False, True])
def test_each_result_is_the_same_alone_and_in_the_mix(merge):
    """merge=True: the requests' BF16x4 block GEMMs go out in shared grouped launches
    (several requests' tile lists in one persistent launch); every tile is computed the
    same way in any launch, so the results equal the lone runs."""
    from paper_2606_04771_b300._lib import merge_count
    from paper_2606_04771_b300.serve import QuenchServer

    reqs = _reqs()
    alone = [_alone(r) for r in reqs]
    m0 = merge_count()
    with QuenchServer(max_active=len(reqs), merge_launches=merge) as s:
        ids = [s.submit(r) for r in reqs]
        for i in ids:
            assert s.wait(i, timeout=600) == "done"
        mix = [s.result(i) for i in ids]
        st = s.stats()
    for r, a, m in zip(reqs, alone, mix):
        for k in KEYS:
            assert np.abs(m[k] - a[k]).max() <= 1e-12, (r, k)
        assert m["energy"] == pytest.approx(a["energy"], abs=1e-12)
        assert m["info"]["steps"] == round(r.t_final / r.dt)
        assert np.abs(m["n"].sum() - (r.L - (1 if r.vacancy else 0))) < 1e-9
    assert st["done"] == len(reqs) and st["failed"] == 0
    assert st["peak_active"] >= 2  # the requests did run side by side
    assert st["latency_p99_s"] >= st["latency_p50_s"] > 0
    if not merge:
        assert merge_count() == m0


def test_merged_launches_carry_several_requests_and_change_nothing():
    """Three BF16x4 requests served side by side with merged launches: some launches
    carry more than one request's tile list, and every result equals the lone run bit
    for bit."""
    from paper_2606_04771_b300._lib import merge_count
    from paper_2606_04771_b300.serve import QuenchServer, Request

    reqs = [Request(L=L, U=4.0, t_final=0.3, chi=128, precision="bf16x4", mode="two") for L in (16, 18, 20)]
    alone = [_alone(r) for r in reqs]
    m0 = merge_count()
    with QuenchServer(max_active=3, merge_launches=True) as s:
        ids = [s.submit(r) for r in reqs]
        for i in ids:
            assert s.wait(i, timeout=600) == "done"
        mix = [s.result(i) for i in ids]
    m1 = merge_count()
    assert m1[0] > m0[0] and m1[1] - m0[1] >= 2 * (m1[0] - m0[0])  # launches that carried >= 2 lists
    for a, m in zip(alone, mix):
        for k in KEYS:
            assert np.array_equal(m[k], a[k]), k


def test_served_request_equals_a_chain():
    from paper_2606_04771_b300 import Chain

    r = _reqs()[2]
    ch = Chain(r.L, r.J, r.U, symmetry=r.symmetry, precision=r.precision)
    for _ in range(round(r.t_final / r.dt)):
        ch.step(r.dt, r.chi, r.eps, mode=r.mode)
    o = ch.measure()
    ch.close()
    m = _alone(r)
    for k in KEYS:
        assert np.abs(m[k] - o[k]).max() <= 1e-12, k


def test_admission_keeps_estimates_within_the_budget():
    from paper_2606_04771_b300.serve import QuenchServer, footprint_bytes

    reqs = _reqs()[:3]
    budget = 1.5 * max(footprint_bytes(r) for r in reqs)  # room for one at a time
    with QuenchServer(hbm_budget_gb=budget / 1e9, max_active=3) as s:
        ids = [s.submit(r) for r in reqs]
        for i in ids:
            assert s.wait(i, timeout=600) == "done"
        spans = sorted((s.info(i)["t_admit"], s.info(i)["t_done"]) for i in ids)
        st = s.stats()
    assert st["peak_active"] == 1 and st["peak_reserved_bytes"] <= budget
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert b0 >= a1  # never two resident at once


def test_footprint_estimate_bounds_the_device_bytes():
    from paper_2606_04771_b300.serve import QuenchServer, Request

    reqs = [Request(L=24, U=4.0, t_final=1.0, chi=256, precision="bf16x4", mode="two", symmetry="u1u1"),
            Request(L=32, U=4.0, t_final=1.0, chi=512, precision="bf16x4", mode="two", symmetry="su2")]
    with QuenchServer(max_active=2) as s:
        ids = [s.submit(r) for r in reqs]
        for i in ids:
            assert s.wait(i, timeout=900) == "done"
        infos = [s.info(i) for i in ids]
    for r, inf in zip(reqs, infos):
        print("footprint", r.L, r.chi, r.symmetry, "chi reached", inf["chi"], "device bytes", inf["device_bytes_peak"],
              "estimate", inf["footprint"])
        assert 0 < inf["device_bytes_peak"] <= inf["footprint"]


def test_cancel_a_running_request():
    from paper_2606_04771_b300._lib import TdvpError
    from paper_2606_04771_b300.serve import QuenchServer, Request

    with QuenchServer(max_active=1) as s:
        i = s.submit(Request(L=24, U=4.0, t_final=50.0, chi=256, precision="bf16x4", mode="two"))
        for _ in range(600):
            if s.poll(i) == "running":
                break
            s.wait(i, timeout=0.01)
        s.cancel(i)
        assert s.wait(i, timeout=600) == "cancelled"
        with pytest.raises(TdvpError, match="ECANCELED"):
            s.result(i)
        assert s.info(i)["steps"] < 1000
        j = s.submit(_reqs()[0])  # the worker serves the next request
        assert s.wait(j, timeout=600) == "done"
