"""Serving: independent quench requests evolved concurrently on one GPU.

Binding of the library's serving loop (tdvp_server_* in include/tdvp.h).  The
scheduler, the workers and every step of every request run in the C library: each
admitted request owns a context (MPS, environments and workspaces resident on the
device) and a worker thread with its own CUDA stream, so the kernels of different
requests overlap on the device; the oldest queued request is admitted as soon as a
worker is free and its HBM footprint estimate fits the budget (continuous
batching).  This module marshals requests and results and, as a command, replays a
seeded stream of mixed requests with Poisson arrivals and reports p50/p99 latency
beside throughput:

    python -m paper_2606_04771_b300.serve --requests 16 --rate 2 --seed 1
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import sys
import time
from dataclasses import dataclass

import numpy as np

from ._lib import MODE, PREC, SYM, RequestC, TdvpError, check, lib, make_opts, vacancy_occupations

STATES = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "cancelled"}


@dataclass
class Request:
    L: int
    U: float
    t_final: float
    chi: int
    J: float = 1.0
    dt: float = 0.05
    eps: float = 1e-9
    mode: str = "adaptive"
    precision: str = "bf16x4"
    symmetry: str = "su2"
    vacancy: bool = False
    arrival: float = 0.0  # seconds after the start of a replayed stream

    def c(self):
        """The C struct and the occupations array it points to (keep both alive)."""
        occ = np.ascontiguousarray(vacancy_occupations(self.L), dtype=np.int32) if self.vacancy else None
        r = RequestC(self.L, self.J, self.U, SYM[self.symmetry], PREC[self.precision], MODE[self.mode], self.dt,
                     self.t_final, int(self.chi), self.eps, occ.ctypes.data if occ is not None else None)
        return r, occ


def footprint_bytes(req: Request, krylov_max=20) -> float:
    """The server's admission estimate for `req` (bytes)."""
    r, _occ = req.c()
    b = C.c_double()
    check(lib().tdvp_server_footprint(C.byref(r), krylov_max, C.byref(b)))
    return b.value


class QuenchServer:
    """A running server (its worker threads start at construction)."""

    def __init__(self, hbm_budget_gb=200.0, max_active=8, krylov_max=20, krylov_tol=1e-12, device=-1,
                 merge_launches=False):
        """merge_launches: the running requests' BF16x4 block GEMMs go out in shared
        grouped launches (tdvp_opts.merge_launches) instead of one launch per request."""
        o = make_opts(krylov_max=krylov_max, krylov_tol=krylov_tol, device=device, merge_launches=merge_launches)
        self.h = C.c_void_p()
        check(lib().tdvp_server_create(hbm_budget_gb * 1e9, int(max_active), C.byref(o), C.byref(self.h)))
        self.requests = {}

    def submit(self, req: Request) -> int:
        r, _occ = req.c()
        i = C.c_longlong()
        check(lib().tdvp_server_submit(self.h, C.byref(r), C.byref(i)))
        self.requests[i.value] = req
        return i.value

    def poll(self, rid) -> str:
        st = C.c_int()
        check(lib().tdvp_server_poll(self.h, rid, C.byref(st)))
        return STATES[st.value]

    def wait(self, rid, timeout=None):
        """Block until the request has ended; returns its state, or None on timeout."""
        ms = -1 if timeout is None else int(timeout * 1000)
        st = C.c_int()
        rc = lib().tdvp_server_wait(self.h, rid, ms, C.byref(st))
        if rc == -7:
            return None
        check(rc)
        return STATES[st.value]

    def info(self, rid):
        """Timings, bond dimension, device bytes and status of a request, in any state."""
        v = np.zeros(10)
        rc = lib().tdvp_server_result(self.h, rid, None, None, None, None, v.ctypes.data, 10)
        if rc == -1:  # unknown id (other codes are the request's own state or error)
            check(rc)
        keys = ["energy", "chi", "steps", "heff_flops", "t_submit", "t_admit", "t_done", "device_bytes_peak",
                "footprint", "status"]
        return dict(zip(keys, v.tolist()))

    def result(self, rid):
        """Observables of a finished request (as Chain.measure) and its info;
        raises TdvpError for a failed or cancelled one."""
        L = self.requests[rid].L
        n, sz, docc, ent = np.zeros(L), np.zeros(L), np.zeros(L), np.zeros(max(L - 1, 1))
        check(lib().tdvp_server_result(self.h, rid, n.ctypes.data, sz.ctypes.data, docc.ctypes.data, ent.ctypes.data,
                                       None, 0))
        inf = self.info(rid)
        return {"n": n, "sz": sz, "docc": docc, "n_up": 0.5 * n + sz, "n_dn": 0.5 * n - sz, "s_ent": ent[: L - 1],
                "energy": inf["energy"], "info": inf}

    def cancel(self, rid):
        check(lib().tdvp_server_cancel(self.h, rid))

    def pause(self, paused=True):
        check(lib().tdvp_server_pause(self.h, 1 if paused else 0))

    def stats(self):
        v = np.zeros(13)
        check(lib().tdvp_server_stats(self.h, v.ctypes.data, 13))
        keys = ["submitted", "done", "failed", "cancelled", "queued", "running", "latency_p50_s", "latency_p99_s",
                "wall_s", "peak_active", "peak_reserved_bytes", "steps", "heff_flops"]
        return dict(zip(keys, v.tolist()))

    def close(self):
        if self.h:
            check(lib().tdvp_server_destroy(self.h))
            self.h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def synthetic_requests(n=16, rate=2.0, seed=1, Ls=(16, 24, 32, 48, 60), Us=(2.0, 4.0, 8.0), ts=(0.5, 1.0),
                       chis=(256, 512), precision="bf16x4", mode="adaptive"):
    """A seeded mixed request stream: Poisson arrivals at `rate` per second, L, U,
    t_final and chi cap drawn uniformly from the given sets."""
    g = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n):
        t += g.exponential(1.0 / rate)
        out.append(Request(L=int(g.choice(Ls)), U=float(g.choice(Us)), t_final=float(g.choice(ts)),
                           chi=int(g.choice(chis)), precision=precision, mode=mode, arrival=t))
    return out


def replay(server: QuenchServer, reqs, log=None):
    """Submit each request at its arrival time (counted from now), wait for all and
    return {id: result}.  A failed request raises."""
    t0 = time.perf_counter()
    ids = []
    for r in sorted(reqs, key=lambda r: r.arrival):
        d = r.arrival - (time.perf_counter() - t0)
        if d > 0:
            time.sleep(d)
        ids.append(server.submit(r))
    out = {}
    for i in ids:
        server.wait(i)
        out[i] = server.result(i)
        if log is not None:
            inf, r = out[i]["info"], server.requests[i]
            print(json.dumps({"id": i, "L": r.L, "U": r.U, "t_final": r.t_final, "chi_cap": r.chi,
                              "chi": int(inf["chi"]), "steps": int(inf["steps"]),
                              "wait_s": inf["t_admit"] - inf["t_submit"], "run_s": inf["t_done"] - inf["t_admit"],
                              "latency_s": inf["t_done"] - inf["t_submit"], "energy": inf["energy"],
                              "device_gb_peak": inf["device_bytes_peak"] / 1e9,
                              "footprint_gb": inf["footprint"] / 1e9}), file=log, flush=True)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description="Serve a seeded stream of mixed quench requests on one GPU.")
    ap.add_argument("--requests", type=int, default=16)
    ap.add_argument("--rate", type=float, default=2.0, help="Poisson arrivals per second")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--t", type=float, nargs="+", default=[0.5, 1.0])
    ap.add_argument("--chi", type=int, nargs="+", default=[256, 512])
    ap.add_argument("--L", type=int, nargs="+", default=[16, 24, 32, 48, 60])
    ap.add_argument("--U", type=float, nargs="+", default=[2.0, 4.0, 8.0])
    ap.add_argument("--max-active", type=int, default=8)
    ap.add_argument("--hbm-gb", type=float, default=200.0)
    ap.add_argument("--precision", default="bf16x4", choices=sorted(PREC))
    ap.add_argument("--mode", default="adaptive", choices=sorted(MODE))
    ap.add_argument("--eps", type=float, default=None, help="truncation threshold (default: the Request default)")
    ap.add_argument("--merge", action="store_true",
                    help="shared grouped launches of the running requests' BF16x4 block GEMMs")
    a = ap.parse_args(argv)
    reqs = synthetic_requests(a.requests, a.rate, a.seed, Ls=tuple(a.L), Us=tuple(a.U), ts=tuple(a.t),
                              chis=tuple(a.chi), precision=a.precision, mode=a.mode)
    if a.eps is not None:
        for r in reqs:
            r.eps = a.eps
    from ._lib import merge_count

    m0 = merge_count()
    with QuenchServer(hbm_budget_gb=a.hbm_gb, max_active=a.max_active, merge_launches=a.merge) as srv:
        try:
            replay(srv, reqs, log=sys.stdout)
        except TdvpError as e:
            print(json.dumps({"error": str(e)}), flush=True)
            raise
        st = srv.stats()
    st["requests_per_s"] = st["done"] / st["wall_s"]
    st["steps_per_s"] = st["steps"] / st["wall_s"]
    st["heff_tflops"] = st["heff_flops"] / st["wall_s"] / 1e12
    m1 = merge_count()
    st["merged_launches"] = m1[0] - m0[0]
    st["merged_task_lists"] = m1[1] - m0[1]
    print(json.dumps({"summary": st, "max_active": a.max_active, "rate_per_s": a.rate, "seed": a.seed,
                      "precision": a.precision, "mode": a.mode, "merge": a.merge}), flush=True)


if __name__ == "__main__":
    main()
