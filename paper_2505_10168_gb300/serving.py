"""Python face of the continuous-batching request server (stmg_server_* in include/stmg.h).

The server (native, in libstmg.so) runs forward and adjoint solves of uneven grids
concurrently on worker streams, admits requests by device footprint into a fixed memory
arena and keeps finished hierarchies resident for reuse.  This module marshals requests,
replays an arrival trace, and summarises latency and throughput.
"""
from __future__ import annotations

import ctypes as C
import time

import numpy as np

from . import _binding as B


ServerOpts, Request, Result = B.ServerOpts, B.Request, B.Result


def _lib():
    return B.lib()


class Server:
    def __init__(self, workers=4, budget_bytes=0, cache=True, max_nu=0):
        """max_nu > 0: a request that reaches its cycle cap or diverges is solved again with
        twice the smoothing sweeps, up to max_nu."""
        L = _lib()
        o = ServerOpts()
        L.stmg_server_default_opts(C.byref(o))
        o.workers, o.budget_bytes, o.cache = int(workers), int(budget_bytes), int(bool(cache))
        o.max_nu = int(max_nu)
        h = C.c_void_p()
        B.check(L.stmg_server_create(C.byref(h), C.byref(o)))
        self._h = h
        self._keep = {}

    def submit(self, nel, nt, L, t_end, k, c, q=None, q_value=1.0, adjoint=False, out=None, **opts):
        """Queue one solve; k, c, q are host float64 arrays; out: host/device result or None."""
        k = np.ascontiguousarray(k, dtype=np.float64)
        c = np.ascontiguousarray(c, dtype=np.float64)
        r = Request(int(nel), int(nt), float(L), float(t_end), k.ctypes.data, c.ctypes.data,
                    None if q is None else B.ptr(q), float(q_value), int(bool(adjoint)),
                    None if out is None else B.ptr(out), B.make_opts(**opts))
        t = C.c_longlong(0)
        B.check(_lib().stmg_server_submit(self._h, C.byref(r), C.byref(t)))
        self._keep[t.value] = (q, out)  # the server reads q and writes out until the request is done
        return t.value

    def result(self, ticket, wait=True):
        r = Result()
        B.check(_lib().stmg_server_result(self._h, int(ticket), int(bool(wait)), C.byref(r)))
        if r.status >= 0:
            self._keep.pop(ticket, None)
        return dict(status=B.STATUS.get(r.status, "pending"), cycles=r.cycles, relres=r.relres, theta=r.theta,
                    t_submit=r.t_submit, t_start=r.t_start, t_end=r.t_end, bytes=r.bytes, worker=r.worker, nu=r.nu)

    def drain(self):
        B.check(_lib().stmg_server_drain(self._h))

    def now(self):
        return _lib().stmg_server_now(self._h)

    @property
    def peak_bytes(self):
        return _lib().stmg_server_peak_bytes(self._h)

    def close(self):
        if getattr(self, "_h", None):
            _lib().stmg_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def replay(server, requests, fields, speed=1.0, **opts):
    """Submit requests at their arrival times (seconds / speed after the first) and wait.

    fields(req) -> (k, c) host arrays.  Returns (results, summary) with latency = finish -
    arrival on the server clock, p50/p99 in seconds, DOF/s = total DOFs / makespan, and the
    finest-level sweep rate = sum of DOFs x cycles x 2 nu / makespan (the smoothing work
    done, comparable across requests that need different numbers of cycles and sweeps).
    """
    t0 = server.now()
    a0 = requests[0]["arrival"] if requests else 0.0
    tickets = []
    for r in requests:
        due = t0 + (r["arrival"] - a0) / speed
        while True:
            dt = due - server.now()
            if dt <= 0:
                break
            time.sleep(min(dt, 0.002))
        k, c = fields(r)
        tickets.append(server.submit(r["N"], r["NT"], r["L"], r["tT"], k, c, q=None, q_value=1.0,
                                     adjoint=r["adjoint"], **opts))
    res = [server.result(t) for t in tickets]
    lat = np.array([x["t_end"] - x["t_submit"] for x in res])
    dofs = np.array([(r["N"] + 1) * (r["NT"] + 1) for r in requests], dtype=np.float64)
    span = max(x["t_end"] for x in res) - min(x["t_submit"] for x in res)
    nu0 = opts.get("nu")
    # smoothing work on the finest level: 2 nu sweeps per V-cycle (the nu of the attempt that
    # returned, so an escalated request's first attempt is not counted)
    sweeps = sum(d * x["cycles"] * 2 * x["nu"] for d, x in zip(dofs, res))
    summary = dict(requests=len(res), ok=sum(x["status"] == "ok" for x in res),
                   nu_raised=sum(1 for x in res if nu0 and x["nu"] > nu0),
                   p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
                   dofs_per_s=float(dofs.sum() / span), makespan_s=float(span),
                   fine_sweep_dofs_per_s=float(sweeps / span),
                   mean_cycles=float(np.mean([x["cycles"] for x in res])), peak_bytes=int(server.peak_bytes))
    return res, summary
