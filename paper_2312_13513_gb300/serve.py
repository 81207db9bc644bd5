"""Python face of the serving loop (chem_serve_*) and of batched advances (chem_advance_batch)."""
from __future__ import annotations

import ctypes

from . import _lib, _ptr, _stream_ptr, check

ROUTE_FP64, ROUTE_SURROGATE = 0, 1
QUEUED, RUNNING, DONE, FAILED = 0, 1, 2, 3


def advance_batch(mech, segments, stream=None):
    """segments: list of dicts(T, p, Y, dt, rtol, atol[, status, nsub, nrej]) of device tensors."""
    arr = (_lib.Segment * len(segments))()
    for i, s in enumerate(segments):
        a = arr[i]
        a.T, a.p, a.Y = s["T"].data_ptr(), s["p"].data_ptr(), s["Y"].data_ptr()
        a.ld = s["Y"].shape[1]
        a.ncells = s["T"].numel()
        a.idx = None
        a.status = s["status"].data_ptr() if s.get("status") is not None else None
        a.nsub = s["nsub"].data_ptr() if s.get("nsub") is not None else None
        a.nrej = s["nrej"].data_ptr() if s.get("nrej") is not None else None
        a.dt, a.rtol, a.atol = float(s["dt"]), float(s.get("rtol", 1e-6)), float(s.get("atol", 1e-10))
    check(_lib.load().chem_advance_batch(mech.handle, arr, len(segments), _stream_ptr(stream)))


def surrogate_advance_batch(model, segments, stream=None):
    """segments: list of dicts(T, p, Y, dt[, rtol, atol, route]) of device tensors, all on the
    model's dt and the same tolerances; one gathered surrogate pass (chem_surrogate_advance_batch)."""
    arr = (_lib.Segment * len(segments))()
    for i, s in enumerate(segments):
        a = arr[i]
        a.T, a.p, a.Y = s["T"].data_ptr(), s["p"].data_ptr(), s["Y"].data_ptr()
        a.ld = s["Y"].shape[1]
        a.ncells = s["T"].numel()
        a.idx = None
        a.status = s["route"].data_ptr() if s.get("route") is not None else None
        a.nsub = None
        a.nrej = None
        a.dt, a.rtol, a.atol = float(s["dt"]), float(s.get("rtol", 1e-6)), float(s.get("atol", 1e-10))
    check(_lib.load().chem_surrogate_advance_batch(model.handle, model.mech.handle, arr, len(segments),
                                                   _stream_ptr(stream)))


class Server:
    def __init__(self, budget_bytes, n_streams=4, idle_poll_us=20.0, slice_ms=0.0, max_pause_ms=0.0):
        """slice_ms: FP64 time slice (0: library default, negative: unsliced jobs); max_pause_ms:
        longest wait of an FP64 job for running surrogate passes (0: default, negative: none)."""
        h = ctypes.c_void_p()
        opt = _lib.ServeOptions(n_streams, idle_poll_us, slice_ms, max_pause_ms)
        check(_lib.load().chem_serve_create(int(budget_bytes), ctypes.byref(opt), ctypes.byref(h)))
        self.handle = h
        self._keep = []

    def register(self, mech, T, p, Y, model=None):
        sid = ctypes.c_int()
        check(_lib.load().chem_serve_register_state(self.handle, mech.handle,
                                                    model.handle if model is not None else None,
                                                    _ptr(T), _ptr(p), _ptr(Y), Y.shape[1], T.numel(),
                                                    ctypes.byref(sid)))
        self._keep.append((T, p, Y))
        return sid.value

    def submit(self, state_id, route, dt, rtol=1e-6, atol=1e-10):
        rid = ctypes.c_uint64()
        check(_lib.load().chem_serve_submit(self.handle, state_id, route, float(dt), float(rtol), float(atol),
                                            ctypes.byref(rid)))
        return rid.value

    def poll(self, req_id):
        st = ctypes.c_int(); lat = ctypes.c_double()
        check(_lib.load().chem_serve_poll(self.handle, req_id, ctypes.byref(st), ctypes.byref(lat)))
        return st.value, lat.value

    def wait(self, req_id, timeout_s):
        return check(_lib.load().chem_serve_wait(self.handle, req_id, float(timeout_s)))

    def stats(self):
        out = (ctypes.c_int64 * 8)()
        check(_lib.load().chem_serve_stats(self.handle, out))
        keys = ("completed", "failed", "launches", "requests_launched", "max_concurrent", "bytes_in_use",
                "slices", "joined")
        return dict(zip(keys, list(out)))

    def close(self):
        if getattr(self, "handle", None):
            _lib.load().chem_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_closed_loop(server, solvers, duration_s=10.0, mean_gap_s=2e-3, seed=0, max_requests=4000):
    """Closed-loop load: each solver submits its next sub-step an Exp(gap) gap after its previous
    result completes, for duration_s seconds or max_requests requests; requests still in flight at
    the end are waited for.  gap = the solver's own "think_s" when it has one (its flow solve
    between chemistry steps; its first submission then comes at a uniform time in [0, think_s)),
    else mean_gap_s.

    solvers: list of dicts(state_id, route, dt, cells[, label, think_s, flow]).  flow (optional) is
    called before each submission of the solver: the solver's own step between two chemistry
    sub-steps (it must leave the state ready on the device).  Returns dict with per-request
    latencies (s) and the label of each request's solver, cells advanced and the wall time.
    """
    import heapq
    import random
    import time as _time
    rng = random.Random(seed)
    t0 = _time.perf_counter()
    gap = [s.get("think_s", mean_gap_s) for s in solvers]
    due = [(t0 + (rng.uniform(0.0, gap[i]) if "think_s" in solvers[i] else rng.expovariate(1.0 / gap[i])), i)
           for i in range(len(solvers))]
    heapq.heapify(due)
    inflight = {}
    lat, labels, cells, submitted = [], [], 0, 0
    end = t0 + duration_s
    while True:
        now = _time.perf_counter()
        while due and due[0][0] <= now and now < end and submitted < max_requests:
            _, i = heapq.heappop(due)
            s = solvers[i]
            if s.get("flow") is not None:
                s["flow"]()
            rid = server.submit(s["state_id"], s["route"], s["dt"])
            inflight[rid] = i
            submitted += 1
        for rid in list(inflight):
            st, l = server.poll(rid)
            if st >= DONE:
                i = inflight.pop(rid)
                if st == DONE:
                    lat.append(l)
                    labels.append(solvers[i].get("label", ""))
                    cells += solvers[i]["cells"]
                heapq.heappush(due, (_time.perf_counter() + rng.expovariate(1.0 / gap[i]), i))
        if (now >= end or submitted >= max_requests) and not inflight:
            break
        _time.sleep(1e-4)
    wall = _time.perf_counter() - t0
    return {"latencies": lat, "labels": labels, "cells": cells, "wall_s": wall, "submitted": submitted}
