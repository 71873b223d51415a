"""Serving: a request loop over resident clouds (sdf_serve_* of include/ptsdf.h).

    srv = Server(mem_budget_bytes=..., max_inflight=8, n_streams=4)
    cid = srv.register(cloud)
    ticket = srv.submit(SDF_REQ_QUERY, cid, x, out)      # x, out: CUDA tensors or numpy arrays
    stats = srv.poll(ticket)                             # waits; timestamps in ns
    srv.shutdown()

Argument marshalling only: admission, scheduling and the kernels run in the
library.  Buffers passed to submit are kept alive here until the request is
polled.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import _abi, _buffers
from ._abi import check, lib, make_opts

SDF_REQ_QUERY, SDF_REQ_GRAD, SDF_REQ_UNION, SDF_REQ_INTERSECT, SDF_REQ_DIFFERENCE, SDF_REQ_TRACE_STEP = range(6)


SDF_SERVE_FIFO, SDF_SERVE_SMALLEST_FIRST = 0, 1


class sdf_serve_config(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("n_streams", ctypes.c_int32), ("device", ctypes.c_int32), ("policy", ctypes.c_int32),
                ("starve_ms", ctypes.c_int32), ("split_gpairs", ctypes.c_int32), ("express_gpairs", ctypes.c_float)]


class sdf_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("cloud_id", ctypes.c_int32), ("cloud_id_b", ctypes.c_int32),
                ("host_buffers", ctypes.c_int32), ("x", ctypes.c_void_p), ("dirs", ctypes.c_void_p),
                ("t", ctypes.c_void_p), ("q", ctypes.c_int64), ("out", ctypes.c_void_p),
                ("opts", _abi.sdf_query_opts)]


class sdf_request_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("chunks", ctypes.c_int32), ("arrive_ns", ctypes.c_int64),
                ("admit_ns", ctypes.c_int64), ("start_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64),
                ("device_ms", ctypes.c_double)]


class Server:
    def __init__(self, mem_budget_bytes: int = 8 << 30, max_inflight: int = 8, n_streams: int = 4,
                 device: int | None = None, policy: int = SDF_SERVE_FIFO, starve_ms: int = 2000,
                 split_gpairs: int = 0, express_gpairs: float = 0.0):
        """split_gpairs: requests above split_gpairs x 1e9 (query, point) pairs
        run as query chunks interleaved with other requests (0: never).
        express_gpairs: requests (and chunks) of at most express_gpairs x 1e9
        pairs run on high-priority streams, the others on low-priority ones
        (0: one priority; > 0 needs n_streams >= 2)."""
        import torch
        cfg = sdf_serve_config(int(mem_budget_bytes), int(max_inflight), int(n_streams),
                               torch.cuda.current_device() if device is None else int(device), int(policy),
                               int(starve_ms), int(split_gpairs), float(express_gpairs))
        h = ctypes.c_void_p()
        check(lib().sdf_serve_create(ctypes.byref(cfg), ctypes.byref(h)), "sdf_serve_create")
        self._h = h
        self._keep = {}
        self._clouds = []
        self._lock = threading.Lock()

    def register(self, cloud) -> int:
        cid = ctypes.c_int32()
        check(lib().sdf_serve_register(self._h, cloud.handle, ctypes.byref(cid)), "sdf_serve_register")
        self._clouds.append(cloud)
        return cid.value

    def submit(self, kind: int, cloud_id: int, x, out, cloud_id_b: int = -1, dirs=None, t=None, **opts) -> int:
        nx = x.size if isinstance(x, np.ndarray) else x.numel()
        if nx % 3:
            raise ValueError("x: must hold q x 3 floats")
        q = nx // 3
        xp, host = _buffers.request_buffer(x, 3 * q, "x")
        # the library reads and writes every buffer of a request in the same memory space
        op, ohost = _buffers.request_buffer(out, 4 * q if int(kind) == SDF_REQ_GRAD else q, "out", writable=True)
        dp, dhost = _buffers.request_buffer(dirs, 3 * q, "dirs") if dirs is not None else (None, host)
        tp, thost = _buffers.request_buffer(t, q, "t") if t is not None else (None, host)
        if not host == ohost == dhost == thost:
            raise ValueError("x, out, dirs and t must all be host or all be device buffers")
        r = sdf_request()
        r.kind, r.cloud_id, r.cloud_id_b, r.host_buffers = int(kind), int(cloud_id), int(cloud_id_b), int(host)
        r.x, r.q, r.out = xp, q, op
        r.dirs, r.t = dp, tp
        r.opts = make_opts(**opts)
        ticket = ctypes.c_uint64()
        check(lib().sdf_serve_submit(self._h, ctypes.byref(r), ctypes.byref(ticket)), "sdf_serve_submit")
        with self._lock:
            self._keep[ticket.value] = (x, out, dirs, t)
        return ticket.value

    def poll(self, ticket: int, timeout_s: float | None = None) -> dict:
        """Waits for a request; raises TimeoutError if it is not finished in time."""
        st = sdf_request_stats()
        us = -1 if timeout_s is None else max(0, int(timeout_s * 1e6))
        s = lib().sdf_serve_poll(self._h, ctypes.c_uint64(ticket), us, ctypes.byref(st))
        if s == _abi.SDF_ETIMEOUT:
            raise TimeoutError(f"request {ticket} not finished")
        with self._lock:
            self._keep.pop(ticket, None)
        check(s, "sdf_serve_poll")
        return {"arrive_ns": st.arrive_ns, "admit_ns": st.admit_ns, "start_ns": st.start_ns,
                "done_ns": st.done_ns, "device_ms": st.device_ms, "chunks": st.chunks}

    def stats(self) -> dict:
        q, f, m = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        check(lib().sdf_serve_stats(self._h, ctypes.byref(q), ctypes.byref(f), ctypes.byref(m)), "sdf_serve_stats")
        return {"queued": q.value, "inflight": f.value, "mem_in_use": m.value}

    def shutdown(self):
        if getattr(self, "_h", None) is not None:
            lib().sdf_serve_shutdown(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.shutdown()
        except Exception:
            pass
