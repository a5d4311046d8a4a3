"""ctypes binding of the serving loop (of_server_* in include/of.h) and an open-loop
load driver. Argument marshalling and timing only: batching, admission, copies and
the flow computation all happen in libof.so.
"""
from __future__ import annotations

import collections
import ctypes
import time

import numpy as np
import torch

from . import of

_lib = of.lib()


class ServerConfig(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("radius", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("in_format", ctypes.c_int32), ("in_bits", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("fp64_cond", ctypes.c_float), ("flags", ctypes.c_uint32), ("hbm_budget_bytes", ctypes.c_uint64),
                ("max_batch", ctypes.c_int32), ("max_inflight", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_int32), ("status", ctypes.c_int32), ("tag", ctypes.c_uint64),
                ("arrival_ns", ctypes.c_int64), ("launch_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64),
                ("batch", ctypes.c_int32), ("has_field", ctypes.c_int32)]


_vp, _i32, _i64, _u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
for _name, _res, _args in [
    ("of_server_config_init", None, [ctypes.POINTER(ServerConfig)]),
    ("of_server_create", ctypes.c_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(_vp)]),
    ("of_server_open_stream", ctypes.c_int, [_vp, _i32, _i32, ctypes.POINTER(_i32)]),
    ("of_server_close_stream", ctypes.c_int, [_vp, _i32]),
    ("of_server_submit", ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _u64, _i64]),
    ("of_server_poll", ctypes.c_int, [_vp, ctypes.POINTER(Result), _i32, ctypes.POINTER(_i32), _i32]),
    ("of_server_drain", ctypes.c_int, [_vp, _i32]),
    ("of_server_stats", ctypes.c_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_u64)]),
    ("of_server_now_ns", _i64, []),
    ("of_server_destroy", ctypes.c_int, [_vp]),
]:
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def now_ns() -> int:
    return _lib.of_server_now_ns()


class Server:
    def __init__(self, levels=3, radius=4, iterations=5, bits=12, storage="f16", hbm_budget_bytes=8 << 30,
                 max_batch=64, max_inflight=2, flags=0, fp64_cond=1e3):
        c = ServerConfig()
        _lib.of_server_config_init(ctypes.byref(c))
        c.levels, c.radius, c.iterations = levels, radius, iterations
        c.in_format = of.OF_U8 if bits <= 8 else of.OF_U16
        c.in_bits = bits
        c.storage = of.STORAGE[storage] if isinstance(storage, str) else storage
        c.fp64_cond = fp64_cond
        c.flags = flags
        c.hbm_budget_bytes = int(hbm_budget_bytes)
        c.max_batch, c.max_inflight = max_batch, max_inflight
        self.config = c
        self.bits = bits
        h = _vp()
        of._check(_lib.of_server_create(ctypes.byref(c), ctypes.byref(h)), "of_server_create")
        self._h = h
        self._buf = (Result * 1024)()
        # Each submitted frame tensor is referenced here until its result is polled: the
        # library copies the frame when its tick runs, so the host memory must not be
        # freed (and handed to another tensor by torch's pinned-memory cache) before that.
        # Results of one stream are reported in submission order.
        self._held = collections.defaultdict(collections.deque)

    def open_stream(self, H, W) -> int:
        i = _i32()
        of._check(_lib.of_server_open_stream(self._h, H, W, ctypes.byref(i)), "of_server_open_stream")
        return i.value

    def try_open_stream(self, H, W):
        i = _i32()
        rc = _lib.of_server_open_stream(self._h, H, W, ctypes.byref(i))
        return rc, i.value

    def close_stream(self, sid):
        of._check(_lib.of_server_close_stream(self._h, sid), "of_server_close_stream")

    def submit(self, sid, frame: torch.Tensor, u=None, v=None, tag=0, arrival_ns=0):
        if frame.is_cuda or not frame.is_contiguous():
            raise ValueError("frame: expected a contiguous host tensor (pinned for full copy speed)")
        rc = _lib.of_server_submit(self._h, sid, frame.data_ptr(), u.data_ptr() if u is not None else None,
                                   v.data_ptr() if v is not None else None, int(tag), int(arrival_ns))
        of._check(rc, "of_server_submit")
        self._held[sid].append(frame)

    def poll(self, timeout_us=0) -> list[dict]:
        n = _i32()
        rc = _lib.of_server_poll(self._h, self._buf, len(self._buf), ctypes.byref(n), int(timeout_us))
        of._check(rc, "of_server_poll")
        out = [{f: getattr(self._buf[i], f) for f, _ in Result._fields_} for i in range(n.value)]
        for r in out:
            held = self._held.get(r["stream"])
            if held:
                held.popleft()
        return out

    def drain(self, timeout_ms=30000):
        of._check(_lib.of_server_drain(self._h, int(timeout_ms)), "of_server_drain")

    def stats(self):
        t, p, u = _i64(), _i64(), _u64()
        of._check(_lib.of_server_stats(self._h, ctypes.byref(t), ctypes.byref(p), ctypes.byref(u)), "of_server_stats")
        return {"ticks": t.value, "pairs": p.value, "hbm_used": u.value}

    def close(self):
        if self._h is not None:
            _lib.of_server_destroy(self._h)
            self._h = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def pinned_frame(a: np.ndarray) -> torch.Tensor:
    t = torch.from_numpy(a.astype(np.int32)).to(torch.uint16) if a.dtype == np.uint16 else torch.from_numpy(a)
    return t.contiguous().pin_memory()


def run_open_loop(server: Server, streams, arrivals, warmup_s=0.0, out_ring=4, poll_us=200, end_s=None, keep=()):
    """Submit frames at their scheduled arrival times (open loop) and collect results.

    streams: list of (sid, frames) with frames a list of pinned host tensors, taken in
    order (cycled if a stream has more arrivals than frames). arrivals: sorted list of
    (t_seconds, stream_index). Each stream's u, v come from a ring of `out_ring` device
    buffer pairs; a slot is reused only after its result has been reported. A result is
    `in_window` when its arrival lies in [warmup_s, end_s). keep: (stream_index,
    frame_number) pairs whose fields are copied out when they are reported. Returns
    (results, t0_ns, kept) with kept[(stream_index, frame_number)] = (u, v)."""
    dev = [[(torch.empty(f[0].shape, dtype=torch.float32, device="cuda"),
             torch.empty(f[0].shape, dtype=torch.float32, device="cuda")) for _ in range(out_ring)]
           for _, f in streams]
    busy = [[False] * out_ring for _ in streams]
    count = [0] * len(streams)
    owner = {}
    results = []
    kept = {}
    keep = set(keep)
    torch.cuda.synchronize()
    t0 = now_ns() + 20_000_000
    end_ns = None if end_s is None else end_s * 1e9

    def take(r):
        si2, slot, fno = owner.pop(r["tag"])
        busy[si2][slot] = False
        if (si2, fno) in keep and r["has_field"]:
            u, v = dev[si2][slot]
            kept[(si2, fno)] = (u.clone(), v.clone())
        r["stream_index"] = si2
        r["frame_number"] = fno
        rel = r["arrival_ns"] - t0
        r["in_window"] = rel >= warmup_s * 1e9 and (end_ns is None or rel < end_ns)
        results.append(r)

    for k, (t, si) in enumerate(arrivals):
        due = t0 + int(t * 1e9)
        while True:
            for r in server.poll(0):
                take(r)
            wait = due - now_ns()
            if wait <= 0:
                break
            time.sleep(min(wait, 200_000) / 1e9)
        sid, frames = streams[si]
        slot = count[si] % out_ring
        while busy[si][slot]:   # output buffer still in use: wait for results
            for r in server.poll(poll_us):
                take(r)
        u, v = dev[si][slot]
        busy[si][slot] = True
        owner[k] = (si, slot, count[si])
        server.submit(sid, frames[count[si] % len(frames)], u, v, tag=k, arrival_ns=due)
        count[si] += 1
    server.drain()
    for r in server.poll(0):
        take(r)
    return results, t0, kept


def summarize(results, window_s):
    lat = np.array([(r["done_ns"] - r["arrival_ns"]) / 1e6 for r in results if r["in_window"] and r["has_field"]])
    fields = int(sum(1 for r in results if r["in_window"] and r["has_field"]))
    batch = np.array([r["batch"] for r in results if r["in_window"] and r["has_field"]])
    return {"fields": fields, "fields_per_s": fields / window_s,
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "max_ms": float(lat.max()) if lat.size else None,
            "mean_batch": float(batch.mean()) if batch.size else None,
            "errors": int(sum(1 for r in results if r["status"] != 0))}
