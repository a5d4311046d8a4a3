"""ctypes binding of libof.so (include/of.h). Argument marshalling only.

Every step of the flow computation runs in the CUDA library; this module checks tensor
shapes and dtypes, passes device pointers and the current CUDA stream, and turns status
codes into exceptions. PyTorch provides device memory and streams. There is no CPU
fallback: if libof.so is missing or cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libof.so")

OF_OK, OF_EINVAL, OF_ENOMEM, OF_ECUDA, OF_EDEVICE, OF_ETIMEOUT, OF_ESTATE, OF_EBUSY = 0, -1, -2, -3, -4, -5, -6, -7
OF_U8, OF_U16 = 0, 1
OF_F32, OF_F16, OF_BF16 = 0, 1, 2
OF_FLAG_NO_GRAPH = 0x1
OF_FLAG_GATHER = 0x2
OF_FLAG_ZNSSD = 0x4
OF_FLAG_I1GRAD = 0x8
STORAGE = {"f32": OF_F32, "f16": OF_F16, "bf16": OF_BF16}


class OfError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {_lib.of_status_string(status).decode()} ({status})")


class Plan(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("radius", ctypes.c_int32), ("iterations", ctypes.c_int32), ("in_format", ctypes.c_int32),
                ("in_bits", ctypes.c_int32), ("storage", ctypes.c_int32), ("fp64_cond", ctypes.c_float),
                ("flags", ctypes.c_uint32)]

    @classmethod
    def make(cls, H, W, levels=3, radius=4, iterations=5, bits=8, storage="f32", fp64_cond=1e3, flags=0):
        p = cls()
        _lib.of_plan_init(ctypes.byref(p), int(H), int(W))
        p.levels, p.radius, p.iterations = int(levels), int(radius), int(iterations)
        p.in_format = OF_U8 if bits <= 8 else OF_U16
        p.in_bits = int(bits)
        p.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        p.fp64_cond = float(fp64_cond)
        p.flags = int(flags)
        return p

    def __repr__(self):
        return (f"Plan(H={self.H}, W={self.W}, levels={self.levels}, radius={self.radius}, "
                f"iterations={self.iterations}, in_format={self.in_format}, in_bits={self.in_bits}, "
                f"storage={self.storage}, fp64_cond={self.fp64_cond}, flags={self.flags})")


class Tuning(ctypes.Structure):
    """of_tuning: how a batched launch runs (see include/of.h)."""
    _fields_ = [("generic_sums", ctypes.c_int32), ("stage_i2", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("phased", ctypes.c_int32), ("prefetch", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("branches", ctypes.c_int32), ("fusion", ctypes.c_int32), ("strip", ctypes.c_int32),
                ("ms", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run `python -m paper_1306_2461_gb300.build` "
                          "(the flow computation has no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    i32, vp, pp = ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)
    P = ctypes.POINTER(Plan)
    sig = {
        "of_plan_init": (None, [P, i32, i32]),
        "of_plan_validate": (ctypes.c_int, [P]),
        "of_plan_check": (ctypes.c_int, [P, ctypes.c_float, ctypes.POINTER(ctypes.c_int)]),
        "of_level_size": (ctypes.c_int, [P, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "of_workspace_bytes": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_size_t)]),
        "of_create": (ctypes.c_int, [P, pp]),
        "of_compute": (ctypes.c_int, [vp, vp, vp, vp, vp, vp]),
        "of_compute_batch": (ctypes.c_int, [i32, pp, pp, pp, pp, pp, vp]),
        "of_sync_status": (ctypes.c_int, [vp]),
        "of_destroy": (ctypes.c_int, [vp]),
        "of_get_level": (ctypes.c_int, [vp, i32, i32, vp, vp]),
        "of_window_sums": (ctypes.c_int, [vp, i32, i32, i32, vp, vp]),
        "of_debug_wait_timeout": (ctypes.c_int, [i32]),
        "of_sbubble_count": (ctypes.c_int, [vp, i32, i32, ctypes.c_float, vp, vp]),
        "of_field_minmax": (ctypes.c_int, [vp, i32, i32, vp, vp]),
        "of_debug_fail_allocs": (ctypes.c_int, [i32]),
        "of_compute_batch_host": (ctypes.c_int, [i32, pp, pp, pp, pp, pp, pp, pp, pp, pp, vp, i32]),
        "of_compute_noalloc": (ctypes.c_int, [P, vp, vp, vp, vp, vp]),
        "of_autotune_batch": (ctypes.c_int, [i32, pp, pp, pp, pp, pp, vp, i32, ctypes.POINTER(Tuning),
                                             ctypes.POINTER(Tuning), i32, ctypes.POINTER(i32)]),
        "of_batch_size_class": (ctypes.c_int, [i32, pp, ctypes.POINTER(i32)]),
        "of_tuning_get": (ctypes.c_int, [P, i32, ctypes.POINTER(Tuning)]),
        "of_tuning_set": (ctypes.c_int, [P, i32, ctypes.POINTER(Tuning)]),
        "of_tuning_clear": (ctypes.c_int, []),
        "of_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "of_version": (ctypes.c_int, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


_lib = _load()


def lib():
    return _lib


def _check(rc: int, what: str):
    if rc != OF_OK:
        raise OfError(rc, what)


def _stream(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


# ------------------------------------------------------------------ host helpers
def plan_validate(p: Plan) -> int:
    return _lib.of_plan_validate(ctypes.byref(p))


def plan_check(p: Plan, max_disp_px: float) -> bool:
    ok = ctypes.c_int()
    _check(_lib.of_plan_check(ctypes.byref(p), float(max_disp_px), ctypes.byref(ok)), "of_plan_check")
    return bool(ok.value)


def level_size(p: Plan, level: int) -> tuple[int, int]:
    h, w = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.of_level_size(ctypes.byref(p), int(level), ctypes.byref(h), ctypes.byref(w)), "of_level_size")
    return h.value, w.value


def workspace_bytes(p: Plan) -> int:
    n = ctypes.c_size_t()
    _check(_lib.of_workspace_bytes(ctypes.byref(p), ctypes.byref(n)), "of_workspace_bytes")
    return n.value


def version() -> int:
    return _lib.of_version()


# ------------------------------------------------------------------- the handle
def _img_ptr(t: torch.Tensor | None, p: Plan, name: str) -> int | None:
    if t is None:
        return None
    want = torch.uint8 if p.in_format == OF_U8 else torch.uint16
    if t.dtype != want or not t.is_cuda or tuple(t.shape) != (p.H, p.W) or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous CUDA {want} tensor of shape ({p.H}, {p.W}), "
                         f"got {t.dtype} {tuple(t.shape)} on {t.device}")
    return t.data_ptr()


def _flow_ptr(t: torch.Tensor, p: Plan, name: str) -> int:
    if t.dtype != torch.float32 or not t.is_cuda or tuple(t.shape) != (p.H, p.W) or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous CUDA float32 tensor of shape ({p.H}, {p.W})")
    return t.data_ptr()


class Flow:
    """One of_create handle: the workspace of one plan on the current device."""

    def __init__(self, plan: Plan):
        self.plan = plan
        h = ctypes.c_void_p()
        _check(_lib.of_create(ctypes.byref(plan), ctypes.byref(h)), "of_create")
        self._h = h

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("handle destroyed")
        return self._h

    def compute(self, I1, I2, u=None, v=None, stream=None):
        """Queue the flow I1 -> I2 on `stream` (default: torch's current stream).
        I1 = None reuses the previous call's I2 pyramid. Returns (u, v)."""
        p = self.plan
        if u is None:
            u = torch.empty((p.H, p.W), dtype=torch.float32, device=I2.device)
        if v is None:
            v = torch.empty((p.H, p.W), dtype=torch.float32, device=I2.device)
        rc = _lib.of_compute(self.handle, _img_ptr(I1, p, "I1"), _img_ptr(I2, p, "I2"), _flow_ptr(u, p, "u"),
                             _flow_ptr(v, p, "v"), _stream(stream))
        _check(rc, "of_compute")
        return u, v

    def sync_status(self) -> int:
        return _lib.of_sync_status(self.handle)

    def get_level(self, which: int, level: int, stream=None) -> torch.Tensor:
        Hl, Wl = level_size(self.plan, level)
        out = torch.empty((Hl, Wl), dtype=torch.float32, device="cuda")
        _check(_lib.of_get_level(self.handle, int(which), int(level), out.data_ptr(), _stream(stream)),
               "of_get_level")
        return out

    def close(self):
        if self._h is not None:
            rc = _lib.of_destroy(self._h)
            self._h = None
            _check(rc, "of_destroy")

    def __del__(self):
        try:
            if getattr(self, "_h", None) is not None:
                _lib.of_destroy(self._h)
                self._h = None
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _ptr_array(vals):
    arr = (ctypes.c_void_p * max(1, len(vals)))()
    for i, x in enumerate(vals):
        arr[i] = x
    return arr


def compute_batch(flows, I1s, I2s, us=None, vs=None, stream=None):
    """of_compute_batch over independent pairs. Returns the lists (us, vs)."""
    n = len(flows)
    if us is None:
        us = [torch.empty((f.plan.H, f.plan.W), dtype=torch.float32, device="cuda") for f in flows]
    if vs is None:
        vs = [torch.empty((f.plan.H, f.plan.W), dtype=torch.float32, device="cuda") for f in flows]
    _check(_lib.of_compute_batch(n, *_batch_ptrs(flows, I1s, I2s, us, vs), _stream(stream)), "of_compute_batch")
    return us, vs


def _batch_ptrs(flows, I1s, I2s, us, vs):
    n = len(flows)
    hs = _ptr_array([f.handle.value for f in flows])
    a1 = _ptr_array([_img_ptr(I1s[i], flows[i].plan, "I1") for i in range(n)])
    a2 = _ptr_array([_img_ptr(I2s[i], flows[i].plan, "I2") for i in range(n)])
    au = _ptr_array([_flow_ptr(us[i], flows[i].plan, "u") for i in range(n)])
    av = _ptr_array([_flow_ptr(vs[i], flows[i].plan, "v") for i in range(n)])
    return hs, a1, a2, au, av


def _host_ptr(t: torch.Tensor | None, dtype, p: Plan, name: str) -> int | None:
    if t is None:
        return None
    if t.is_cuda or t.dtype != dtype or tuple(t.shape) != (p.H, p.W) or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous host {dtype} tensor of shape ({p.H}, {p.W}) "
                         "(pinned for asynchronous copies)")
    return t.data_ptr()


def compute_batch_host(flows, hI1s, hI2s, hus, hvs, dI1s, dI2s, dus, dvs, stream=None, chunk=0):
    """of_compute_batch_host: frames from host tensors, fields into host tensors, the
    copies overlapped with the batched launches (chunks of `chunk` pairs, 0 = about
    8 Mpx per chunk, smaller at either end of the batch). hI1s[i] = None reuses the previous pyramid. Synchronise `stream` before
    reading hus/hvs."""
    n = len(flows)
    img = [torch.uint8 if f.plan.in_format == OF_U8 else torch.uint16 for f in flows]
    arrs = [
        _ptr_array([f.handle.value for f in flows]),
        _ptr_array([_host_ptr(hI1s[i], img[i], flows[i].plan, "hI1") for i in range(n)]),
        _ptr_array([_host_ptr(hI2s[i], img[i], flows[i].plan, "hI2") for i in range(n)]),
        _ptr_array([_host_ptr(hus[i], torch.float32, flows[i].plan, "hu") for i in range(n)]),
        _ptr_array([_host_ptr(hvs[i], torch.float32, flows[i].plan, "hv") for i in range(n)]),
        _ptr_array([_img_ptr(dI1s[i], flows[i].plan, "dI1") if hI1s[i] is not None else None for i in range(n)]),
        _ptr_array([_img_ptr(dI2s[i], flows[i].plan, "dI2") for i in range(n)]),
        _ptr_array([_flow_ptr(dus[i], flows[i].plan, "du") for i in range(n)]),
        _ptr_array([_flow_ptr(dvs[i], flows[i].plan, "dv") for i in range(n)]),
    ]
    _check(_lib.of_compute_batch_host(n, *arrs, _stream(stream), int(chunk)), "of_compute_batch_host")


def autotune_batch(flows, I1s, I2s, us=None, vs=None, stream=None, reps=3):
    """of_autotune_batch: time every candidate tuning on this batch and record the
    fastest in the library's table. Returns (best, [each candidate]) as dicts."""
    n = len(flows)
    if us is None:
        us = [torch.empty((f.plan.H, f.plan.W), dtype=torch.float32, device="cuda") for f in flows]
    if vs is None:
        vs = [torch.empty((f.plan.H, f.plan.W), dtype=torch.float32, device="cuda") for f in flows]
    best = Tuning()
    res = (Tuning * 32)()
    nres = ctypes.c_int32()
    _check(_lib.of_autotune_batch(n, *_batch_ptrs(flows, I1s, I2s, us, vs), _stream(stream), int(reps),
                                  ctypes.byref(best), res, len(res), ctypes.byref(nres)), "of_autotune_batch")
    return best.as_dict(), [res[i].as_dict() for i in range(nres.value)]


def batch_size_class(flows) -> int:
    sc = ctypes.c_int32()
    _check(_lib.of_batch_size_class(len(flows), _ptr_array([f.handle.value for f in flows]), ctypes.byref(sc)),
           "of_batch_size_class")
    return sc.value


def tuning_get(method: Plan, size_class: int) -> dict | None:
    t = Tuning()
    rc = _lib.of_tuning_get(ctypes.byref(method), int(size_class), ctypes.byref(t))
    if rc == OF_ESTATE:
        return None
    _check(rc, "of_tuning_get")
    return t.as_dict()


def tuning_set(method: Plan, size_class: int, generic_sums=0, stage_i2=1, blocks_per_sm=0, phased=1, prefetch=0,
               tile_h=0, branches=0, fusion=1, strip=4):
    """of_tuning_set; the defaults are the library's tuning without a table entry."""
    t = Tuning(int(generic_sums), int(stage_i2), int(blocks_per_sm), int(phased), int(prefetch), int(tile_h),
               int(branches), int(fusion), int(strip), 0.0)
    _check(_lib.of_tuning_set(ctypes.byref(method), int(size_class), ctypes.byref(t)), "of_tuning_set")


def tuning_clear():
    _check(_lib.of_tuning_clear(), "of_tuning_clear")


def compute_noalloc(plan: Plan, I1: torch.Tensor, I2: torch.Tensor, u: torch.Tensor, v: torch.Tensor,
                    stream=None):
    """of_compute_noalloc: one pair with no handle and no device allocation (a static
    32 MiB device scratch shared by all calls; overlapping calls race). Fills u, v."""
    _check(_lib.of_compute_noalloc(ctypes.byref(plan), _img_ptr(I1, plan, "I1"), _img_ptr(I2, plan, "I2"),
                                   _flow_ptr(u, plan, "u"), _flow_ptr(v, plan, "v"), _stream(stream)),
           "of_compute_noalloc")
    return u, v


def window_sums(ch: torch.Tensor, r: int, stream=None) -> torch.Tensor:
    """Box sums of 5 planes (5, H, W) float32 over the (2r+1)^2 window (zero outside)."""
    if ch.dtype != torch.float32 or not ch.is_cuda or ch.dim() != 3 or ch.shape[0] != 5 or not ch.is_contiguous():
        raise ValueError("ch: expected a contiguous CUDA float32 tensor of shape (5, H, W)")
    out = torch.empty_like(ch)
    _check(_lib.of_window_sums(ch.data_ptr(), ch.shape[1], ch.shape[2], int(r), out.data_ptr(), _stream(stream)),
           "of_window_sums")
    return out


def sbubble(u: torch.Tensor, Tv: float, stream=None) -> torch.Tensor:
    """Eq. 3: device count of vectors with u <= Tv (int64 tensor of one element);
    S_bubble = count / u.numel()."""
    if u.dtype != torch.float32 or not u.is_cuda or u.dim() != 2 or not u.is_contiguous():
        raise ValueError("u: expected a contiguous 2-D CUDA float32 tensor")
    out = torch.empty(1, dtype=torch.int64, device=u.device)
    _check(_lib.of_sbubble_count(u.data_ptr(), u.shape[0], u.shape[1], float(Tv), out.data_ptr(), _stream(stream)),
           "of_sbubble_count")
    return out


def field_minmax(f: torch.Tensor, stream=None) -> torch.Tensor:
    """(min, max) of a 2-D CUDA float32 field, as a device tensor of two floats."""
    if f.dtype != torch.float32 or not f.is_cuda or f.dim() != 2 or not f.is_contiguous():
        raise ValueError("f: expected a contiguous 2-D CUDA float32 tensor")
    out = torch.empty(2, dtype=torch.float32, device=f.device)
    _check(_lib.of_field_minmax(f.data_ptr(), f.shape[0], f.shape[1], out.data_ptr(), _stream(stream)),
           "of_field_minmax")
    return out


def debug_wait_timeout(timeout_us: int) -> int:
    return _lib.of_debug_wait_timeout(int(timeout_us))
