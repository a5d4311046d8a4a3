"""FP64 CPU oracle for the pyramidal Lucas-Kanade flow (arXiv:1306.2461, Sect. 2.4).

TEST INFRASTRUCTURE. Only the tests, the package smoke check and the benchmark's CPU
baseline may import this module. The product library never calls it, and it shares no
code with the CUDA path: the arithmetic lives in `of_oracle.c` (plain double loops),
this file only compiles it with gcc and marshals numpy arrays through ctypes.

Each wrapper names the step of the method it computes; the C file states the readings
taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "of_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboforacle.so")
# A prebuilt oracle library to load instead (the mutation tests point this at a copy
# of the oracle with a planted mistake).
_LIB_OVERRIDE = os.environ.get("OF_ORACLE_LIB")
_lock = threading.Lock()
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile of_oracle.c with gcc (-O2, OpenMP, no FP contraction). Returns the .so path."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    os.makedirs(_OUT_DIR, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
            _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)   # no OpenMP on this host
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(_LIB_OVERRIDE or build())
            i, d = ctypes.c_int, ctypes.c_double
            L.ofo_pyr_down.argtypes = [_dp, i, i, _dp]
            L.ofo_bilinear.argtypes = [_dp, i, i, d, d]
            L.ofo_bilinear.restype = d
            L.ofo_upsample_flow.argtypes = [_dp, i, i, _dp, i, i]
            L.ofo_warp_grad.argtypes = [_dp, _dp, _dp, i, i, _dp, _dp, _dp]
            L.ofo_window_sum.argtypes = [_dp, i, i, i, _dp]
            L.ofo_solve.argtypes = [_dp] * 7 + [i, _dp, _dp, _dp,
                                                 np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")]
            L.ofo_lk_iteration.argtypes = [_dp, _dp, i, i, i, _dp, _dp, _dp, _dp, _dp]
            L.ofo_lk_iteration.restype = i
            L.ofo_flow.argtypes = [_dp, _dp, i, i, i, i, i, _dp, _dp, ctypes.c_void_p]
            L.ofo_flow.restype = i
            L.ofo_flow_variant.argtypes = [_dp, _dp, i, i, i, i, i, _dp, _dp, ctypes.c_void_p, i]
            L.ofo_flow_variant.restype = i
            L.ofo_lk_iteration_i1grad.argtypes = [_dp, _dp, i, i, i, _dp, _dp, _dp, _dp, _dp]
            L.ofo_lk_iteration_i1grad.restype = i
            L.ofo_znssd.argtypes = [_dp, i, i, i, d, _dp]
            fp = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
            L.ofo_sbubble_count.argtypes = [fp, i, i, ctypes.c_float]
            L.ofo_sbubble_count.restype = ctypes.c_longlong
            L.ofo_sbubble_threshold.argtypes = [fp, i, i]
            L.ofo_sbubble_threshold.restype = d
            L.ofo_threads.restype = i
            L.ofo_set_threads.argtypes = [i]
            _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def threads() -> int:
    return int(lib().ofo_threads())


def set_threads(n: int) -> None:
    lib().ofo_set_threads(int(n))


def level_size(H: int, W: int, level: int) -> tuple[int, int]:
    for _ in range(level):
        H, W = (H + 1) // 2, (W + 1) // 2
    return H, W


def pyr_down(img) -> np.ndarray:
    """One pyramid reduction: binomial 5x5 low-pass (clamped taps), keep even samples."""
    a = _f64(img)
    H, W = a.shape
    out = np.empty(((H + 1) // 2, (W + 1) // 2), np.float64)
    lib().ofo_pyr_down(a, H, W, out)
    return out


def pyramid(img, levels: int) -> list[np.ndarray]:
    out = [_f64(img)]
    for _ in range(levels - 1):
        out.append(pyr_down(out[-1]))
    return out


def bilinear(img, x: float, y: float) -> float:
    a = _f64(img)
    return float(lib().ofo_bilinear(a, a.shape[0], a.shape[1], float(x), float(y)))


def upsample_flow(fc, H: int, W: int) -> np.ndarray:
    """u_l(x, y) = 2 * bilinear(u_{l+1}; x/2, y/2)."""
    a = _f64(fc)
    out = np.empty((H, W), np.float64)
    lib().ofo_upsample_flow(a, a.shape[0], a.shape[1], out, H, W)
    return out


def warp_grad(I2, u, v):
    """I2 warped by (u, v) and the gradient of I2 at the displaced positions: (Iw, gx, gy)."""
    a = _f64(I2)
    Iw, gx, gy = (np.empty_like(a) for _ in range(3))
    lib().ofo_warp_grad(a, _f64(u), _f64(v), a.shape[0], a.shape[1], Iw, gx, gy)
    return Iw, gx, gy


def window_sum(c, r: int) -> np.ndarray:
    a = _f64(c)
    out = np.empty_like(a)
    lib().ofo_window_sum(a, a.shape[0], a.shape[1], int(r), out)
    return out


def solve(Sa, Sb, Sc, Sd, Se, fu=None, fv=None):
    """Per-pixel 2x2 normal equations [Sa Sb; Sb Sc] x = [Sd; Se].

    Returns (xu, xv, det/tr^2 (-1 when tr <= 0), solved). Where the singular guard
    fails, x takes the fallback (fu, fv), zero by default.
    """
    arrs = [_f64(x).ravel() for x in (Sa, Sb, Sc, Sd, Se)]
    n = arrs[0].size
    fu = np.zeros(n) if fu is None else _f64(fu).ravel()
    fv = np.zeros(n) if fv is None else _f64(fv).ravel()
    xu, xv, q = (np.empty(n) for _ in range(3))
    ok = np.empty(n, np.int32)
    lib().ofo_solve(*arrs, fu, fv, n, xu, xv, q, ok)
    shp = np.shape(Sa)
    return xu.reshape(shp), xv.reshape(shp), q.reshape(shp), ok.reshape(shp).astype(bool)


def lk_iteration(P1, P2, u, v, r: int):
    """One Jacobi Gauss-Newton iteration at one level. Returns (u', v', det/tr^2)."""
    a, b = _f64(P1), _f64(P2)
    H, W = a.shape
    un, vn, q = (np.empty((H, W)) for _ in range(3))
    if lib().ofo_lk_iteration(a, b, H, W, int(r), _f64(u), _f64(v), un, vn, q):
        raise MemoryError("oracle iteration failed")
    return un, vn, q


def lk_iteration_i1grad(P1, P2, u, v, r: int):
    """One iteration of the variant linearised with the first image's gradient (window
    matrix fixed per level). Returns (u', v', det/tr^2)."""
    a, b = _f64(P1), _f64(P2)
    H, W = a.shape
    un, vn, q = (np.empty((H, W)) for _ in range(3))
    if lib().ofo_lk_iteration_i1grad(a, b, H, W, int(r), _f64(u), _f64(v), un, vn, q):
        raise MemoryError("oracle iteration failed")
    return un, vn, q


def flow(I1, I2, levels: int, radius: int, iterations: int, want_ratio: bool = False, i1grad: bool = False):
    """Dense coarse-to-fine flow at level 0. Returns (u, v) or (u, v, min det/tr^2 at level 0).
    i1grad=True: the variant with the first image's gradient (window matrix fixed per level)."""
    a, b = _f64(I1), _f64(I2)
    if a.shape != b.shape or a.ndim != 2:
        raise ValueError("I1 and I2 must be 2-D arrays of one shape")
    H, W = a.shape
    u = np.empty((H, W))
    v = np.empty((H, W))
    q = np.empty((H, W)) if want_ratio else None
    rc = lib().ofo_flow_variant(a, b, H, W, int(levels), int(radius), int(iterations), u, v,
                                q.ctypes.data if q is not None else None, 1 if i1grad else 0)
    if rc:
        raise ValueError("oracle flow failed (bad arguments or out of memory)")
    return (u, v, q) if want_ratio else (u, v)


def flow_stored(I1, I2, levels: int, radius: int, iterations: int, storage: str = "f16"):
    """The coarse-to-fine flow (Sect. 2.4) in FP64 on a pyramid whose reduced levels are
    rounded to a storage precision after each reduction ("f32", "f16" or "bf16", round to
    nearest even), level 0 kept exact: the method run on the inputs a storage-limited
    implementation holds. The steps are this module's pyr_down, upsample_flow and
    lk_iteration, in the order of flow(). Returns (u, v)."""
    def bf16(a):
        x = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
        r = ((x + 0x7FFF + ((x >> 16) & 1)) >> 16) << 16
        return r.astype(np.uint32).view(np.float32).astype(np.float64)
    rnd = {"f32": lambda a: np.asarray(a, np.float32).astype(np.float64),
           "f16": lambda a: np.asarray(a, np.float64).astype(np.float16).astype(np.float64),
           "bf16": bf16}[storage]
    P1, P2 = [_f64(I1)], [_f64(I2)]
    for _ in range(levels - 1):
        P1.append(rnd(pyr_down(P1[-1])))
        P2.append(rnd(pyr_down(P2[-1])))
    u = v = None
    for l in range(levels - 1, -1, -1):
        Hl, Wl = P1[l].shape
        if l == levels - 1:
            u, v = np.zeros((Hl, Wl)), np.zeros((Hl, Wl))
        else:
            u, v = upsample_flow(u, Hl, Wl), upsample_flow(v, Hl, Wl)
        for _ in range(iterations):
            u, v, _ = lk_iteration(P1[l], P2[l], u, v, radius)
    return u, v


ZNSSD_RADIUS = 5      # Sect. 2.4: local statistics over a radius of 5 pixels
ZNSSD_EPS = 1.0       # added to the local variance (intensity units squared)


def znssd(img, rho: int = ZNSSD_RADIUS, eps: float = ZNSSD_EPS) -> np.ndarray:
    """Eq. 2 local normalisation: (I - local mean) / sqrt(local variance + eps)."""
    a = _f64(img)
    out = np.empty_like(a)
    lib().ofo_znssd(a, a.shape[0], a.shape[1], int(rho), float(eps), out)
    return out


def sbubble_count(u, Tv: float) -> int:
    """Eq. 3 numerator: vectors with streamwise component u <= Tv (FP32 comparison)."""
    a = np.ascontiguousarray(u, dtype=np.float32)
    return int(lib().ofo_sbubble_count(a, a.shape[0], a.shape[1], float(np.float32(Tv))))


def sbubble_threshold(mean_u) -> float:
    """Eq. 3 threshold T_v = (min + max)/2 of the mean streamwise field."""
    a = np.ascontiguousarray(mean_u, dtype=np.float32)
    return float(lib().ofo_sbubble_threshold(a, a.shape[0], a.shape[1]))


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
