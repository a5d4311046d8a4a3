"""Seeded synthetic inputs: particle-image pairs with an analytic displacement field.

The paper measures real laser-sheet particle images of a backward-facing-step flow
(Sect. 2.2: 8-bit camera, 20 um particles; Sect. 2.4: ROI 1792x384). Those images are
not available, so every workload here is rendered: Gaussian particles (sigma 1 px)
point-sampled at pixel centres, a second frame with every particle moved by a known
displacement field, additive Gaussian noise, rounding half-even and clipping to the
camera's bit depth.

Convention: the displacement u(x) maps frame 1 onto frame 2, I1(x) ~ I2(x + u(x)),
with x the column index, y the row index, u positive to the right and down.

This module holds input generation only. It contains none of the flow method's
arithmetic (no pyramid, warp, gradient, window sum or solve), so the oracle and the
CUDA path can both be fed from it without sharing any of the method's code.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable

import numpy as np

FlowFn = Callable[[np.ndarray, np.ndarray], tuple[np.ndarray, np.ndarray]]


def _rngs(seed: int, n: int) -> list[np.random.Generator]:
    """Independent child generators (PCG64) from one seed."""
    return [np.random.Generator(np.random.PCG64(s))
            for s in np.random.SeedSequence(seed).spawn(n)]


# --------------------------------------------------------------------------- flows
def _lamb_oseen_norm() -> tuple[float, float]:
    """max_t (1 - exp(-t^2)) / t and its argmax; the peak of the Lamb-Oseen profile."""
    t = np.linspace(1.0, 1.3, 300001)
    f = (1.0 - np.exp(-t * t)) / t
    k = int(np.argmax(f))
    return float(f[k]), float(t[k])


LAMB_OSEEN_PEAK, LAMB_OSEEN_PEAK_RADIUS = _lamb_oseen_norm()  # 0.638..., 1.1209...


def lamb_oseen(x, y, cx, cy, peak, rc, sign=1.0):
    """Lamb-Oseen vortex velocity whose azimuthal speed peaks at `peak` px at rho = 1.1209 rc."""
    dx = x - cx
    dy = y - cy
    rho2 = dx * dx + dy * dy
    rho = np.sqrt(rho2)
    with np.errstate(divide="ignore", invalid="ignore"):
        vt = peak * (rc / rho) * (1.0 - np.exp(-rho2 / (rc * rc))) / LAMB_OSEEN_PEAK
        ux = np.where(rho > 0, -sign * vt * dy / rho, 0.0)
        uy = np.where(rho > 0, sign * vt * dx / rho, 0.0)
    return ux, uy


def uniform_flow(du: float, dv: float) -> FlowFn:
    def f(x, y):
        return np.full(np.shape(x), du, dtype=np.float64), np.full(np.shape(y), dv, dtype=np.float64)
    return f


def vortex_shear_flow(H: int, W: int, peak=6.0, rc=80.0, dU=8.0, thickness=40.0) -> FlowFn:
    """Lamb-Oseen vortex at the image centre plus a tanh shear layer u_x += dU/2 tanh(2(y-H/2)/delta).

    The vortex turns with the layer's own vorticity (a Kelvin-Helmholtz roller), so the
    two add up to ~peak + dU/2 = 10 px above and below the core.
    """
    def f(x, y):
        ux, uy = lamb_oseen(x, y, W / 2.0, H / 2.0, peak, rc, sign=-1.0)
        ux = ux + 0.5 * dU * np.tanh(2.0 * (y - H / 2.0) / thickness)
        return ux, uy
    return f


def band_limited_flow(H: int, W: int, kmax: float, umax: float, rng: np.random.Generator) -> FlowFn:
    """Random periodic flow with complex Gaussian Fourier coefficients for |k| <= kmax.

    Integer wavenumbers on the H x W torus; the grid field is scaled so that max |u| = umax,
    and evaluated off-grid by cubic spline interpolation with periodic wrap (the field has
    no energy above kmax/min(H,W) cycles/px, so the interpolation error is negligible).
    """
    from scipy import ndimage

    ky = np.fft.fftfreq(H) * H
    kx = np.fft.fftfreq(W) * W
    KX, KY = np.meshgrid(kx, ky)
    mask = (KX * KX + KY * KY) <= kmax * kmax
    comp = []
    for _ in range(2):
        c = (rng.standard_normal((H, W)) + 1j * rng.standard_normal((H, W))) * mask
        comp.append(np.real(np.fft.ifft2(c)))
    mag = np.sqrt(comp[0] ** 2 + comp[1] ** 2).max()
    gu = comp[0] * (umax / mag)
    gv = comp[1] * (umax / mag)
    cu = ndimage.spline_filter(gu, order=3, mode="grid-wrap")
    cv = ndimage.spline_filter(gv, order=3, mode="grid-wrap")

    def f(x, y):
        coords = np.stack([np.asarray(y, np.float64).ravel(), np.asarray(x, np.float64).ravel()])
        shp = np.shape(x)
        ux = ndimage.map_coordinates(cu, coords, order=3, mode="grid-wrap", prefilter=False)
        uy = ndimage.map_coordinates(cv, coords, order=3, mode="grid-wrap", prefilter=False)
        return ux.reshape(shp), uy.reshape(shp)
    return f


def karman_flow(H: int, W: int, t: float, U=3.0, drift=2.0, peak=2.5, spacing=0.3, offset=0.1,
                rc_frac=0.04) -> FlowFn:
    """Vortex-street velocity (px/frame) at frame time t: freestream U plus two rows of
    Lamb-Oseen vortices at y = H/2 +- offset*H, alternating sign, spaced spacing*W,
    drifting +drift px/frame (the street wraps around the image width)."""
    L = spacing * W
    rc = rc_frac * min(H, W)
    nv = int(math.ceil(W / L)) + 3

    def f(x, y):
        ux = np.full(np.shape(x), U, np.float64)
        uy = np.zeros(np.shape(x), np.float64)
        for k in range(-1, nv):
            for row, sgn in ((0, 1.0), (1, -1.0)):
                cx = ((k + 0.5 * row) * L + drift * t) % (nv * L) - L
                cy = H / 2.0 + (offset * H if row else -offset * H)
                a, b = lamb_oseen(x, y, cx, cy, peak, rc, sgn)
                ux += a
                uy += b
        return ux, uy
    return f


# ----------------------------------------------------------------------- rendering
def render_particles(H: int, W: int, px: np.ndarray, py: np.ndarray, peak: float,
                     sigma: float = 1.0) -> np.ndarray:
    """Sum of point-sampled Gaussians peak*exp(-|x-p|^2/(2 sigma^2)) at pixel centres (float64).
    Every (particle, tap) contribution is gathered first, offset by offset, and summed into
    the image by one bincount."""
    rad = int(math.ceil(4.0 * sigma))
    ix = np.rint(px).astype(np.int64)
    iy = np.rint(py).astype(np.int64)
    inv = 1.0 / (2.0 * sigma * sigma)
    idx, wts = [], []
    for dy in range(-rad, rad + 1):
        yy = iy + dy
        wy = np.exp(-((yy - py) ** 2) * inv)
        oky = (yy >= 0) & (yy < H)
        for dx in range(-rad, rad + 1):
            xx = ix + dx
            ok = oky & (xx >= 0) & (xx < W)
            idx.append(yy[ok] * W + xx[ok])
            wts.append(peak * wy[ok] * np.exp(-((xx[ok] - px[ok]) ** 2) * inv))
    img = np.bincount(np.concatenate(idx), weights=np.concatenate(wts), minlength=H * W)
    return img.astype(np.float64).reshape(H, W)


def quantise(img: np.ndarray, noise: float, bits: int, rng: np.random.Generator) -> np.ndarray:
    """Add N(0, noise), round half-even, clip to [0, 2^bits - 1], store as uint8/uint16."""
    out = np.rint(img + rng.normal(0.0, noise, img.shape)) if noise > 0 else np.rint(img)
    out = np.clip(out, 0, (1 << bits) - 1)
    return out.astype(np.uint8 if bits <= 8 else np.uint16)


def sample_positions(H, W, density, pad, rng, density_fn=None):
    """Uniform particle positions over [-pad, W+pad) x [-pad, H+pad), `density` particles/px.

    `density_fn(y)` (optional) gives a per-row density; rejection sampling thins the
    uniform draw down to it.
    """
    area = (W + 2 * pad) * (H + 2 * pad)
    dmax = density
    n = rng.poisson(dmax * area)
    x = rng.uniform(-pad, W + pad, n)
    y = rng.uniform(-pad, H + pad, n)
    if density_fn is not None:
        keep = rng.uniform(0, dmax, n) < density_fn(y)
        x, y = x[keep], y[keep]
    return x, y


@dataclasses.dataclass
class Pair:
    I1: np.ndarray          # uint8 / uint16, H x W
    I2: np.ndarray
    u_gt: np.ndarray        # float64 H x W, analytic displacement at pixel centres
    v_gt: np.ndarray
    bits: int
    meta: dict

    @property
    def shape(self):
        return self.I1.shape


def particle_pair(H, W, flow: FlowFn, *, density, peak, noise, bits, seed, sigma=1.0,
                  umax=None, density_fn=None, meta=None, gain=None, background=None) -> Pair:
    r_pos, r_n1, r_n2 = _rngs(seed, 3)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    ug, vg = flow(xx, yy)
    if umax is None:
        umax = float(np.sqrt(ug * ug + vg * vg).max())
    pad = umax + 4.0 * sigma + 1.0
    px, py = sample_positions(H, W, density, pad, r_pos, density_fn)
    du, dv = flow(px, py)
    f1 = render_particles(H, W, px, py, peak, sigma)
    f2 = render_particles(H, W, px + du, py + dv, peak, sigma)
    if gain is not None:          # illumination that does not move with the particles
        f1, f2 = f1 * gain, f2 * gain
    if background is not None:
        f1, f2 = f1 + background, f2 + background
    return Pair(quantise(f1, noise, bits, r_n1), quantise(f2, noise, bits, r_n2),
                np.asarray(ug, np.float64), np.asarray(vg, np.float64), bits,
                dict(meta or {}, H=H, W=W, density=density, peak=peak, noise=noise, seed=seed,
                     n_particles=int(px.size)))


# -------------------------------------------------------------- named workloads
@dataclasses.dataclass(frozen=True)
class Workload:
    """A workload shape: image size, bit depth, and the flow parameters (levels, radius, iterations)."""
    name: str
    H: int
    W: int
    bits: int
    levels: int
    radius: int
    iterations: int
    seed: int


C1 = Workload("pair256_u8_translate", 256, 256, 8, 2, 5, 4, 0)
C2 = Workload("pair1024_u16_vortex_shear", 1024, 1024, 12, 3, 4, 5, 1)
C3 = Workload("pair2048_u16_lowseed_bandlimited", 2048, 2048, 12, 4, 3, 6, 2)
WORKLOADS = {w.name: w for w in (C1, C2, C3)}


def make_c1(H=256, W=256, seed=0) -> Pair:
    """256^2 uint8, 0.02 particles/px, peak 200, noise 2, uniform (1.3, -0.7) px."""
    return particle_pair(H, W, uniform_flow(1.3, -0.7), density=0.02, peak=200.0, noise=2.0,
                         bits=8, seed=seed, meta={"workload": C1.name})


def make_c2(H=1024, W=1024, seed=1, rc=80.0, thickness=40.0) -> Pair:
    """12-bit, 0.03 particles/px, Lamb-Oseen vortex (peak 6 px, rc 80) + tanh shear (dU 8, 40 px).

    12-bit peak 3200 and noise std 32 (the 8-bit values x16). Smaller H, W keep the same
    physical parameters, so a reduced-size case has the same displacement magnitudes.
    """
    return particle_pair(H, W, vortex_shear_flow(H, W, 6.0, rc, 8.0, thickness), density=0.03,
                         peak=3200.0, noise=32.0, bits=12, seed=seed, meta={"workload": C2.name})


def make_c2_uneven_light(H=1024, W=1024, seed=1) -> Pair:
    """The 1024^2 vortex + shear workload under uneven illumination, the case the local
    normalisation of Eq. 2 is for: 0.05 particles/px, a laser-sheet-like gain varying
    smoothly from 0.4 to 1.6 across the image and a background rising from 300 to 900
    counts (12-bit), so that no pixel clips at zero."""
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    gain = 1.0 + 0.6 * np.cos(np.pi * xx / W) * np.cos(0.5 * np.pi * yy / H)
    background = 300.0 + 600.0 * (yy / max(H - 1, 1))
    return particle_pair(H, W, vortex_shear_flow(H, W, 6.0, 80.0, 8.0, 40.0), density=0.05, peak=2400.0,
                         noise=24.0, bits=12, seed=seed, gain=gain, background=background,
                         meta={"workload": "pair1024_u16_uneven_light"})


def bfs_flow(H: int, W: int, U=8.0, back=-1.0, y_layer=0.6, delta=20.0, n_vort=5, peak=2.0, rc=20.0) -> FlowFn:
    """A flow shaped like the region downstream of a backward-facing step (Sect. 2.3): a
    shear layer at y = y_layer*H between the free stream (U px/frame, upper part of the
    image) and a slow recirculation (back px/frame, lower part), with a row of vortices
    rolled up along the layer. Max |u| ~ U + peak."""
    yl = y_layer * H

    def f(x, y):
        ux = back + 0.5 * (U - back) * (1.0 - np.tanh((y - yl) / delta))
        uy = np.zeros(np.shape(y), np.float64)
        for k in range(n_vort):
            a, b = lamb_oseen(x, y, (k + 0.5) * W / n_vort, yl, peak, rc, sign=1.0)
            ux = ux + a
            uy = uy + b
        return ux, uy
    return f


def make_bfs(H=384, W=1792, seed=5) -> Pair:
    """The region of interest of the paper's setup (1792 x 384, 8-bit camera, Sect. 2.4)
    with particles as the 256^2 workload, displaced by bfs_flow()."""
    return particle_pair(H, W, bfs_flow(H, W), density=0.02, peak=200.0, noise=2.0, bits=8, seed=seed,
                         meta={"workload": "roi1792x384_u8_bfs"})


def make_c3(H=2048, W=2048, seed=2, umax=10.0) -> Pair:
    """12-bit, 0.03 particles/px except 0.002 in rows [0.4H, 0.6H); band-limited flow
    with wavenumbers |k| <= min(H,W)/64 (cutoff 1/64 px^-1), max |u| = 10 px."""
    r_flow, = _rngs(seed + 1000, 1)
    flow = band_limited_flow(H, W, min(H, W) / 64.0, umax, r_flow)

    def dens(y):
        return np.where((y >= 0.4 * H) & (y < 0.6 * H), 0.002, 0.03)
    return particle_pair(H, W, flow, density=0.03, peak=3200.0, noise=32.0, bits=12, seed=seed,
                         umax=umax, density_fn=dens, meta={"workload": C3.name})


BATCH_SIZES = ((256, 256), (512, 512), (1024, 1024), (1024, 2048))  # (H, W)


def make_batch(n=64, seed=3, sizes=BATCH_SIZES) -> list[Pair]:
    """Mixed-size uint8 pairs; per pair U[-3,3]^2 uniform flow plus a random Lamb-Oseen vortex."""
    rng, = _rngs(seed, 1)
    out = []
    for i in range(n):
        H, W = sizes[int(rng.integers(len(sizes)))]
        du, dv = rng.uniform(-3, 3, 2)
        cx, cy = rng.uniform(0.25, 0.75) * W, rng.uniform(0.25, 0.75) * H
        pk = rng.uniform(1, 5)
        rc = rng.uniform(0.05, 0.15) * min(H, W)
        sg = 1.0 if rng.uniform() < 0.5 else -1.0

        def flow(x, y, du=du, dv=dv, cx=cx, cy=cy, pk=pk, rc=rc, sg=sg):
            a, b = lamb_oseen(x, y, cx, cy, pk, rc, sg)
            return a + du, b + dv
        out.append(particle_pair(H, W, flow, density=0.02, peak=200.0, noise=2.0, bits=8,
                                 seed=seed * 100003 + i, meta={"batch_index": i}))
    return out


def same_size_batch(n: int, make=make_c2, seed0=1, **kw) -> list[Pair]:
    """n pairs of one workload with consecutive seeds."""
    return [make(seed=seed0 + 7919 * i, **kw) for i in range(n)]


# --------------------------------------------------------- time-resolved streams
class ParticleStream:
    """A time-resolved sequence of frames: particles advected by RK4 over one frame in a
    vortex-street field, re-seeded at the inflow edge. Ground truth for the pair
    (k, k+1) is the RK4 one-frame displacement from each grid point."""

    def __init__(self, H, W, seed, bits=12, density=0.03, peak=3200.0, noise=32.0, sigma=1.0):
        self.H, self.W, self.bits = H, W, bits
        self.density, self.peak, self.noise, self.sigma = density, peak, noise, sigma
        self.rng, self.nrng = _rngs(seed, 2)
        self.pad = 12.0
        self.t = 0.0
        self.px, self.py = sample_positions(H, W, density, self.pad, self.rng)

    def _rk4(self, x, y, t):
        def vel(xx, yy, tt):
            return karman_flow(self.H, self.W, tt)(xx, yy)
        k1 = vel(x, y, t)
        k2 = vel(x + 0.5 * k1[0], y + 0.5 * k1[1], t + 0.5)
        k3 = vel(x + 0.5 * k2[0], y + 0.5 * k2[1], t + 0.5)
        k4 = vel(x + k3[0], y + k3[1], t + 1.0)
        return ((k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0]) / 6.0,
                (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1]) / 6.0)

    def frame(self) -> np.ndarray:
        img = render_particles(self.H, self.W, self.px, self.py, self.peak, self.sigma)
        return quantise(img, self.noise, self.bits, self.nrng)

    def ground_truth(self):
        yy, xx = np.mgrid[0:self.H, 0:self.W].astype(np.float64)
        return self._rk4(xx, yy, self.t)

    def advance(self):
        dx, dy = self._rk4(self.px, self.py, self.t)
        self.px, self.py = self.px + dx, self.py + dy
        self.t += 1.0
        out = self.px >= self.W + self.pad
        n = int(out.sum())
        if n:
            self.px[out] = self.rng.uniform(-self.pad, -self.pad + 3.0 * 3.0, n)
            self.py[out] = self.rng.uniform(-self.pad, self.H + self.pad, n)


SERVE_MIX = ((512, 512, 8), (1024, 1024, 6), (2048, 2048, 2))  # (H, W, streams): ratio 4:3:1


def serving_streams(seed=4, mix=SERVE_MIX):
    """The 16-stream serving mix: (H, W) per stream and a ParticleStream for each."""
    out = []
    k = 0
    for H, W, n in mix:
        for _ in range(n):
            out.append(ParticleStream(H, W, seed * 1009 + k))
            k += 1
    return out


def poisson_arrivals(n_streams: int, rate_per_stream: float, duration: float, seed: int):
    """Open-loop arrival schedule: list of (time_s, stream) sorted by time."""
    rng, = _rngs(seed + 77, 1)
    ev = []
    for s in range(n_streams):
        t = rng.exponential(1.0 / rate_per_stream)
        while t < duration:
            ev.append((t, s))
            t += rng.exponential(1.0 / rate_per_stream)
    ev.sort()
    return ev


# ----------------------------------------------------------- textures for pins
def band_limited_texture(n_waves=16, fmax=1.0 / 16.0, seed=0, amp=50.0, offset=128.0):
    """T(x, y) = offset + sum of n_waves cosines with random direction, frequency <= fmax
    cycles/px and random phase. Returns a callable evaluated analytically (no interpolation)."""
    rng, = _rngs(seed, 1)
    f = rng.uniform(0.3 * fmax, fmax, n_waves)
    th = rng.uniform(0, 2 * np.pi, n_waves)
    ph = rng.uniform(0, 2 * np.pi, n_waves)
    a = rng.uniform(0.5, 1.0, n_waves) * amp / math.sqrt(n_waves)
    kx = 2 * np.pi * f * np.cos(th)
    ky = 2 * np.pi * f * np.sin(th)

    def T(x, y):
        x = np.asarray(x, np.float64)[..., None]
        y = np.asarray(y, np.float64)[..., None]
        return offset + (a * np.cos(kx * x + ky * y + ph)).sum(-1)
    return T


def translated_texture_pair(H, W, d, seed=0, **kw):
    """I1 = T, I2(x) = T(x - d) (float64), so that I1(x) = I2(x + d) exactly."""
    T = band_limited_texture(seed=seed, **kw)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    return T(xx, yy), T(xx - d[0], yy - d[1])
