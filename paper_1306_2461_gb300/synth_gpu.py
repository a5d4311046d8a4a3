"""Time-resolved particle-image streams generated on the GPU (input generation only; no
part of the flow method).

The physics is that of synth.ParticleStream: particles seeded uniformly (synth.
sample_positions), advected by a fourth-order Runge-Kutta step over one frame in the
vortex street of synth.karman_flow (freestream plus two rows of Lamb-Oseen vortices of
alternating sign drifting downstream), re-seeded at the inflow edge when they leave on
the right, rendered as point-sampled Gaussians at pixel centres, with Gaussian noise,
rounded half-even and clipped to the bit depth. Ground truth for the pair (k, k+1) is the
RK4 one-frame displacement from each grid point at frame time k.

The CPU generator takes about half a second per 2048^2 frame and its RK4 step a third of
a second; serving benchmarks need thousands of consecutive frames, so this module runs
the same steps with torch on the device (float64), vectorised over particles and
vortices, and copies each finished frame to a pinned host buffer (the server takes
frames from host memory, as from a camera). Rendering accumulates with atomic adds, so
the summation order (and, rarely, a rounding of the quantised value) may differ from the
CPU generator and between runs; the frames of one run are what every served and
alone-computed field of that run is computed from.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import synth


class GpuParticleStream:
    def __init__(self, H, W, seed, bits=12, density=0.03, peak=3200.0, noise=32.0, sigma=1.0, device="cuda",
                 U=3.0, drift=2.0, vpeak=2.5, spacing=0.3, offset=0.1, rc_frac=0.04):
        self.H, self.W, self.bits = H, W, bits
        self.peak, self.noise, self.sigma = peak, noise, sigma
        self.dev = torch.device(device)
        self.pad = 12.0
        self.t = 0.0
        rng, _ = synth._rngs(seed, 2)
        px, py = synth.sample_positions(H, W, density, self.pad, rng)
        f64 = dict(dtype=torch.float64, device=self.dev)
        self.px = torch.as_tensor(px, **f64)
        self.py = torch.as_tensor(py, **f64)
        self.gen = torch.Generator(device=self.dev)
        self.gen.manual_seed(int(seed) * 7919 + 17)
        # the vortex street of synth.karman_flow
        self.U, self.drift, self.vpeak = U, drift, vpeak
        self.L = spacing * W
        self.rc = rc_frac * min(H, W)
        self.nv = int(math.ceil(W / self.L)) + 3
        cx0, cy, sgn = [], [], []
        for k in range(-1, self.nv):
            for row, s in ((0, 1.0), (1, -1.0)):
                cx0.append((k + 0.5 * row) * self.L)
                cy.append(H / 2.0 + (offset * H if row else -offset * H))
                sgn.append(s)
        self.cx0 = torch.tensor(cx0, **f64)
        self.cy = torch.tensor(cy, **f64)
        self.sgn = torch.tensor(sgn, **f64)

    def velocity(self, x, y, t):
        """Vortex-street velocity (px/frame) at frame time t, at points (x, y)."""
        cx = torch.remainder(self.cx0 + self.drift * t, self.nv * self.L) - self.L
        dx = x[:, None] - cx[None, :]
        dy = y[:, None] - self.cy[None, :]
        rho2 = dx * dx + dy * dy
        rho = torch.sqrt(rho2)
        safe = torch.where(rho > 0, rho, torch.ones_like(rho))
        vt = self.vpeak * (self.rc / safe) * (1.0 - torch.exp(-rho2 / (self.rc * self.rc))) / synth.LAMB_OSEEN_PEAK
        vt = torch.where(rho > 0, vt, torch.zeros_like(vt))
        ux = self.U + (-self.sgn * vt * dy / safe).sum(1)
        uy = (self.sgn * vt * dx / safe).sum(1)
        return ux, uy

    def _rk4(self, x, y, t):
        k1 = self.velocity(x, y, t)
        k2 = self.velocity(x + 0.5 * k1[0], y + 0.5 * k1[1], t + 0.5)
        k3 = self.velocity(x + 0.5 * k2[0], y + 0.5 * k2[1], t + 0.5)
        k4 = self.velocity(x + k3[0], y + k3[1], t + 1.0)
        return ((k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0]) / 6.0,
                (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1]) / 6.0)

    def frame(self) -> torch.Tensor:
        """The current frame on the device, (H, W) uint16 (uint8 for bits <= 8)."""
        H, W = self.H, self.W
        rad = int(math.ceil(4.0 * self.sigma))
        offs = torch.arange(-rad, rad + 1, device=self.dev, dtype=torch.int64)
        ix = torch.round(self.px).to(torch.int64)
        iy = torch.round(self.py).to(torch.int64)
        inv = 1.0 / (2.0 * self.sigma * self.sigma)
        xx = ix[:, None] + offs[None, :]
        yy = iy[:, None] + offs[None, :]
        wx = torch.exp(-((xx.to(torch.float64) - self.px[:, None]) ** 2) * inv)
        wy = torch.exp(-((yy.to(torch.float64) - self.py[:, None]) ** 2) * inv)
        w = (self.peak * wy)[:, :, None] * wx[:, None, :]
        ok = ((yy >= 0) & (yy < H))[:, :, None] & ((xx >= 0) & (xx < W))[:, None, :]
        idx = yy[:, :, None] * W + xx[:, None, :]
        img = torch.zeros(H * W, dtype=torch.float64, device=self.dev)
        img.index_add_(0, idx[ok], w[ok])
        if self.noise > 0:
            img = img + self.noise * torch.randn(H * W, generator=self.gen, dtype=torch.float64, device=self.dev)
        q = torch.clamp(torch.round(img), 0, (1 << self.bits) - 1).to(torch.int32).reshape(H, W)
        return q.to(torch.uint8 if self.bits <= 8 else torch.uint16)

    def ground_truth(self, step=1):
        """RK4 one-frame displacement from the grid points (every `step`-th row and column)
        at the current frame time, float32 (H/step, W/step) tensors on the device."""
        ys = torch.arange(0, self.H, step, dtype=torch.float64, device=self.dev)
        xs = torch.arange(0, self.W, step, dtype=torch.float64, device=self.dev)
        yy, xx = torch.meshgrid(ys, xs, indexing="ij")
        u, v = self._rk4(xx.reshape(-1), yy.reshape(-1), self.t)
        return u.reshape(yy.shape).float(), v.reshape(yy.shape).float()

    def advance(self):
        dx, dy = self._rk4(self.px, self.py, self.t)
        self.px = self.px + dx
        self.py = self.py + dy
        self.t += 1.0
        out = self.px >= self.W + self.pad
        n = int(out.sum())
        if n:
            nx = torch.rand(n, generator=self.gen, dtype=torch.float64, device=self.dev) * 9.0 - self.pad
            ny = torch.rand(n, generator=self.gen, dtype=torch.float64, device=self.dev) * (self.H + 2 * self.pad) \
                - self.pad
            self.px[out] = nx
            self.py[out] = ny


def render_sequence(stream: GpuParticleStream, n: int, gt_at=(), gt_step=1):
    """n consecutive frames of `stream` in pinned host memory, and the ground truth of the
    pairs (k, k+1) for k in gt_at: ({k: (u, v)} on the device)."""
    gts = {}
    buf = None
    for k in range(n):
        f = stream.frame()
        if buf is None:   # one pinned allocation for the whole sequence
            buf = torch.empty((n,) + tuple(f.shape), dtype=f.dtype, pin_memory=True)
        buf[k].copy_(f)
        if k in gt_at:
            gts[k] = stream.ground_truth(gt_step)
        stream.advance()
    return [buf[k] for k in range(n)], gts


def per_stream_arrivals(n_streams: int, n_frames: int, rate_per_stream: float, seed: int):
    """Open-loop Poisson arrivals with exactly n_frames per stream: list of (time_s,
    stream) sorted by time, and each stream's last arrival time."""
    rng, = synth._rngs(seed + 91, 1)
    ev, last = [], []
    for s in range(n_streams):
        t = np.cumsum(rng.exponential(1.0 / rate_per_stream, n_frames))
        ev += [(float(x), s) for x in t]
        last.append(float(t[-1]))
    ev.sort()
    return ev, last
