"""Seeded input generators: determinism, shapes, value ranges, flow magnitudes."""
import numpy as np

from paper_1306_2461_gb300 import synth


def test_pairs_are_seeded_and_typed():
    a = synth.make_c1(64, 80, seed=3)
    b = synth.make_c1(64, 80, seed=3)
    c = synth.make_c1(64, 80, seed=4)
    assert a.I1.dtype == np.uint8 and a.I1.shape == (64, 80)
    assert np.array_equal(a.I1, b.I1) and np.array_equal(a.I2, b.I2)
    assert not np.array_equal(a.I1, c.I1)
    assert np.all(a.u_gt == 1.3) and np.all(a.v_gt == -0.7)


def test_12bit_pair_range_and_flow_peak():
    p = synth.make_c2(256, 256, seed=1)
    assert p.I1.dtype == np.uint16 and int(p.I1.max()) <= 4095
    speed = np.sqrt(p.u_gt ** 2 + p.v_gt ** 2)
    assert 8.0 < speed.max() < 11.0      # 6 px vortex peak on top of a +-4 px shear


def test_lamb_oseen_peak():
    rc = 80.0
    rho = synth.LAMB_OSEEN_PEAK_RADIUS * rc
    ux, uy = synth.lamb_oseen(np.array([rho]), np.array([0.0]), 0.0, 0.0, 6.0, rc)
    assert abs(np.hypot(ux, uy)[0] - 6.0) < 1e-9
    assert abs(synth.LAMB_OSEEN_PEAK_RADIUS - 1.1209) < 1e-3


def test_single_particle_render():
    img = synth.render_particles(9, 9, np.array([4.0]), np.array([4.0]), 200.0, 1.0)
    assert img[4, 4] == 200.0 and abs(img[4, 5] - 200.0 * np.exp(-0.5)) < 1e-12


def test_band_limited_flow_max_and_low_seeding():
    p = synth.make_c3(256, 256, seed=2)
    s = np.sqrt(p.u_gt ** 2 + p.v_gt ** 2)
    assert abs(s.max() - 10.0) < 1e-6
    band = p.I1[int(0.4 * 256) + 8:int(0.6 * 256) - 8].astype(float)
    rest = p.I1[:int(0.4 * 256) - 8].astype(float)
    assert band.mean() < rest.mean()


def test_batch_mix_and_arrivals():
    b = synth.make_batch(8, seed=3)
    assert len(b) == 8 and all(p.I1.shape in synth.BATCH_SIZES for p in b)
    ev = synth.poisson_arrivals(4, 100.0, 0.5, seed=4)
    assert all(ev[i][0] <= ev[i + 1][0] for i in range(len(ev) - 1))
    assert 100 < len(ev) < 300


def test_stream_frames_advance():
    s = synth.ParticleStream(64, 96, seed=1)
    f0 = s.frame()
    u, v = s.ground_truth()
    s.advance()
    f1 = s.frame()
    assert f0.shape == (64, 96) and f0.dtype == np.uint16 and not np.array_equal(f0, f1)
    assert 1.0 < u.mean() < 5.0


def test_device_stream_generator_has_the_cpu_generators_physics():
    # synth_gpu runs the time-resolved stream with torch; run on the CPU here, its
    # vortex-street velocity and RK4 one-frame displacement equal synth's, and its
    # frames are seeded, typed and advance in time
    import torch
    from paper_1306_2461_gb300 import synth_gpu
    H, W = 64, 96
    g = synth_gpu.GpuParticleStream(H, W, seed=1, device="cpu")
    c = synth.ParticleStream(H, W, seed=1)
    rng = np.random.default_rng(0)
    x = rng.uniform(-10, W + 10, 500)
    y = rng.uniform(-10, H + 10, 500)
    for t in (0.0, 3.5, 40.0):
        ug, vg = g.velocity(torch.from_numpy(x), torch.from_numpy(y), t)
        uc, vc = synth.karman_flow(H, W, t)(x, y)
        assert np.allclose(ug.numpy(), uc, atol=1e-12) and np.allclose(vg.numpy(), vc, atol=1e-12)
    dg = g._rk4(torch.from_numpy(x), torch.from_numpy(y), 2.0)
    dc = c._rk4(x, y, 2.0)
    assert np.allclose(dg[0].numpy(), dc[0], atol=1e-12) and np.allclose(dg[1].numpy(), dc[1], atol=1e-12)
    assert np.allclose(g.px.numpy(), c.px) and np.allclose(g.py.numpy(), c.py)   # same seeding
    f0 = g.frame()
    g.advance()
    f1 = g.frame()
    a0, a1 = f0.to(torch.int32), f1.to(torch.int32)
    assert f0.shape == (H, W) and f0.dtype == torch.uint16 and int(a0.max()) <= 4095
    assert not torch.equal(a0, a1)
    u, v = g.ground_truth()
    assert u.shape == (H, W) and 1.0 < float(u.mean()) < 5.0
