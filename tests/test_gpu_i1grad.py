"""The variant linearised with the first image's gradient (OF_FLAG_I1GRAD): the window
matrix is summed once per level from I1, each iteration sums two channels. Parity with
the oracle's variant on the same inputs, to the same tolerances as the main path."""
import numpy as np
import pytest

from paper_1306_2461_gb300 import synth
from helpers import gpu_flow, parity_check, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def of():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_2461_gb300 import build
    build.build()
    from paper_1306_2461_gb300 import of as ofmod
    return ofmod


def run(of, p, L, r, n, storage, bits=None, extra=0):
    return gpu_flow(p, L, r, n, storage, bits=bits, flags=of.OF_FLAG_I1GRAD | extra)


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("H,W,L,r,n", [(256, 256, 2, 5, 4), (77, 301, 3, 4, 2), (1, 1, 1, 1, 1)])
def test_identical_images_exactly_zero(of, storage, H, W, L, r, n):
    rng = np.random.default_rng(H + W)
    I = rng.integers(0, 4096, (H, W)).astype(np.uint16)
    u, v = run(of, (I, I), L, r, n, storage, bits=12)
    assert np.all(u == 0.0) and np.all(v == 0.0)


def test_integer_translation_exact(of):
    I1, I2 = synth.translated_texture_pair(128, 160, (3.0, -2.0), seed=1)
    I1 = np.rint(I1).astype(np.uint16)
    I2 = np.rint(I2).astype(np.uint16)
    u, v = run(of, (I1, I2), 3, 4, 15, "f32", bits=12)
    m = 24
    assert np.abs(u[m:-m, m:-m] - 3.0).max() < 1e-4 and np.abs(v[m:-m, m:-m] + 2.0).max() < 1e-4


def test_c1_pair256_fp32(of, oracle_mod):
    p = synth.make_c1()
    u, v = run(of, p, 2, 5, 4, "f32")
    parity_check(u, v, p, oracle_mod, 2, 5, 4, "f32", "256^2 u8 (I1 gradient)", i1grad=True)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_c2_vortex_shear(of, oracle_mod, storage):
    p = synth.make_c2(384, 320, seed=1)
    u, v = run(of, p, 3, 4, 5, storage)
    parity_check(u, v, p, oracle_mod, 3, 4, 5, storage, "384x320 u16 (I1 gradient)", i1grad=True)


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("H,W,L,r,n", [(200, 150, 3, 4, 3), (37, 301, 2, 3, 2), (64, 64, 1, 10, 3),
                                       (130, 66, 4, 2, 1), (97, 33, 2, 7, 2), (2, 9, 2, 2, 2), (5, 3, 4, 10, 2)])
def test_ragged_and_degenerate_shapes_every_pixel(of, oracle_mod, storage, H, W, L, r, n):
    # fixed and generic radii (7 has no specialised kernel), ragged tiles, tiny images
    I1, I2 = synth.translated_texture_pair(H, W, (0.4, -0.3), seed=H + W, amp=800.0, offset=2000.0,
                                           fmax=1.0 / 6.0)
    I1 = np.rint(I1).astype(np.uint16)
    I2 = np.rint(I2).astype(np.uint16)
    u, v = run(of, (I1, I2), L, r, n, storage, bits=12)
    parity_check(u, v, (I1, I2), oracle_mod, L, r, n, storage, f"{H}x{W} (I1 gradient)", margin=0,
                 workload=False, i1grad=True)


def test_differs_from_second_image_gradient(of):
    p = synth.make_c2(256, 256, seed=2)
    ua, va = gpu_flow(p, 3, 4, 3, "f32")
    ub, vb = run(of, p, 3, 4, 3, "f32")
    assert np.abs(ua - ub).max() > 1e-3


def test_graph_replay_and_reuse_equal_direct(of):
    import torch
    s = synth.ParticleStream(160, 224, seed=4)
    frames = []
    for _ in range(3):
        frames.append(s.frame())
        s.advance()
    d = [to_dev(x) for x in frames]
    pg = of.Plan.make(160, 224, 3, 4, 3, bits=12, storage="f16", flags=of.OF_FLAG_I1GRAD)
    pd = of.Plan.make(160, 224, 3, 4, 3, bits=12, storage="f16", flags=of.OF_FLAG_I1GRAD | of.OF_FLAG_NO_GRAPH)
    st = torch.cuda.Stream()
    with of.Flow(pg) as f, of.Flow(pd) as g, torch.cuda.stream(st):
        for _ in range(2):     # the second call replays the cached graph
            u1, v1 = f.compute(d[0], d[1], stream=st)
        u1, v1 = u1.clone(), v1.clone()
        u2, v2 = g.compute(d[0], d[1], stream=st)
        u3, v3 = f.compute(None, d[2], stream=st)    # frame 1's pyramid reused
        u4, v4 = g.compute(d[1], d[2], stream=st)
        st.synchronize()
        assert torch.equal(u1, u2) and torch.equal(v1, v2)
        assert torch.equal(u3, u4) and torch.equal(v3, v4)


def test_noalloc_entry_accepts_the_variant(of):
    import torch
    p = synth.make_c1(128, 160, seed=9)
    plan = of.Plan.make(128, 160, 2, 4, 3, bits=8, storage="f32", flags=of.OF_FLAG_I1GRAD)
    u = torch.empty(128, 160, device="cuda")
    v = torch.empty(128, 160, device="cuda")
    of.compute_noalloc(plan, to_dev(p.I1), to_dev(p.I2), u, v)
    torch.cuda.synchronize()
    ua, va = run(of, p, 2, 4, 3, "f32", bits=8)
    assert np.array_equal(u.cpu().numpy().astype(np.float64), ua)
    assert np.array_equal(v.cpu().numpy().astype(np.float64), va)


def test_batched_host_and_served_variant_equal_per_pair(of):
    # the variant through of_compute_batch (with a reused pyramid), of_compute_batch_host
    # and the serving loop: of_compute's bits
    import torch
    from paper_1306_2461_gb300 import serve
    sizes = [(160, 224), (96, 128), (200, 136)]
    frames = []
    for k, (H, W) in enumerate(sizes):
        st = synth.ParticleStream(H, W, seed=60 + k)
        fr = []
        for _ in range(3):
            fr.append(st.frame())
            st.advance()
        frames.append(fr)
    fl = of.OF_FLAG_I1GRAD
    plans = [of.Plan.make(H, W, 3, 4, 3, bits=12, storage="f16", flags=fl) for H, W in sizes]

    def alone(k, j):
        with of.Flow(plans[k]) as f:
            u, v = f.compute(to_dev(frames[k][j - 1]), to_dev(frames[k][j]))
            torch.cuda.synchronize()
        return u, v

    flows = [of.Flow(p) for p in plans]
    of.compute_batch(flows, [to_dev(f[0]) for f in frames], [to_dev(f[1]) for f in frames])
    ub, vb = of.compute_batch(flows, [None, to_dev(frames[1][1]), None], [to_dev(f[2]) for f in frames])
    torch.cuda.synchronize()
    for k in range(3):
        u1, v1 = alone(k, 2)
        assert torch.equal(ub[k], u1) and torch.equal(vb[k], v1), k
    hu = [torch.empty(s_, dtype=torch.float32).pin_memory() for s_ in sizes]
    hv = [torch.empty(s_, dtype=torch.float32).pin_memory() for s_ in sizes]
    du = [torch.empty(s_, device="cuda") for s_ in sizes]
    dv = [torch.empty(s_, device="cuda") for s_ in sizes]
    hf = [[serve.pinned_frame(x) for x in fr] for fr in frames]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        of.compute_batch_host(flows, [h[0] for h in hf], [h[1] for h in hf], hu, hv,
                              [to_dev(f[0]) for f in frames], [to_dev(f[1]) for f in frames], du, dv, stream=s)
    s.synchronize()
    for k in range(3):
        u1, v1 = alone(k, 1)
        assert torch.equal(hu[k], u1.cpu()) and torch.equal(hv[k], v1.cpu()), k
    with serve.Server(levels=3, radius=4, iterations=3, bits=12, storage="f16", max_batch=8, flags=fl) as srv:
        sids = [srv.open_stream(H, W) for H, W in sizes]
        outs = {}
        for j in range(3):
            for k, sid in enumerate(sids):
                outs[(k, j)] = (torch.empty(sizes[k], device="cuda"), torch.empty(sizes[k], device="cuda"))
                srv.submit(sid, hf[k][j], *outs[(k, j)], tag=10 * k + j)
        srv.drain()
        assert all(r["status"] == 0 for r in srv.poll(0))
    for k in range(3):
        for j in (1, 2):
            u1, v1 = alone(k, j)
            assert torch.equal(outs[(k, j)][0], u1) and torch.equal(outs[(k, j)][1], v1), (k, j)
    best, cands = of.autotune_batch(flows, [to_dev(f[0]) for f in frames], [to_dev(f[1]) for f in frames], reps=1)
    assert len(cands) == 8 and all(c["phased"] == 1 and c["stage_i2"] == 0 for c in cands)
    assert sum(c["branches"] == 2 for c in cands) == 2
    of.tuning_clear()
    for f in flows:
        f.close()
