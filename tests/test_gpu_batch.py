"""The batched persistent form (of_compute_batch): the same fields as one of_compute per
pair, bit for bit, and the oracle on sampled pairs, at the full sizes of the
benchmark's launch configuration and of the mixed-size batch."""
import numpy as np
import pytest

from paper_1306_2461_gb300 import synth
from helpers import parity_check, to_dev

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


def single(of, plan, I1, I2):
    import torch
    with of.Flow(plan) as f:
        u, v = f.compute(I1, I2)
        torch.cuda.synchronize()
        assert f.sync_status() == of.OF_OK
    return u, v


def oracle_check(oracle_mod, pair, u, v, L, r, n, storage):
    parity_check(u.cpu().double().numpy(), v.cpu().double().numpy(), pair, oracle_mod, L, r, n, storage,
                 f"{pair.I1.shape[0]}x{pair.I1.shape[1]}")


@pytest.mark.parametrize("branches", [1, 2])
def test_bench_configuration_full_size(of, oracle_mod, branches):
    # 64 pairs of 1024^2 12-bit frames, FP16 storage, 3 levels, r = 4, 5 iterations:
    # the launch the benchmark times (8 distinct pairs cycled, as there), in one launch
    # sequence (the default) and in the two concurrent sequences the autotuner picks
    import torch
    B, D = 64, 8
    src = [synth.make_c2(1024, 1024, seed=1 + 7919 * i) for i in range(D)]
    plan = of.Plan.make(1024, 1024, 3, 4, 5, bits=12, storage="f16")
    flows = [of.Flow(plan) for _ in range(B)]
    of.tuning_clear()
    of.tuning_set(plan, of.batch_size_class(flows), branches=branches)
    I1 = [to_dev(src[i % D].I1) for i in range(B)]
    I2 = [to_dev(src[i % D].I2) for i in range(B)]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(2):                    # second call replays the cached graph
            us, vs = of.compute_batch(flows, I1, I2, stream=s)
    s.synchronize()
    assert all(f.sync_status() == of.OF_OK for f in flows)
    for i in range(D):
        u1, v1 = single(of, plan, I1[i], I2[i])
        for j in range(i, B, D):               # every copy of pair i
            assert torch.equal(us[j], u1) and torch.equal(vs[j], v1), j
    for i in (0, 5):
        oracle_check(oracle_mod, src[i], us[i], vs[i], 3, 4, 5, "f16")
    of.tuning_clear()
    for f in flows:
        f.close()


def test_mixed_size_batch_64_pairs(of, oracle_mod):
    # 64 uint8 pairs drawn from 256^2, 512^2, 1024^2 and 1024x2048, uniform + vortex
    # flows, 3 levels, r = 4, 5 iterations, FP16 storage
    import torch
    pairs = synth.make_batch(64, seed=3)
    plans = [of.Plan.make(*p.shape, 3, 4, 5, bits=8, storage="f16") for p in pairs]
    flows = [of.Flow(pl) for pl in plans]
    I1 = [to_dev(p.I1) for p in pairs]
    I2 = [to_dev(p.I2) for p in pairs]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        us, vs = of.compute_batch(flows, I1, I2, stream=s)
    s.synchronize()
    assert all(f.sync_status() == of.OF_OK for f in flows)
    for i in range(0, 64, 5):
        u1, v1 = single(of, plans[i], I1[i], I2[i])
        assert torch.equal(us[i], u1) and torch.equal(vs[i], v1), i
    smallest = min(range(64), key=lambda i: pairs[i].I1.size)
    for i in (smallest, 7):
        oracle_check(oracle_mod, pairs[i], us[i], vs[i], 3, 4, 5, "f16")
    for f in flows:
        f.close()


def test_batch_staged_i2_equals_single(of):
    import torch
    pairs = synth.make_batch(5, seed=9, sizes=((160, 256), (256, 256), (96, 320)))
    flows = [of.Flow(of.Plan.make(*p.shape, 3, 4, 4, bits=8, storage="f16", flags=of.OF_FLAG_GATHER))
             for p in pairs]
    I1 = [to_dev(p.I1) for p in pairs]
    I2 = [to_dev(p.I2) for p in pairs]
    ub, vb = of.compute_batch(flows, I1, I2)
    torch.cuda.synchronize()
    for i, p in enumerate(pairs):
        u1, v1 = single(of, of.Plan.make(*p.shape, 3, 4, 4, bits=8, storage="f16"), I1[i], I2[i])
        assert torch.equal(ub[i], u1) and torch.equal(vb[i], v1), i
    for f in flows:
        f.close()


def test_batch_with_reused_first_image(of):
    # scheme 1 inside a batch: half the pairs reuse their previous second image
    import torch
    streams = [synth.ParticleStream(160, 224, seed=k) for k in range(4)]
    frames = []
    for st in streams:
        fr = []
        for _ in range(3):
            fr.append(to_dev(st.frame()))
            st.advance()
        frames.append(fr)
    plan = of.Plan.make(160, 224, 3, 4, 3, bits=12, storage="f16")
    flows = [of.Flow(plan) for _ in range(4)]
    of.compute_batch(flows, [f[0] for f in frames], [f[1] for f in frames])
    ub, vb = of.compute_batch(flows, [None, frames[1][1], None, frames[3][1]], [f[2] for f in frames])
    torch.cuda.synchronize()
    for k in range(4):
        u1, v1 = single(of, plan, frames[k][1], frames[k][2])
        assert torch.equal(ub[k], u1) and torch.equal(vb[k], v1), k
    for f in flows:
        f.close()


def test_batch_rejects_mixed_methods_and_repeats(of):
    import torch
    a = of.Flow(of.Plan.make(64, 64, 3, 4, 5))
    b = of.Flow(of.Plan.make(64, 64, 3, 5, 5))
    I = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(of.OfError) as ei:
        of.compute_batch([a, b], [I, I], [I, I])
    assert ei.value.status == of.OF_EINVAL
    with pytest.raises(of.OfError) as ei:
        of.compute_batch([a, a], [I, I], [I, I])
    assert ei.value.status == of.OF_EINVAL
    c = of.Flow(of.Plan.make(64, 64, 3, 4, 5))
    with pytest.raises(of.OfError) as ei:
        of.compute_batch([a, c], [I, None], [I, I])
    assert ei.value.status == of.OF_ESTATE


def test_empty_and_degenerate_batches(of, oracle_mod):
    import torch
    # n = 0: a no-op in both batched forms; the autotuner needs at least one pair
    assert of.compute_batch([], [], []) == ([], [])
    of.compute_batch_host([], [], [], [], [], [], [], [], [])
    with pytest.raises(of.OfError) as ei:
        of.autotune_batch([], [], [], [], [])
    assert ei.value.status == of.OF_EINVAL
    # 1x1, 1xW and Hx1 images (every level 1x1 or a single row/column) batched with a
    # normal pair: the fields equal one of_compute per pair, and the oracle's
    shapes = [(1, 1), (1, 37), (29, 1), (64, 96)]
    rng = np.random.default_rng(8)
    imgs = [(rng.integers(0, 4096, s_).astype(np.uint16), rng.integers(0, 4096, s_).astype(np.uint16))
            for s_ in shapes]
    plans = [of.Plan.make(*s_, 3, 2, 3, bits=12, storage="f32") for s_ in shapes]
    flows = [of.Flow(p_) for p_ in plans]
    ub, vb = of.compute_batch(flows, [to_dev(a) for a, _ in imgs], [to_dev(b) for _, b in imgs])
    torch.cuda.synchronize()
    for k, (a, b) in enumerate(imgs):
        u1, v1 = single(of, plans[k], to_dev(a), to_dev(b))
        assert torch.equal(ub[k], u1) and torch.equal(vb[k], v1), shapes[k]
        if shapes[k][0] * shapes[k][1] < 64:
            uo, vo = oracle_mod.flow(a.astype(np.float64), b.astype(np.float64), 3, 2, 3)
            assert np.abs(ub[k].cpu().numpy() - uo).max() <= 1e-3 and np.abs(vb[k].cpu().numpy() - vo).max() <= 1e-3
    for f in flows:
        f.close()


@pytest.mark.parametrize("branches", [1, 2])
@pytest.mark.parametrize("chunk", [0, 1, 3, 64])
def test_host_buffer_pipeline_equals_device_batch(of, chunk, branches):
    # frames from pinned host memory, fields back to pinned host memory, copies
    # overlapped with the chunked launches (alternating between two compute streams, each
    # chunk in one or two concurrent launch sequences): the same bits as
    # of_compute_batch, including pairs that reuse their previous pyramid
    import torch
    from paper_1306_2461_gb300 import serve
    streams = [synth.ParticleStream(*hw, seed=20 + k) for k, hw in
               enumerate([(160, 224), (96, 128), (160, 224), (200, 136), (96, 128)])]
    frames = []
    for st in streams:
        fr = []
        for _ in range(3):
            fr.append(st.frame())
            st.advance()
        frames.append(fr)
    n = len(streams)
    plans = [of.Plan.make(*fr[0].shape, 3, 4, 3, bits=12, storage="f16") for fr in frames]
    of.tuning_clear()
    if branches > 1:     # every size class a chunk of these pairs can have
        for sc in range(8, 20):
            of.tuning_set(plans[0], sc, branches=branches)
    fa = [of.Flow(p) for p in plans]
    fb = [of.Flow(p) for p in plans]
    hI = [[serve.pinned_frame(x) for x in fr] for fr in frames]
    dI1 = [to_dev(fr[0]) for fr in frames]
    dI2 = [to_dev(fr[1]) for fr in frames]
    hu = [torch.empty(fr[0].shape, dtype=torch.float32).pin_memory() for fr in frames]
    hv = [torch.empty(fr[0].shape, dtype=torch.float32).pin_memory() for fr in frames]
    du = [torch.empty(fr[0].shape, dtype=torch.float32, device="cuda") for fr in frames]
    dv = [torch.empty(fr[0].shape, dtype=torch.float32, device="cuda") for fr in frames]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        of.compute_batch_host(fa, [h[0] for h in hI], [h[1] for h in hI], hu, hv, dI1, dI2, du, dv,
                              stream=s, chunk=chunk)
        ub, vb = of.compute_batch(fb, [to_dev(fr[0]) for fr in frames], [to_dev(fr[1]) for fr in frames],
                                  stream=s)
    s.synchronize()
    for i in range(n):
        assert torch.equal(hu[i], ub[i].cpu()) and torch.equal(hv[i], vb[i].cpu()), i
    # second step: odd pairs reuse their previous pyramid
    reuse = [None if i % 2 else hI[i][1] for i in range(n)]
    dI1b = [to_dev(frames[i][1]) for i in range(n)]
    with torch.cuda.stream(s):
        of.compute_batch_host(fa, reuse, [h[2] for h in hI], hu, hv, dI1b, dI2, du, dv, stream=s, chunk=chunk)
        ub, vb = of.compute_batch(fb, [None if i % 2 else to_dev(frames[i][1]) for i in range(n)],
                                  [to_dev(fr[2]) for fr in frames], stream=s)
    s.synchronize()
    for i in range(n):
        assert torch.equal(hu[i], ub[i].cpu()) and torch.equal(hv[i], vb[i].cpu()), i
    with pytest.raises(of.OfError):       # a handle twice
        of.compute_batch_host([fa[0], fa[0]], [hI[0][0]] * 2, [hI[0][1]] * 2, hu[:1] * 2, hv[:1] * 2,
                              dI1[:1] * 2, dI2[:1] * 2, du[:1] * 2, dv[:1] * 2, stream=s)
    for f in fa + fb:
        f.close()
    of.tuning_clear()


def test_host_pipeline_default_chunks_ramp(of):
    # 24 pairs of 1024^2 with the default chunking: chunks of 2, 4, 8, 4, 4 and 2 pairs
    # (smaller at either end of the batch) give the same bits as of_compute_batch
    import torch
    src = [synth.make_c2(1024, 1024, seed=50 + k) for k in range(4)]
    n = 24
    plan = of.Plan.make(1024, 1024, 3, 4, 3, bits=12, storage="f16")
    fa = [of.Flow(plan) for _ in range(n)]
    fb = [of.Flow(plan) for _ in range(n)]
    pin = lambda a: torch.from_numpy(a.astype(np.int32)).to(torch.uint16).pin_memory()
    h1 = [pin(src[i % 4].I1) for i in range(n)]
    h2 = [pin(src[i % 4].I2) for i in range(n)]
    dI1 = [torch.empty((1024, 1024), dtype=torch.uint16, device="cuda") for _ in range(n)]
    dI2 = [torch.empty((1024, 1024), dtype=torch.uint16, device="cuda") for _ in range(n)]
    hu = [torch.empty((1024, 1024), dtype=torch.float32).pin_memory() for _ in range(n)]
    hv = [torch.empty((1024, 1024), dtype=torch.float32).pin_memory() for _ in range(n)]
    du = [torch.empty((1024, 1024), dtype=torch.float32, device="cuda") for _ in range(n)]
    dv = [torch.empty((1024, 1024), dtype=torch.float32, device="cuda") for _ in range(n)]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        of.compute_batch_host(fa, h1, h2, hu, hv, dI1, dI2, du, dv, stream=s, chunk=0)
        ub, vb = of.compute_batch(fb, [to_dev(src[i % 4].I1) for i in range(n)],
                                  [to_dev(src[i % 4].I2) for i in range(n)], stream=s)
    s.synchronize()
    for i in range(n):
        assert torch.equal(hu[i], ub[i].cpu()) and torch.equal(hv[i], vb[i].cpu()), i
    for f in fa + fb:
        f.close()


def test_more_pairs_than_one_phase_launch_holds(of):
    # 70 small pairs: each phase is split into launches of at most 64 pairs; every
    # field equals of_compute's, including pairs that reuse their previous pyramid
    import torch
    n = 70
    rng = np.random.default_rng(5)
    sizes = [(int(rng.integers(24, 96)), int(rng.integers(24, 96))) for _ in range(n)]
    frames = []
    for k, (H, W) in enumerate(sizes):
        st = synth.ParticleStream(H, W, seed=100 + k)
        fr = []
        for _ in range(3):
            fr.append(st.frame())
            st.advance()
        frames.append(fr)
    plans = [of.Plan.make(H, W, 2, 3, 2, bits=12, storage="f16") for H, W in sizes]
    flows = [of.Flow(p) for p in plans]
    of.compute_batch(flows, [to_dev(f[0]) for f in frames], [to_dev(f[1]) for f in frames])
    reuse = [None if k % 3 == 0 else to_dev(frames[k][1]) for k in range(n)]
    ub, vb = of.compute_batch(flows, reuse, [to_dev(f[2]) for f in frames])
    torch.cuda.synchronize()
    assert all(f.sync_status() == of.OF_OK for f in flows)
    for k in range(n):
        u1, v1 = single(of, plans[k], to_dev(frames[k][1]), to_dev(frames[k][2]))
        assert torch.equal(ub[k], u1) and torch.equal(vb[k], v1), k
    for f in flows:
        f.close()


def test_host_pipelines_in_two_threads(of):
    # two threads run host-buffer pipelines at once, each with its own handles, buffers and
    # stream (and its own internal compute stream, on which its chunks' launch sequences are
    # captured): every field equals the single-threaded device batch's
    import threading
    import torch
    sizes = [(160, 224), (96, 128), (200, 136), (128, 128)]
    n = len(sizes)
    frames = [[synth.make_c1(H, W, seed=70 + 10 * t + k) for k, (H, W) in enumerate(sizes)] for t in range(2)]
    plans = [of.Plan.make(H, W, 3, 4, 3, bits=8, storage="f16") for H, W in sizes]
    results, errors = [None, None], []

    def worker(t):
        try:
            fl = [of.Flow(p) for p in plans]
            h1 = [torch.from_numpy(p.I1).pin_memory() for p in frames[t]]
            h2 = [torch.from_numpy(p.I2).pin_memory() for p in frames[t]]
            hu = [torch.empty(s, dtype=torch.float32).pin_memory() for s in sizes]
            hv = [torch.empty(s, dtype=torch.float32).pin_memory() for s in sizes]
            d1 = [torch.empty(s, dtype=torch.uint8, device="cuda") for s in sizes]
            d2 = [torch.empty(s, dtype=torch.uint8, device="cuda") for s in sizes]
            du = [torch.empty(s, dtype=torch.float32, device="cuda") for s in sizes]
            dv = [torch.empty(s, dtype=torch.float32, device="cuda") for s in sizes]
            s = torch.cuda.Stream()
            for _ in range(20):
                with torch.cuda.stream(s):
                    of.compute_batch_host(fl, h1, h2, hu, hv, d1, d2, du, dv, stream=s, chunk=1)
                s.synchronize()
                for f in fl:
                    assert f.sync_status() == of.OF_OK
            results[t] = ([x.clone() for x in hu], [x.clone() for x in hv])
            for f in fl:
                f.close()
        except Exception as e:      # reported by the main thread
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(2)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    for t in range(2):
        fb = [of.Flow(p) for p in plans]
        ub, vb = of.compute_batch(fb, [to_dev(p.I1) for p in frames[t]], [to_dev(p.I2) for p in frames[t]])
        torch.cuda.synchronize()
        for k in range(n):
            assert torch.equal(results[t][0][k], ub[k].cpu()) and torch.equal(results[t][1][k], vb[k].cpu()), (t, k)
        for f in fb:
            f.close()
