"""The serving loop: continuous batching of camera streams with resident pyramids.

Every served field must equal the field of_compute gives for the same two frames
alone (bit for bit: the batched launch runs the same tile code), streams are admitted
against the HBM budget, and latencies are reported from the scheduled arrivals.
"""
import numpy as np
import pytest

from paper_1306_2461_gb300 import synth
from helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_2461_gb300 import build
    build.build()
    from paper_1306_2461_gb300 import of, serve
    return of, serve


def stream_frames(H, W, seed, n):
    s = synth.ParticleStream(H, W, seed=seed)
    out = []
    for _ in range(n):
        out.append(s.frame())
        s.advance()
    return out


def test_served_fields_equal_alone(mods):
    import torch
    of, serve = mods
    sizes = [(160, 224), (96, 128), (192, 160)]
    frames = [stream_frames(H, W, 10 + k, 5) for k, (H, W) in enumerate(sizes)]
    with serve.Server(levels=3, radius=4, iterations=3, bits=12, storage="f16", max_batch=8) as srv:
        sids = [srv.open_stream(H, W) for H, W in sizes]
        outs = {}
        pinned = [[serve.pinned_frame(f) for f in fr] for fr in frames]
        # interleave the streams, several frames queued at once
        tag = 0
        for k in range(5):
            for j, sid in enumerate(sids):
                u = torch.full(sizes[j], float("nan"), device="cuda")
                v = torch.full(sizes[j], float("nan"), device="cuda")
                outs[tag] = (j, k, u, v)
                srv.submit(sid, pinned[j][k], u, v, tag=tag)
                tag += 1
        srv.drain()
        res = srv.poll(0)
        assert len(res) == 15 and all(r["status"] == 0 for r in res)
        assert sum(r["has_field"] for r in res) == 12
        st = srv.stats()
        assert st["pairs"] == 12 and st["ticks"] >= 5
    for r in res:
        j, k, u, v = outs[r["tag"]]
        if k == 0:
            assert r["has_field"] == 0
            continue
        plan = of.Plan.make(*sizes[j], 3, 4, 3, bits=12, storage="f16")
        with of.Flow(plan) as f:
            ua, va = f.compute(to_dev(frames[j][k - 1]), to_dev(frames[j][k]))
            torch.cuda.synchronize()
        assert torch.equal(u, ua) and torch.equal(v, va), (j, k)


def test_admission_by_hbm_budget(mods):
    of, serve = mods
    plan = of.Plan.make(512, 512, 3, 4, 5, bits=12, storage="f16")
    need = of.workspace_bytes(plan) + 2 * 512 * 512 * 2
    with serve.Server(hbm_budget_bytes=int(need * 1.5)) as srv:
        a = srv.open_stream(512, 512)
        rc, _ = srv.try_open_stream(512, 512)
        assert rc == of.OF_ENOMEM
        assert srv.stats()["hbm_used"] == need
        rc, b = srv.try_open_stream(128, 128)       # a small stream still fits
        assert rc == of.OF_OK
        srv.close_stream(a)
        rc, c = srv.try_open_stream(512, 512)       # memory freed: admitted
        assert rc == of.OF_OK


def test_open_loop_latency_and_throughput(mods):
    of, serve = mods
    sizes = [(256, 256), (256, 256), (384, 384), (128, 192)]
    with serve.Server(levels=3, radius=4, iterations=5, bits=12, storage="f16", max_batch=16) as srv:
        streams = []
        for k, (H, W) in enumerate(sizes):
            fr = [serve.pinned_frame(f) for f in stream_frames(H, W, 30 + k, 3)]
            streams.append((srv.open_stream(H, W), fr))
        arrivals = synth.poisson_arrivals(len(sizes), 200.0, 0.3, seed=5)
        results, _, _ = serve.run_open_loop(srv, streams, arrivals, warmup_s=0.05)
        s = serve.summarize(results, 0.25)
        print(s)
        assert len(results) == len(arrivals)
        assert s["errors"] == 0 and s["fields"] > 0
        assert all(r["done_ns"] >= r["launch_ns"] > 0 for r in results)
        assert 0 < s["p50_ms"] <= s["p99_ms"] < 1000


def test_continuous_batching_under_load_equals_alone(mods):
    # eight time-resolved streams of mixed sizes whose next frames all arrive while ticks
    # are running: the ticks batch several streams' frames (mean batch > 4), frames
    # arriving during a tick join a later one, and every served field equals the field of
    # the same two frames computed alone
    import torch
    of, serve = mods
    sizes = [(160, 224), (96, 128), (192, 160), (128, 128), (224, 96), (160, 160), (96, 256), (200, 136)]
    nfr = 6
    frames = [stream_frames(H, W, 50 + k, nfr) for k, (H, W) in enumerate(sizes)]
    outs = {}
    with serve.Server(levels=3, radius=4, iterations=3, bits=12, storage="f16", max_batch=16,
                      max_inflight=2) as srv:
        sids = [srv.open_stream(H, W) for H, W in sizes]
        pinned = [[serve.pinned_frame(f) for f in fr] for fr in frames]
        for j, sid in enumerate(sids):                  # every stream's first frame
            srv.submit(sid, pinned[j][0], tag=100 * j)
        srv.drain()
        srv.poll(0)
        bufs = {(j, k): (torch.full(sizes[j], float("nan"), device="cuda"),
                         torch.full(sizes[j], float("nan"), device="cuda")) for j in range(len(sizes))
                for k in range(1, nfr)}
        torch.cuda.synchronize()
        for k in range(1, nfr):                         # then all the other frames at once
            for j, sid in enumerate(sids):
                u, v = bufs[(j, k)]
                srv.submit(sid, pinned[j][k], u, v, tag=100 * j + k)
        srv.drain()
        res = srv.poll(0)
    assert len(res) == (nfr - 1) * len(sizes) and all(r["status"] == 0 and r["has_field"] for r in res)
    mean_batch = float(np.mean([r["batch"] for r in res]))
    print(f"mean batch {mean_batch:.2f} over {len(res)} fields")
    assert mean_batch > 4
    for j, (H, W) in enumerate(sizes):
        plan = of.Plan.make(H, W, 3, 4, 3, bits=12, storage="f16")
        with of.Flow(plan) as f:
            for k in range(1, nfr):
                ua, va = f.compute(to_dev(frames[j][k - 1]), to_dev(frames[j][k]))
                torch.cuda.synchronize()
                u, v = bufs[(j, k)]
                assert torch.equal(u, ua) and torch.equal(v, va), (j, k)
