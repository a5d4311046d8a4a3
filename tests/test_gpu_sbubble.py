"""Eq. 3 reductions on the device: the count of vectors at or below T_v (exact integer,
compared with the oracle bit for bit) and the min/max giving T_v."""
import numpy as np
import pytest

from paper_1306_2461_gb300 import synth

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


@pytest.mark.parametrize("H,W", [(1, 1), (7, 13), (384, 1792), (1024, 1024), (2048, 2048)])
def test_count_matches_oracle(of, oracle_mod, H, W):
    import torch
    rng = np.random.default_rng(H + W)
    u = rng.normal(0.0, 2.0, (H, W)).astype(np.float32)
    u.flat[::97] = 0.25                                      # exact ties at a threshold
    ud = torch.from_numpy(u).cuda()
    for Tv in (-1.0, 0.25, 0.0, 3.5, -100.0):
        c = int(of.sbubble(ud, Tv).item())
        assert c == oracle_mod.sbubble_count(u, Tv), (H, W, Tv)


def test_minmax_and_threshold(of, oracle_mod):
    import torch
    rng = np.random.default_rng(1)
    m = rng.normal(-1.0, 4.0, (333, 517)).astype(np.float32)
    mm = of.field_minmax(torch.from_numpy(m).cuda()).cpu().numpy()
    assert mm[0] == m.min() and mm[1] == m.max()
    assert 0.5 * (float(mm[0]) + float(mm[1])) == oracle_mod.sbubble_threshold(m)
    nan = np.full((4, 5), np.nan, np.float32)
    nan[2, 3] = -7.5
    mm = of.field_minmax(torch.from_numpy(nan).cuda()).cpu().numpy()
    assert mm[0] == -7.5 and mm[1] == -7.5


def test_sbubble_on_a_computed_field(of, oracle_mod):
    # the bubble of a computed vortex-street field: GPU flow -> GPU count, vs the same
    # count by the oracle on the GPU flow (the decision is taken in FP32 on both sides)
    import torch
    from helpers import gpu_flow
    s = synth.ParticleStream(256, 384, seed=2)
    f0 = s.frame()
    s.advance()
    f1 = s.frame()
    u, v = gpu_flow((f0, f1), 3, 4, 5, "f16", bits=12)
    u32 = u.astype(np.float32)
    ud = torch.from_numpy(u32).cuda()
    mm = of.field_minmax(ud).cpu().numpy()
    Tv = 0.5 * (float(mm[0]) + float(mm[1]))
    c = int(of.sbubble(ud, Tv).item())
    assert c == oracle_mod.sbubble_count(u32, Tv)
    assert 0 < c < u32.size
