"""The autotuner of the batched launch: every candidate gives the per-pair results (bit
for bit with the grouped sums, within the FP32 tolerance with the per-output sums), the
fastest is recorded and used, and the JSON cache restores it in a later process."""
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
    yield ofmod
    ofmod.tuning_clear()


def batch(of, sizes, storage="f32", seed=0):
    pairs = [synth.make_c1(H, W, seed=seed + k) for k, (H, W) in enumerate(sizes)]
    plans = [of.Plan.make(H, W, 3, 4, 3, bits=8, storage=storage) for H, W in sizes]
    flows = [of.Flow(p) for p in plans]
    I1 = [to_dev(p.I1) for p in pairs]
    I2 = [to_dev(p.I2) for p in pairs]
    return pairs, flows, I1, I2


def test_every_candidate_matches_the_per_pair_path(of, oracle_mod):
    import torch
    sizes = [(256, 256), (192, 320), (128, 96), (256, 256)]
    pairs, flows, I1, I2 = batch(of, sizes)
    ref = []
    for k, (H, W) in enumerate(sizes):
        with of.Flow(of.Plan.make(H, W, 3, 4, 3, bits=8, storage="f32")) as f:
            u, v = f.compute(I1[k], I2[k])
            ref.append((u.clone(), v.clone()))
    torch.cuda.synchronize()
    best, cands = of.autotune_batch(flows, I1, I2, reps=2)
    print(best, cands)
    assert len(cands) == 9 and best["ms"] == min(c["ms"] for c in cands)
    sc = of.batch_size_class(flows)
    t = of.tuning_get(flows[0].plan, sc)
    assert (t["generic_sums"], t["stage_i2"], t["blocks_per_sm"]) == \
        (best["generic_sums"], best["stage_i2"], best["blocks_per_sm"])
    for c in cands:
        of.tuning_set(flows[0].plan, sc, c["generic_sums"], c["stage_i2"], c["blocks_per_sm"])
        us, vs = of.compute_batch(flows, I1, I2)
        torch.cuda.synchronize()
        for k in range(len(sizes)):
            if c["generic_sums"] == 0:
                assert torch.equal(us[k], ref[k][0]) and torch.equal(vs[k], ref[k][1]), (c, k)
            else:
                m = 24
                d = max(float((us[k] - ref[k][0])[m:-m, m:-m].abs().max()),
                        float((vs[k] - ref[k][1])[m:-m, m:-m].abs().max()))
                assert d <= 1e-3, (c, k, d)
                if k == 0:      # and the oracle's parity holds for the per-output sums too
                    parity_check(us[k].cpu().double().numpy(), vs[k].cpu().double().numpy(), pairs[k],
                                 oracle_mod, 3, 4, 3, "f32", "per-output sums")
    of.tuning_clear()
    for f in flows:
        f.close()


def test_cache_file_round_trip(of, tmp_path):
    from paper_1306_2461_gb300 import autotune
    sizes = [(128, 128), (128, 160)]
    _, flows, I1, I2 = batch(of, sizes, storage="f16", seed=5)
    path = str(tmp_path / "tune.json")
    ent = autotune.tune(flows, I1, I2, reps=1, path=path)
    sc = of.batch_size_class(flows)
    assert ent["size_class"] == sc and len(ent["candidates"]) == 9
    of.tuning_clear()
    assert of.tuning_get(flows[0].plan, sc) is None
    assert autotune.load(path) == 1
    t = of.tuning_get(flows[0].plan, sc)
    assert (t["generic_sums"], t["stage_i2"], t["blocks_per_sm"]) == \
        (ent["best"]["generic_sums"], ent["best"]["stage_i2"], ent["best"]["blocks_per_sm"])
    again = autotune.ensure(flows, I1, I2, path=path)      # known: no new timing
    assert again["candidates"] == [] and again["best"]["generic_sums"] == ent["best"]["generic_sums"]
    of.tuning_clear()
    for f in flows:
        f.close()


def test_autotune_refuses_reused_pyramids(of):
    _, flows, I1, I2 = batch(of, [(64, 64)])
    with pytest.raises(of.OfError) as ei:
        of.autotune_batch(flows, [None], I2, reps=1)
    assert ei.value.status == of.OF_EINVAL
    flows[0].close()
