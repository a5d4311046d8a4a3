"""The C-ABI library: it loads, exports every entry point include/of.h declares, and its
host-only calls (plan validation, Eq. 1, level sizes, workspace size) behave. No GPU."""
import ctypes
import os
import re

import pytest

from paper_1306_2461_gb300 import build as of_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def of():
    of_build.build()
    from paper_1306_2461_gb300 import of as ofmod
    return ofmod


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(of_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol(of):
    syms = declared_symbols()
    assert "of_create" in syms and "of_compute" in syms and "of_destroy" in syms
    lib = ctypes.CDLL(of.LIB_PATH)
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, f"declared but not exported: {missing}"


def test_plan_defaults_and_validation(of):
    p = of.Plan.make(1024, 1024, 3, 4, 5, bits=12, storage="f16")
    assert of.plan_validate(p) == of.OF_OK
    for field, bad in [("H", 0), ("W", -3), ("levels", 0), ("levels", 17), ("radius", 0), ("radius", 17),
                       ("iterations", 0), ("in_bits", 17), ("storage", 7), ("in_format", 5), ("flags", 0x80)]:
        q = of.Plan.make(64, 64)
        setattr(q, field, bad)
        assert of.plan_validate(q) == of.OF_EINVAL, field
    q = of.Plan.make(64, 64)
    q.fp64_cond = float("nan")
    assert of.plan_validate(q) == of.OF_EINVAL
    q = of.Plan.make(32768, 32768)          # 2^30 pixels: above the 2^28 limit
    assert of.plan_validate(q) == of.OF_EINVAL
    assert of.plan_validate(of.Plan.make(1, 1, levels=1, radius=16)) == of.OF_OK


def test_eq1_level_rule_matches_golden(of):
    rows = [l.split() for l in open(os.path.join(ROOT, "tests", "golden", "nlevels.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) >= 10
    for disp, levels, ok in rows:
        p = of.Plan.make(512, 512, levels=int(levels))
        assert of.plan_check(p, float(disp)) == bool(int(ok)), (disp, levels)


def test_level_sizes_and_workspace(of):
    p = of.Plan.make(383, 1791, levels=3)
    assert [of.level_size(p, l) for l in range(3)] == [(383, 1791), (192, 896), (96, 448)]
    with pytest.raises(of.OfError):
        of.level_size(p, 3)
    N = 1024 * 1024
    flows = 2 * N * 8
    # two pyramids: level 0 in the camera format (1 or 2 B/px), levels 1 and 2
    # (1/4 + 1/16 of the pixels) at the storage precision (4 or 2 B/px)
    for bits, raw in ((8, 1), (12, 2)):
        for storage, s in (("f32", 4), ("f16", 2), ("bf16", 2)):
            b = of.workspace_bytes(of.Plan.make(1024, 1024, bits=bits, storage=storage))
            assert abs((b - flows) - 2 * N * (raw + s * 0.3125)) < 1e5, (bits, storage)


def test_status_strings_and_version(of):
    for s in range(-7, 1):
        assert of.lib().of_status_string(s)
    assert of.version() >= 100


def test_i1grad_flag_validates_and_adds_one_float4_per_pixel(of):
    p = of.Plan.make(1024, 1024, bits=12, storage="f16")
    q = of.Plan.make(1024, 1024, bits=12, storage="f16", flags=of.OF_FLAG_I1GRAD)
    assert of.plan_validate(q) == of.OF_OK
    assert of.workspace_bytes(q) - of.workspace_bytes(p) == 1024 * 1024 * 16
    assert of.plan_validate(of.Plan.make(64, 64, flags=0x10)) == of.OF_EINVAL


def test_tuning_table_host_calls(of):
    m = of.Plan.make(64, 64, 3, 4, 5, bits=12, storage="f16")
    of.tuning_clear()
    assert of.tuning_get(m, 20) is None
    of.tuning_set(m, 20, generic_sums=0, stage_i2=1, blocks_per_sm=2, phased=0, prefetch=0)
    t = of.tuning_get(m, 20)
    assert (t["generic_sums"], t["stage_i2"], t["blocks_per_sm"], t["phased"]) == (0, 1, 2, 0)
    assert of.tuning_get(m, 19) is None                                   # another size class
    assert of.tuning_get(of.Plan.make(64, 64, 3, 4, 4, bits=12, storage="f16"), 20) is None   # another method
    with pytest.raises(of.OfError):
        of.tuning_set(m, 20, generic_sums=1, stage_i2=1)                  # staging needs the grouped kernel
    with pytest.raises(of.OfError):
        of.tuning_set(m, 20, blocks_per_sm=-1, phased=0)
    with pytest.raises(of.OfError):
        of.tuning_set(m, 20, prefetch=17)
    with pytest.raises(of.OfError):
        of.tuning_set(m, 20, blocks_per_sm=2, phased=1)                   # occupancy is a persistent-launch knob
    with pytest.raises(of.OfError):
        of.tuning_set(m, 20, tile_h=20)                                   # tile heights 24 and 32 only
    with pytest.raises(of.OfError):
        of.tuning_set(m, 20, tile_h=32, phased=0)                         # the persistent launch has one
    with pytest.raises(of.OfError):
        of.tuning_set(m, 20, tile_h=32, generic_sums=1)                   # the taller tile is grouped-sums only
    with pytest.raises(of.OfError):
        of.tuning_set(m, 20, branches=5)                                  # at most 4 concurrent sequences
    with pytest.raises(of.OfError):
        of.tuning_set(m, 20, branches=2, phased=0)                        # a phase-launch knob
    with pytest.raises(of.OfError):
        of.tuning_set(m, 20, fusion=3)                                    # fusion depth 1 or 2
    with pytest.raises(of.OfError):
        of.tuning_set(m, 20, fusion=2, tile_h=32)                         # at the default tile height
    with pytest.raises(of.OfError):
        of.tuning_set(m, 20, fusion=2, generic_sums=1, stage_i2=0)        # with the grouped sums
    with pytest.raises(of.OfError):
        of.tuning_set(m, 20, fusion=2, phased=0)                          # of the phase launches
    with pytest.raises(of.OfError):
        of.tuning_set(of.Plan.make(64, 64, 3, 7, 3, bits=12), 20, fusion=2)   # a fixed-radius kernel
    with pytest.raises(of.OfError):
        of.tuning_set(m, 20, strip=3)                                     # strips of 1, 2 or 4 tiles
    with pytest.raises(of.OfError):
        of.tuning_set(m, 20, strip=2, generic_sums=1, stage_i2=0)         # of the grouped sums
    with pytest.raises(of.OfError):
        of.tuning_set(m, 20, strip=2, phased=0)                           # of the phase launches
    of.tuning_set(m, 20, strip=1)
    assert of.tuning_get(m, 20)["strip"] == 1
    of.tuning_set(m, 20, strip=0)                                         # 0: the default
    assert of.tuning_get(m, 20)["strip"] == 4
    of.tuning_set(m, 20, fusion=2)
    assert of.tuning_get(m, 20)["fusion"] == 2
    of.tuning_set(m, 20, branches=3)
    assert of.tuning_get(m, 20)["branches"] == 3 and of.tuning_get(m, 20)["fusion"] == 1
    of.tuning_set(m, 20, tile_h=32, prefetch=1)
    assert (of.tuning_get(m, 20)["tile_h"], of.tuning_get(m, 20)["prefetch"]) == (32, 1)
    v = of.Plan.make(64, 64, 3, 4, 5, bits=12, storage="f16", flags=of.OF_FLAG_I1GRAD)
    of.tuning_set(v, 20, branches=2)                                      # the variant keeps its own entry
    assert of.tuning_get(v, 20)["branches"] == 2 and of.tuning_get(m, 20)["tile_h"] == 32
    of.tuning_set(m, 20)
    assert of.tuning_get(v, 20)["branches"] == 2
    t = of.tuning_get(m, 20)
    assert (t["phased"], t["prefetch"], t["tile_h"], t["branches"]) == (1, 0, 24, 1)
    of.tuning_clear()
    assert of.tuning_get(m, 20) is None
