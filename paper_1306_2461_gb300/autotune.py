"""Persistent cache of the batched launch's autotuning.

libof keeps a process-wide table, keyed by the method and the batch's size class, of
how a batched launch runs: the window-sum strategy, I2 staging, the iteration tile's
height, and phase launches (with or without an L2 prefetch, in one or several concurrent
sequences) or the persistent launch at some resident blocks per SM (of_tuning in
include/of.h). of_autotune_batch fills an entry by timing every
candidate on a real batch. This module keeps those entries in a JSON file per GPU
model, so that a later process starts from the measured choice:

    autotune.load()                       # apply the saved entries for this GPU
    autotune.ensure(flows, I1s, I2s)      # tune this batch shape unless already known

Marshalling and file I/O only; the timing and the choice happen in the library.
"""
from __future__ import annotations

import json
import os
import tempfile

import torch

from . import of

DEFAULT_PATH = os.path.join(os.path.expanduser("~"), ".cache", "paper_1306_2461_gb300", "autotune.json")


def _device() -> str:
    return torch.cuda.get_device_name()


def _method(plan: of.Plan) -> dict:
    return {"in_format": plan.in_format, "in_bits": plan.in_bits, "storage": plan.storage, "radius": plan.radius,
            "levels": plan.levels, "iterations": plan.iterations, "znssd": int(bool(plan.flags & of.OF_FLAG_ZNSSD)),
            "i1grad": int(bool(plan.flags & of.OF_FLAG_I1GRAD))}


def _key(method: dict, size_class: int) -> str:
    m = method
    return (f"fmt{m['in_format']}/st{m['storage']}/r{m['radius']}/L{m['levels']}/n{m['iterations']}"
            f"/zn{m['znssd']}/i1{m.get('i1grad', 0)}/sc{size_class}")


def _plan_of(method: dict) -> of.Plan:
    flags = (of.OF_FLAG_ZNSSD if method["znssd"] else 0) | (of.OF_FLAG_I1GRAD if method.get("i1grad") else 0)
    p = of.Plan.make(64, 64, method["levels"], method["radius"], method["iterations"], bits=method["in_bits"],
                     storage=method["storage"], flags=flags)
    p.in_format = method["in_format"]
    return p


def _read(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _write(path: str, data: dict):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(path) or ".", suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def load(path: str | None = None) -> int:
    """Apply the saved entries for this GPU model to the library's table. Returns how many."""
    data = _read(path or DEFAULT_PATH).get(_device(), {})
    for ent in data.values():
        b = ent["best"]
        of.tuning_set(_plan_of(ent["method"]), ent["size_class"], b["generic_sums"], b["stage_i2"],
                      b["blocks_per_sm"], b.get("phased", 0), b.get("prefetch", 0), b.get("tile_h", 0),
                      b.get("branches", 0), b.get("fusion", 1), b.get("strip", 4))
    return len(data)


def tune(flows, I1s, I2s, us=None, vs=None, stream=None, reps: int = 3, path: str | None = None,
         save: bool = True) -> dict:
    """Time every candidate on this batch (of_autotune_batch), record the choice in the
    library and, when save is set, in the cache file. Returns the entry."""
    best, cands = of.autotune_batch(flows, I1s, I2s, us, vs, stream=stream, reps=reps)
    method = _method(flows[0].plan)
    sc = of.batch_size_class(flows)
    ent = {"method": method, "size_class": sc, "batch": len(flows), "best": best, "candidates": cands}
    if save:
        p = path or DEFAULT_PATH
        data = _read(p)
        data.setdefault(_device(), {})[_key(method, sc)] = ent
        _write(p, data)
    return ent


def ensure(flows, I1s, I2s, us=None, vs=None, stream=None, reps: int = 3, path: str | None = None) -> dict:
    """The table's tuning for this batch shape, tuning it first when there is none."""
    t = of.tuning_get(flows[0].plan, of.batch_size_class(flows))
    if t is not None:
        return {"method": _method(flows[0].plan), "size_class": of.batch_size_class(flows), "best": t,
                "candidates": []}
    return tune(flows, I1s, I2s, us, vs, stream=stream, reps=reps, path=path)
