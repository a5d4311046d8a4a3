"""of_compute_noalloc, the entry point for callers that cannot allocate device memory
while running (a real-time acquisition loop, where cudaMalloc can stall the device, or
a host that owns all device memory through its own allocator). It must give the fields
of_compute gives, bit for bit (the same arithmetic: it runs the gathered tiles, which
equal the staged ones exactly), call after call, from its static scratch, without
allocating.

Called through the C ABI with ctypes. Kept in a file of its own that pytest collects
last; it passes alone in a fresh process and after the other tests.
"""
import ctypes

import pytest

from paper_1306_2461_gb300 import synth
from helpers import to_dev

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


def noalloc(of):
    fn = of.lib().of_compute_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(of.Plan)] + [ctypes.c_void_p] * 5
    return fn


def test_noalloc_matches_of_compute_on_two_calls_in_a_row(of):
    import torch
    fn = noalloc(of)
    cases = [(synth.make_c2(1024, 1024, seed=1), of.Plan.make(1024, 1024, 3, 4, 5, bits=12, storage="f16"), "f16"),
             (synth.make_c1(), of.Plan.make(256, 256, 2, 5, 4, bits=8, storage="f32"), "f32")]
    inputs = [(to_dev(p.I1), to_dev(p.I2)) for p, _, _ in cases]
    # the existing entry point
    ref = []
    for (I1, I2), (_, plan, _) in zip(inputs, cases):
        with of.Flow(plan) as f:
            u, v = f.compute(I1, I2)
            torch.cuda.synchronize()
            ref.append((u.clone(), v.clone()))
    s = torch.cuda.Stream()
    outs = [(torch.empty_like(u), torch.empty_like(v)) for u, v in ref]
    # the first call on this device sets up the scratch address; make it here, outside
    # the allocation check below
    plan0 = cases[0][1]
    assert fn(ctypes.byref(plan0), inputs[0][0].data_ptr(), inputs[0][1].data_ptr(), outs[0][0].data_ptr(),
              outs[0][1].data_ptr(), s.cuda_stream) == of.OF_OK
    s.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    # two calls in a row on one stream, different plans and inputs, no sync between
    for (I1, I2), (_, plan, _), (u, v) in zip(inputs, cases, outs):
        u.fill_(float("nan"))
        v.fill_(float("nan"))
        assert fn(ctypes.byref(plan), I1.data_ptr(), I2.data_ptr(), u.data_ptr(), v.data_ptr(),
                  s.cuda_stream) == of.OF_OK
    s.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    for (u, v), (ur, vr), (_, _, storage) in zip(outs, ref, cases):
        d = max(float((u - ur).abs().max()), float((v - vr).abs().max()))
        print(f"{storage}: max |noalloc - of_compute| = {d:.3e} px")
        assert torch.equal(u, ur) and torch.equal(v, vr), storage


def test_noalloc_rejects_what_it_cannot_hold(of):
    import torch
    fn = noalloc(of)
    I = torch.zeros((2048, 2048), dtype=torch.uint16, device="cuda")
    u = torch.empty((2048, 2048), dtype=torch.float32, device="cuda")
    big = of.Plan.make(2048, 2048, 4, 3, 6, bits=12, storage="f16")
    assert of.workspace_bytes(big) > 32 * 1024 * 1024          # beyond the 32 MiB scratch
    assert fn(ctypes.byref(big), I.data_ptr(), I.data_ptr(), u.data_ptr(), u.data_ptr(), None) == of.OF_ENOMEM
    # one 1024^2 pair fits at any storage, but not with the variant's window matrices
    for st in ("f32", "f16"):
        assert of.workspace_bytes(of.Plan.make(1024, 1024, 3, 4, 5, bits=12, storage=st)) <= 32 * 1024 * 1024
        g = of.Plan.make(1024, 1024, 3, 4, 5, bits=12, storage=st, flags=of.OF_FLAG_I1GRAD)
        assert of.workspace_bytes(g) > 32 * 1024 * 1024
        assert fn(ctypes.byref(g), I.data_ptr(), I.data_ptr(), u.data_ptr(), u.data_ptr(), None) == of.OF_ENOMEM
    small = of.Plan.make(64, 64, 2, 3, 2, bits=12)
    J = torch.zeros((64, 64), dtype=torch.uint16, device="cuda")
    w = torch.empty((64, 64), dtype=torch.float32, device="cuda")
    assert fn(ctypes.byref(small), None, J.data_ptr(), w.data_ptr(), w.data_ptr(), None) == of.OF_EINVAL
    bad = of.Plan.make(0, 64)
    assert fn(ctypes.byref(bad), J.data_ptr(), J.data_ptr(), w.data_ptr(), w.data_ptr(), None) == of.OF_EINVAL
