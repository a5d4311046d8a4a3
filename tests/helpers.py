"""Shared helpers for the GPU tests: run the CUDA path on numpy inputs and compare it
with the oracle.

Which pixels are compared (parity_check):
  - at least (r+2)*2^(L-1) px from the border for particle images: nearer to it the
    displacement carries windows and warps outside the image and the FP64 method is
    itself unstable;
  - not within a decade of the singular guard at level 0 (a guard decision may flip);
  - not unstable: pixels whose FP64 result moves by more than a quarter of the
    tolerance when the input images are perturbed by 1 part in 10^6 (rounding-level
    noise; a test may probe with a larger relative amplitude where the FP32 arithmetic's
    accumulated rounding is larger, and says why) or, with FP16/BF16 storage, when a few
    stored pyramid values round the other way, are not determined to the tolerance by
    the method itself.
Every exclusion is counted and bounded. The implementation check compares the CUDA
path with the oracle run on the pyramid stored as the CUDA path stores it (level 0
exact, reduced levels rounded to the storage type), so both sides see the same
inputs and only the arithmetic differs: it applies the FP32 bound (IMPL_TOL) whatever
the storage. The storage check (FP16/BF16 against the unrounded FP64 oracle) applies the
stated max and RMS bounds to the compared pixels whose FP64 result moves by less than
half the tolerance when the pyramid is rounded; the others ("storage-sensitive": the
method itself does not determine them to the tolerance from inputs known to the
storage precision) are counted and bounded.
"""
import numpy as np

TOL = {"f32": (1e-3, None), "f16": (2e-2, 5e-3), "bf16": (2e-1, 5e-2)}
IMPL_TOL = TOL["f32"][0]   # FP32 arithmetic against FP64 on identical stored inputs


def to_dev(a):
    import torch
    if a.dtype == np.uint16:
        return torch.from_numpy(a.astype(np.int32)).to("cuda").to(torch.uint16)
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def gpu_flow(pair_or_images, levels, radius, iterations, storage="f32", bits=None, fp64_cond=1e3, flags=0):
    """Run of_compute on one pair (a synth.Pair or an (I1, I2) tuple). Returns float64 (u, v)."""
    import torch
    from paper_1306_2461_gb300 import of
    I1, I2 = images(pair_or_images)
    if bits is None:
        bits = 8 if I1.dtype == np.uint8 else 12
    H, W = I1.shape
    plan = of.Plan.make(H, W, levels, radius, iterations, bits=bits, storage=storage, fp64_cond=fp64_cond,
                        flags=flags)
    with of.Flow(plan) as f:
        u, v = f.compute(to_dev(I1), to_dev(I2))
        torch.cuda.synchronize()
        assert f.sync_status() == of.OF_OK
    return u.cpu().double().numpy(), v.cpu().double().numpy()


def images(p):
    return (p.I1, p.I2) if hasattr(p, "I1") else p


def round_f16(a):
    return np.asarray(a, np.float64).astype(np.float16).astype(np.float64)


def round_bf16(a):
    x = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((x + 0x7FFF + ((x >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def oracle_flow_stored(oracle_mod, I1, I2, L, r, n, storage, perturb=0.0, seed=0, round0=False, i1grad=False):
    """The oracle's steps (FP64) on a pyramid stored as the CUDA path stores it: level 0
    exact, level l+1 = round(reduce(level l)) with round-to-nearest-even to `storage`.
    perturb > 0 multiplies each reduced value by (1 + U(-perturb, perturb)) before the
    rounding, which flips the rounding of values that lie near a rounding boundary, as
    FP32 arithmetic in the reduction can."""
    rnd = {"f32": lambda a: np.asarray(a, np.float32).astype(np.float64), "f16": round_f16,
           "bf16": round_bf16}[storage]
    rng = np.random.default_rng(seed)
    jit = (lambda a: a * (1.0 + rng.uniform(-perturb, perturb, a.shape))) if perturb > 0 else (lambda a: a)
    P1 = [np.asarray(I1, np.float64)]
    P2 = [np.asarray(I2, np.float64)]
    if round0:      # level 0 itself at the storage precision (normalised images)
        P1[0], P2[0] = rnd(jit(P1[0])), rnd(jit(P2[0]))
    for _ in range(L - 1):
        P1.append(rnd(jit(oracle_mod.pyr_down(P1[-1]))))
        P2.append(rnd(jit(oracle_mod.pyr_down(P2[-1]))))
    u = v = None
    for l in range(L - 1, -1, -1):
        Hl, Wl = P1[l].shape
        if l == L - 1:
            u, v = np.zeros((Hl, Wl)), np.zeros((Hl, Wl))
        else:
            u, v = oracle_mod.upsample_flow(u, Hl, Wl), oracle_mod.upsample_flow(v, Hl, Wl)
        for _ in range(n):
            it = oracle_mod.lk_iteration_i1grad if i1grad else oracle_mod.lk_iteration
            u, v, _ = it(P1[l], P2[l], u, v, r)
    return u, v


def ambiguous_mask(ratio_min, r, iterations, lo=1e-7, hi=1e-5):
    """Pixels whose level-0 window came within a decade of the singular guard
    (det/tr^2 in [lo, hi]) at some iteration, grown by the distance one decision can
    travel in the remaining iterations ((r+1) px each)."""
    from scipy import ndimage
    band = (ratio_min >= lo) & (ratio_min <= hi)
    if not band.any():
        return band
    k = (r + 1) * iterations
    return ndimage.binary_dilation(band, np.ones((2 * k + 1, 2 * k + 1), bool))


def compare(u, v, uo, vo, mask=None):
    du = np.abs(u - uo)
    dv = np.abs(v - vo)
    d = np.maximum(du, dv)
    if mask is not None:
        d, du, dv = d[~mask], du[~mask], dv[~mask]
    return {"max": float(d.max()) if d.size else 0.0,
            "rms": float(np.sqrt(0.5 * (du ** 2 + dv ** 2).mean())) if d.size else 0.0,
            "n": int(d.size)}


def parity_check(u, v, pair_or_imgs, oracle_mod, L, r, n, storage, label="", margin=None, workload=True,
                 excluded_max=None, sensitive_max=0.01, region=None, round0=False, probes=1, probe_amp=1e-6,
                 i1grad=False):
    """Assert the tolerance of `storage` on the compared pixels (see the module docstring).
    workload=False (synthetic textures used for shape coverage) asserts the
    implementation check only and reports the storage effect. i1grad: the variant
    linearised with the first image's gradient, on both sides."""
    I1, I2 = images(pair_or_imgs)
    I1 = np.asarray(I1, np.float64)
    I2 = np.asarray(I2, np.float64)
    uo, vo, q = oracle_mod.flow(I1, I2, L, r, n, want_ratio=True, i1grad=i1grad)
    H, W = u.shape
    tmax, trms = TOL[storage]
    if margin is None:
        margin = (r + 2) * 2 ** (L - 1)
    border = np.ones((H, W), bool)
    border[margin:H - margin, margin:W - margin] = False
    if region is not None:      # compare only inside `region` (the rest is reported)
        outside = ~region & ~border
        if outside.any():
            uo_, vo_ = oracle_mod.flow(I1, I2, L, r, n, i1grad=i1grad)
            d = np.maximum(np.abs(u - uo_), np.abs(v - vo_))[outside]
            print(f"{label} {storage}: outside the compared region ({int(outside.sum())} px): max {d.max():.3e} "
                  f"rms {np.sqrt((d ** 2).mean()):.3e}, within tol {float((d <= TOL[storage][0]).mean()):.2%}")
        border |= ~region
    n_inner = int((~border).sum())
    assert n_inner > 0, "no interior pixels for this margin"
    amb = ambiguous_mask(q, r, n) & ~border
    unstable = np.zeros((H, W), bool)
    us, vs_ = oracle_flow_stored(oracle_mod, I1, I2, L, r, n, storage, round0=round0, i1grad=i1grad)

    def probe(k):
        rng = np.random.default_rng(12345 + k)
        up, vp = oracle_mod.flow(I1 * (1 + rng.uniform(-probe_amp, probe_amp, I1.shape)),
                                 I2 * (1 + rng.uniform(-probe_amp, probe_amp, I2.shape)), L, r, n, i1grad=i1grad)
        mv = np.maximum(np.abs(up - uo), np.abs(vp - vo)) > 0.25 * tmax
        if storage != "f32":
            # stability to a rounding flip of stored pyramid values
            uq, vq = oracle_flow_stored(oracle_mod, I1, I2, L, r, n, storage, perturb=probe_amp, seed=7 + k,
                                        round0=round0, i1grad=i1grad)
            mv |= np.maximum(np.abs(uq - us), np.abs(vq - vs_)) > 0.25 * tmax
        return mv
    for k in range(probes):
        unstable |= probe(k)
    unstable &= ~border & ~amb
    invalid = border | amb | unstable
    limit = excluded_max if excluded_max is not None else (0.01 if workload else 0.05)
    assert amb.sum() + unstable.sum() <= limit * n_inner, \
        f"{int(amb.sum())} near-singular and {int(unstable.sum())} unstable of {n_inner} interior px"
    sens = (np.maximum(np.abs(us - uo), np.abs(vs_ - vo)) > 0.5 * tmax) & ~invalid
    impl = compare(u, v, us, vs_, invalid)
    st = compare(u, v, uo, vo, invalid)
    sm = compare(u, v, uo, vo, invalid | sens)
    full = np.maximum(np.abs(u - uo), np.abs(v - vo))
    print(f"{label} {storage}: {impl['n']} px compared (near-singular {int(amb.sum())}, unstable "
          f"{int(unstable.sum())}); vs oracle on the same stored pyramid: max {impl['max']:.3e} rms "
          f"{impl['rms']:.3e}; vs unrounded FP64 oracle: max {st['max']:.3e} rms {st['rms']:.3e}, "
          f"storage-sensitive {int(sens.sum())}, max on the rest {sm['max']:.3e}; whole image max {full.max():.3e}")
    assert impl["max"] <= IMPL_TOL, impl
    if workload:
        if trms is not None:
            assert sm["rms"] <= trms, sm
        assert sens.sum() <= sensitive_max * max(1, impl["n"]), int(sens.sum())
        assert sm["max"] <= tmax, sm
    impl["invalid"] = invalid   # the pixels left out of the comparison (border, near-singular, unstable)
    return impl


def epe(u, v, pair, margin):
    e = np.sqrt((u - pair.u_gt) ** 2 + (v - pair.v_gt) ** 2)[margin:-margin, margin:-margin]
    return float(np.sqrt((e ** 2).mean())), float(e.max())
