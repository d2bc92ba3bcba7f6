"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle on seeded inputs."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_1308_4908_gb300 import synth
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_4908_gb300 import hdr
    c = hdr.Context(0)
    yield c
    c.close()


def upload(frame):
    return [torch.from_numpy(s.raw).cuda() for s in frame.sensors]


def run(ctx, frame, params=None, rig_id=0, levels=False):
    p = params or frame.params
    ctx.set_rig(rig_id, frame.sensors)
    raws = upload(frame)
    choice = torch.empty((3, p.out_h, p.out_w), dtype=torch.uint8, device="cuda")
    lv = None
    if levels:
        NL = len(p.sigmas) + p.order
        lv = torch.empty((3, NL, p.out_h, p.out_w, 2), dtype=torch.float32, device="cuda")
    out = ctx.reconstruct(rig_id, p, raws, choice=choice, levels=lv)
    ctx.check()
    res = dict(out=out.float().cpu().numpy(), choice=choice.cpu().numpy())
    if levels:
        res["levels"] = lv.cpu().numpy()
    return res


def check_frame(ctx, frame, params=None, pixels=None, rel_tol=parity.REL_TOL, extra=0.0, levels=False):
    """Run the frame on the GPU and compare with the oracle (tolerance in tests/parity.py)."""
    p = params or frame.params
    g = run(ctx, frame, p, levels=levels)
    if pixels is None:
        vv, uu = np.mgrid[0:p.out_h, 0:p.out_w]
        pixels = np.stack([uu.ravel(), vv.ravel()], axis=1)
    o = oracle.reconstruct(frame.sensors, p, pixels, levels=True, kappa=True)
    gu = g["out"][:, pixels[:, 1], pixels[:, 0]]
    gc = g["choice"][:, pixels[:, 1], pixels[:, 0]]
    stats = parity.compare(gu, gc, o, pixels, len(p.sigmas), p.order, p.ici_gamma, p.min_pivot,
                           rel_tol=rel_tol, extra_rel=extra)
    return stats, g, o


# ------------------------------------------------------------------ workloads

def test_tiny_full_frame(ctx):
    """2 sensors of 64x64, order 0, one scale: every output pixel against the oracle."""
    stats, _, _ = check_frame(ctx, synth.tiny())
    assert stats["n"] > 3 * 64 * 64 * 0.9
    assert stats["mismatched_choice"] == 0


@pytest.mark.parametrize("order", [0, 1, 2])
def test_paper_rig_small_all_orders(ctx, order):
    """The paper-scale recipe (3 sensors, affine misalignment, 4 scales with ICI) on a 96x96
    frame - six tiles per side with a ragged tail - for every order, all pixels."""
    fr = synth.paper_scale(size=96)
    p = dataclasses.replace(fr.params, order=order)
    stats, _, _ = check_frame(ctx, fr, p)
    assert stats["n"] > 0


def test_paper_scale_full_size_sampled(ctx):
    """Full 3 x 2048^2 frame, order 2, ICI over 4 scales, in the benchmark's launch
    configuration; the oracle checks 3000 sampled pixels plus the frame border."""
    fr = synth.paper_scale()
    r = np.random.default_rng(0)
    pix = r.integers(0, 2048, (2400, 2))
    edge = np.concatenate([np.stack([np.arange(0, 2048, 17), np.zeros(121, int)], 1),
                           np.stack([np.full(121, 2047), np.arange(0, 2048, 17)], 1),
                           np.stack([np.arange(0, 2048, 17), np.full(121, 2047)], 1),
                           np.stack([np.zeros(121, int), np.arange(0, 2048, 17)], 1)])
    pix = np.concatenate([pix, edge, [[0, 0], [2047, 2047], [0, 2047], [2047, 0]]])
    stats, g, _ = check_frame(ctx, fr, pixels=pix)
    assert stats["n"] > 3 * 2400
    assert np.isfinite(g["out"]).mean() > 0.999


def check_levels(ctx, fr):
    """C_0 and Var C_0 of every level from the diagnostic entry point against the oracle's."""
    p = fr.params
    g = run(ctx, fr, p, levels=True)
    vv, uu = np.mgrid[0:64, 0:64]
    pix = np.stack([uu.ravel(), vv.ravel()], axis=1)
    o = oracle.reconstruct(fr.sensors, p, pix, levels=True, kappa=True)
    lv = g["levels"]  # [3, NL, H, W, 2]
    NL = lv.shape[1]
    n_cmp = 0
    for c in range(3):
        for l in range(NL):
            gc0 = lv[c, l, pix[:, 1], pix[:, 0], 0]
            gv = lv[c, l, pix[:, 1], pix[:, 0], 1]
            ov, oc0, ovar, piv = o["valid"][:, c, l], o["c0"][:, c, l], o["var"][:, c, l], o["pivot"][:, c, l]
            clear = np.abs(piv - p.min_pivot) > 0.02 * p.min_pivot + parity.pivot_band(piv, o["kappa"][:, c, l])
            both = clear & (ov == 1)
            assert np.all(np.isfinite(gc0[both])), (c, l)
            assert np.all(np.isnan(gc0[clear & (ov == 0)])), (c, l)
            tol = parity.level_tol(oc0[both], o["efit"][both, c, l], o["ew"][both, c, l])
            err = np.abs(gc0[both] - oc0[both])
            assert np.all(err <= tol), (c, l, float((err / tol).max()))
            # Var C_0 is a quadratic form in the same fit: allow 10x the C_0 tolerance, relative
            ev = np.abs(gv[both] - ovar[both]) / np.abs(ovar[both])
            assert np.all(ev <= 10 * tol / np.maximum(np.abs(oc0[both]), parity.TAU) + 1e-4), (c, l, float(ev.max()))
            n_cmp += both.sum()
    assert n_cmp > 3 * 64 * 64 * 3


def test_levels_match_oracle(ctx):
    """Every level (each scale at order M, then the lower orders at the largest scale):
    C_0 and Var C_0 from the diagnostic entry point against the oracle's."""
    check_levels(ctx, synth.paper_scale(size=64, seed=1010))


def test_levels_on_a_translational_rig(ctx):
    """A rig whose plain reconstruction reads tabulated weights: the diagnostic entry point plans
    the searched window instead, and every level matches the oracle."""
    check_levels(ctx, translational(64, 1011, [(0.0, 0.0), (0.4, 0.45), (-1.3, 0.7)]))


# ------------------------------------------------------------------ rigs and mappings

@pytest.mark.parametrize("case", ["aligned", "translated", "rotated6", "upsampled"])
def test_rigs(ctx, case):
    """Perfectly aligned sensors, the [0.4, 0.45] px middle-sensor offset, 6 degree rotations
    (Section 7.2) and a 1.5x upsampled output (Section 4.2: arbitrary output resolution)."""
    fr = synth.paper_scale(size=80, seed=1020)
    W = 80
    if case == "aligned":
        affs = [synth.affine_about_center(W, W)] * 3
    elif case == "translated":
        affs = [synth.affine_about_center(W, W), synth.affine_about_center(W, W, 0.4, 0.45),
                synth.affine_about_center(W, W)]
    elif case == "rotated6":
        affs = [synth.affine_about_center(W, W), synth.affine_about_center(W, W, 0.3, -0.2, 6.0),
                synth.affine_about_center(W, W, -0.5, 0.1, -6.0)]
    else:
        affs = [s.affine for s in fr.sensors]
    for s, a in zip(fr.sensors, affs):
        s.affine = np.asarray(a)
        s.raw = synth.simulate_raw(fr.scene, s, 1020, int(s.nd * 1000))
    p = fr.params
    if case == "upsampled":
        p = dataclasses.replace(p, out_w=120, out_h=120, out_affine=synth.output_affine(W, W, 120, 120))
    if case == "aligned":
        p = dataclasses.replace(p, order=1)
    check_frame(ctx, fr, p)


def translational(size, seed, shifts):
    """The paper rig with pure translations (Section 8's aligned/translational case) at 1x output."""
    fr = synth.paper_scale(size=size, seed=seed)
    for s, (tx, ty) in zip(fr.sensors, shifts):
        s.affine = np.asarray(synth.affine_about_center(size, size, tx, ty))
        s.raw = synth.simulate_raw(fr.scene, s, seed, int(s.nd * 1000))
    return fr


@pytest.mark.parametrize("order", [0, 1, 2])
def test_tabulated_weights_match_the_oracle(ctx, order):
    """Translation-only rigs at 1x output read their windows from the per-frame table (Section 8):
    every pixel within tolerance of the oracle; the searched path gives the same fit up to
    rounding (the two paths are different code: their outputs are not bit-identical)."""
    fr = translational(96, 1040 + order, [(0.0, 0.0), (0.4, 0.45), (-1.3, 0.7)])
    p = dataclasses.replace(fr.params, order=order)
    _, g, _ = check_frame(ctx, fr, p)
    q = dataclasses.replace(p, tab_weights=0)
    _, h, _ = check_frame(ctx, fr, q)
    assert not np.array_equal(g["out"], h["out"])


def test_tabulated_weights_other_shifts_and_scales(ctx):
    """Integer, negative and half-pixel shifts, one scale and eight scales, FP16 output."""
    fr = translational(80, 1050, [(-2.0, 3.0), (0.5, -0.5), (1.999, -0.001)])
    check_frame(ctx, fr, dataclasses.replace(fr.params, sigmas=(0.7,)))
    check_frame(ctx, fr, dataclasses.replace(fr.params, order=1, sigmas=tuple(0.5 + 0.2 * i for i in range(8))))
    check_frame(ctx, fr, dataclasses.replace(fr.params, out_dtype=1), extra=parity.HALF_TOL)


@pytest.mark.parametrize("order,sigmas,extra", [
    (2, (0.6, 0.9, 1.3), {}),                       # two scales per pass: a short first pass
    (0, (0.5, 0.7, 0.9, 1.2, 1.6), {}),             # four per pass: passes of 1 and 4 scales
    (2, (1.1,), {}),                                # one scale in the second slot of one pass
    (1, (0.6, 0.9, 1.3, 1.8), {"accum": 1}),        # compensated sums: one scale per pass
    (1, (0.6, 0.9, 1.3, 1.8), {"cond_fallback": 1.0}),  # the FP64 re-solve compiled in
])
def test_tabulated_weights_passes(ctx, order, sigmas, extra):
    """The table holds the cells of each pass's largest window, nearest first, with one weight per
    scale of the pass: scale counts that leave the first pass short, a single scale, compensated
    sums (one scale per pass) and the FP64 re-solve variant all match the oracle, and differ from
    the searched path only by rounding."""
    fr = translational(72, 1070 + order, [(0.25, -0.6), (-1.4, 0.35), (0.9, 1.2)])
    p = dataclasses.replace(fr.params, order=order, sigmas=sigmas, **extra)
    _, g, _ = check_frame(ctx, fr, p)
    _, h, _ = check_frame(ctx, fr, dataclasses.replace(p, tab_weights=0))
    assert not np.array_equal(g["out"], h["out"])


def test_tabulated_weights_only_for_translations(ctx):
    """A rotated rig or a resampled output keeps the searched window: the switch changes nothing."""
    fr = synth.paper_scale(size=64, seed=1060)
    a = run(ctx, fr, fr.params)
    b = run(ctx, fr, dataclasses.replace(fr.params, tab_weights=0))
    np.testing.assert_array_equal(a["out"], b["out"])
    fr = translational(64, 1061, [(0.3, 0.2), (0.1, -0.4), (0.0, 0.0)])
    p = dataclasses.replace(fr.params, out_w=96, out_h=96, out_affine=synth.output_affine(64, 64, 96, 96))
    a = run(ctx, fr, p)
    b = run(ctx, fr, dataclasses.replace(p, tab_weights=0))
    np.testing.assert_array_equal(a["out"], b["out"])


def test_ragged_and_tiny_outputs(ctx):
    """Output sizes that are not multiples of the tile, a 1x1 output, and an output that
    extends past the sensors (NaN where no sample exists)."""
    fr = synth.paper_scale(size=48, seed=1030)
    for (w, h) in ((37, 23), (1, 1), (17, 16)):
        check_frame(ctx, fr, dataclasses.replace(fr.params, out_w=w, out_h=h))
    p = dataclasses.replace(fr.params, out_w=64, out_h=64,
                            out_affine=np.array([[1.0, 0, -8.0], [0, 1.0, -8.0]]))
    _, g, o = check_frame(ctx, fr, p)
    assert np.isnan(g["out"][:, 0, 0]).all()


def test_empty_output_is_a_noop(ctx):
    fr = synth.tiny()
    p = dataclasses.replace(fr.params, out_w=0, out_h=0)
    ctx.set_rig(0, fr.sensors)
    out = torch.empty((3, 0, 0), device="cuda")
    ctx.reconstruct(0, p, upload(fr), out=out)
    ctx.check()


@pytest.mark.parametrize("n_scales", [1, 8])
def test_scale_counts(ctx, n_scales):
    fr = synth.paper_scale(size=40, seed=1040)
    sig = (1.1,) if n_scales == 1 else tuple(0.4 + 0.25 * k for k in range(8))
    check_frame(ctx, fr, dataclasses.replace(fr.params, sigmas=sig))


def test_one_and_eight_sensors(ctx):
    fr = synth.paper_scale(size=40, seed=1050)
    one = synth.Frame(fr.sensors[:1], dataclasses.replace(fr.params, order=1), fr.scene)
    check_frame(ctx, one)
    r = np.random.default_rng(3)
    sens = []
    for k in range(8):
        s = synth.Sensor(40, 40, 2.0 ** (-2 * k), synth.affine_about_center(40, 40, *r.uniform(-1, 1, 2),
                                                                           r.uniform(-3, 3)))
        s.raw = synth.simulate_raw(fr.scene, s, 1050, k)
        sens.append(s)
    check_frame(ctx, synth.Frame(sens, fr.params, fr.scene))


def test_saturated_sensor_and_calibration_frames(ctx):
    """A fully saturated sensor contributes nothing; per-pixel bias / non-uniformity /
    read-noise / saturation frames (Sections 4.1, 6) follow the oracle."""
    fr = synth.paper_scale(size=48, seed=1060)
    fr.sensors[0].raw[:] = synth.CLIP_DN
    check_frame(ctx, fr)
    r = np.random.default_rng(4)
    for s in fr.sensors:
        s.bias_frame = (s.black + r.uniform(-2, 2, (48, 48))).astype(np.float32)
        s.prnu_frame = r.uniform(0.95, 1.05, (48, 48)).astype(np.float32)
        s.read_var_frame = r.uniform(6, 12, (48, 48)).astype(np.float32)
        s.sat_frame = np.full((48, 48), 4000, np.uint16)
    check_frame(ctx, fr)


def test_sensor_order_independence_gpu(ctx):
    """Permuting the sensors changes only the FP32 summation order: both orders meet the oracle,
    and where they used the same level they differ by at most twice its tolerance."""
    fr = synth.paper_scale(size=64, seed=1070)
    sa, a, o = check_frame(ctx, fr)
    fr2 = synth.Frame(fr.sensors[::-1], fr.params, fr.scene)
    sb, b, _ = check_frame(ctx, fr2)
    same = a["choice"] == b["choice"]
    assert same.mean() > 0.99
    vv, uu = np.mgrid[0:64, 0:64]
    lvl = np.where(a["choice"] == 255, 0, a["choice"]).astype(int)          # [3, H, W]
    ochoice = o["choice"].T.reshape(3, 64, 64) if o["choice"].ndim == 2 else o["choice"]
    for c in range(3):
        m = same[c] & (a["choice"][c] != 255)
        idx = (vv[m] * 64 + uu[m])
        l = lvl[c][m]
        tol = parity.level_tol(o["c0"][idx, c, l], o["efit"][idx, c, l], o["ew"][idx, c, l])
        assert np.all(np.abs(a["out"][c][m] - b["out"][c][m]) <= 2 * tol)


# ------------------------------------------------------------------ precision variants and APIs

@pytest.mark.parametrize("out_dtype,accum", [(0, 1), (1, 0), (1, 1)])
def test_precision_variants(ctx, out_dtype, accum):
    fr = synth.paper_scale(size=64, seed=1080)
    p = dataclasses.replace(fr.params)
    p.out_dtype = out_dtype
    p.accum = accum
    extra = parity.HALF_TOL if out_dtype == 1 else 0.0
    check_frame(ctx, fr, p, extra=extra)


def test_host_buffer_entry_point_matches(ctx):
    fr = synth.paper_scale(size=64, seed=1090)
    a = run(ctx, fr)
    out = np.empty((3, 64, 64), np.float32)
    ch = np.empty((3, 64, 64), np.uint8)
    ctx.reconstruct_host(0, fr.params, [np.ascontiguousarray(s.raw) for s in fr.sensors], out, ch)
    np.testing.assert_array_equal(out, a["out"])
    np.testing.assert_array_equal(ch, a["choice"])


@pytest.mark.parametrize("case", ["paper", "rotated6", "upsampled", "half"])
def test_host_buffer_bands_match_the_device_path(ctx, case):
    """Outputs of 32+ tile rows go through the host-buffer entry point in row bands (copies in and
    out overlapped with the reconstruction): results equal the device-buffer entry point's, also
    for rotated rigs and resampled outputs whose windows reach rows of the next band."""
    fr = synth.paper_scale(size=640, seed=1095)
    W = 640
    p = fr.params
    if case == "rotated6":
        affs = [synth.affine_about_center(W, W), synth.affine_about_center(W, W, 0.3, -0.2, 6.0),
                synth.affine_about_center(W, W, -0.5, 0.1, -6.0)]
        for s, a in zip(fr.sensors, affs):
            s.affine = np.asarray(a)
            s.raw = synth.simulate_raw(fr.scene, s, 1095, int(s.nd * 1000))
    elif case == "upsampled":
        p = dataclasses.replace(p, out_w=960, out_h=720, out_affine=synth.output_affine(W, W, 960, 720))
    elif case == "half":
        p = dataclasses.replace(p, out_dtype=1)
    a = run(ctx, fr, p)
    dt = np.float16 if case == "half" else np.float32
    out = np.full((3, p.out_h, p.out_w), -7.0, dt)
    ch = np.zeros((3, p.out_h, p.out_w), np.uint8)
    ctx.reconstruct_host(0, p, [np.ascontiguousarray(s.raw) for s in fr.sensors], out, ch)
    ctx.check()
    np.testing.assert_array_equal(out.astype(np.float32), a["out"])
    np.testing.assert_array_equal(ch, a["choice"])


def test_invalid_arguments_are_rejected(ctx):
    from paper_1308_4908_gb300 import hdr
    fr = synth.tiny()
    ctx.set_rig(0, fr.sensors)
    raws = upload(fr)
    for bad in (dict(order=3), dict(sigmas=(0.8, 0.5)), dict(sigmas=(-1.0,)), dict(trunc_k=0.0)):
        p = dataclasses.replace(fr.params, **bad)
        with pytest.raises(hdr.HdrError) as ei:
            ctx.reconstruct(0, p, raws)
        assert ei.value.status == hdr.HDR_E_INVALID
    with pytest.raises(hdr.HdrError):
        ctx.reconstruct(5, fr.params, raws)          # undefined rig
    bad_sensor = dataclasses.replace(fr.sensors[0], pitch=63)
    with pytest.raises(hdr.HdrError):
        ctx.set_rig(2, [bad_sensor])
    ctx.check()


def test_printed_noise_weight_with_compensated_sums(ctx):
    """weight_mode 1 with compensated moment sums (its own instantiation), order 2, every pixel."""
    fr = synth.paper_scale(size=64, seed=1074)
    check_frame(ctx, fr, dataclasses.replace(fr.params, weight_mode=1, accum=1))


@pytest.mark.parametrize("order", [0, 1, 2])
def test_printed_noise_weight(ctx, order):
    """weight_mode 1, the noise weight K / s as printed in Section 5.2 (Var C_0 with w^2 s2 = K^2),
    against the oracle in the same mode on every pixel of the 96x96 paper rig; the default weight
    gives a different result, and the host-buffer entry point the same bits."""
    fr = synth.paper_scale(size=96, seed=1070 + order)
    p = dataclasses.replace(fr.params, order=order, weight_mode=1)
    _, g, _ = check_frame(ctx, fr, p)
    h = run(ctx, fr, dataclasses.replace(p, weight_mode=0))
    assert not np.array_equal(g["out"], h["out"])
    out = np.empty((3, p.out_h, p.out_w), np.float32)
    ctx.reconstruct_host(0, p, [np.ascontiguousarray(s.raw) for s in fr.sensors], out)
    np.testing.assert_array_equal(out, g["out"])


def test_printed_noise_weight_rejected_where_unsupported(ctx):
    """The level maps, batches, the serving loop and the adaptive passes use the inverse-variance
    weight only: weight_mode 1 is refused there with HDR_E_UNSUPPORTED, before any work."""
    from paper_1308_4908_gb300 import hdr
    fr = synth.paper_scale(size=64, seed=1075)
    p = dataclasses.replace(fr.params, weight_mode=1)
    ctx.set_rig(0, fr.sensors)
    raws = upload(fr)
    out = torch.empty((3, p.out_h, p.out_w), dtype=torch.float32, device="cuda")
    lv = torch.empty((3, len(p.sigmas) + p.order, p.out_h, p.out_w, 2), dtype=torch.float32, device="cuda")
    calls = [
        lambda: ctx.reconstruct(0, p, raws, out=out, levels=lv),
        lambda: ctx.reconstruct_batch([ctx.frame(0, p, raws, out, keep=keep)]),
        lambda: ctx.calpa_gradients(0, p, hdr.hdr_calpa_params_default(), raws),
        lambda: ctx.reconstruct_adaptive(0, p, hdr.hdr_calpa_params_default(), raws, out=out),
    ]
    keep = []
    for call in calls:
        with pytest.raises(hdr.HdrError) as e:
            call()
        assert e.value.status == hdr.HDR_E_UNSUPPORTED
    srv = hdr.Server(ctx, pool_bytes=64 << 20)
    try:
        with pytest.raises(hdr.HdrError) as e:
            srv.submit(0, p, [np.ascontiguousarray(s.raw) for s in fr.sensors], np.empty((3, 64, 64), np.float32))
        assert e.value.status == hdr.HDR_E_UNSUPPORTED
    finally:
        srv.close()
    ctx.check()


def test_largest_output(ctx):
    """The largest output the library accepts, 2^29 pixels (23168 x 23168, the paper rig upsampled
    about 11.3x: 2.1M tiles, planar offsets beyond 2^30), against the oracle on sampled pixels
    including the far corner; five rows more exceed 2^29 and are refused with HDR_E_UNSUPPORTED
    before any work."""
    from paper_1308_4908_gb300 import hdr
    fr = synth.paper_scale(size=2048)
    n = 23168
    assert n * (n + 4) <= 2 ** 29 < n * (n + 5)
    p = dataclasses.replace(fr.params, out_w=n, out_h=n, out_affine=synth.output_affine(2048, 2048, n, n))
    ctx.set_rig(0, fr.sensors)
    raws = upload(fr)
    out = torch.empty((3, n, n), dtype=torch.float32, device="cuda")
    ch = torch.empty((3, n, n), dtype=torch.uint8, device="cuda")
    ctx.reconstruct(0, p, raws, out=out, choice=ch)
    ctx.check()
    r = np.random.default_rng(11)
    pix = np.concatenate([r.integers(0, n, (150, 2)), [[n - 1, n - 1], [0, n - 1], [n - 1, 0], [0, 0]]])
    iy, ix = torch.from_numpy(pix[:, 1]).cuda(), torch.from_numpy(pix[:, 0]).cuda()
    gu = out[:, iy, ix].cpu().numpy()
    gc = ch[:, iy, ix].cpu().numpy()
    del out, ch
    o = oracle.reconstruct(fr.sensors, p, pix, levels=True, kappa=True)
    parity.compare(gu, gc, o, pix, len(p.sigmas), p.order, p.ici_gamma, p.min_pivot)
    with pytest.raises(hdr.HdrError) as e:
        ctx.reconstruct(0, dataclasses.replace(p, out_h=n + 5), raws, out=torch.empty(1, device="cuda"))
    assert e.value.status == hdr.HDR_E_UNSUPPORTED
    torch.cuda.empty_cache()
