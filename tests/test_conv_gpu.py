"""Frames converted ahead of the reconstruction.

The single-frame entry points convert a frame of at least one wave of tiles in one pass (Eq. 18
and the inverse of Eq. 20, once per sample, into colour-phase planes in device memory) and the
reconstruction then copies converted footprints; the batched launch, the no-allocation entry
point and small frames convert each staged footprint inside the kernel. Both use the same
per-sample arithmetic, so their outputs are identical. Cases: odd sensor sizes (a padding column
and row in the converted planes), per-pixel calibration frames with saturated pixels, the printed
weight K / s (square root of the inverse variance), the host-buffer entry point (rows converted
band by band behind their copies), and calls on two streams sharing the context's conversion
buffer.
"""
import dataclasses

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


def _odd_frame(seed=1201, order=2, w=225, h=209):
    """3 sensors of w x h (odd sizes), small rotations, (w - 1) x (h - 1) output (224 x 208 =
    46592 pixels by default: more than one wave of 16 x 16 tiles), 4 scales; sensor 1 with per-pixel
    calibration frames whose saturation level is low in a band of rows."""
    p = synth.Params(order=order, sigmas=synth.PAPER_SCALES, out_w=w - 1, out_h=h - 1)
    fr = synth._build_frame(seed, 3, w, h, (1.0, 1 / 8, 1 / 64), 1.0, 0.3, 0.0, p, f"odd-3x{w}x{h}")
    r = np.random.default_rng(seed)
    s = fr.sensors[1]
    s.bias_frame = (s.black + r.uniform(-2, 2, (h, w))).astype(np.float32)
    s.prnu_frame = r.uniform(0.95, 1.05, (h, w)).astype(np.float32)
    s.read_var_frame = r.uniform(6, 12, (h, w)).astype(np.float32)
    sat = np.full((h, w), 4095, np.uint16)
    sat[60:90] = 300
    s.sat_frame = sat
    return fr


def _single(ctx, rig, fr, p=None):
    p = p or fr.params
    raws = [torch.from_numpy(s.raw).cuda() for s in fr.sensors]
    ch = torch.empty((3, p.out_h, p.out_w), dtype=torch.uint8, device="cuda")
    out = ctx.reconstruct(rig, p, raws, choice=ch)
    ctx.check()
    return out.cpu().numpy(), ch.cpu().numpy()


def test_converted_equals_in_kernel_conversion(ctx):
    from paper_1308_4908_gb300 import hdr
    fr = _odd_frame()
    ctx.set_rig(0, fr.sensors)
    p = fr.params
    assert p.out_w * p.out_h >= 152 * 256
    conv = _single(ctx, 0, fr)
    raws = [torch.from_numpy(s.raw).cuda() for s in fr.sensors]
    out = torch.full((3, p.out_h, p.out_w), -7.0, device="cuda")
    ch = torch.empty((3, p.out_h, p.out_w), dtype=torch.uint8, device="cuda")
    keep = [raws]
    ctx.reconstruct_batch([ctx.frame(0, p, raws, out, ch, keep)], hdr.hdr_batch_config(16, 0, 1, 0))
    ctx.check()
    np.testing.assert_array_equal(conv[1], ch.cpu().numpy())
    np.testing.assert_array_equal(conv[0], out.cpu().numpy())
    r = np.random.default_rng(3)
    pix = np.concatenate([np.stack([r.integers(0, 224, 250), r.integers(0, 208, 250)], 1),
                          [[0, 0], [223, 207], [223, 0], [0, 207], [100, 37], [100, 40]]])
    o = oracle.reconstruct(fr.sensors, p, pix, levels=True, kappa=True)
    parity.compare(conv[0][:, pix[:, 1], pix[:, 0]], conv[1][:, pix[:, 1], pix[:, 0]], o, pix, len(p.sigmas),
                   p.order, p.ici_gamma, p.min_pivot)


def test_printed_weight_converted(ctx):
    """weight_mode 1 stages 1 / s: the conversion pass takes the square root as the kernel does
    (against the no-allocation entry point, which converts in the kernel)."""
    from paper_1308_4908_gb300 import hdr
    fr = _odd_frame(seed=1202, order=1)
    p = dataclasses.replace(fr.params, weight_mode=1)
    ctx.set_rig(1, fr.sensors)
    conv = _single(ctx, 1, fr, p)
    raws = [torch.from_numpy(s.raw).cuda() for s in fr.sensors]
    keep = []
    descs = [hdr.sensor_desc(s, keep) for s in fr.sensors]
    out = torch.full((3, p.out_h, p.out_w), -7.0, device="cuda")
    ch = torch.empty((3, p.out_h, p.out_w), dtype=torch.uint8, device="cuda")
    hdr.hdr_reconstruct_noalloc(0, descs, hdr.params_struct(p), [int(t.data_ptr()) for t in raws], out.data_ptr(),
                                ch.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(conv[1], ch.cpu().numpy())
    np.testing.assert_array_equal(conv[0], out.cpu().numpy())


def test_host_buffers_convert_band_by_band(ctx):
    """hdr_reconstruct_host copies and converts each band's new raw rows behind the previous band:
    the same result as converting the whole frame before one launch."""
    fr = synth.paper_scale(size=512, seed=1203)
    ctx.set_rig(2, fr.sensors)
    p = fr.params
    ref = _single(ctx, 2, fr)
    raws = [np.ascontiguousarray(s.raw) for s in fr.sensors]
    out = np.full((3, p.out_h, p.out_w), -7.0, np.float32)
    ch = np.zeros((3, p.out_h, p.out_w), np.uint8)
    ctx.reconstruct_host(2, p, raws, out, ch)
    np.testing.assert_array_equal(ch, ref[1])
    np.testing.assert_array_equal(out, ref[0])


def test_host_buffers_odd_sizes_and_calibration_frames(ctx):
    """The host-buffer path on 3 sensors of 513 x 387 (odd sizes; 25 tile rows: three bands, whose
    row ranges end inside the frame and, for the last, at the padding row of the odd height) with
    per-pixel calibration frames: identical to the device-buffer call."""
    fr = _odd_frame(seed=1206, order=1, w=513, h=387)
    ctx.set_rig(5, fr.sensors)
    p = fr.params
    ref = _single(ctx, 5, fr)
    raws = [np.ascontiguousarray(s.raw) for s in fr.sensors]
    out = np.full((3, p.out_h, p.out_w), -7.0, np.float32)
    ch = np.zeros((3, p.out_h, p.out_w), np.uint8)
    ctx.reconstruct_host(5, p, raws, out, ch)
    np.testing.assert_array_equal(ch, ref[1])
    np.testing.assert_array_equal(out, ref[0])


def test_calls_on_two_streams_share_the_buffer(ctx):
    """Frames of two rigs reconstructed alternately on two streams with no synchronisation between
    the calls: each call converts into the context's one buffer only after the previous call that
    used it, whatever its stream."""
    a = _odd_frame(seed=1204)
    b = synth.paper_scale(size=256, seed=1205)
    ctx.set_rig(3, a.sensors)
    ctx.set_rig(4, b.sensors)
    ref_a, ref_b = _single(ctx, 3, a), _single(ctx, 4, b)
    ra = [torch.from_numpy(s.raw).cuda() for s in a.sensors]
    rb = [torch.from_numpy(s.raw).cuda() for s in b.sensors]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    outs = []
    for k in range(3):
        for st, rig, fr, raws in ((s1, 3, a, ra), (s2, 4, b, rb)):
            p = fr.params
            with torch.cuda.stream(st):
                o = torch.empty((3, p.out_h, p.out_w), device="cuda")
                c = torch.empty((3, p.out_h, p.out_w), dtype=torch.uint8, device="cuda")
                ctx.reconstruct(rig, p, raws, out=o, choice=c, stream=st)
            outs.append((rig, o, c))
    torch.cuda.synchronize()
    ctx.check()
    for rig, o, c in outs:
        ro, rc = ref_a if rig == 3 else ref_b
        np.testing.assert_array_equal(c.cpu().numpy(), rc)
        np.testing.assert_array_equal(o.cpu().numpy(), ro)
