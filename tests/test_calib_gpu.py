"""Calibration estimates (Section 6.2) on the GPU against the FP64 oracle: stack statistics
bit-exact (both sides evaluate the same exact-integer formula), the pooled gain and the exposure
scaling within 1e-12 relative (FP64 sums in another order), the non-uniformity frame within one
FP32 rounding."""
import numpy as np
import pytest

from oracle import calib
from paper_1308_4908_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_4908_gb300 import hdr
    c = hdr.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("n,w,h", [(2, 8, 1), (37, 61, 17), (64, 256, 96), (5, 3, 2)])
def test_stack_stats_bit_exact(ctx, n, w, h):
    r = np.random.default_rng(n * 1000 + w)
    pitch = synth.pitch_for(w)
    frames = np.zeros((n, h, pitch), np.uint16)
    frames[:, :, :w] = r.integers(0, 65536, (n, h, w))
    frames[:, :, w:] = 65535                     # padding must not leak into the statistics
    mean, var = ctx.calib_stack_stats(torch.from_numpy(frames).cuda(), w)
    om, ov = calib.stack_stats(frames, w)
    np.testing.assert_array_equal(mean.cpu().numpy(), om)
    np.testing.assert_array_equal(var.cpu().numpy(), ov)


def test_gain_and_exposure_match_the_oracle(ctx):
    g = 2.0
    prnu = (1.0 + 0.02 * np.random.default_rng(3).standard_normal((96, 128))).clip(0.9, 1.1)
    black = synth.flat_stack(31, 16, 128, 96, 0.0, g, 9.0, 64.0)
    flat = synth.flat_stack(32, 16, 128, 96, 700.0, g, 9.0, 64.0)
    ref = synth.flat_stack(33, 16, 128, 96, 1200.0, g, 9.0, 64.0)
    sen = synth.flat_stack(34, 16, 128, 96, 9600.0, g, 9.0, 64.0, nd=1 / 8, prnu=prnu)
    dev = {k: ctx.calib_stack_stats(torch.from_numpy(v).cuda(), 128) for k, v in
           dict(black=black, flat=flat, ref=ref, sen=sen).items()}
    orc = {k: calib.stack_stats(v, 128) for k, v in dict(black=black, flat=flat, ref=ref, sen=sen).items()}
    est, used = ctx.calib_gain(dev["flat"][0], dev["flat"][1], dev["black"][0], dev["black"][1], 20.0, 3800.0)
    oest, oused = calib.gain(*orc["flat"], *orc["black"], 20.0, 3800.0)
    assert used == oused == 128 * 96
    assert abs(est - oest) <= 1e-12 * abs(oest)
    assert abs(est - g) / g < 0.03
    nd, a, used = ctx.calib_exposure(dev["sen"][0], dev["black"][0], g, 1.0, dev["ref"][0], dev["black"][0], g, 1 / 8)
    ond, oa, oused = calib.exposure(orc["sen"][0], orc["black"][0], g, 1.0, orc["ref"][0], orc["black"][0], g, 1 / 8,
                                    20.0, 3800.0)
    assert used == oused
    assert abs(nd - ond) <= 1e-12 * abs(ond)
    a = a.cpu().numpy()
    assert np.all(np.abs(a - oa) <= np.spacing(oa))          # one FP32 rounding apart at most
    assert repr(ctx.calib_gain(dev["flat"][0], dev["flat"][1], dev["black"][0], dev["black"][1])) == \
        repr(ctx.calib_gain(dev["flat"][0], dev["flat"][1], dev["black"][0], dev["black"][1]))


def test_no_usable_pixel_and_invalid_arguments(ctx):
    from paper_1308_4908_gb300 import hdr
    z = torch.zeros((4, 8), device="cuda")
    est, used = ctx.calib_gain(z, z, z, z)
    assert used == 0 and np.isnan(est)
    nd, a, used = ctx.calib_exposure(z, z, 2.0, 1.0, z, z, 2.0, 1.0)
    assert used == 0 and np.isnan(nd) and bool((a == 1).all())
    frames = torch.zeros((1, 4, 8), dtype=torch.uint16, device="cuda")
    with pytest.raises(hdr.HdrError):
        ctx.calib_stack_stats(frames, 8)                       # one frame has no variance
    frames = torch.zeros((3, 4, 12), dtype=torch.uint16, device="cuda")
    with pytest.raises(hdr.HdrError):
        ctx.calib_stack_stats(frames, 8)                       # pitch not a multiple of 8
    with pytest.raises(hdr.HdrError):
        ctx.calib_exposure(z, z, 0.0, 1.0, z, z, 2.0, 1.0)
