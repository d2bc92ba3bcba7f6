"""hdr_reconstruct_noalloc: reconstruction for callers that may not allocate device memory.

A real-time capture thread, or a program whose GPU memory belongs to another runtime's pool,
cannot call cudaMalloc; this entry point keeps its scratch (the kernel's status word and the
rig's per-pixel calibration frames) in a fixed device array inside the library. The test calls
it through the C ABI twice in a row - first a rig with per-pixel calibration frames, then a
different rig with scalar calibration, so the second call runs over the first call's leftovers -
and checks each result against the context-based entry point within the parity tolerance used by
the other GPU tests; one result is also checked against the FP64 oracle, and the free device memory
is checked to stay the same across a call. This file is named to be collected last.
"""
import dataclasses

import numpy as np
import pytest

from paper_1308_4908_gb300 import synth
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _frames_rig():
    fr = synth.paper_scale(size=96, seed=1110)
    r = np.random.default_rng(11)
    for s in fr.sensors:
        s.bias_frame = (s.black + r.uniform(-2, 2, (96, 96))).astype(np.float32)
        s.prnu_frame = r.uniform(0.95, 1.05, (96, 96)).astype(np.float32)
        s.read_var_frame = r.uniform(6, 12, (96, 96)).astype(np.float32)
        s.sat_frame = np.full((96, 96), 4000, np.uint16)
    return fr


def _scalar_rig():
    fr = synth.paper_scale(size=80, seed=1111)
    return synth.Frame(fr.sensors, dataclasses.replace(fr.params, order=1), fr.scene)


def _run_both(hdr, ctx, fr):
    p = fr.params
    hp = hdr.params_struct(p)
    raws = [torch.from_numpy(s.raw).cuda() for s in fr.sensors]
    ptrs = [int(t.data_ptr()) for t in raws]
    ctx.set_rig(0, fr.sensors)
    ref = torch.empty((3, p.out_h, p.out_w), device="cuda")
    ref_choice = torch.empty((3, p.out_h, p.out_w), dtype=torch.uint8, device="cuda")
    ctx.reconstruct(0, p, raws, out=ref, choice=ref_choice)
    ctx.check()
    out = torch.full((3, p.out_h, p.out_w), -1.0, device="cuda")
    choice = torch.empty((3, p.out_h, p.out_w), dtype=torch.uint8, device="cuda")
    keep = []
    descs = [hdr.sensor_desc(s, keep) for s in fr.sensors]
    stream = torch.cuda.current_stream().cuda_stream
    hdr.hdr_reconstruct_noalloc(0, descs, hp, ptrs, out.data_ptr(), choice.data_ptr(), stream)
    return ref.cpu().numpy(), ref_choice.cpu().numpy(), out.cpu().numpy(), choice.cpu().numpy()


def _within_tolerance(ref, ref_choice, out, choice):
    """Same level and a value within the parity tolerance (the tolerance's rounding-scale term is
    bounded here by the reference value's own magnitude, since both paths run identical FP32
    arithmetic)."""
    assert np.array_equal(choice, ref_choice)
    assert np.array_equal(np.isnan(out), np.isnan(ref))
    fin = np.isfinite(ref)
    tol = parity.REL_TOL * np.maximum(np.abs(ref[fin]), parity.TAU)
    assert np.all(np.abs(out[fin] - ref[fin]) <= tol)


def _printed_weight_rig():
    fr = _scalar_rig()
    return synth.Frame(fr.sensors, dataclasses.replace(fr.params, weight_mode=1), fr.scene)


def test_noalloc_matches_context_entry_point_twice():
    from paper_1308_4908_gb300 import hdr
    ctx = hdr.Context(0)
    try:
        for fr in (_frames_rig(), _scalar_rig(), _printed_weight_rig()):
            _within_tolerance(*_run_both(hdr, ctx, fr))
    finally:
        ctx.close()


def test_noalloc_rejects_frames_beyond_its_scratch():
    from paper_1308_4908_gb300 import hdr
    fr = synth.paper_scale(size=512, seed=1112)
    for s in fr.sensors:                      # 3 x 512^2 x 4 bytes x 2 frames > 4 MiB
        s.bias_frame = np.full((512, 512), s.black, np.float32)
        s.read_var_frame = np.full((512, 512), s.read_var, np.float32)
    keep = []
    descs = [hdr.sensor_desc(s, keep) for s in fr.sensors]
    raws = [torch.from_numpy(s.raw).cuda() for s in fr.sensors]
    out = torch.empty((3, 512, 512), device="cuda")
    with pytest.raises(hdr.HdrError) as ei:
        hdr.hdr_reconstruct_noalloc(0, descs, hdr.params_struct(fr.params), [int(t.data_ptr()) for t in raws],
                                    out.data_ptr())
    assert ei.value.status == hdr.HDR_E_UNSUPPORTED
    assert "scratch" in str(ei.value)


def test_noalloc_output_matches_the_oracle_and_allocates_nothing():
    """The entry point's own result against the FP64 oracle on sampled pixels (parity rule), and
    the device memory the driver reports free is the same before and after a call: a first call
    with the same configuration loads the kernels, the second may allocate nothing."""
    import oracle
    from paper_1308_4908_gb300 import hdr
    fr = _frames_rig()
    p = fr.params
    hp = hdr.params_struct(p)
    raws = [torch.from_numpy(s.raw).cuda() for s in fr.sensors]
    ptrs = [int(t.data_ptr()) for t in raws]
    keep = []
    descs = [hdr.sensor_desc(s, keep) for s in fr.sensors]
    out = torch.full((3, p.out_h, p.out_w), -1.0, device="cuda")
    choice = torch.empty((3, p.out_h, p.out_w), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    hdr.hdr_reconstruct_noalloc(0, descs, hp, ptrs, out.data_ptr(), choice.data_ptr(), stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    hdr.hdr_reconstruct_noalloc(0, descs, hp, ptrs, out.data_ptr(), choice.data_ptr(), stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    r = np.random.default_rng(12)
    pix = np.stack([r.integers(0, p.out_w, 400), r.integers(0, p.out_h, 400)], axis=1)
    o = oracle.reconstruct(fr.sensors, p, pix, levels=True)
    g, gc = out.cpu().numpy(), choice.cpu().numpy()
    parity.compare(g[:, pix[:, 1], pix[:, 0]], gc[:, pix[:, 1], pix[:, 0]], o, pix, len(p.sigmas), p.order,
                   p.ici_gamma, p.min_pivot)
