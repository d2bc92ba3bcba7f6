"""Adaptive windows (Sections 5.4-5.5) in the batched launch and in the serving loop.

A frame with adaptive parameters runs the gradient pass, the steering-matrix pass and the steered
fit, exactly as the one-call entry point hdr_reconstruct_adaptive runs them; in a batch and in a
served step it must give that entry point's result bit for bit (same kernels, same plans), alone
and next to isotropic frames, whichever steps its tiles land in. One frame is also checked against
the oracle with the GPU's steering matrices (the steered fit's parity rule of the adaptive tests).
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


def _frames():
    """Three small frames of the serving streams (orders 2, scales with the interval rule), one
    with a 1.5x output, and an order-1 batching frame."""
    fr = [synth.serving_stream_frame(m, 0, size_cap=128) for m in (0, 2, 7)]
    b = synth.batching(n_frames=1, size_cap=96, seed=2201)[0]
    return fr + [dataclasses.replace(b, params=dataclasses.replace(b.params, order=1))]


def _single(ctx, rig, fr, calpa):
    p = fr.params
    raws = [torch.from_numpy(s.raw).cuda() for s in fr.sensors]
    ch = torch.empty((3, p.out_h, p.out_w), dtype=torch.uint8, device="cuda")
    if calpa is None:
        out = ctx.reconstruct(rig, p, raws, choice=ch)
    else:
        out = ctx.reconstruct_adaptive(rig, p, calpa, raws, choice=ch)
    ctx.check()
    return out.cpu().numpy(), ch.cpu().numpy()


def test_batch_mixes_adaptive_and_isotropic_frames(ctx):
    from paper_1308_4908_gb300 import hdr
    frames = _frames()
    calpa = hdr.hdr_calpa_params_default()
    kinds = [calpa, None, calpa, calpa]
    keep, hf, outs, refs = [], [], [], []
    for k, (fr, cp) in enumerate(zip(frames, kinds)):
        ctx.set_rig(k, fr.sensors)
        refs.append(_single(ctx, k, fr, cp))
        p = fr.params
        raws = [torch.from_numpy(s.raw).cuda() for s in fr.sensors]
        keep.append(raws)
        out = torch.full((3, p.out_h, p.out_w), -7.0, device="cuda")
        ch = torch.empty((3, p.out_h, p.out_w), dtype=torch.uint8, device="cuda")
        outs.append((out, ch))
        hf.append(ctx.frame(k, p, raws, out, ch, keep, calpa=cp))
    for cfg in (hdr.hdr_batch_config(16, 0, 1, 0), hdr.hdr_batch_config(8, 0, 0, 0), hdr.hdr_batch_config(16, 0, 1, 1)):
        for o, _ in outs:
            o.fill_(-7.0)
        ctx.reconstruct_batch(hf, cfg)            # form 1 with adaptive frames runs as form 0
        ctx.check()
        for (o, ch), (ro, rc) in zip(outs, refs):
            np.testing.assert_array_equal(ch.cpu().numpy(), rc)
            np.testing.assert_array_equal(o.cpu().numpy(), ro)
    # the adaptive frame at 1.5x output against the oracle with the GPU's steering matrices
    fr = frames[2]
    p = fr.params
    raws = [torch.from_numpy(s.raw).cuda() for s in fr.sensors]
    q = ctx.calpa_metric(calpa, ctx.calpa_gradients(2, p, calpa, raws)).cpu().numpy().astype(np.float64)
    r = np.random.default_rng(5)
    pix = np.stack([r.integers(0, p.out_w, 300), r.integers(0, p.out_h, 300)], axis=1)
    o = oracle.reconstruct(fr.sensors, p, pix, levels=True, kappa=True, metric=q)
    g, gc = refs[2]
    parity.compare(g[:, pix[:, 1], pix[:, 0]], gc[:, pix[:, 1], pix[:, 0]], o, pix, len(p.sigmas), p.order,
                   p.ici_gamma, p.min_pivot)


def test_serving_adaptive_requests_alone_and_in_the_mix(ctx):
    """Adaptive and isotropic requests submitted together, in small steps so that every frame's
    tiles span several steps (the steering matrices outlive the step that computed them)."""
    from paper_1308_4908_gb300 import hdr
    frames = _frames()[:3]
    calpa = hdr.hdr_calpa_params_default(alpha=0.5)
    refs = []
    for k, fr in enumerate(frames):
        ctx.set_rig(10 + k, fr.sensors)
        refs.append((_single(ctx, 10 + k, fr, calpa), _single(ctx, 10 + k, fr, None)))
    for step_tiles in (0, 37):
        srv = hdr.Server(ctx, pool_bytes=256 << 20, step_tiles=step_tiles)
        try:
            bufs, tickets = [], []
            for k, fr in enumerate(frames):
                for cp in (calpa, None):
                    p = fr.params
                    raws = [np.ascontiguousarray(s.raw) for s in fr.sensors]
                    out = np.full((3, p.out_h, p.out_w), -7.0, np.float32)
                    ch = np.zeros((3, p.out_h, p.out_w), np.uint8)
                    bufs.append((out, ch))
                    tickets.append(srv.submit(10 + k, p, raws, out, ch, stream_id=k, calpa=cp))
            for t in tickets:
                assert srv.poll(t, -1).status == 0
        finally:
            srv.close()
        for k in range(len(frames)):
            for i in range(2):
                out, ch = bufs[2 * k + i]
                ro, rc = refs[k][i]
                np.testing.assert_array_equal(ch, rc)
                np.testing.assert_array_equal(out, ro)


def test_adaptive_requests_rejected_where_unsupported(ctx):
    from paper_1308_4908_gb300 import hdr
    fr = _frames()[0]
    ctx.set_rig(20, fr.sensors)
    raws = [np.ascontiguousarray(s.raw) for s in fr.sensors]
    p = fr.params
    out = np.zeros((3, p.out_h, p.out_w), np.float32)
    srv = hdr.Server(ctx, pool_bytes=64 << 20)
    try:
        with pytest.raises(hdr.HdrError) as e:
            srv.submit(20, p, raws, out, calpa=hdr.hdr_calpa_params_default(min_eig=-1.0))
        assert e.value.status == hdr.HDR_E_INVALID
        with pytest.raises(hdr.HdrError) as e:
            srv.submit(20, dataclasses.replace(p, weight_mode=1), raws, out, calpa=hdr.hdr_calpa_params_default())
        assert e.value.status == hdr.HDR_E_UNSUPPORTED
    finally:
        srv.close()
    srv8 = hdr.Server(ctx, pool_bytes=64 << 20, batch=hdr.hdr_batch_config(8, 0, 1, 0))
    try:
        with pytest.raises(hdr.HdrError) as e:
            srv8.submit(20, p, raws, out, calpa=hdr.hdr_calpa_params_default())
        assert e.value.status == hdr.HDR_E_UNSUPPORTED
    finally:
        srv8.close()
    keep = []
    t = torch.zeros((3, p.out_h, p.out_w), device="cuda")
    hf = [ctx.frame(20, p, [torch.from_numpy(s.raw).cuda() for s in fr.sensors], t, None, keep,
                    calpa=hdr.hdr_calpa_params_default(window_sigma=-1.0))]
    with pytest.raises(hdr.HdrError) as e:
        ctx.reconstruct_batch(hf)
    assert e.value.status == hdr.HDR_E_INVALID
