"""Batched reconstruction: many uneven frames in one graph-recorded launch.

Form 0 (one grid per frame) runs each frame's single-frame kernel, so its results must equal the
single-frame reconstruction bit for bit, for every launch configuration the autotuner may pick.
Form 1 (persistent kernels over a tile list) walks the window once per scale where the
single-frame kernel feeds several scales from one walk, so its sums round differently: its
frames must equal the oracle within the parity tolerance. One frame of each batch is also checked
against the oracle.
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


def _prepare(ctx, frames, base_rig=0):
    """Rigs, device raws and output buffers for a list of synth frames."""
    items = []
    for k, fr in enumerate(frames):
        ctx.set_rig(base_rig + k, fr.sensors)
        raws = [torch.from_numpy(s.raw).cuda() for s in fr.sensors]
        p = fr.params
        out = torch.full((3, p.out_h, p.out_w), -7.0, device="cuda")
        ch = torch.empty((3, p.out_h, p.out_w), dtype=torch.uint8, device="cuda")
        items.append((base_rig + k, fr, raws, out, ch))
    return items


def _single(ctx, items):
    refs = []
    for rig, fr, raws, _, _ in items:
        ch = torch.empty((3, fr.params.out_h, fr.params.out_w), dtype=torch.uint8, device="cuda")
        out = ctx.reconstruct(rig, fr.params, raws, choice=ch)
        refs.append((out.cpu().numpy(), ch.cpu().numpy()))
    ctx.check()
    return refs


def _batch(ctx, items, cfg=None):
    keep = []
    hf = [ctx.frame(rig, fr.params, raws, out, ch, keep) for rig, fr, raws, out, ch in items]
    ctx.reconstruct_batch(hf, cfg)
    ctx.check()
    return [(out.cpu().numpy(), ch.cpu().numpy()) for _, _, _, out, ch in items]


def _same(a, b):
    for (oa, ca), (ob, cb) in zip(a, b):
        np.testing.assert_array_equal(ca, cb)
        np.testing.assert_array_equal(oa, ob)


def _against_oracle(items, got, n_pix=200):
    for (rig, fr, _, _, _), (out, ch) in zip(items, got):
        p = fr.params
        if p.out_w * p.out_h == 0:
            assert out.size == 0
            continue
        r = np.random.default_rng(rig)
        pix = np.stack([r.integers(0, p.out_w, n_pix), r.integers(0, p.out_h, n_pix)], axis=1)
        o = oracle.reconstruct(fr.sensors, p, pix, levels=True, kappa=True)
        parity.compare(out[:, pix[:, 1], pix[:, 0]], ch[:, pix[:, 1], pix[:, 0]], o, pix, len(p.sigmas), p.order,
                       p.ici_gamma, p.min_pivot)


def _check(items, got, refs, form):
    """Form 0: bit for bit the single-frame results; form 1: the oracle within tolerance."""
    if form == 0:
        _same(got, refs)
    else:
        _against_oracle(items, got)


def test_batch_equals_single_frames_for_every_configuration(ctx):
    """Uneven frames (sizes, sensor counts 2-4, orders 0-2, 1x and 1.5x outputs) in one launch."""
    from paper_1308_4908_gb300 import hdr
    frames = synth.batching(n_frames=8, size_cap=160)
    items = _prepare(ctx, frames)
    refs = _single(ctx, items)
    cfgs = [hdr.hdr_batch_config(th, per_sm, order, 1) for th in (16, 8) for per_sm in (0, 1) for order in (1, 0)]
    cfgs += [hdr.hdr_batch_config(th, 0, order, 0) for th in (16, 8) for order in (1, 0)]
    cfgs += [hdr.hdr_batch_config(16, 0, order, 0, 2) for order in (1, 0)]   # two pixels per thread
    cfgs += [hdr.hdr_batch_config(th, 0, 1, 0, 1, 2) for th in (16, 8)]      # two staging buffers
    for cfg in cfgs:
        for _, _, _, out, _ in items:
            out.fill_(-7.0)
        _check(items, _batch(ctx, items, cfg), refs, cfg.form)


@pytest.mark.parametrize("form", [0, 1])
def test_batch_replays_with_new_contents(ctx, form):
    """The recorded graph is replayed with fresh tables or node parameters: a second batch of the
    same shapes but other frames (other rigs and raws) gives those frames' results."""
    from paper_1308_4908_gb300 import hdr
    a = synth.batching(n_frames=4, size_cap=96, seed=2001)
    b = synth.batching(n_frames=4, size_cap=96, seed=2002)
    ia = _prepare(ctx, a, base_rig=10)
    ib = _prepare(ctx, b, base_rig=20)
    ra, rb = _single(ctx, ia), _single(ctx, ib)
    cfg = hdr.hdr_batch_config(16, 0, 1, form)
    _check(ia, _batch(ctx, ia, cfg), ra, form)
    _check(ib, _batch(ctx, ib, cfg), rb, form)
    _check(ia, _batch(ctx, ia, cfg), ra, form)


def test_tuner_picks_a_configuration_and_batch_uses_it(ctx):
    frames = synth.batching(n_frames=6, size_cap=128, seed=2003)
    items = _prepare(ctx, frames, base_rig=30)
    refs = _single(ctx, items)
    keep = []
    hf = [ctx.frame(rig, fr.params, raws, out, ch, keep) for rig, fr, raws, out, ch in items]
    best = ctx.tune_batch(hf)
    assert best.tile_h in (8, 16) and 0 <= best.ctas_per_sm <= 8 and best.cost_order in (0, 1) and best.form in (0, 1)
    assert best.px_per_thread in (1, 2) and best.stages in (1, 2)
    _check(items, _batch(ctx, items), refs, best.form)        # cfg None -> the tuned configuration


def test_batch_frame_against_oracle(ctx):
    frames = synth.batching(n_frames=3, size_cap=72, seed=2004)
    items = _prepare(ctx, frames, base_rig=40)
    got = _batch(ctx, items)
    for (rig, fr, _, _, _), (out, ch) in zip(items, got):
        p = fr.params
        r = np.random.default_rng(rig)
        pix = np.stack([r.integers(0, p.out_w, 300), r.integers(0, p.out_h, 300)], axis=1)
        o = oracle.reconstruct(fr.sensors, p, pix, levels=True, kappa=True)
        parity.compare(out[:, pix[:, 1], pix[:, 0]], ch[:, pix[:, 1], pix[:, 0]], o, pix, len(p.sigmas), p.order,
                       p.ici_gamma, p.min_pivot)


def test_batch_rejects_bad_input(ctx):
    from paper_1308_4908_gb300 import hdr
    frames = synth.batching(n_frames=2, size_cap=64, seed=2005)
    items = _prepare(ctx, frames, base_rig=50)
    keep = []
    hf = [ctx.frame(rig, fr.params, raws, out, ch, keep) for rig, fr, raws, out, ch in items]
    hf[1].rig_id = 63                      # undefined rig
    with pytest.raises(hdr.HdrError):
        ctx.reconstruct_batch(hf)
    with pytest.raises(hdr.HdrError):
        ctx.reconstruct_batch(hf[:0])
    with pytest.raises(hdr.HdrError):
        ctx.reconstruct_batch(hf[:1], hdr.hdr_batch_config(12, 0, 1, 0))
    with pytest.raises(hdr.HdrError):
        ctx.reconstruct_batch(hf[:1], hdr.hdr_batch_config(16, 0, 1, 2))
    with pytest.raises(hdr.HdrError):
        ctx.reconstruct_batch(hf[:1], hdr.hdr_batch_config(8, 0, 1, 0, 2))    # two pixels per thread: 16 rows
    with pytest.raises(hdr.HdrError):
        ctx.reconstruct_batch(hf[:1], hdr.hdr_batch_config(16, 0, 1, 1, 2))   # and form 0 only
    for bad in (hdr.hdr_batch_config(16, 0, 1, 0, 1, 3), hdr.hdr_batch_config(16, 0, 1, 0, 1, -1),
                hdr.hdr_batch_config(16, 0, 1, 1, 1, 2),                     # two staging buffers: form 0
                hdr.hdr_batch_config(16, 0, 1, 0, 2, 2)):                    # and one pixel per thread
        with pytest.raises(hdr.HdrError):
            ctx.reconstruct_batch(hf[:1], bad)


@pytest.mark.parametrize("stages", [1, 2])
def test_staging_depth_spans_and_ranges(ctx, stages):
    """Two staging buffers: each CTA takes four tiles strided over the launch's tile range and
    copies the next tile while it computes the current one. Frames of 1 to 16 tiles (fewer tiles
    than a CTA takes, ragged last CTA), tile heights 16 and 8, and served steps of 7 tiles (tile
    sub-ranges of frames): every result bit-identical to the single-frame kernel."""
    import dataclasses
    from paper_1308_4908_gb300 import hdr
    frames = synth.batching(n_frames=5, size_cap=64, seed=2010)
    sizes = [(16, 16), (20, 9), (48, 17), (33, 40), (64, 64)]
    # the frames' own output mappings, cropped to these sizes
    frames = [dataclasses.replace(fr, params=dataclasses.replace(fr.params, out_w=w, out_h=h))
              for fr, (w, h) in zip(frames, sizes)]
    items = _prepare(ctx, frames, base_rig=0)
    refs = _single(ctx, items)
    for th in (16, 8):
        _same(_batch(ctx, items, hdr.hdr_batch_config(th, 0, 1, 0, 1, stages)), refs)
    srv = hdr.Server(ctx, pool_bytes=64 << 20, step_tiles=7, batch=hdr.hdr_batch_config(16, 0, 1, 0, 1, stages))
    try:
        bufs, tickets = [], []
        for rig, fr, _, _, _ in items:
            p = fr.params
            out = np.full((3, p.out_h, p.out_w), -7.0, np.float32)
            ch = np.zeros((3, p.out_h, p.out_w), np.uint8)
            bufs.append((out, ch))
            tickets.append(srv.submit(rig, p, [np.ascontiguousarray(s.raw) for s in fr.sensors], out, ch))
        for t in tickets:
            assert srv.poll(t, -1).status == 0
    finally:
        srv.close()
    for (out, ch), (ro, rc) in zip(bufs, refs):
        np.testing.assert_array_equal(ch, rc)
        np.testing.assert_array_equal(out, ro)


@pytest.mark.parametrize("form", [0, 1])
def test_batch_with_empty_and_one_pixel_frames(ctx, form):
    import dataclasses
    from paper_1308_4908_gb300 import hdr
    frames = synth.batching(n_frames=3, size_cap=64, seed=2006)
    frames[0] = dataclasses.replace(frames[0], params=dataclasses.replace(frames[0].params, out_w=0, out_h=0))
    frames[1] = dataclasses.replace(frames[1], params=dataclasses.replace(frames[1].params, out_w=1, out_h=1))
    items = _prepare(ctx, frames, base_rig=56)
    refs = _single(ctx, items)
    _check(items, _batch(ctx, items, hdr.hdr_batch_config(16, 0, 1, form)), refs, form)


@pytest.mark.parametrize("form,stages,px", [(0, 1, 1), (0, 2, 1), (0, 1, 2), (1, 1, 1)])
def test_batch_with_translational_frames(ctx, form, stages, px):
    """Frames whose rigs are pure translations use tabulated weights in form 0 (one or two staging
    buffers, one or two pixels per thread) and the searched window in the persistent form: each
    equals its single-frame result within the parity tolerance and is bit-identical to it in
    form 0."""
    import dataclasses
    from paper_1308_4908_gb300 import hdr
    frames = synth.batching(n_frames=3, size_cap=96, seed=2007)
    for k, fr in enumerate(frames):
        w, h = fr.sensors[0].width, fr.sensors[0].height
        for i, s in enumerate(fr.sensors):
            s.affine = np.asarray(synth.affine_about_center(w, h, 0.3 * i - 0.2, 0.1 * k))
            s.raw = synth.simulate_raw(fr.scene, s, 2007, 100 * k + i)
        frames[k] = dataclasses.replace(fr, params=dataclasses.replace(fr.params, out_w=w, out_h=h,
                                                                        out_affine=synth.output_affine(w, h, w, h)))
    items = _prepare(ctx, frames, base_rig=60 - 3)
    refs = _single(ctx, items)
    got = _batch(ctx, items, hdr.hdr_batch_config(16, 0, 1, form, px, stages))
    if form == 0:
        _same(got, refs)
    else:
        for (rig, fr, _, _, _), (out, ch) in zip(items, got):
            p = fr.params
            r = np.random.default_rng(rig)
            pix = np.stack([r.integers(0, p.out_w, 200), r.integers(0, p.out_h, 200)], axis=1)
            o = oracle.reconstruct(fr.sensors, p, pix, levels=True, kappa=True)
            parity.compare(out[:, pix[:, 1], pix[:, 0]], ch[:, pix[:, 1], pix[:, 0]], o, pix, len(p.sigmas), p.order,
                           p.ici_gamma, p.min_pivot)
