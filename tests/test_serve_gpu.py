"""Serving loop: continuous batching of frames from several streams through hdr_server_*.

A frame's result must be the same alone and in the mix (every pixel is computed by the same
per-pixel arithmetic, whatever shares its step), equal to the plain per-frame launch, and within
the oracle's tolerance on sampled pixels. Admission by memory, tile budgets, polling and invalid
requests are covered too.
"""
import numpy as np
import pytest

import oracle
from paper_1308_4908_gb300 import synth
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CAP = 192                         # raw size cap: every stream shape, a few hundred tiles per frame


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_4908_gb300 import hdr
    c = hdr.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def streams(ctx):
    """Two frames of each of the 8 serving streams (rig id = stream id)."""
    out = {}
    for m in range(len(synth.SERVING_STREAMS)):
        frames = [synth.serving_stream_frame(m, k, size_cap=CAP) for k in range(2)]
        ctx.set_rig(m, frames[0].sensors)
        out[m] = frames
    return out


def _host(fr):
    p = fr.params
    raws = [np.ascontiguousarray(s.raw) for s in fr.sensors]
    return raws, np.full((3, p.out_h, p.out_w), -7.0, np.float32), np.zeros((3, p.out_h, p.out_w), np.uint8)


def _plain(ctx, rig, fr):
    p = fr.params
    ch = torch.empty((3, p.out_h, p.out_w), dtype=torch.uint8, device="cuda")
    out = ctx.reconstruct(rig, p, [torch.from_numpy(s.raw).cuda() for s in fr.sensors], choice=ch)
    ctx.check()
    return out.cpu().numpy(), ch.cpu().numpy()


def _serve(ctx, items, **kw):
    """Submit (rig, frame) items all at once; returns [(out, choice, result)] in item order."""
    from paper_1308_4908_gb300 import hdr
    srv = hdr.Server(ctx, **kw)
    try:
        bufs, tickets = [], []
        for rig, fr in items:
            raws, out, ch = _host(fr)
            tickets.append(srv.submit(rig, fr.params, raws, out, ch, stream_id=rig))
            bufs.append((out, ch))
        res = [srv.poll(t, -1) for t in tickets]
        stats = srv.stats()
    finally:
        srv.close()
    assert stats.completed == len(items) and stats.submitted == len(items)
    return [(o, c, r) for (o, c), r in zip(bufs, res)], stats


def test_alone_and_in_the_mix_are_identical(ctx, streams):
    items = [(m, streams[m][k]) for k in range(2) for m in streams]
    probe = (5, streams[5][1])
    alone, _ = _serve(ctx, [probe])
    mixed, stats = _serve(ctx, items, step_tiles=96)
    plain = _plain(ctx, *probe)
    i = next(k for k, it in enumerate(items) if it[0] == probe[0] and it[1] is probe[1])
    np.testing.assert_array_equal(alone[0][0], mixed[i][0])
    np.testing.assert_array_equal(alone[0][1], mixed[i][1])
    np.testing.assert_array_equal(alone[0][0], plain[0])
    np.testing.assert_array_equal(alone[0][1], plain[1])
    assert stats.steps > 1 and max(r.steps for _, _, r in mixed) > 1
    for (rig, fr), (out, ch, r) in zip(items, mixed):
        assert r.status == 0 and r.total_ms >= r.queue_ms >= 0
        ref = _plain(ctx, rig, fr)
        np.testing.assert_array_equal(out, ref[0])
        np.testing.assert_array_equal(ch, ref[1])


@pytest.mark.parametrize("step_tiles", [96, 0])
def test_least_remaining_work_order(ctx, streams, step_tiles):
    """order 1 (the least remaining work first) changes which tiles share a step, not what a pixel
    computes: every frame of a mix equals its plain reconstruction."""
    items = [(m, streams[m][k]) for k in range(2) for m in streams]
    mixed, stats = _serve(ctx, items, step_tiles=step_tiles, order=1)
    for (rig, fr), (out, ch, r) in zip(items, mixed):
        assert r.status == 0
        ref = _plain(ctx, rig, fr)
        np.testing.assert_array_equal(out, ref[0])
        np.testing.assert_array_equal(ch, ref[1])


def test_served_frame_against_oracle(ctx, streams):
    fr = streams[7][0]                     # the upsampled stream
    (out, ch, _), = _serve(ctx, [(7, fr)])[0]
    p = fr.params
    r = np.random.default_rng(77)
    pix = np.stack([r.integers(0, p.out_w, 400), r.integers(0, p.out_h, 400)], axis=1)
    o = oracle.reconstruct(fr.sensors, p, pix, levels=True, kappa=True)
    parity.compare(out[:, pix[:, 1], pix[:, 0]], ch[:, pix[:, 1], pix[:, 0]], o, pix, len(p.sigmas), p.order,
                   p.ici_gamma, p.min_pivot)


def test_admission_by_memory(ctx, streams):
    """A pool that holds about one frame at a time still serves every request, in order."""
    items = [(m, streams[m][0]) for m in (5, 6, 2, 0, 7)]
    biggest = 0
    for _, fr in items:
        p = fr.params
        need = sum(s.raw.nbytes for s in fr.sensors) + p.out_w * p.out_h * 3 * 5 + 4096
        if p.out_w * p.out_h >= 152 * 256:     # converted ahead: four colour-phase planes of float2
            need += sum(4 * ((s.height + 1) // 2) * ((((s.width + 1) // 2) + 1) & ~1) * 8 + 256 for s in fr.sensors)
        biggest = max(biggest, need)
    res, stats = _serve(ctx, items, max_frames=8, pool_bytes=int(biggest * 1.2))
    for (rig, fr), (out, ch, r) in zip(items, res):
        ref = _plain(ctx, rig, fr)
        np.testing.assert_array_equal(out, ref[0])
    # one slot: each frame is admitted only after the previous one completed (the submissions
    # themselves are microseconds apart)
    res, _ = _serve(ctx, items, max_frames=1)
    for (rig, fr), (out, ch, r) in zip(items, res):
        np.testing.assert_array_equal(out, _plain(ctx, rig, fr)[0])
    for prev, cur in zip(res, res[1:]):
        assert cur[2].queue_ms >= prev[2].total_ms - 5.0


def test_poll_and_rejections(ctx, streams):
    from paper_1308_4908_gb300 import hdr
    fr = streams[6][0]
    raws, out, ch = _host(fr)
    srv = hdr.Server(ctx, pool_bytes=64 << 20)
    try:
        t = srv.submit(6, fr.params, raws, out, ch)
        r = srv.poll(t, -1)
        assert r is not None and r.status == 0
        with pytest.raises(hdr.HdrError):          # a result is returned once
            srv.poll(t, 0)
        with pytest.raises(hdr.HdrError):          # undefined rig
            srv.submit(60, fr.params, raws, out, ch)
        bad = hdr.params_struct(fr.params)
        bad.order = 3
        with pytest.raises(hdr.HdrError):
            srv.submit(6, bad, raws, out, ch)
    finally:
        srv.close()
    for order in (-1, 2):
        with pytest.raises(hdr.HdrError) as e:
            hdr.Server(ctx, pool_bytes=64 << 20, order=order)
        assert e.value.status == hdr.HDR_E_INVALID
    small = hdr.Server(ctx, pool_bytes=1 << 16)
    try:
        with pytest.raises(hdr.HdrError) as e:
            small.submit(6, fr.params, raws, out, ch)
        assert e.value.status == hdr.HDR_E_UNSUPPORTED
    finally:
        small.close()


def test_busy_until_done_and_fp16_output(ctx, streams):
    from paper_1308_4908_gb300 import hdr
    big = synth.serving_stream_frame(5, 0)         # full-size 2048^2 3-sensor frame
    ctx.set_rig(20, big.sensors)
    hp = hdr.params_struct(big.params)
    hp.out_dtype = 1
    raws = [np.ascontiguousarray(s.raw) for s in big.sensors]
    out = np.zeros((3, hp.out_h, hp.out_w), np.float16)
    srv = hdr.Server(ctx)
    try:
        t = srv.submit(20, hp, raws, out)
        assert srv.poll(t, 0) is None               # a 4-Mpixel frame takes milliseconds
        r = srv.poll(t, -1)
        assert r.status == 0 and r.steps == 1
    finally:
        srv.close()
    ref = torch.empty((3, hp.out_h, hp.out_w), dtype=torch.float16, device="cuda")
    ctx.reconstruct(20, hp, [torch.from_numpy(s.raw).cuda() for s in big.sensors], out=ref)
    ctx.check()
    np.testing.assert_array_equal(out, ref.cpu().numpy())


def test_empty_and_tiny_outputs(ctx, streams):
    """A 0x0 output completes without a step; a 1x1 output is one ragged tile."""
    import dataclasses
    from paper_1308_4908_gb300 import hdr
    fr = streams[0][0]
    raws = [np.ascontiguousarray(s.raw) for s in fr.sensors]
    srv = hdr.Server(ctx, pool_bytes=64 << 20)
    try:
        p0 = dataclasses.replace(fr.params, out_w=0, out_h=0)
        t0 = srv.submit(0, p0, raws, np.zeros((3, 0, 0), np.float32))
        p1 = dataclasses.replace(fr.params, out_w=1, out_h=1)
        one = np.full((3, 1, 1), -7.0, np.float32)
        t1 = srv.submit(0, p1, raws, one)
        assert srv.poll(t0, -1).steps == 0
        assert srv.poll(t1, -1).steps == 1
    finally:
        srv.close()
    ref = _plain(ctx, 0, dataclasses.replace(fr, params=p1))
    np.testing.assert_array_equal(one, ref[0])


def test_translational_frames_use_their_tables_in_the_mix(ctx, streams):
    """Frames whose rigs are pure translations at 1x output read tabulated weights (Section 8) in
    the serving steps as in a plain launch: served alone, in a mix with other streams, and by
    hdr_reconstruct, the same bits."""
    from tests.test_parity_gpu import translational
    tr = [translational(80, 1090 + k, [(0.0, 0.0), (0.4 * k, -0.3), (-1.2, 0.7 * k)]) for k in range(2)]
    for k, fr in enumerate(tr):
        ctx.set_rig(40 + k, fr.sensors)
    items = [(40 + k, fr) for k, fr in enumerate(tr)] + [(m, streams[m][0]) for m in (0, 3)]
    mixed, _ = _serve(ctx, items, step_tiles=64)
    for (rig, fr), (out, ch, r) in zip(items, mixed):
        ref = _plain(ctx, rig, fr)
        np.testing.assert_array_equal(out, ref[0])
        np.testing.assert_array_equal(ch, ref[1])
