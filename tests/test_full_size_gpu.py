"""Parity at the full sizes of the batching and serving workloads, in the launch configurations
the benchmark times.

* Batching: the 16 uneven frames (raw 512^2 to 2048^2, 2-4 sensors, orders 0-2, 1x and 1.5x
  outputs) in one launch of the graph of per-frame grids with 16-row tiles, the configuration the
  tuner picks for this batch.
* Serving: one frame of each of the 8 streams (up to a 2048^2 rig upsampled to 3840x2160),
  submitted together to a server with the benchmark's settings (8192-tile steps, 48 slots).

Each frame is checked against the oracle on random pixels plus its four corners (the tolerance
and the admissible-level rule of tests/parity.py).
"""
import numpy as np
import pytest

import oracle
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def frames():
    import bench
    from paper_1308_4908_gb300 import synth
    jobs = [("batch", s) for s in synth.batching_specs()] + [("serve", m) for m in range(len(synth.SERVING_STREAMS))]
    made = bench.make_frames(jobs)
    n = len(synth.batching_specs())
    return made[:n], made[n:]


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_4908_gb300 import hdr
    c = hdr.Context(0)
    yield c
    c.close()


def _pixels(p, n, seed):
    r = np.random.default_rng(seed)
    pix = np.stack([r.integers(0, p.out_w, n), r.integers(0, p.out_h, n)], axis=1)
    corners = np.array([[0, 0], [p.out_w - 1, 0], [0, p.out_h - 1], [p.out_w - 1, p.out_h - 1]])
    return np.concatenate([pix, corners])


def _check(fr, out, ch, seed, n=120):
    p = fr.params
    pix = _pixels(p, n, seed)
    o = oracle.reconstruct(fr.sensors, p, pix, levels=True, kappa=True)
    return parity.compare(out[:, pix[:, 1], pix[:, 0]], ch[:, pix[:, 1], pix[:, 0]], o, pix, len(p.sigmas), p.order,
                          p.ici_gamma, p.min_pivot)


def test_batching_workload_full_size(ctx, frames):
    from paper_1308_4908_gb300 import hdr
    batch, _ = frames
    keep, hf, bufs = [], [], []
    for k, fr in enumerate(batch):
        ctx.set_rig(k, fr.sensors)
        p = fr.params
        raws = [torch.from_numpy(s.raw).cuda() for s in fr.sensors]
        out = torch.full((3, p.out_h, p.out_w), -7.0, device="cuda")
        ch = torch.empty((3, p.out_h, p.out_w), dtype=torch.uint8, device="cuda")
        hf.append(ctx.frame(k, p, raws, out, ch, keep))
        keep.append(raws)
        bufs.append((out, ch))
    ctx.reconstruct_batch(hf, hdr.hdr_batch_config(16, 0, 1, 0))
    ctx.check()
    assert len({fr.params.order for fr in batch}) == 3
    for k, (fr, (out, ch)) in enumerate(zip(batch, bufs)):
        _check(fr, out.cpu().numpy(), ch.cpu().numpy(), seed=500 + k)


def test_serving_mix_full_size(ctx, frames):
    from paper_1308_4908_gb300 import hdr
    _, streams = frames
    for m, fr in enumerate(streams):
        ctx.set_rig(32 + m, fr.sensors)
    srv = hdr.Server(ctx, max_frames=48, pool_bytes=6 << 30, step_tiles=8192)
    try:
        bufs, tickets = [], []
        for m, fr in enumerate(streams):
            p = fr.params
            out = np.full((3, p.out_h, p.out_w), -7.0, np.float32)
            ch = np.zeros((3, p.out_h, p.out_w), np.uint8)
            bufs.append((out, ch))
            tickets.append(srv.submit(32 + m, p, [np.ascontiguousarray(s.raw) for s in fr.sensors], out, ch,
                                      stream_id=m))
        res = [srv.poll(t, -1) for t in tickets]
    finally:
        srv.close()
    assert all(r.status == 0 for r in res)
    assert max(r.steps for r in res) > 1          # the 3840x2160 frame spans several steps
    for m, (fr, (out, ch)) in enumerate(zip(streams, bufs)):
        _check(fr, out, ch, seed=700 + m)
