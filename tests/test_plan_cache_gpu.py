"""The host-side planning caches stay correct when what they cache changes.

A context caches whole single-frame plans (by rig generation, parameters and raw pointers),
encoded tensor maps and the device tables of tabulated window weights (Section 8). These tests
change a rig under the same id and raw buffers, force the weight-table cache to evict (a context
created with HDR_LPA_MAX_TABLES set keeps that many tables), and evict in the middle of a batch,
whose frames are all planned before its one launch: every result is checked against the oracle or
against the single-frame result that is checked against it elsewhere.
"""
import dataclasses
import os

import numpy as np
import pytest

import oracle
from paper_1308_4908_gb300 import synth
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ctx(max_tables=None):
    from paper_1308_4908_gb300 import hdr
    old = os.environ.get("HDR_LPA_MAX_TABLES")
    if max_tables is not None:
        os.environ["HDR_LPA_MAX_TABLES"] = str(max_tables)
    try:
        return hdr.Context(0)
    finally:
        if max_tables is not None:
            if old is None:
                del os.environ["HDR_LPA_MAX_TABLES"]
            else:
                os.environ["HDR_LPA_MAX_TABLES"] = old


def _translational(n, seed):
    """n small frames whose sensors are pure translations (distinct per frame), 1x output, orders
    0, 1, 2 in turn: each plans a tabulated weight table of its own."""
    frames = synth.batching(n_frames=n, size_cap=80, seed=seed)
    for k, fr in enumerate(frames):
        w, h = fr.sensors[0].width, fr.sensors[0].height
        for i, s in enumerate(fr.sensors):
            s.affine = np.asarray(synth.affine_about_center(w, h, 0.31 * i - 0.23 + 0.07 * k, 0.11 * k - 0.4 * i))
            s.raw = synth.simulate_raw(fr.scene, s, seed, 100 * k + i)
        frames[k] = dataclasses.replace(fr, params=dataclasses.replace(fr.params, out_w=w, out_h=h, order=k % 3,
                                                                        out_affine=synth.output_affine(w, h, w, h)))
    return frames


def _check(out, choice, fr, n_pix=300, seed=0):
    p = fr.params
    r = np.random.default_rng(seed)
    pix = np.stack([r.integers(0, p.out_w, n_pix), r.integers(0, p.out_h, n_pix)], axis=1)
    o = oracle.reconstruct(fr.sensors, p, pix, levels=True)
    parity.compare(out[:, pix[:, 1], pix[:, 0]], choice[:, pix[:, 1], pix[:, 0]], o, pix, len(p.sigmas), p.order,
                   p.ici_gamma, p.min_pivot)


def _run(ctx, rig, fr, raws):
    p = fr.params
    ch = torch.empty((3, p.out_h, p.out_w), dtype=torch.uint8, device="cuda")
    out = ctx.reconstruct(rig, p, raws, choice=ch)
    ctx.check()
    return out.cpu().numpy(), ch.cpu().numpy()


def test_plan_cache_follows_rig_changes():
    """Same rig id, same raw buffers, same parameters: replacing the rig's transforms or adding
    per-pixel calibration frames must not reuse the cached plan of the old rig."""
    ctx = _ctx()
    try:
        fr = synth.paper_scale(size=64, seed=311)
        p = dataclasses.replace(fr.params, order=1)
        fr = dataclasses.replace(fr, params=p)
        raws = [torch.from_numpy(s.raw).cuda() for s in fr.sensors]
        ctx.set_rig(3, fr.sensors)
        _check(*_run(ctx, 3, fr, raws), fr, seed=1)
        # another misalignment of the same sensors (the raw values stay; only the rig changes)
        moved = [dataclasses.replace(s) for s in fr.sensors]
        for i, s in enumerate(moved):
            s.affine = np.asarray(synth.affine_about_center(64, 64, 0.7 - 0.5 * i, -0.6 + 0.3 * i, 0.15 * i))
        fr2 = dataclasses.replace(fr, sensors=moved)
        ctx.set_rig(3, moved)
        _check(*_run(ctx, 3, fr2, raws), fr2, seed=2)
        # per-pixel frames on the same rig id
        r = np.random.default_rng(5)
        cal = [dataclasses.replace(s) for s in moved]
        for s in cal:
            s.bias_frame = 64.0 + r.normal(0.0, 2.0, (s.height, s.width))
            s.prnu_frame = 1.0 + r.normal(0.0, 0.02, (s.height, s.width))
        fr3 = dataclasses.replace(fr, sensors=cal)
        ctx.set_rig(3, cal)
        _check(*_run(ctx, 3, fr3, raws), fr3, seed=3)
    finally:
        ctx.close()


def test_reconstruct_after_table_eviction():
    """A context that keeps one weight table: frame A, then frame B (evicts A's table), then A
    again with the same buffers and parameters (its cached plan pointed at the freed table)."""
    ctx = _ctx(max_tables=1)
    try:
        fa, fb = _translational(2, seed=4101)
        ra = [torch.from_numpy(s.raw).cuda() for s in fa.sensors]
        rb = [torch.from_numpy(s.raw).cuda() for s in fb.sensors]
        ctx.set_rig(0, fa.sensors)
        ctx.set_rig(1, fb.sensors)
        first = _run(ctx, 0, fa, ra)
        _check(*first, fa, seed=4)
        _check(*_run(ctx, 1, fb, rb), fb, seed=5)
        again = _run(ctx, 0, fa, ra)
        np.testing.assert_array_equal(again[0], first[0])
        np.testing.assert_array_equal(again[1], first[1])
    finally:
        ctx.close()


def test_batch_survives_table_eviction():
    """Six translational frames, each with its own weight table, in one batch of a context that
    keeps two tables: the cache evicts twice while the batch is planned, before its launch. The
    tables the earlier plans hold must stay allocated until the launch: every frame equals its
    single-frame result, and one is checked against the oracle."""
    from paper_1308_4908_gb300 import hdr
    frames = _translational(6, seed=4202)
    ref_ctx = _ctx()
    ctx = _ctx(max_tables=2)
    try:
        items = []
        refs = []
        for k, fr in enumerate(frames):
            raws = [torch.from_numpy(s.raw).cuda() for s in fr.sensors]
            ref_ctx.set_rig(k, fr.sensors)
            refs.append(_run(ref_ctx, k, fr, raws))
            ctx.set_rig(k, fr.sensors)
            p = fr.params
            out = torch.full((3, p.out_h, p.out_w), -7.0, device="cuda")
            ch = torch.empty((3, p.out_h, p.out_w), dtype=torch.uint8, device="cuda")
            items.append((k, fr, raws, out, ch))
        for rep in range(2):
            keep = []
            hf = [ctx.frame(rig, fr.params, raws, out, ch, keep) for rig, fr, raws, out, ch in items]
            ctx.reconstruct_batch(hf, hdr.hdr_batch_config(16, 0, 1, 0))
            ctx.check()
            for (_, fr, _, out, ch), (ro, rc) in zip(items, refs):
                np.testing.assert_array_equal(ch.cpu().numpy(), rc)
                np.testing.assert_array_equal(out.cpu().numpy(), ro)
        _check(refs[3][0], refs[3][1], frames[3], seed=6)
    finally:
        ctx.close()
        ref_ctx.close()
