"""Failure detection without a GPU fault: the bounded-wait self-test makes a wait run out (an
mbarrier expecting bytes that no copy delivers) and sets the device status a reconstruction whose
staging never lands would set. Every path must report HDR_E_TIMEOUT through the host API, write
nothing after the failure, and leave the context usable.
"""
import numpy as np
import pytest

from paper_1308_4908_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_4908_gb300 import hdr
    c = hdr.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def frame(ctx):
    fr = synth.paper_scale(size=64, seed=3001)
    ctx.set_rig(0, fr.sensors)
    raws = [torch.from_numpy(s.raw).cuda() for s in fr.sensors]
    ref = ctx.reconstruct(0, fr.params, raws).cpu().numpy()
    ctx.check()
    return fr, raws, ref


def test_timeout_is_reported_once_and_the_context_recovers(ctx, frame):
    from paper_1308_4908_gb300 import hdr
    fr, raws, ref = frame
    ctx.selftest_timeout()
    with pytest.raises(hdr.HdrError) as e:
        ctx.check()
    assert e.value.status == hdr.HDR_E_TIMEOUT
    ctx.check()                                        # the status was cleared
    out = ctx.reconstruct(0, fr.params, raws)
    ctx.check()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)


def test_launches_after_a_timeout_retire_without_writing(ctx, frame):
    from paper_1308_4908_gb300 import hdr
    fr, raws, ref = frame
    p = fr.params
    ctx.selftest_timeout()
    out = torch.full((3, p.out_h, p.out_w), -7.0, device="cuda")
    ctx.reconstruct(0, p, raws, out=out)
    with pytest.raises(hdr.HdrError) as e:
        ctx.check()
    assert e.value.status == hdr.HDR_E_TIMEOUT
    assert bool((out == -7.0).all())
    ctx.reconstruct(0, p, raws, out=out)
    ctx.check()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("form", [0, 1])
def test_batched_launch_after_a_timeout(ctx, frame, form):
    from paper_1308_4908_gb300 import hdr
    fr, raws, ref = frame
    p = fr.params
    outs = [torch.full((3, p.out_h, p.out_w), -7.0, device="cuda") for _ in range(3)]
    keep = []
    hf = [ctx.frame(0, p, raws, o, None, keep) for o in outs]
    cfg = hdr.hdr_batch_config(16, 0, 1, form)
    # the form's own result first (form 0 equals the single-frame result bit for bit; the
    # persistent form 1 walks once per scale and rounds its sums differently)
    ctx.reconstruct_batch(hf, cfg)
    ctx.check()
    want = [o.cpu().numpy() for o in outs]
    if form == 0:
        for w in want:
            np.testing.assert_array_equal(w, ref)
    for o in outs:
        o.fill_(-7.0)
    ctx.selftest_timeout()
    ctx.reconstruct_batch(hf, cfg)
    with pytest.raises(hdr.HdrError) as e:
        ctx.check()
    assert e.value.status == hdr.HDR_E_TIMEOUT
    assert all(bool((o == -7.0).all()) for o in outs)
    ctx.reconstruct_batch(hf, cfg)
    ctx.check()
    for o, w in zip(outs, want):
        np.testing.assert_array_equal(o.cpu().numpy(), w)


def test_serving_fails_the_requests_on_the_device_and_recovers(ctx, frame):
    from paper_1308_4908_gb300 import hdr
    fr, raws, ref = frame
    p = fr.params
    host_raws = [np.ascontiguousarray(s.raw) for s in fr.sensors]
    ctx.selftest_timeout()
    torch.cuda.synchronize()                           # the status word is set before serving starts
    srv = hdr.Server(ctx, pool_bytes=64 << 20)
    try:
        bad = np.zeros((3, p.out_h, p.out_w), np.float32)
        t = srv.submit(0, p, host_raws, bad)
        with pytest.raises(hdr.HdrError) as e:
            srv.poll(t, -1)
        assert e.value.status == hdr.HDR_E_TIMEOUT
        good = np.zeros((3, p.out_h, p.out_w), np.float32)
        t = srv.submit(0, p, host_raws, good)
        r = srv.poll(t, -1)
        assert r.status == 0
        np.testing.assert_array_equal(good, ref)
        st = srv.stats()
        assert st.completed == 1 and st.submitted == 2
    finally:
        srv.close()
