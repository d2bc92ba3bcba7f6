"""Adaptive windows (CALPA, Sections 5.4-5.5) on the GPU, pass by pass against the oracle.

Each pass is compared on the GPU's own input to it, so that a difference points at that pass:
pass 1 (gradients of the order-1 green fit) against the oracle's gradients; pass 2 (steering
matrices) against the oracle's steering_metric of the GPU's gradients; pass 3 (the steered
reconstruction) against the oracle's reconstruction with the GPU's matrices.

Tolerances. Pass 1: a gradient is a linear coefficient of one FP32 fit, so it carries the same
rounding as C_0 does (tests/parity.py) with the coefficient's own rounding scales (the oracle
reports them): |g - o| <= REL_TOL |o| + U32 (C_FIT efit + C_W ew); where the fit's smallest
pivot lies within 2 % of min_pivot either usability decision is correct (0 or the gradient).
Pass 2 sums the structure tensor and forms its eigenvalues in FP64 like the oracle; the rest
(square roots, normalisation, elongation, the power, the matrix) runs in FP32 with no
cancellation: a few ulp on each eigenvalue of C and on its direction, together at most about 20
U32 of the trace for alpha <= 1, so 32 U32 of the trace. Pass 3: the
reconstruction tolerance of tests/parity.py (the window's FP32 quadratic form perturbs the weights
by a few U32 relative, inside C_W).
"""
import numpy as np
import pytest

import oracle
from paper_1308_4908_gb300 import synth
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PIVOT_BAND = 0.02
Q_TOL = 32 * parity.U32


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_4908_gb300 import hdr
    c = hdr.Context(0)
    yield c
    c.close()


def _calpa(**over):
    from paper_1308_4908_gb300 import hdr
    return hdr.hdr_calpa_params_default(**over)


def _raws(frame):
    return [torch.from_numpy(s.raw).cuda() for s in frame.sensors]


def _passes(ctx, fr, c, rig_id=0, params=None):
    """The three passes on the GPU; returns (grad, metric, out, choice) as numpy arrays."""
    p = params or fr.params
    ctx.set_rig(rig_id, fr.sensors)
    raws = _raws(fr)
    g = ctx.calpa_gradients(rig_id, p, c, raws)
    q = ctx.calpa_metric(c, g)
    ch = torch.empty((3, p.out_h, p.out_w), dtype=torch.uint8, device="cuda")
    out = ctx.reconstruct_steered(rig_id, p, c, raws, q, choice=ch)
    ctx.check()
    return g.cpu().numpy(), q.cpu().numpy(), out.float().cpu().numpy(), ch.cpu().numpy()


def check_gradients(fr, p, c, g_gpu, pixels=None):
    """Pass 1 against the oracle; returns the largest error / tolerance."""
    d = oracle.gradients(fr.sensors, p, c.grad_sigma, pixels=pixels, diagnostics=True)
    if pixels is not None:
        g_gpu = g_gpu[pixels[:, 1], pixels[:, 0]]
    o = d["grad"]
    g = g_gpu.astype(np.float64)
    near = np.abs(d["pivot"] - p.min_pivot) <= PIVOT_BAND * p.min_pivot + 1e-5
    zero = np.all(g == 0.0, axis=-1)
    tol = parity.REL_TOL * np.abs(o) + parity.U32 * (parity.C_FIT * d["efit"] + parity.C_W * d["ew"])
    ok = np.abs(g - o) <= tol
    ok = ok | (near[..., None] & zero[..., None])
    bad = np.argwhere(~ok)
    assert bad.size == 0, (f"{len(bad)} gradient components off; first {bad[:5].tolist()}: "
                           f"gpu {[g[tuple(b[:-1])].tolist() for b in bad[:3]]} "
                           f"oracle {[o[tuple(b[:-1])].tolist() for b in bad[:3]]}")
    clear = ~near
    assert np.all(np.isfinite(g))
    ratio = np.abs(g - o)[clear] / np.maximum(tol[clear], 1e-300)
    return float(ratio.max()) if ratio.size else 0.0


def check_metric(q_gpu, q_orc):
    norm = np.abs(q_orc[..., 0]) + np.abs(q_orc[..., 2])
    err = np.abs(q_gpu.astype(np.float64) - q_orc).max(axis=-1)
    assert np.all(err <= Q_TOL * norm), float((err / norm).max())


@pytest.fixture(scope="module")
def small():
    """The paper-scale recipe (3 sensors, affine misalignment, order 2, 4 scales) at 80x72:
    several tiles per side with ragged tails."""
    fr = synth.paper_scale(size=96, out_size=None, seed=1021)
    import dataclasses
    p = dataclasses.replace(fr.params, out_w=80, out_h=72)
    return dataclasses.replace(fr, params=p)


@pytest.fixture(scope="module")
def small_run(ctx, small):
    c = _calpa()
    return c, _passes(ctx, small, c)


def test_pass1_gradients(small, small_run):
    c, (g, _, _, _) = small_run
    r = check_gradients(small, small.params, c, g)
    assert r <= 1.0


def test_pass2_metric(small_run):
    c, (g, q, _, _) = small_run
    q_orc = oracle.steering_metric(g.astype(np.float64), c.window_sigma, c.alpha, c.lambda1, c.lambda2, c.min_eig,
                                   c.max_eig, c.grad_scale)
    check_metric(q, q_orc)
    # eigenvalues inside the clamp, up to FP32 rounding: the entries' own rounding and the unit
    # direction's squared norm (1 within a few ulp) scale the clamped eigenvalues
    q64 = q.astype(np.float64)
    tr, det = q64[..., 0] + q64[..., 2], q64[..., 0] * q64[..., 2] - q64[..., 1] ** 2
    disc = np.sqrt(np.maximum(tr * tr / 4 - det, 0))
    slack = 8 * parity.U32 * (np.abs(q64[..., 0]) + np.abs(q64[..., 2]) + 2 * np.abs(q64[..., 1]))
    assert np.all(tr / 2 - disc >= c.min_eig - slack) and np.all(tr / 2 + disc <= c.max_eig + slack)


def test_pass3_steered_reconstruction(small, small_run):
    c, (_, q, out, ch) = small_run
    p = small.params
    vv, uu = np.mgrid[0:p.out_h, 0:p.out_w]
    pix = np.stack([uu.ravel(), vv.ravel()], axis=1)
    o = oracle.reconstruct(small.sensors, p, pix, levels=True, kappa=True, metric=q.astype(np.float64))
    stats = parity.compare(out[:, pix[:, 1], pix[:, 0]], ch[:, pix[:, 1], pix[:, 0]], o, pix, len(p.sigmas), p.order,
                           p.ici_gamma, p.min_pivot)
    assert stats["n"] > 0.9 * 3 * p.out_w * p.out_h


def test_adaptive_entry_point_is_the_three_passes(ctx, small, small_run):
    c, (_, _, out, ch) = small_run
    p = small.params
    ch2 = torch.empty((3, p.out_h, p.out_w), dtype=torch.uint8, device="cuda")
    out2 = ctx.reconstruct_adaptive(0, p, c, _raws(small), choice=ch2)
    ctx.check()
    np.testing.assert_array_equal(out2.cpu().numpy(), out)
    np.testing.assert_array_equal(ch2.cpu().numpy(), ch)
    # the host-buffer entry point: same bits
    out3 = np.full((3, p.out_h, p.out_w), -7.0, np.float32)
    ch3 = np.zeros((3, p.out_h, p.out_w), np.uint8)
    ctx.reconstruct_adaptive_host(0, p, c, [np.ascontiguousarray(s.raw) for s in small.sensors], out3, ch3)
    ctx.check()
    np.testing.assert_array_equal(out3, out)
    np.testing.assert_array_equal(ch3, ch)


@pytest.mark.parametrize("order", [0, 1])
def test_lower_orders_steered(ctx, small, order):
    import dataclasses
    p = dataclasses.replace(small.params, order=order, out_w=40, out_h=36)
    c = _calpa(alpha=0.3, window_sigma=1.5)
    g, q, out, ch = _passes(ctx, small, c, params=p)
    check_gradients(small, p, c, g)
    vv, uu = np.mgrid[0:p.out_h, 0:p.out_w]
    pix = np.stack([uu.ravel(), vv.ravel()], axis=1)
    o = oracle.reconstruct(small.sensors, p, pix, levels=True, kappa=True, metric=q.astype(np.float64))
    parity.compare(out[:, pix[:, 1], pix[:, 0]], ch[:, pix[:, 1], pix[:, 0]], o, pix, len(p.sigmas), p.order,
                   p.ici_gamma, p.min_pivot)


def test_identity_metric_is_the_isotropic_window(ctx):
    """C = I turns the steered window into Eq. 8's: on the affine paper rig the steered kernel must
    match the oracle's isotropic reconstruction to the parity tolerance, as the searched isotropic
    kernel does (the two kernels derive the traversal box differently, from the FP32 quadratic
    form or from FP64 unit extents, so a row may start one cell apart and offsets round
    differently)."""
    import dataclasses
    fr = synth.paper_scale(size=96, seed=1060)
    p = dataclasses.replace(fr.params, out_w=88, out_h=70)
    ctx.set_rig(0, fr.sensors)
    raws = _raws(fr)
    q = torch.zeros((p.out_h, p.out_w, 3), dtype=torch.float32, device="cuda")
    q[..., 0] = 1.0
    q[..., 2] = 1.0
    ch1 = torch.empty((3, p.out_h, p.out_w), dtype=torch.uint8, device="cuda")
    ch2 = torch.empty_like(ch1)
    a = ctx.reconstruct_steered(0, p, _calpa(), raws, q, choice=ch1).cpu().numpy()
    b = ctx.reconstruct(0, p, raws, choice=ch2).cpu().numpy()
    ctx.check()
    vv, uu = np.mgrid[0:p.out_h, 0:p.out_w]
    pix = np.stack([uu.ravel(), vv.ravel()], axis=1)
    o = oracle.reconstruct(fr.sensors, p, pix, levels=True, kappa=True)
    for out, ch in ((a, ch1.cpu().numpy()), (b, ch2.cpu().numpy())):
        parity.compare(out[:, pix[:, 1], pix[:, 0]], ch[:, pix[:, 1], pix[:, 0]], o, pix, len(p.sigmas), p.order,
                       p.ici_gamma, p.min_pivot)


def test_empty_tiny_and_rejected(ctx, small):
    import dataclasses
    from paper_1308_4908_gb300 import hdr
    ctx.set_rig(0, small.sensors)
    raws = _raws(small)
    c = _calpa()
    p0 = dataclasses.replace(small.params, out_w=0, out_h=0)
    ctx.reconstruct_adaptive(0, p0, c, raws)                       # nothing to do
    p1 = dataclasses.replace(small.params, out_w=1, out_h=1)
    g, q, out, ch = _passes(ctx, small, c, params=p1)             # one ragged tile, M = 1
    o = oracle.adaptive(small.sensors, p1, c.grad_sigma, c.window_sigma, c.alpha, c.lambda1, c.lambda2, c.min_eig,
                        c.max_eig, pixels=np.array([[0, 0]]), levels=True, kappa=True)
    check_gradients(small, p1, c, g)
    check_metric(q, oracle.steering_metric(g.astype(np.float64), c.window_sigma, c.alpha, c.lambda1, c.lambda2,
                                           c.min_eig, c.max_eig, c.grad_scale))
    assert np.isfinite(out).all() and o["out"].shape == (1, 3)
    with pytest.raises(hdr.HdrError) as e:
        ctx.reconstruct_adaptive(0, small.params, _calpa(window_sigma=4.0), raws)
    assert e.value.status == hdr.HDR_E_INVALID
    with pytest.raises(hdr.HdrError) as e:
        ctx.reconstruct_adaptive(0, small.params, _calpa(min_eig=0.0), raws)
    assert e.value.status == hdr.HDR_E_INVALID
    with pytest.raises(hdr.HdrError) as e:                         # the window would outgrow the staging box
        ctx.reconstruct_adaptive(0, small.params, _calpa(min_eig=1e-4), raws)
    assert e.value.status == hdr.HDR_E_UNSUPPORTED


def test_full_size_sampled(ctx):
    """The paper-scale 3 x 2048^2 frame, order 2, 4 scales: each pass on sampled pixels (pass 2 on
    the crop of the GPU's gradients that holds each sampled pixel's disc)."""
    fr = synth.paper_scale()
    p = fr.params
    c = _calpa()
    g, q, out, ch = _passes(ctx, fr, c)
    r = np.random.default_rng(5)
    pix = np.concatenate([r.integers(0, 2048, (300, 2)), [[0, 0], [2047, 2047], [0, 2047], [2047, 0], [5, 1000]]])
    check_gradients(fr, p, c, g, pixels=pix)
    rad = int(np.floor(3.0 * c.window_sigma))
    for u, v in pix[:60]:
        v0, v1, u0, u1 = max(0, v - rad), min(p.out_h, v + rad + 1), max(0, u - rad), min(p.out_w, u + rad + 1)
        qo = oracle.steering_metric(g[v0:v1, u0:u1].astype(np.float64), c.window_sigma, c.alpha, c.lambda1,
                                    c.lambda2, c.min_eig, c.max_eig, c.grad_scale)[v - v0, u - u0]
        check_metric(q[v, u][None], qo[None])
    o = oracle.reconstruct(fr.sensors, p, pix, levels=True, kappa=True, metric=q.astype(np.float64))
    parity.compare(out[:, pix[:, 1], pix[:, 0]], ch[:, pix[:, 1], pix[:, 0]], o, pix, len(p.sigmas), p.order,
                   p.ici_gamma, p.min_pivot)


@pytest.mark.parametrize("accum,out_dtype", [(1, 0), (0, 1)])
def test_steered_compensated_sums_and_fp16_output(ctx, small, accum, out_dtype):
    """The steered kernel with compensated moment sums (its own instantiation) and with FP16
    output, against the oracle with the same matrices (FP16 adds its 2^-11 rounding)."""
    import dataclasses
    p = dataclasses.replace(small.params, accum=accum, out_dtype=out_dtype, out_w=48, out_h=40)
    c = _calpa()
    g, q, out, ch = _passes(ctx, small, c, params=p)
    check_gradients(small, p, c, g)
    vv, uu = np.mgrid[0:p.out_h, 0:p.out_w]
    pix = np.stack([uu.ravel(), vv.ravel()], axis=1)
    o = oracle.reconstruct(small.sensors, p, pix, levels=True, kappa=True, metric=q.astype(np.float64))
    parity.compare(out[:, pix[:, 1], pix[:, 0]], ch[:, pix[:, 1], pix[:, 0]], o, pix, len(p.sigmas), p.order,
                   p.ici_gamma, p.min_pivot, extra_rel=parity.HALF_TOL if out_dtype == 1 else 0.0)


def test_metric_with_a_gradient_unit(ctx, small_run):
    """grad_scale (the unit of the radiant power for the fixed regularisers) against the oracle."""
    c0, (g, _, _, _) = small_run
    c = _calpa(grad_scale=1e-3, alpha=0.3)
    q = ctx.calpa_metric(c, torch.from_numpy(g).cuda()).cpu().numpy()
    ctx.check()
    check_metric(q, oracle.steering_metric(g.astype(np.float64), c.window_sigma, c.alpha, c.lambda1, c.lambda2,
                                           c.min_eig, c.max_eig, c.grad_scale))


def test_four_sensors_and_an_upsampled_output(ctx):
    """A 4-sensor rig (ND 1 .. 1/512) reconstructed 1.5x upsampled with steered windows, order 2,
    against the oracle on every pixel."""
    fr = synth.batching_frame((1004, 99, 4, 64, 48, 2, 1.5))
    p = fr.params
    c = _calpa()
    g, q, out, ch = _passes(ctx, fr, c)
    check_gradients(fr, p, c, g)
    check_metric(q, oracle.steering_metric(g.astype(np.float64), c.window_sigma, c.alpha, c.lambda1, c.lambda2,
                                           c.min_eig, c.max_eig, c.grad_scale))
    vv, uu = np.mgrid[0:p.out_h, 0:p.out_w]
    pix = np.stack([uu.ravel(), vv.ravel()], axis=1)
    o = oracle.reconstruct(fr.sensors, p, pix, levels=True, kappa=True, metric=q.astype(np.float64))
    parity.compare(out[:, pix[:, 1], pix[:, 0]], ch[:, pix[:, 1], pix[:, 0]], o, pix, len(p.sigmas), p.order,
                   p.ici_gamma, p.min_pivot)


def test_metric_of_a_tall_thin_output(ctx):
    """An output of one column and 600000 rows (more block rows than a grid's second dimension
    allows): the matrix pass against the oracle."""
    r = np.random.default_rng(21)
    g = r.normal(0.0, 20.0, (600000, 1, 2)).astype(np.float32)
    g[::97, 0, 0] += 300.0
    c = _calpa()
    q = ctx.calpa_metric(c, torch.from_numpy(g).cuda()).cpu().numpy()
    ctx.check()
    check_metric(q, oracle.steering_metric(g.astype(np.float64), c.window_sigma, c.alpha, c.lambda1, c.lambda2,
                                           c.min_eig, c.max_eig, c.grad_scale))
