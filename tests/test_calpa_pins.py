"""Pins of the adaptive (CALPA) oracle, Sections 5.4-5.5: gradients from the order-1 green fit,
the steering matrix from the local gradient structure, and the fit with the steered window."""
import numpy as np
import pytest

import oracle
from paper_1308_4908_gb300 import synth
from tests.test_oracle_pins import _poly, value_rig


def _plane(gx, gy):
    def fn(c, X, Y):
        return 300.0 + 40.0 * c + gx * (X - 12.0) + gy * (Y - 12.0)
    return fn


def test_gradients_of_a_plane_are_exact():
    """An order-1 fit reproduces a plane exactly (Sections 5.1-5.2), so its linear coefficients
    are the plane's gradient at every pixel with a usable fit, for any rig."""
    sensors = value_rig(_plane(3.0, -2.0))
    p = synth.Params(order=2, sigmas=(1.0,), out_w=24, out_h=24)
    g = oracle.gradients(sensors, p, 1.2)
    inner = g[6:18, 6:18]
    np.testing.assert_allclose(inner[..., 0], 3.0, rtol=0, atol=1e-9)
    np.testing.assert_allclose(inner[..., 1], -2.0, rtol=0, atol=1e-9)


def test_metric_of_a_flat_region_is_isotropic():
    """Zero gradients: s1 = s2 = 0, elongation 1, scaling (lambda2 / M)^alpha (M window pixels)."""
    q = oracle.steering_metric(np.zeros((21, 21, 2)), 1.0, 0.5, min_eig=1e-9, max_eig=1e9)
    M = sum(1 for i in range(-3, 4) for j in range(-3, 4) if i * i + j * j <= 9)
    want = (0.001 / M) ** 0.5
    np.testing.assert_allclose(q[10, 10], [want, 0.0, want], rtol=1e-12, atol=0)


def test_metric_of_a_constant_gradient():
    """A constant gradient g: rank-one structure, s1 = |g| sqrt(sum w), s2 = 0; the window is
    narrow along g (eigenvalue gamma sigma_j) and long across it (gamma / sigma_j)."""
    g = np.zeros((15, 15, 2))
    g[..., 0], g[..., 1] = 3.0, 4.0
    ws, alpha = 1.0, 0.3
    q = oracle.steering_metric(g, ws, alpha, min_eig=1e-12, max_eig=1e12)
    offs = [(i, j) for i in range(-3, 4) for j in range(-3, 4) if i * i + j * j <= 9]
    sw = sum(np.exp(-(i * i + j * j) / 2.0) for i, j in offs)
    s1 = 5.0 * np.sqrt(sw)
    el = (s1 + 1.0) / 1.0
    gam = (0.001 / len(offs)) ** alpha
    u = np.array([0.6, 0.8])
    C = gam * el * np.outer(u, u) + gam / el * np.outer([-0.8, 0.6], [-0.8, 0.6])
    np.testing.assert_allclose(q[7, 7], [C[0, 0], C[0, 1], C[1, 1]], rtol=1e-10)


def test_metric_follows_an_edge():
    """Gradients of a vertical step edge point along x: the steered window is narrow in x (across
    the edge) and long in y (along it); the eigenvalues are clamped to the bounds."""
    g = np.zeros((21, 21, 2))
    g[:, 9:12, 0] = 50.0
    q = oracle.steering_metric(g, 1.0, 0.5)
    c11, c12, c22 = q[10, 10]
    assert c11 > c22 and abs(c12) < 1e-9
    assert 0.25 <= c22 <= c11 <= 16.0


def test_scaled_identity_metric_is_the_isotropic_fit_at_a_scaled_sigma():
    """Q = c I gives the window exp(-c |d|^2 / (2 sigma^2)) on |d| < k sigma / sqrt(c): the
    isotropic fit at sigma / sqrt(c) (Eq. 8)."""
    r = np.random.default_rng(2)
    sensors = value_rig(lambda c, X, Y: 100 + 30 * np.sin(0.4 * X + c) * np.cos(0.3 * Y), var_fn=None)
    p = synth.Params(order=2, sigmas=(1.2, 2.0, 3.0), out_w=24, out_h=24, min_pivot=1e-9)
    cfac = 2.25
    q = np.zeros((24, 24, 3))
    q[..., 0] = q[..., 2] = cfac
    pix = np.array([[u, v] for u in range(5, 19, 3) for v in range(5, 19, 3)])
    a = oracle.reconstruct(sensors, p, pix, levels=True, metric=q)
    import dataclasses
    b = oracle.reconstruct(sensors, dataclasses.replace(p, sigmas=tuple(s / np.sqrt(cfac) for s in p.sigmas)), pix,
                           levels=True)
    np.testing.assert_array_equal(a["count"], b["count"])
    np.testing.assert_allclose(a["c0"], b["c0"], rtol=1e-10, atol=1e-10)
    np.testing.assert_array_equal(a["choice"], b["choice"])


@pytest.mark.parametrize("order", [1, 2])
def test_steered_window_reproduces_polynomials(order):
    """Any positive window reproduces polynomials of degree <= M (Sections 5.1-5.2): so does the
    steered one, with a different random orientation and elongation at every pixel."""
    fn = _poly(order, 20 + order)
    sensors = value_rig(fn)
    p = synth.Params(order=order, sigmas=(1.2, 1.8), out_w=24, out_h=24, min_pivot=1e-12)
    r = np.random.default_rng(4)
    th = r.uniform(0, np.pi, (24, 24))
    e1, e2 = r.uniform(0.5, 2.0, (24, 24)), r.uniform(0.5, 2.0, (24, 24))
    c, s = np.cos(th), np.sin(th)
    q = np.stack([e1 * c * c + e2 * s * s, (e1 - e2) * c * s, e1 * s * s + e2 * c * c], axis=2)
    pix = np.array([[u, v] for u in range(7, 17, 3) for v in range(7, 17, 3)])
    res = oracle.reconstruct(sensors, p, pix, levels=True, metric=q)
    for i, (u, v) in enumerate(pix):
        for ch in range(3):
            for lvl in range(2):
                assert res["valid"][i, ch, lvl]
                assert res["c0"][i, ch, lvl] == pytest.approx(fn(ch, float(u), float(v)), rel=1e-9)


def test_steered_window_area_follows_the_determinant():
    """The support d^T Q d < R^2 has area pi R^2 / sqrt(det Q): Q = 4 I holds about a quarter of
    the samples of the isotropic window, Q = diag(4, 1/4) about as many."""
    sensors = value_rig(lambda c, X, Y: 100.0 + 0 * X, size=40, rot=0.0, trans=0.5)
    p = synth.Params(order=0, sigmas=(3.0,), out_w=40, out_h=40)
    pix = np.array([[20, 20], [19, 21]])
    iso = oracle.reconstruct(sensors, p, pix, levels=True)["count"]
    q4 = np.zeros((40, 40, 3))
    q4[..., 0] = q4[..., 2] = 4.0
    small = oracle.reconstruct(sensors, p, pix, levels=True, metric=q4)["count"]
    qa = np.zeros((40, 40, 3))
    qa[..., 0], qa[..., 2] = 4.0, 0.25
    aniso = oracle.reconstruct(sensors, p, pix, levels=True, metric=qa)["count"]
    assert np.all(np.abs(small / iso - 0.25) < 0.06)
    assert np.all(np.abs(aniso / iso - 1.0) < 0.12)
    with pytest.raises(ValueError):
        oracle.reconstruct(sensors, p, pix, metric=-q4)


def test_gradient_unit_scaling():
    """Gradients in a unit s times larger: the elongation is unchanged when lambda1 is scaled by s,
    and the scaling parameter grows by s^(2 alpha) when lambda2 is scaled by s^2, so the matrix
    computed with grad_scale = s equals s^(2 alpha) times the one with the regularisers rescaled."""
    r = np.random.default_rng(4)
    g = r.normal(0.0, 3.0, (17, 19, 2))
    g[:, 8:11, 0] += 40.0
    s, alpha = 1e-3, 0.4
    a = oracle.steering_metric(g, 1.3, alpha, 1.0, 1e-3, 1e-12, 1e12, grad_scale=s)
    b = oracle.steering_metric(g, 1.3, alpha, 1.0 / s, 1e-3 / s ** 2, 1e-12, 1e12)
    np.testing.assert_allclose(a, s ** (2 * alpha) * b, rtol=1e-10, atol=0)


def test_gradient_rounding_scale_bounds_a_perturbation():
    """The rounding scale the oracle reports for each gradient component bounds how far it moves
    when every sample value is perturbed by a relative eps (first order): with f_k -> f_k (1 + eps
    s_k), |s_k| <= 1, the coefficient moves by sum_k w_k (A^-1 phi_k)_1 f_k eps s_k, at most
    eps efit. Random signs come close to it; the scale must never be exceeded."""
    import copy
    rng = np.random.default_rng(12)

    def fn(c, X, Y):
        return 200.0 + 30.0 * np.sin(0.4 * X) + 10.0 * np.cos(0.3 * Y) + 5.0 * c
    sensors = value_rig(fn, seed=9)
    p = synth.Params(order=2, sigmas=(1.0,), out_w=24, out_h=24)
    pix = np.array([[u, v] for u in range(6, 18, 3) for v in range(6, 18, 3)])
    base = oracle.gradients(sensors, p, 1.2, pixels=pix, diagnostics=True)
    eps = 1e-6
    worst = 0.0
    for trial in range(4):
        pert = copy.deepcopy(sensors)
        for s in pert:
            s.value_f = s.value_f * (1.0 + eps * rng.choice([-1.0, 1.0], s.value_f.shape))
        g = oracle.gradients(pert, p, 1.2, pixels=pix)
        ratio = np.abs(g - base["grad"]) / (eps * base["efit"])
        worst = max(worst, float(ratio.max()))
    assert worst <= 1.0 + 1e-6, worst
    assert worst > 0.05, worst    # the scale is not loose by orders of magnitude
