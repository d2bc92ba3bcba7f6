"""Pins of the oracle quantities that set the parity tolerance (tests/parity.py).

The GPU value of C_0 may differ from the oracle's by U32 (C_FIT efit + C_W ew) beyond the 1e-5
relative term. efit and ew are reported by the oracle per fit:

* efit = sum_k w_k L1_k (|f_k| + F1_k) bounds how far C_0 moves per unit relative perturbation of
  the moment sums (right-hand side and normal matrix), L1_k = sum_m |l_m phi_m(d_k)|,
  l = A^{-1} e_0, F1_k = sum_m |c_m phi_m(d_k)|, c = A^{-1} b;
* ew = sum_k G_k (1 + r_k^2 / sigma^2) / s2_k L1_k |f_k - phi(d_k)^T c| bounds how far it moves per
  unit relative perturbation of the Gaussian G at every sample (its ex2 evaluation) and of r_k^2
  (the rounding of the sample position).

Section 5.2 fixes what they must bound: the estimate is a linear filter of the samples,
C_0 = sum_k l_k f_k with the equivalent kernel l_k = w_k e_0^T A^{-1} phi(d_k), and a relative
change of one sample's weight moves C_0 by l_k (f_k - phi(d_k)^T c). The sensitivities are taken
here from the oracle as a black box (central differences of its C_0 with respect to one sample's
value or variance), never from its formulas. At order 0 (L1_k = |l_k| / w_k) both scales equal
the worst case of those first-order changes exactly; at orders 1 and 2 they bound it. The
condition number the oracle reports (cyclic Jacobi eigen-iteration) is pinned on matrices whose
spectrum is known in closed form.
"""
import copy
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_1308_4908_gb300 import synth
from tests.test_oracle_pins import value_rig

SIGMA = 1.2
K_TRUNC = 3.0
PIXELS = [(10, 11), (12, 12), (13, 9)]


def _scene(c, X, Y):
    return 200.0 + 30.0 * np.sin(0.45 * X + 0.2 * Y) + 12.0 * np.cos(0.3 * Y) + 25.0 * c + 0.8 * X * Y / 10.0


def _signed_scene(c, X, Y):
    # crosses zero inside the windows: |f| and the residuals differ in sign from sample to sample
    return 40.0 * np.sin(0.7 * X - 0.4 * Y + c) + 5.0


def _window_samples(sensors, P, c, sigma_c):
    """(sensor, x, y, r^2) of every sample of colour c within k sigma_c of the point P, from the
    sensors' transforms (the test's own enumeration)."""
    out = []
    for s, sen in enumerate(sensors):
        y, x = np.mgrid[0:sen.height, 0:sen.width]
        X, Y = synth.apply_affine(np.asarray(sen.affine), x.astype(float), y.astype(float))
        r2 = (X - P[0]) ** 2 + (Y - P[1]) ** 2
        sel = (synth.cfa_color(x, y) == c) & (r2 < (K_TRUNC * sigma_c) ** 2)
        for yy, xx in zip(*np.nonzero(sel)):
            out.append((s, int(xx), int(yy), float(r2[yy, xx])))
    return out


def _c0(sensors, p, pix, c):
    r = oracle.reconstruct(sensors, p, np.array([pix]), levels=True)
    return float(r["c0"][0, c, 0]), float(r["efit"][0, c, 0]), float(r["ew"][0, c, 0]), bool(r["valid"][0, c, 0])


def _sensitivities(sensors, p, pix, c, samples):
    """Per sample k: l_k f_k = f_k dC_0/df_k and b_k = dC_0/dln w_k (w = K / s2, so a relative
    change of s2 by exp(-t) is a change of ln w by t), by central differences of the oracle."""
    work = copy.deepcopy(sensors)
    lf, lw = [], []
    for (s, x, y, _) in samples:
        sen = work[s]
        f0, v0 = sen.value_f[y, x], sen.value_var[y, x]
        h = 1e-6 * max(abs(f0), 1.0)
        sen.value_f[y, x] = f0 + h
        up = _c0(work, p, pix, c)[0]
        sen.value_f[y, x] = f0 - h
        dn = _c0(work, p, pix, c)[0]
        sen.value_f[y, x] = f0
        lf.append((up - dn) / (2 * h) * f0)
        t = 1e-5
        sen.value_var[y, x] = v0 * math.exp(-t)
        up = _c0(work, p, pix, c)[0]
        sen.value_var[y, x] = v0 * math.exp(t)
        dn = _c0(work, p, pix, c)[0]
        sen.value_var[y, x] = v0
        lw.append((up - dn) / (2 * t))
    return np.array(lf), np.array(lw)


def _window_factor(samples, sigma_c):
    """(G_k / K_k)(1 + r_k^2 / sigma^2): a relative change of G_k by e and of r_k^2 by e changes
    K_k = G_k - exp(-k^2/2) relatively by at most e times this."""
    r2 = np.array([smp[3] for smp in samples])
    G = np.exp(-r2 / (2 * sigma_c ** 2))
    K = G - math.exp(-0.5 * K_TRUNC ** 2)
    return G / K * (1.0 + r2 / sigma_c ** 2)


def _cases(order, scene):
    sensors = value_rig(scene, seed=11)
    p = synth.Params(order=order, sigmas=(SIGMA,), out_w=24, out_h=24, trunc_k=K_TRUNC, min_pivot=1e-9)
    for pix in PIXELS:
        for c in range(3):
            sigma_c = SIGMA * (p.green_ratio if c == 1 else 1.0)
            samples = _window_samples(sensors, pix, c, sigma_c)
            yield sensors, p, pix, c, sigma_c, samples


@pytest.mark.parametrize("scene", [_scene, _signed_scene])
def test_order0_rounding_scales_are_the_worst_case(scene):
    """Order 0 (Eq. 7): l_k = w_k / sum w, so a relative perturbation e of every value moves C_0 by
    at most e sum_k |l_k f_k|, one of the normal matrix (the sum of weights) by e |C_0|: their sum
    is efit exactly. A relative perturbation e of every Gaussian and every r^2 changes each weight
    by at most e (G/K)(1 + r^2/sigma^2), moving C_0 by at most e sum_k |b_k| (G_k/K_k)(1 + r_k^2/
    sigma^2): that is ew exactly."""
    n = 0
    for sensors, p, pix, c, sigma_c, samples in _cases(0, scene):
        c0, efit, ew, valid = _c0(sensors, p, pix, c)
        assert valid and len(samples) >= 8
        lf, lw = _sensitivities(sensors, p, pix, c, samples)
        assert efit == pytest.approx(np.abs(lf).sum() + abs(c0), rel=1e-7)
        assert ew == pytest.approx((np.abs(lw) * _window_factor(samples, sigma_c)).sum(), rel=1e-6)
        # the sensitivities themselves: the weights sum to one, and sum_k b_k = 0 (a common
        # relative change of every weight leaves the weighted mean where it is)
        assert abs(lw.sum()) <= 1e-6 * np.abs(lw).sum()
        n += 1
    assert n == 3 * len(PIXELS)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("scene", [_scene, _signed_scene])
def test_rounding_scales_bound_the_worst_case(order, scene):
    """Orders 1 and 2: efit bounds the worst first-order change of C_0 under relative perturbations
    of the sample values and under relative perturbations of the sample weights (both enter the
    moment sums), ew the one under relative perturbations of each Gaussian and each r^2; neither is
    loose by more than a factor 20 (L1_k sums the basis terms of l_k in absolute value, and the
    matrix and right-hand side perturbations are bounded separately)."""
    tight_fit, tight_w = [], []
    for sensors, p, pix, c, sigma_c, samples in _cases(order, scene):
        c0, efit, ew, valid = _c0(sensors, p, pix, c)
        assert valid
        lf, lw = _sensitivities(sensors, p, pix, c, samples)
        worst_f = np.abs(lf).sum()
        worst_wt = np.abs(lw).sum()
        worst_win = (np.abs(lw) * _window_factor(samples, sigma_c)).sum()
        assert worst_f <= efit * (1 + 1e-6)
        assert worst_wt <= efit * (1 + 1e-6)
        assert worst_win <= ew * (1 + 1e-6)
        tight_fit.append(max(worst_f, worst_wt) / efit)
        tight_w.append(worst_win / ew)
    # measured: efit 0.1-0.45 of the worst case, ew 0.2-0.94 (orders 1 and 2, both scenes)
    assert min(tight_fit) > 0.05, tight_fit
    assert min(tight_w) > 0.1, tight_w


@pytest.mark.parametrize("order", [0, 1, 2])
def test_rounding_scales_are_invariant_to_the_unit_of_length(order):
    """Rounding of C_0 does not depend on the unit of length: a rig, its output mapping and its
    window scale all multiplied by s give the same samples, weights and C_0 (the basis coefficients
    scale by powers of s, their products with the basis do not), so efit and ew are unchanged."""
    sensors = value_rig(_scene, seed=5)
    p = synth.Params(order=order, sigmas=(0.9, 1.6), out_w=24, out_h=24, min_pivot=1e-9)
    pix = np.array([[u, v] for u in (7, 12, 16) for v in (8, 13)])
    base = oracle.reconstruct(sensors, p, pix, levels=True)
    for s in (0.37, 3.1):
        big = copy.deepcopy(sensors)
        for sen in big:
            sen.affine = np.asarray(sen.affine) * s
        ps = dataclasses.replace(p, sigmas=tuple(sg * s for sg in p.sigmas), out_affine=p.out_affine * s)
        r = oracle.reconstruct(big, ps, pix, levels=True)
        ok = base["valid"].astype(bool)
        assert ok.sum() > 20
        np.testing.assert_array_equal(r["count"], base["count"])
        np.testing.assert_allclose(r["c0"][ok], base["c0"][ok], rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(r["efit"][ok], base["efit"][ok], rtol=1e-9)
        np.testing.assert_allclose(r["ew"][ok], base["ew"][ok], rtol=1e-9)


def test_random_sign_perturbation_stays_within_the_scales():
    """Every value of a whole frame perturbed by a relative eps with random signs, then every
    variance: each C_0 moves by at most eps efit (first order); the random signs reach a fair part
    of it somewhere."""
    rng = np.random.default_rng(21)
    sensors = value_rig(_scene, seed=13)
    p = synth.Params(order=2, sigmas=(0.8, 1.2, 1.8), out_w=24, out_h=24, min_pivot=1e-9)
    pix = np.array([[u, v] for u in range(5, 19, 2) for v in range(5, 19, 3)])
    base = oracle.reconstruct(sensors, p, pix, levels=True)
    ok = base["valid"].astype(bool)
    eps = 1e-7
    worst = 0.0
    for field in ("value_f", "value_var"):
        for trial in range(3):
            pert = copy.deepcopy(sensors)
            for sen in pert:
                arr = getattr(sen, field)
                setattr(sen, field, arr * (1.0 + eps * rng.choice([-1.0, 1.0], arr.shape)))
            r = oracle.reconstruct(pert, p, pix, levels=True)
            ratio = np.abs(r["c0"][ok] - base["c0"][ok]) / (eps * base["efit"][ok])
            assert ratio.max() <= 1.0 + 1e-4, (field, ratio.max())
            worst = max(worst, float(ratio.max()))
    assert worst > 0.05, worst


# ------------------------------------------------------------------ condition number

def _reflector(rng, n):
    u = rng.normal(size=(n, 1))
    return np.eye(n) - 2.0 * (u @ u.T) / float((u.T @ u)[0, 0])


def test_condition_2x2_closed_form():
    """Symmetric 2 x 2: eigenvalues (a + c)/2 +- sqrt(((a - c)/2)^2 + b^2)."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        a, b, c = rng.normal(size=3) * rng.choice([1e-3, 1.0, 1e3])
        h, d = 0.5 * (a + c), math.hypot(0.5 * (a - c), b)
        lam = np.abs([h + d, h - d])
        want = lam.max() / lam.min()
        got = oracle.condition(np.array([[a, b], [b, c]]))
        assert got == pytest.approx(want, rel=1e-9 * max(1.0, want))


def test_condition_diagonal_plus_rank_one():
    """D + rho v v^T with distinct diagonal d: the eigenvalues are the roots of the secular equation
    1 + rho sum_i v_i^2 / (d_i - lambda), one in each gap between the d_i and one beyond, found
    here by bisection."""
    rng = np.random.default_rng(8)
    for _ in range(20):
        d = np.sort(rng.uniform(0.1, 5.0, 3))
        v = rng.normal(size=3)
        rho = rng.uniform(0.2, 3.0)
        f = lambda lam: 1.0 + rho * np.sum(v * v / (d - lam))
        edges = [d[0], d[1], d[2], d[2] + rho * float(v @ v) + 1.0]
        roots = []
        for lo, hi in zip(edges[:-1], edges[1:]):
            lo, hi = lo + 1e-14 * (1 + abs(lo)), hi - 1e-14 * (1 + abs(hi))
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                if f(mid) < 0:
                    lo = mid
                else:
                    hi = mid
            roots.append(0.5 * (lo + hi))
        A = np.diag(d) + rho * np.outer(v, v)
        want = max(roots) / min(roots)
        assert oracle.condition(A) == pytest.approx(want, rel=1e-9)


@pytest.mark.parametrize("n", [3, 6])
def test_condition_known_spectrum(n):
    """Q diag(lambda) Q^T with Q a product of Householder reflections: condition max|lambda| /
    min|lambda|, including indefinite spectra and conditions up to 1e12."""
    rng = np.random.default_rng(n)
    for kappa in (1.0, 37.0, 1e4, 1e8, 1e12):
        lam = np.geomspace(1.0, kappa, n) * rng.choice([-1.0, 1.0], n)
        rng.shuffle(lam)
        Q = _reflector(rng, n) @ _reflector(rng, n) @ _reflector(rng, n)
        A = Q @ np.diag(lam) @ Q.T
        A = 0.5 * (A + A.T)
        got = oracle.condition(A)
        # the matrix entries carry rounding of eps |lambda|_max: the smallest eigenvalue only to
        # eps kappa relative
        assert got == pytest.approx(kappa, rel=1e-12 * kappa + 1e-9)
    assert oracle.condition(np.diag([1.0, 0.0, 2.0])) == math.inf


def test_value_mode_from_raw_reproduces_the_raw_fit():
    """Eq. 18's f and Eq. 20's s2 written out per pixel (saturated pixels excluded) and fed back in
    value mode give the raw-mode result to rounding, including per-pixel calibration frames and a
    saturated region; rounded to FP32 they move C_0 by a few units of FP32 rounding of its terms."""
    fr = synth.paper_scale(size=40, seed=91)
    r = np.random.default_rng(2)
    s0 = fr.sensors[0]
    s0.bias_frame = 64.0 + r.normal(0.0, 1.5, (s0.height, s0.width))
    s0.prnu_frame = 1.0 + r.normal(0.0, 0.02, (s0.height, s0.width))
    s0.raw[10:14, 5:30] = 4095
    pix = np.array([[u, v] for u in range(2, 40, 5) for v in range(1, 40, 4)])
    base = oracle.reconstruct(fr.sensors, fr.params, pix, levels=True)
    val = oracle.reconstruct(oracle.value_sensors(fr.sensors), fr.params, pix, levels=True)
    np.testing.assert_array_equal(val["choice"], base["choice"])
    np.testing.assert_array_equal(val["count"], base["count"])
    np.testing.assert_allclose(val["out"], base["out"], rtol=1e-12, atol=1e-12)
    r32 = oracle.reconstruct(oracle.value_sensors(fr.sensors, round_to=np.float32), fr.params, pix, levels=True)
    same = (r32["choice"] == base["choice"]) & np.isfinite(base["out"])
    lvl = np.clip(base["choice"], 0, None)[..., None]
    efit = np.take_along_axis(base["efit"], lvl, axis=2)[..., 0]
    dev = np.abs(r32["out"] - base["out"])[same] / (2.0 ** -24 * efit[same])
    assert same.mean() > 0.95 and dev.max() < 4.0, (same.mean(), dev.max())
