"""FP64 CPU oracle for noise-aware multi-sensor LPA reconstruction (test infrastructure).

Only `tests/`, `__graft_entry__.smoke()` and `bench.py`'s CPU-baseline leg may
import this package. The product path (the CUDA library and its binding) never
does; the two share no code. Two independent routes live here:

* `lpa_oracle.c` (loaded through ctypes): the definition per output pixel in
  double precision - bounding-box gather, normal equations, Jacobi
  equilibration, LDL^T, scale choice by intersection of confidence intervals,
  order fallback (see its header for the passages followed and the readings).
* `bruteforce.py`: every sample of every sensor, weighted least squares by
  Householder QR (numpy), for tiny rigs - an independent check of the C route.

Parity of `lpa_oracle.c` with the paper is pinned by `tests/test_oracle_*.py`
against closed forms, invariants and brute force (the paper prints no numeric
results). The paper's own code is not available, so parity with that code is
unpinned (noise-weight exponent and window truncation are readings).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lpa_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblpa_oracle.so")

MAX_SCALES = 8


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP); returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Sensor(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("pitch", ctypes.c_int32),
                ("raw", ctypes.c_void_p), ("value_f", ctypes.c_void_p), ("value_var", ctypes.c_void_p),
                ("gain", ctypes.c_double), ("exposure", ctypes.c_double), ("nd", ctypes.c_double),
                ("read_var", ctypes.c_double), ("black", ctypes.c_double), ("sat", ctypes.c_double),
                ("bias_px", ctypes.c_void_p), ("prnu_px", ctypes.c_void_p),
                ("read_var_px", ctypes.c_void_p), ("sat_px", ctypes.c_void_p),
                ("affine", ctypes.c_double * 6)]


class _Params(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("n_scales", ctypes.c_int32),
                ("sigma", ctypes.c_double * MAX_SCALES), ("green_ratio", ctypes.c_double),
                ("trunc_k", ctypes.c_double), ("ici_gamma", ctypes.c_double),
                ("min_pivot", ctypes.c_double), ("out_affine", ctypes.c_double * 6),
                ("weight_mode", ctypes.c_int32)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.orc_reconstruct.argtypes = [P, ctypes.c_int, P, ctypes.c_int64] + [P] * 14
        lib.orc_reconstruct.restype = ctypes.c_int
        lib.orc_radiometry.argtypes = [ctypes.c_double] * 8 + [P, P]
        lib.orc_radiometry.restype = ctypes.c_int
        lib.orc_ici.argtypes = [ctypes.c_int, P, P, P, ctypes.c_double, P]
        lib.orc_gradients.argtypes = [P, ctypes.c_int, P, ctypes.c_double, ctypes.c_int64, P, P, P, P, P, P, P, P]
        lib.orc_gradients.restype = ctypes.c_int
        lib.orc_ici.restype = ctypes.c_int
        lib.orc_equivalent_kernel.argtypes = [P, ctypes.c_int, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_double, ctypes.c_int32, ctypes.c_int32] + [P] * 7
        lib.orc_equivalent_kernel.restype = ctypes.c_int
        lib.orc_radiometry_frame.argtypes = [P, P, P]
        lib.orc_radiometry_frame.restype = ctypes.c_int
        lib.orc_condition.argtypes = [P, ctypes.c_int32]
        lib.orc_condition.restype = ctypes.c_double
        _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _f64(a) -> Optional[np.ndarray]:
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class _Marshal:
    """Keeps the numpy buffers alive while the C structs point at them."""

    def __init__(self, sensors, params):
        self.keep: List[np.ndarray] = []
        n = len(sensors)
        self.arr = (_Sensor * max(n, 1))()
        for i, s in enumerate(sensors):
            d = self.arr[i]
            d.width, d.height = int(s.width), int(s.height)
            vf = getattr(s, "value_f", None)
            if vf is not None:
                f = _f64(vf)
                v = _f64(s.value_var)
                self.keep += [f, v]
                d.value_f, d.value_var = _ptr(f), _ptr(v)
                d.pitch = int(s.width)
                d.raw = None
            else:
                raw = np.ascontiguousarray(s.raw, dtype=np.uint16)
                self.keep.append(raw)
                d.raw = _ptr(raw)
                d.pitch = int(raw.shape[1])
            d.gain, d.exposure, d.nd = float(s.gain), float(s.exposure), float(s.nd)
            d.read_var, d.black, d.sat = float(s.read_var), float(s.black), float(s.sat)
            for name, field in (("bias_frame", "bias_px"), ("prnu_frame", "prnu_px"),
                                ("read_var_frame", "read_var_px"), ("sat_frame", "sat_px")):
                fr = getattr(s, name, None)
                if fr is not None:
                    fr = _f64(fr)
                    self.keep.append(fr)
                setattr(d, field, _ptr(fr))
            d.affine[:] = [float(x) for x in np.asarray(s.affine, dtype=np.float64).reshape(6)]
        self.n = n
        p = _Params()
        p.order = int(params.order)
        p.n_scales = len(params.sigmas)
        for j, sg in enumerate(params.sigmas):
            p.sigma[j] = float(sg)
        p.green_ratio = float(params.green_ratio)
        p.trunc_k = float(params.trunc_k)
        p.ici_gamma = float(params.ici_gamma)
        p.min_pivot = float(params.min_pivot)
        p.out_affine[:] = [float(x) for x in np.asarray(params.out_affine, dtype=np.float64).reshape(6)]
        p.weight_mode = int(getattr(params, "weight_mode", 0))
        self.params = p


def n_levels(params) -> int:
    return len(params.sigmas) + int(params.order)


def reconstruct(sensors: Sequence, params, pixels: Optional[np.ndarray] = None,
                levels: bool = False, kappa: bool = False, metric: Optional[np.ndarray] = None) -> Dict[str, np.ndarray]:
    """Run the oracle on output pixels `pixels` ([n, 2] of (u, v); default: the whole output grid).

    Returns a dict with `out` [n, 3] (or [3, H, W] for the whole grid), `choice`, `margin` and, when
    `levels`, the per-level arrays `c0`, `var`, `pivot`, `count`, `valid` ([n, 3, J+M]), the
    rounding scales `efit` and `ew` (see lpa_oracle.c) and, with `kappa`, the condition numbers.
    `metric` ([out_h, out_w, 3] of {Q11, Q12, Q22}, optional) steers the window of every pixel
    (Section 5.4; see `steering_metric`).
    """
    lib = _load()
    grid = pixels is None
    if grid:
        vv, uu = np.mgrid[0:params.out_h, 0:params.out_w]
        pixels = np.stack([uu.ravel(), vv.ravel()], axis=1)
    pixels = np.asarray(pixels, dtype=np.int64)
    n = pixels.shape[0]
    pu = np.ascontiguousarray(pixels[:, 0], dtype=np.int32)
    pv = np.ascontiguousarray(pixels[:, 1], dtype=np.int32)
    m = _Marshal(sensors, params)
    NL = n_levels(params)
    out = np.empty((n, 3))
    choice = np.empty((n, 3), dtype=np.int32)
    margin = np.empty((n, 3))
    lv = {}
    if levels or kappa:
        lv = dict(c0=np.empty((n, 3, NL)), var=np.empty((n, 3, NL)), pivot=np.empty((n, 3, NL)),
                  count=np.empty((n, 3, NL), dtype=np.int32), valid=np.empty((n, 3, NL), dtype=np.int32),
                  efit=np.empty((n, 3, NL)), ew=np.empty((n, 3, NL)))
        if kappa:
            lv["kappa"] = np.empty((n, 3, NL))
    q = None
    if metric is not None:
        metric = np.asarray(metric, dtype=np.float64)
        q = np.ascontiguousarray(metric[pv, pu].reshape(n, 3))
    rc = lib.orc_reconstruct(ctypes.byref(m.arr), m.n, ctypes.byref(m.params), n, _ptr(pu), _ptr(pv), _ptr(q),
                             _ptr(out), _ptr(choice), _ptr(margin), _ptr(lv.get("c0")), _ptr(lv.get("var")),
                             _ptr(lv.get("pivot")), _ptr(lv.get("kappa")), _ptr(lv.get("count")),
                             _ptr(lv.get("valid")), _ptr(lv.get("efit")), _ptr(lv.get("ew")))
    if rc != 0:
        raise ValueError(f"orc_reconstruct rejected its arguments (code {rc})")
    res = dict(out=out, choice=choice, margin=margin, **lv)
    if grid:
        H, W = params.out_h, params.out_w
        res["out"] = out.reshape(H, W, 3).transpose(2, 0, 1).copy()
        res["choice"] = choice.reshape(H, W, 3).transpose(2, 0, 1).copy()
        res["margin"] = margin.reshape(H, W, 3).transpose(2, 0, 1).copy()
    res["pixels"] = pixels
    return res


def gradients(sensors: Sequence, params, grad_sigma: float, pixels: Optional[np.ndarray] = None,
              diagnostics: bool = False):
    """First pass of the adaptive reconstruction (Section 5.4, green channel as in Section 5.5):
    the gradient (c1, c2) of the isotropic order-1 G fit at scale grad_sigma (R/B units) at each
    output pixel; 0 where the fit is not usable. Whole grid: [out_h, out_w, 2]; `pixels` ([n, 2] of
    (u, v)): [n, 2]. With `diagnostics`, returns a dict with `grad` and, per pixel, the fit's
    smallest equilibrated pivot `pivot`, sample `count` and the rounding scales `efit`, `ew` of c1
    and c2 ([..., 2], as reconstruct() reports them for C_0)."""
    lib = _load()
    grid = pixels is None
    if grid:
        vv, uu = np.mgrid[0:params.out_h, 0:params.out_w]
        pixels = np.stack([uu.ravel(), vv.ravel()], axis=1)
    pixels = np.asarray(pixels, dtype=np.int64)
    pu = np.ascontiguousarray(pixels[:, 0], dtype=np.int32)
    pv = np.ascontiguousarray(pixels[:, 1], dtype=np.int32)
    n = pu.size
    m = _Marshal(sensors, params)
    gx = np.empty(n)
    gy = np.empty(n)
    dg = {}
    if diagnostics:
        dg = dict(pivot=np.empty(n), count=np.empty(n, dtype=np.int32), efit=np.empty((n, 2)), ew=np.empty((n, 2)))
    rc = lib.orc_gradients(ctypes.byref(m.arr), m.n, ctypes.byref(m.params), float(grad_sigma), n, _ptr(pu), _ptr(pv),
                           _ptr(gx), _ptr(gy), _ptr(dg.get("pivot")), _ptr(dg.get("count")), _ptr(dg.get("efit")),
                           _ptr(dg.get("ew")))
    if rc != 0:
        raise ValueError(f"orc_gradients rejected its arguments (code {rc})")
    shape = (params.out_h, params.out_w) if grid else (n,)
    g = np.stack([gx, gy], axis=1).reshape(*shape, 2)
    if not diagnostics:
        return g
    return dict(grad=g, pivot=dg["pivot"].reshape(shape), count=dg["count"].reshape(shape),
                efit=dg["efit"].reshape(*shape, 2), ew=dg["ew"].reshape(*shape, 2))


def steering_metric(grad: np.ndarray, window_sigma: float, alpha: float, lambda1: float = 1.0,
                    lambda2: float = 0.001, min_eig: float = 0.25, max_eig: float = 16.0,
                    grad_scale: float = 1.0) -> np.ndarray:
    """Second pass (Section 5.4): per output pixel the steering matrix C_j (as {C11, C12, C22}) from
    the gradients `grad` [H, W, 2] of the output pixels within 3 window_sigma (Gaussian weights
    w_i, pixels inside the image only; M = their number). The singular values s1 >= s2 and right
    singular vectors u1, u2 of the weighted gradient matrix (rows sqrt(w_i) g_i) are those of
    T = sum_i w_i g_i g_i^T; elongation sigma_j = (s1 + lambda1) / (s2 + lambda1), scaling
    gamma_j = ((s1 s2 + lambda2) / M)^alpha, and C_j = gamma_j (sigma_j u1 u1^T + u2 u2^T / sigma_j)
    (reading: the window exp(-d^T C_j d / (2 sigma^2)) is narrow across the dominant gradient and
    long along it), its two eigenvalues clamped to [min_eig, max_eig] (reading: bounds the window).
    `grad_scale` multiplies the gradients first (the unit of the radiant power, which the paper's
    fixed lambda1 and lambda2 presuppose but do not state)."""
    g = np.asarray(grad, dtype=np.float64) * grad_scale
    H, W = g.shape[:2]
    r = int(np.floor(3.0 * window_sigma))
    T = np.zeros((H, W, 3))
    M = np.zeros((H, W))
    for dj in range(-r, r + 1):
        for di in range(-r, r + 1):
            if di * di + dj * dj > (3.0 * window_sigma) ** 2:
                continue
            w = np.exp(-(di * di + dj * dj) / (2.0 * window_sigma ** 2))
            v0, v1 = max(0, -dj), min(H, H - dj)
            u0, u1 = max(0, -di), min(W, W - di)
            gs = g[v0 + dj:v1 + dj, u0 + di:u1 + di]
            T[v0:v1, u0:u1, 0] += w * gs[..., 0] * gs[..., 0]
            T[v0:v1, u0:u1, 1] += w * gs[..., 0] * gs[..., 1]
            T[v0:v1, u0:u1, 2] += w * gs[..., 1] * gs[..., 1]
            M[v0:v1, u0:u1] += 1.0
    a, b, c = T[..., 0], T[..., 1], T[..., 2]
    h = 0.5 * (a + c)
    d = np.sqrt((0.5 * (a - c)) ** 2 + b * b)
    l1, l2 = h + d, np.maximum(h - d, 0.0)
    s1, s2 = np.sqrt(l1), np.sqrt(l2)
    # eigenvector of l1: (b, l1 - a) or (l1 - c, b), whichever is longer; (1, 0) if T is diagonal with a >= c
    e1x, e1y = b, l1 - a
    f1x, f1y = l1 - c, b
    use_f = f1x * f1x + f1y * f1y > e1x * e1x + e1y * e1y
    ux = np.where(use_f, f1x, e1x)
    uy = np.where(use_f, f1y, e1y)
    nrm = np.sqrt(ux * ux + uy * uy)
    iso = nrm == 0.0
    ux = np.where(iso, 1.0, ux / np.where(iso, 1.0, nrm))
    uy = np.where(iso, 0.0, uy / np.where(iso, 1.0, nrm))
    elong = (s1 + lambda1) / (s2 + lambda1)
    gamma = ((s1 * s2 + lambda2) / M) ** alpha
    ea = np.clip(gamma * elong, min_eig, max_eig)   # along u1 (across the edge)
    eb = np.clip(gamma / elong, min_eig, max_eig)   # along u2 = (-uy, ux)
    C11 = ea * ux * ux + eb * uy * uy
    C12 = (ea - eb) * ux * uy
    C22 = ea * uy * uy + eb * ux * ux
    return np.stack([C11, C12, C22], axis=2)


def condition(A: np.ndarray) -> float:
    """2-norm condition number max|lambda| / min|lambda| of a symmetric matrix (at most 6 x 6) by the
    oracle's cyclic Jacobi eigen-iteration (the routine behind the `kappa` diagnostics)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("square matrix expected")
    return float(_load().orc_condition(_ptr(A), A.shape[0]))


class ValueSensor:
    """A sensor in value mode: the radiant power estimate and its variance per pixel (excluded
    pixels: variance +inf) with the sensor's transform."""

    def __init__(self, width, height, affine, value_f, value_var):
        self.width, self.height = int(width), int(height)
        self.affine = np.asarray(affine, dtype=np.float64).reshape(2, 3)
        self.value_f, self.value_var = value_f, value_var
        self.gain = self.exposure = self.nd = self.read_var = 1.0
        self.black, self.sat = 0.0, 1e300
        self.bias_frame = self.prnu_frame = self.read_var_frame = self.sat_frame = None


def value_sensors(sensors: Sequence, round_to=None) -> List[ValueSensor]:
    """The value-mode sensors of raw sensors: Eq. 18's f and Eq. 20's s2 of every pixel (Section 6,
    saturated pixels excluded). With `round_to` (e.g. np.float32) f and the inverse variance 1/s2
    (the factor the weight uses) are rounded to that type: the inputs a lower-precision path
    starts from."""
    lib = _load()
    out = []
    for s in sensors:
        m = _Marshal([s], _DefaultParams())
        f = np.empty((s.height, s.width))
        s2 = np.empty((s.height, s.width))
        if lib.orc_radiometry_frame(ctypes.byref(m.arr), _ptr(f), _ptr(s2)) != 0:
            raise ValueError("value_sensors needs raw sensors")
        if round_to is not None:
            f = f.astype(round_to).astype(np.float64)
            with np.errstate(divide="ignore"):
                iv = (1.0 / s2).astype(round_to).astype(np.float64)
                s2 = np.where(iv > 0, 1.0 / iv, np.inf)
        out.append(ValueSensor(s.width, s.height, s.affine, f, s2))
    return out


class _DefaultParams:
    order, sigmas, green_ratio, trunc_k, ici_gamma, min_pivot = 0, (1.0,), 1.0, 3.0, 2.0, 1e-3
    out_affine = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])


def radiometry(y, b, g, t, a, n, read_var, sat):
    """Eqs. 18 and 20 for one digital value; returns (excluded, f, s2)."""
    lib = _load()
    f = ctypes.c_double()
    s2 = ctypes.c_double()
    ex = lib.orc_radiometry(float(y), float(b), float(g), float(t), float(a), float(n), float(read_var),
                            float(sat), ctypes.addressof(f), ctypes.addressof(s2))
    return bool(ex), f.value, s2.value


def ici(c0: Sequence[float], var: Sequence[float], valid: Sequence[int], gamma: float):
    """The scale-choice rule on given intervals; returns (chosen index or -1, margin)."""
    lib = _load()
    c0 = np.ascontiguousarray(c0, dtype=np.float64)
    var = np.ascontiguousarray(var, dtype=np.float64)
    valid = np.ascontiguousarray(valid, dtype=np.int32)
    mg = ctypes.c_double()
    ch = lib.orc_ici(len(c0), _ptr(c0), _ptr(var), _ptr(valid), float(gamma), ctypes.addressof(mg))
    return ch, mg.value


def equivalent_kernel(sensors, params, u: int, v: int, c: int, sigma: float, order: int, cap: int = 4096):
    """Equivalent kernel of one fit: dict of per-sample arrays, or None if the fit is not usable."""
    lib = _load()
    m = _Marshal(sensors, params)
    bufs = dict(sensor=np.zeros(cap, np.int32), x=np.zeros(cap, np.int32), y=np.zeros(cap, np.int32),
                dx=np.zeros(cap), dy=np.zeros(cap), f=np.zeros(cap), ell=np.zeros(cap))
    k = lib.orc_equivalent_kernel(ctypes.byref(m.arr), m.n, ctypes.byref(m.params), int(u), int(v), int(c),
                                  float(sigma), int(order), cap, *(_ptr(bufs[x]) for x in
                                                                   ("sensor", "x", "y", "dx", "dy", "f", "ell")))
    if k == -1:
        return None
    if k < 0:
        raise ValueError(f"orc_equivalent_kernel rejected its arguments (code {k})")
    k = min(k, cap)
    return {key: val[:k] for key, val in bufs.items()}


def adaptive(sensors: Sequence, params, grad_sigma: float, window_sigma: float, alpha: float,
             lambda1: float = 1.0, lambda2: float = 0.001, min_eig: float = 0.25, max_eig: float = 16.0,
             pixels: Optional[np.ndarray] = None, levels: bool = False, kappa: bool = False,
             grad_scale: float = 1.0):
    """The adaptive reconstruction of Sections 5.4-5.5 (CALPA): gradients of the green channel,
    the steering matrix per output pixel, then the fit of every channel with the steered window.
    Returns reconstruct()'s dict plus `grad` and `metric` (whole output grid)."""
    g = gradients(sensors, params, grad_sigma)
    q = steering_metric(g, window_sigma, alpha, lambda1, lambda2, min_eig, max_eig, grad_scale)
    res = reconstruct(sensors, params, pixels, levels=levels, kappa=kappa, metric=q)
    res["grad"] = g
    res["metric"] = q
    return res
