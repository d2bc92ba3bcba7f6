"""Seeded synthetic inputs: scene, sensor rig and raw Bayer frames.

This module is the camera *simulator* (the forward model of Section 3 and the
noise model of Section 6, Eqs. 16-17). It holds none of the reconstruction's
arithmetic: no radiometric inversion, no window weights, no fitting. Both the
CUDA path's tests/benchmark and the FP64 oracle draw their inputs from here.

Recipe (stands in for the paper's simulated Kodak KAI-04050 / Canon rigs of
Section 7 and the 4-Mpixel camera of Section 8, whose HR scenes and captures
are not available):

* scene: log10-radiance L = -2 + 6*clip(S, 0, 1), S = 1/2 + 5/4 * (a normalised
  sum of three random linear ramps and two low-frequency separable cosines),
  plus eight random straight step edges, each a jump of +-U(0.5, 2) decades
  split evenly across the edge (-jump/2 on one side, +jump/2 on the other), so
  that L covers [-2, 4] roughly uniformly; every channel gets its own
  tint U(-0.3, 0.3) decades per region (base tint plus a per-edge tint jump);
  clipped to [-2, 4], so the radiance spans 1e-2 .. 1e4 (electrons per unit time
  at n = 1).
* rig: per-sensor affine T_s (sensor px -> reference px) made of a rotation and
  isotropic scale about the sensor centre ((W-1)/2, (H-1)/2) plus a translation.
* noise: e ~ Poisson(t * a * n * f) (Eq. 16), y = round(g*e + N(0, Var r) + b)
  clipped to [0, 4095] (Eq. 17 with a black pedestal b so read noise is not
  clipped at zero), gain g = 2 DN/e- ("0.5 e-/DN"), read noise sigma 3 DN,
  b = 64 DN, 12-bit clip level 4095 which is also the saturation threshold.
* CFA: RGGB Bayer, (x even, y even) = R, (x odd, y odd) = B, other sites G
  (Section 2.5).

Seeds: configuration i uses base seed 1000 + i; sub-streams are derived with
numpy's SeedSequence spawning keyed by (seed, purpose, index).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

CLIP_DN = 4095
BLACK_DN = 64.0
GAIN_DN_PER_E = 2.0
READ_SIGMA_DN = 3.0


def _rng(seed: int, *key: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed), *map(int, key)]))


def pitch_for(width: int) -> int:
    """Row pitch in uint16 elements: a multiple of 8 (16 bytes) for bulk tensor copies."""
    return (int(width) + 7) // 8 * 8


def affine_about_center(width: int, height: int, tx: float = 0.0, ty: float = 0.0,
                        rot_deg: float = 0.0, scale: float = 1.0) -> np.ndarray:
    """2x3 row-major affine sensor px -> reference px: rotate/scale about the sensor centre, then translate."""
    cx, cy = (width - 1) / 2.0, (height - 1) / 2.0
    th = math.radians(rot_deg)
    c, s = math.cos(th) * scale, math.sin(th) * scale
    m = np.array([[c, -s, 0.0], [s, c, 0.0]], dtype=np.float64)
    m[0, 2] = cx + tx - (c * cx - s * cy)
    m[1, 2] = cy + ty - (s * cx + c * cy)
    return m


def apply_affine(m: np.ndarray, x: np.ndarray, y: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    m = np.asarray(m, dtype=np.float64).reshape(2, 3)
    return m[0, 0] * x + m[0, 1] * y + m[0, 2], m[1, 0] * x + m[1, 1] * y + m[1, 2]


def cfa_color(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """RGGB colour index per sensor pixel: 0 = R, 1 = G, 2 = B."""
    x = np.asarray(x) & 1
    y = np.asarray(y) & 1
    return np.where((x == 0) & (y == 0), 0, np.where((x == 1) & (y == 1), 2, 1))


# --------------------------------------------------------------------------- scenes

@dataclasses.dataclass
class Scene:
    """Analytic HDR scene in reference coordinates. `radiance(c, X, Y)` is point-sampled."""
    width: float
    height: float
    ramps: np.ndarray        # [3, 3] (amplitude, angle, unused)
    cosines: np.ndarray      # [2, 5] (amplitude, fx, phx, fy, phy)
    edges: np.ndarray        # [8, 4] (px, py, angle, jump)
    edge_tint: np.ndarray    # [8, 3]
    base_tint: np.ndarray    # [3]
    constant: Optional[float] = None    # constant-radiance scene (all channels)

    def log_radiance(self, c: int, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
        X = np.asarray(X, dtype=np.float64)
        Y = np.asarray(Y, dtype=np.float64)
        if self.constant is not None:
            return np.full(np.broadcast(X, Y).shape, math.log10(self.constant))
        u = X / self.width
        v = Y / self.height
        acc = np.zeros(np.broadcast(u, v).shape)
        norm = 0.0
        for amp, ang, _ in self.ramps:
            acc = acc + amp * (np.cos(ang) * (u - 0.5) + np.sin(ang) * (v - 0.5))
            norm += abs(amp) * 0.75
        for amp, fx, phx, fy, phy in self.cosines:
            acc = acc + amp * np.cos(2 * np.pi * (fx * u + phx)) * np.cos(2 * np.pi * (fy * v + phy))
            norm += abs(amp)
        s = 0.5 + 1.25 * acc / norm
        L = -2.0 + 6.0 * np.clip(s, 0.0, 1.0) + self.base_tint[c]
        for k, (px, py, ang, jump) in enumerate(self.edges):
            side = np.where((np.cos(ang) * (u - px) + np.sin(ang) * (v - py)) > 0, 0.5, -0.5)
            L = L + side * (jump + self.edge_tint[k, c])
        return np.clip(L, -2.0, 4.0)

    def radiance(self, c: int, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
        return np.power(10.0, self.log_radiance(c, X, Y))


def make_scene(seed: int, width: float, height: float) -> Scene:
    r = _rng(seed, 1)
    ramps = np.stack([r.uniform(0.5, 1.0, 3), r.uniform(0, 2 * np.pi, 3), np.zeros(3)], axis=1)
    cos = np.stack([r.uniform(0.3, 0.7, 2), r.uniform(0.5, 3.0, 2), r.uniform(0, 1, 2),
                    r.uniform(0.5, 3.0, 2), r.uniform(0, 1, 2)], axis=1)
    jumps = r.uniform(0.5, 2.0, 8) * r.choice([-1.0, 1.0], 8)
    edges = np.stack([r.uniform(0.1, 0.9, 8), r.uniform(0.1, 0.9, 8), r.uniform(0, 2 * np.pi, 8), jumps], axis=1)
    edge_tint = r.uniform(-0.3, 0.3, (8, 3))
    base_tint = r.uniform(-0.3, 0.3, 3)
    return Scene(float(width), float(height), ramps, cos, edges, edge_tint, base_tint)


def constant_scene(value: float, width: float = 1.0, height: float = 1.0) -> Scene:
    z = np.zeros((0, 3))
    return Scene(float(width), float(height), z, np.zeros((0, 5)), np.zeros((0, 4)), np.zeros((0, 3)),
                 np.zeros(3), constant=float(value))


# --------------------------------------------------------------------------- rig

@dataclasses.dataclass
class Sensor:
    """One sensor s: raw layout, exposure/noise parameters and its transform T_s (Sections 3, 4.2, 6)."""
    width: int
    height: int
    nd: float                         # exposure scaling n_s
    affine: np.ndarray                # T_s, 2x3 sensor px -> reference px
    gain: float = GAIN_DN_PER_E       # g_s in DN per electron
    exposure: float = 1.0             # t_s
    read_var: float = READ_SIGMA_DN ** 2
    black: float = BLACK_DN
    sat: int = CLIP_DN
    pitch: int = 0
    raw: Optional[np.ndarray] = None  # uint16 [height, pitch]
    # optional per-pixel calibration frames [height, width]
    bias_frame: Optional[np.ndarray] = None
    prnu_frame: Optional[np.ndarray] = None
    read_var_frame: Optional[np.ndarray] = None
    sat_frame: Optional[np.ndarray] = None

    def __post_init__(self):
        if not self.pitch:
            self.pitch = pitch_for(self.width)
        self.affine = np.asarray(self.affine, dtype=np.float64).reshape(2, 3)


def simulate_raw(scene: Scene, sensor: Sensor, seed: int, index: int, noise: bool = True) -> np.ndarray:
    """Raw uint16 frame [height, pitch] of `scene` seen through `sensor` (Eqs. 16-17)."""
    H, W = sensor.height, sensor.width
    ys, xs = np.mgrid[0:H, 0:W]
    X, Y = apply_affine(sensor.affine, xs.astype(np.float64), ys.astype(np.float64))
    col = cfa_color(xs, ys)
    f = np.empty((H, W))
    for c in range(3):
        m = col == c
        f[m] = scene.radiance(c, X[m], Y[m])
    a = sensor.prnu_frame if sensor.prnu_frame is not None else 1.0
    b = sensor.bias_frame if sensor.bias_frame is not None else sensor.black
    rv = sensor.read_var_frame if sensor.read_var_frame is not None else sensor.read_var
    mean_e = sensor.exposure * a * sensor.nd * f
    if noise:
        r = _rng(seed, 2, index)
        e = r.poisson(mean_e).astype(np.float64)
        y = sensor.gain * e + r.standard_normal((H, W)) * np.sqrt(rv) + b
    else:
        y = sensor.gain * mean_e + b
    y = np.clip(np.rint(y), 0, CLIP_DN).astype(np.uint16)
    out = np.zeros((H, sensor.pitch), dtype=np.uint16)
    out[:, :W] = y
    return out


@dataclasses.dataclass
class Params:
    """Reconstruction parameters (Section 5.3; scale selection rule for several scales)."""
    order: int = 2
    sigmas: Tuple[float, ...] = (0.7,)
    green_ratio: float = 1.0 / math.sqrt(2.0)
    trunc_k: float = 3.0
    ici_gamma: float = 2.0
    out_w: int = 0
    out_h: int = 0
    out_affine: Optional[np.ndarray] = None   # output px -> reference px
    min_pivot: float = 1e-3
    cond_fallback: float = 1e6
    out_dtype: int = 0        # 0 float32, 1 float16
    accum: int = 0            # 0 plain, 1 compensated
    tab_weights: int = 1      # 1 tabulated window weights where the rig allows, 0 never
    weight_mode: int = 0      # 0 noise weight K / s2, 1 the printed K / s (Eq. 6)

    def __post_init__(self):
        if self.out_affine is None:
            self.out_affine = np.array([[1.0, 0, 0], [0, 1.0, 0]])
        self.out_affine = np.asarray(self.out_affine, dtype=np.float64).reshape(2, 3)
        self.sigmas = tuple(float(s) for s in self.sigmas)


def output_affine(ref_w: int, ref_h: int, out_w: int, out_h: int) -> np.ndarray:
    """Centre-aligned output grid: P = (u + 0.5)/s - 0.5 per axis, s = out/ref."""
    sx, sy = out_w / ref_w, out_h / ref_h
    return np.array([[1 / sx, 0.0, 0.5 / sx - 0.5], [0.0, 1 / sy, 0.5 / sy - 0.5]])


@dataclasses.dataclass
class Frame:
    sensors: List[Sensor]
    params: Params
    scene: Scene
    name: str = ""


def _build_frame(seed: int, n_sensors: int, w: int, h: int, nds: Sequence[float],
                 trans: float, rot_deg: float, scale_eps: float, params: Params,
                 name: str, noise: bool = True, scene: Optional[Scene] = None,
                 frame_index: int = 0, rig_index: Optional[int] = None) -> Frame:
    r = _rng(seed, 0, frame_index if rig_index is None else rig_index)
    scene = scene if scene is not None else make_scene(seed, w, h)
    sensors = []
    for s in range(n_sensors):
        tx, ty = r.uniform(-trans, trans, 2) if trans > 0 else (0.0, 0.0)
        rot = r.uniform(-rot_deg, rot_deg) if rot_deg > 0 else 0.0
        sc = 1.0 + (r.uniform(-scale_eps, scale_eps) if scale_eps > 0 else 0.0)
        sen = Sensor(w, h, nds[s], affine_about_center(w, h, tx, ty, rot, sc))
        sen.raw = simulate_raw(scene, sen, seed, 100 * frame_index + s, noise=noise)
        sensors.append(sen)
    return Frame(sensors, params, scene, name)


# --------------------------------------------------------------------------- the workloads

PAPER_SCALES = (0.5, 0.8, 1.2, 1.8)


def tiny(seed: int = 1001) -> Frame:
    """2 sensors of 64x64, ND 1 and 1/8, translation U(-1,1) px, order 0, one scale 0.7 px, 64x64 output."""
    p = Params(order=0, sigmas=(0.7,), out_w=64, out_h=64)
    return _build_frame(seed, 2, 64, 64, (1.0, 1 / 8), 1.0, 0.0, 0.0, p, "tiny-2x64x64-M0")


def paper_scale(seed: int = 1002, size: int = 2048, out_size: Optional[int] = None) -> Frame:
    """3 sensors of size^2 (2048^2 at full scale), ND 1, 1/16, 1/256, affine misalignment, order 2, 4 scales."""
    o = out_size or size
    p = Params(order=2, sigmas=PAPER_SCALES, out_w=o, out_h=o,
               out_affine=output_affine(size, size, o, o))
    return _build_frame(seed, 3, size, size, (1.0, 1 / 16, 1 / 256), 1.5, 0.2, 1e-3, p,
                        f"paper-3x{size}x{size}-M2-ICI4")


PAPER_CAMERA_SIZE = (2336, 1752)


def paper_camera(seed: int = 1009, translational: bool = True, sigma: float = 0.7) -> Frame:
    """The four-sensor camera of Section 8 as a synthetic rig: 4 x 2336x1752 RGGB 12-bit sensors
    whose exposure scalings span 1 : 2^12 (ND 1, 1/16, 1/256, 1/4096), gain 0.27 DN/e- and read
    noise 72 e- (Section 8), exposure time 2 / 0.27 (the raw levels of the other workloads, whose
    sensors have 2 DN/e-); misaligned by translations of up to 3 px and, unless `translational`,
    rotations of up to 0.3 degrees; order 0, one scale `sigma`, output 2336x1752 at 1x."""
    w, h = PAPER_CAMERA_SIZE
    r = _rng(seed, 0, 0 if translational else 1)
    scene = make_scene(seed, w, h)
    sensors = []
    for s, nd in enumerate((1.0, 1 / 16, 1 / 256, 1 / 4096)):
        tx, ty = r.uniform(-3.0, 3.0, 2)
        rot = 0.0 if translational else r.uniform(-0.3, 0.3)
        sen = Sensor(w, h, nd, affine_about_center(w, h, tx, ty, rot), gain=0.27, exposure=2.0 / 0.27,
                     read_var=(72.0 * 0.27) ** 2)
        sen.raw = simulate_raw(scene, sen, seed, s)
        sensors.append(sen)
    p = Params(order=0, sigmas=(sigma,), out_w=w, out_h=h)
    return Frame(sensors, p, scene, f"paper-camera-4x{w}x{h}-M0-{'translational' if translational else 'rotated'}")


def precision(seed: int = 1003, size: int = 2048, order: int = 0) -> Frame:
    """Tiny recipe (2 sensors, ND 1 and 1/8, U(-1,1) translation, sigma 0.7) at size^2 raw -> 2x upsampled output."""
    o = 2 * size
    p = Params(order=order, sigmas=(0.7,), out_w=o, out_h=o, out_affine=output_affine(size, size, o, o))
    return _build_frame(seed, 2, size, size, (1.0, 1 / 8), 1.0, 0.0, 0.0, p, f"precision-2x{size}->{o}-M{order}")


BATCH_SIZES = ((512, 512), (1280, 720), (1920, 1080), (2048, 2048))
BATCH_NDS = (1.0, 1 / 8, 1 / 64, 1 / 512)


def batching_specs(seed: int = 1004, n_frames: int = 16, size_cap: Optional[int] = None) -> List[tuple]:
    """The drawn shape of each batching frame: (seed, k, sensors, w, h, order, output scale)."""
    r = _rng(seed, 5)
    specs = []
    for k in range(n_frames):
        w, h = BATCH_SIZES[r.integers(0, len(BATCH_SIZES))]
        if size_cap:
            w, h = min(w, size_cap), min(h, size_cap)
        ns = int(r.integers(2, 5))
        order = int(r.integers(0, 3))
        osc = (1.0, 1.5)[r.integers(0, 2)]
        specs.append((seed, k, ns, int(w), int(h), order, osc))
    return specs


def batching_frame(spec: tuple) -> Frame:
    seed, k, ns, w, h, order, osc = spec
    ow, oh = int(round(w * osc)), int(round(h * osc))
    p = Params(order=order, sigmas=PAPER_SCALES, out_w=ow, out_h=oh, out_affine=output_affine(w, h, ow, oh))
    return _build_frame(seed * 100 + k, ns, w, h, BATCH_NDS[:ns], 1.5, 0.2, 1e-3, p,
                        f"batch{k}-{ns}x{w}x{h}-M{order}-x{osc}", frame_index=k)


def batching(seed: int = 1004, n_frames: int = 16, size_cap: Optional[int] = None) -> List[Frame]:
    """16 frames of drawn size, 2-4 sensors, order 0-2, output scale 1 or 1.5; 4 scales with ICI."""
    return [batching_frame(sp) for sp in batching_specs(seed, n_frames, size_cap)]


SERVING_STREAMS = (
    # (raw w, raw h, sensors, out w, out h)
    (1280, 720, 2, 1280, 720), (1280, 720, 2, 1280, 720),
    (1920, 1080, 3, 1920, 1080), (1920, 1080, 3, 1920, 1080), (1920, 1080, 3, 1920, 1080),
    (2048, 2048, 3, 2048, 2048), (2048, 2048, 3, 2048, 2048),
    (2048, 2048, 3, 3840, 2160),
)


def serving_stream_frame(stream: int, k: int, seed: int = 1005, size_cap: Optional[int] = None) -> Frame:
    """Frame k of serving stream m: one scene and one rig geometry per stream (seed 100*seed + m),
    fresh noise per frame; order 2, 4 scales with ICI. size_cap shrinks the raw and output sizes."""
    w, h, ns, ow, oh = SERVING_STREAMS[stream]
    if size_cap:
        sx, sy = min(1.0, size_cap / w), min(1.0, size_cap / h)
        w, h, ow, oh = int(w * sx) // 8 * 8, int(h * sy) // 2 * 2, int(ow * sx) // 8 * 8, int(oh * sy) // 2 * 2
    p = Params(order=2, sigmas=PAPER_SCALES, out_w=ow, out_h=oh, out_affine=output_affine(w, h, ow, oh))
    return _build_frame(100 * seed + stream, ns, w, h, (1.0, 1 / 16, 1 / 256)[:ns], 1.5, 0.2, 1e-3, p,
                        f"serve{stream}.{k}", frame_index=k, rig_index=0)


# --------------------------------------------------------------------------- calibration stacks

def flat_stack(seed: int, n_frames: int, width: int, height: int, electrons: float, gain: float = 2.0,
               read_var: float = 9.0, bias: float = 64.0, nd: float = 1.0,
               prnu: Optional[np.ndarray] = None) -> np.ndarray:
    """n_frames raw frames [n, height, pitch] of a uniform flat field (Eqs. 16-17): per pixel
    Poisson(electrons * nd * a) photo-electrons times `gain`, plus N(0, read_var) read noise and
    the `bias` pedestal, rounded and clipped to 12 bits. electrons = 0 gives black frames."""
    r = _rng(seed, 7)
    pitch = pitch_for(width)
    out = np.zeros((n_frames, height, pitch), dtype=np.uint16)
    a = prnu if prnu is not None else 1.0
    for k in range(n_frames):
        e = r.poisson(electrons * nd * a * np.ones((height, width))).astype(np.float64)
        y = gain * e + r.standard_normal((height, width)) * np.sqrt(read_var) + bias
        out[k, :, :width] = np.clip(np.rint(y), 0, CLIP_DN).astype(np.uint16)
    return out
