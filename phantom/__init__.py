"""Seeded synthetic CT phantoms: the inputs shared by the tests, the oracle runs
and the benchmark.

This module holds none of the registration arithmetic (no trilinear warp, no
gradient, no force, no smoothing).  Every image is an analytic function of the
continuous position -- layered ellipsoids with 0.5-voxel logistic edges -- so
the moving image is produced by evaluating that function at deformed
positions, never by resampling a voxel grid.

Stand-ins for the paper's clinical data (Sec. 2.3: planning / treatment CT of
head-and-neck and pelvic patients, 1.97 x 1.97 x 2.5 mm voxels; HN4 was
240 x 160 x 70, Sec. 3), which is not available:

* ``phantom64``     64x64x32, air / body / bone shell / two brighter organs,
                    noise sigma 20 HU, 4 bumps <= 4 voxels, 1 level x 100
                    iterations, contour weight 1.
* ``headneck256``   256x256x96, fat / soft tissue / mandible / vertebra ring,
                    cord, two parotids and a target at tissue +-15 HU,
                    noise 25 HU, 8 bumps <= 8 voxels, 3 levels 100/50/25.
* ``pelvis512``     512x512x160, bladder / prostate / rectum / femoral heads /
                    target; the moving image is CBCT-like (noise 40 HU, a
                    +-5% smooth multiplicative bias and radial streaks),
                    bumps <= 12 voxels on bladder and rectum, 3 levels.
* ``batch_mix``     the uneven-size mix {128x128x64, 256x256x96, 384x384x128,
                    512x512x160}, 2-8 masks, bumps <= 10 voxels.

Deformation model: the ground-truth DVF ``u_gt`` is a sum of Gaussian bumps in
voxel units (component order x, y, z).  The warp convention is pull-back:
the moving image satisfies ``moving(x + u_gt(x)) == static_clean(x)``.  To
build it, ``w`` = the inverse of ``u_gt`` is found by the fixed-point
iteration ``w(y) = -u_gt(y + w(y))`` and the analytic phantom is evaluated at
``y + w(y)``.  Bump amplitudes are capped so the displacement gradient stays
below 0.5, which keeps that iteration a contraction.

Arrays are C-ordered ``[nz][ny][nx]`` (x fastest); DVFs are ``[3][nz][ny][nx]``.
Seeds: case seed = 1000 * config number + case index (NumPy PCG64).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
import torch

__all__ = ["Case", "CONFIGS", "make_case", "make_case_device", "config_names", "batch_mix_cases",
           "batch_mix_specs", "voxel_iters"]

AIR = -1000.0


@dataclasses.dataclass
class Layer:
    """One painted structure.  ``centre`` and ``axes`` are fractions of the
    volume extent per axis (x, y, z); ``shell`` > 0 makes a hollow shell of that
    many voxels; ``cut`` = (axis, direction, position) keeps one side of a plane."""
    name: str
    hu: float
    centre: Tuple[float, float, float]
    axes: Tuple[float, float, float]
    shell: float = 0.0
    cut: Optional[Tuple[int, float, float]] = None
    painted: bool = True      # False: a mask-only structure (e.g. a target margin)


@dataclasses.dataclass
class Config:
    number: int
    name: str
    shape: Tuple[int, int, int]          # (nz, ny, nx)
    layers: List[Layer]
    masks: List[str]                      # layer names used as structure masks
    body: str                             # layer whose interior receives the bumps
    noise_static: float
    noise_moving: float
    n_bumps: int
    cap: float                            # max |u_gt| in voxels at the default shape
    levels: int
    iters: Tuple[int, ...]                # coarse -> fine
    lam: float                            # contour weight, one value for every mask
    bump_sites: Optional[List[str]] = None  # bump centres near these layers (else body)
    cbct: bool = False                    # CBCT-like moving image (bias + streaks)
    spacing_mm: Tuple[float, float, float] = (1.97, 1.97, 2.5)


def _hn_layers() -> List[Layer]:
    return [
        Layer("fat", -100.0, (0.5, 0.5, 0.5), (0.44, 0.38, 0.62)),
        Layer("tissue", 40.0, (0.5, 0.5, 0.5), (0.40, 0.34, 0.62)),
        Layer("mandible", 700.0, (0.5, 0.40, 0.38), (0.24, 0.20, 0.14), shell=2.0,
              cut=(1, -1.0, 0.40)),
        Layer("vertebra", 700.0, (0.5, 0.70, 0.5), (0.075, 0.075, 0.70), shell=2.0),
        Layer("cord", 35.0, (0.5, 0.70, 0.5), (0.040, 0.040, 0.70)),
        Layer("parotid_l", 55.0, (0.30, 0.52, 0.56), (0.075, 0.085, 0.13)),
        Layer("parotid_r", 55.0, (0.70, 0.52, 0.56), (0.075, 0.085, 0.13)),
        Layer("target", 25.0, (0.44, 0.44, 0.46), (0.065, 0.065, 0.09)),
    ]


def _pelvis_layers() -> List[Layer]:
    return [
        Layer("fat", -100.0, (0.5, 0.5, 0.5), (0.46, 0.36, 0.70)),
        Layer("tissue", 40.0, (0.5, 0.5, 0.5), (0.42, 0.32, 0.70)),
        Layer("femoral_l", 700.0, (0.27, 0.55, 0.50), (0.075, 0.075, 0.10)),
        Layer("femoral_r", 700.0, (0.73, 0.55, 0.50), (0.075, 0.075, 0.10)),
        Layer("bladder", 10.0, (0.5, 0.42, 0.62), (0.11, 0.085, 0.14)),
        Layer("prostate", 48.0, (0.5, 0.53, 0.42), (0.045, 0.04, 0.06)),
        Layer("rectum", 22.0, (0.5, 0.64, 0.45), (0.04, 0.04, 0.18)),
        Layer("target", 48.0, (0.5, 0.53, 0.42), (0.06, 0.055, 0.08), painted=False),
    ]


def _phantom64_layers() -> List[Layer]:
    return [
        Layer("body", -50.0, (0.5, 0.5, 0.5), (0.42, 0.38, 0.42)),
        Layer("bone", 700.0, (0.5, 0.5, 0.5), (0.36, 0.32, 0.38), shell=2.0),
        Layer("organ1", 20.0, (0.38, 0.45, 0.5), (0.11, 0.12, 0.20)),
        Layer("organ2", 40.0, (0.62, 0.55, 0.5), (0.10, 0.10, 0.18)),
    ]


CONFIGS: Dict[str, Config] = {
    "phantom64": Config(1, "phantom64", (32, 64, 64), _phantom64_layers(),
                        ["organ1", "organ2"], "body", 20.0, 20.0, 4, 4.0,
                        1, (100,), 1.0),
    "headneck256": Config(2, "headneck256", (96, 256, 256), _hn_layers(),
                          ["cord", "parotid_l", "parotid_r", "mandible", "target"],
                          "tissue", 25.0, 25.0, 8, 8.0, 3, (100, 50, 25), 1e-3),
    "pelvis512": Config(3, "pelvis512", (160, 512, 512), _pelvis_layers(),
                        ["prostate", "bladder", "rectum", "femoral_l", "femoral_r",
                         "target"], "tissue", 25.0, 40.0, 8, 12.0, 3, (100, 50, 25),
                        1e-3, bump_sites=["bladder", "rectum"], cbct=True),
}

BATCH_SHAPES = [(64, 128, 128), (96, 256, 256), (128, 384, 384), (160, 512, 512)]


def config_names() -> List[str]:
    return list(CONFIGS)


@dataclasses.dataclass
class Case:
    name: str
    seed: int
    static: np.ndarray          # float32 [nz,ny,nx], HU
    moving: np.ndarray          # float32 [nz,ny,nx], HU
    static_masks: np.ndarray    # uint8 [k,nz,ny,nx], 1 = inside
    moving_masks: np.ndarray    # uint8 [k,nz,ny,nx]
    u_gt: np.ndarray            # float32 [3,nz,ny,nx], voxel units, (x,y,z)
    body: np.ndarray            # uint8 [nz,ny,nx], static-space body region
    signs: List[int]            # +1 if the structure is brighter than its surroundings
    mask_names: List[str]
    spacing_mm: Tuple[float, float, float]
    levels: int
    iters: Tuple[int, ...]
    lam: List[float]

    @property
    def shape(self) -> Tuple[int, int, int]:
        return tuple(self.static.shape)

    @property
    def k(self) -> int:
        return int(self.static_masks.shape[0])


# --------------------------------------------------------------------------- #
# analytic phantom
# --------------------------------------------------------------------------- #
def _logistic(t):
    return 0.5 * (1.0 + torch.tanh(0.5 * t))


def _ellipsoid_signed_distance(px, py, pz, c, r):
    """Approximate signed distance (voxels) to an axis-aligned ellipsoid:
    exact along rays from the centre."""
    dx = (px - c[0]) / r[0]
    dy = (py - c[1]) / r[1]
    dz = (pz - c[2]) / r[2]
    rho = torch.sqrt(dx * dx + dy * dy + dz * dz)
    dist = torch.sqrt((px - c[0]) ** 2 + (py - c[1]) ** 2 + (pz - c[2]) ** 2)
    safe = torch.clamp(rho, min=1e-12)
    d = dist * (1.0 - 1.0 / safe)
    return torch.where(rho < 1e-9, torch.full_like(d, -min(r)), d)


def _layer_occupancy(layer: Layer, px, py, pz, shape, width=0.5):
    """Smooth occupancy in [0,1] of one layer at continuous voxel positions."""
    nz, ny, nx = shape
    ext = (nx, ny, nz)
    c = [layer.centre[a] * (ext[a] - 1) for a in range(3)]
    r = [max(layer.axes[a] * ext[a], 0.75) for a in range(3)]
    s = _logistic(-_ellipsoid_signed_distance(px, py, pz, c, r) / width)
    if layer.shell > 0:
        ri = [max(r[a] - layer.shell, 0.25) for a in range(3)]
        s = s * (1.0 - _logistic(-_ellipsoid_signed_distance(px, py, pz, c, ri) / width))
    if layer.cut is not None:
        axis, direction, pos = layer.cut
        p = (px, py, pz)[axis]
        s = s * _logistic(direction * (p - pos * (ext[axis] - 1)) / width)
    return s


def _paint(layers: Sequence[Layer], px, py, pz, shape) -> np.ndarray:
    v = torch.full(px.shape, AIR, dtype=torch.float64, device=px.device)
    for layer in layers:
        if not layer.painted:
            continue
        s = _layer_occupancy(layer, px, py, pz, shape)
        v = v * (1.0 - s) + layer.hu * s
    return v


def _grid(shape, device=None):
    nz, ny, nx = shape
    z, y, x = torch.meshgrid(torch.arange(nz, dtype=torch.float64, device=device),
                             torch.arange(ny, dtype=torch.float64, device=device),
                             torch.arange(nx, dtype=torch.float64, device=device), indexing="ij")
    return x, y, z


# --------------------------------------------------------------------------- #
# ground-truth deformation
# --------------------------------------------------------------------------- #
def _bump_field(bumps, px, py, pz):
    out = torch.zeros((3,) + tuple(px.shape), dtype=torch.float64, device=px.device)
    for (c, sig, amp) in bumps:
        g = torch.exp(-((px - c[0]) ** 2 + (py - c[1]) ** 2 + (pz - c[2]) ** 2)
                      / (2.0 * sig * sig))
        for a in range(3):
            out[a] += float(amp[a]) * g
    return out


def _sample_in_layer(rng, layer: Layer, shape, count, shrink=0.8):
    nz, ny, nx = shape
    ext = (nx, ny, nz)
    c = [layer.centre[a] * (ext[a] - 1) for a in range(3)]
    r = [layer.axes[a] * ext[a] * shrink for a in range(3)]
    pts = []
    while len(pts) < count:
        d = rng.uniform(-1.0, 1.0, size=3)
        if float(np.sum(d * d)) <= 1.0:
            pts.append([c[a] + d[a] * r[a] for a in range(3)])
    return pts


def _make_bumps(rng, cfg: Config, shape, cap):
    layers = {l.name: l for l in cfg.layers}
    sites = cfg.bump_sites or [cfg.body]
    centres = []
    for i in range(cfg.n_bumps):
        centres += _sample_in_layer(rng, layers[sites[i % len(sites)]], shape, 1,
                                    shrink=0.8 if cfg.bump_sites is None else 1.2)
    bumps = []
    for c in centres:
        sig = float(rng.uniform(max(2.0, 2.0 * cap), max(3.0, 3.0 * cap)))
        d = rng.normal(size=3)
        d /= max(np.linalg.norm(d), 1e-12)
        bumps.append((c, sig, d * float(rng.uniform(0.5, 1.0))))
    return bumps


def _scale_bumps(bumps, shape, cap, device=None):
    """Scale amplitudes so max |u_gt| == cap and the displacement gradient <= 0.5."""
    x, y, z = _grid(shape, device)
    u = _bump_field(bumps, x, y, z)
    mag = float(torch.sqrt((u * u).sum(dim=0)).max())
    if mag <= 0:
        return bumps, u
    scale = cap / mag
    grad = 0.0
    for a in range(3):
        for ax in range(3):
            if u.shape[3 - ax] > 1:
                grad = max(grad, float(torch.diff(u[a], dim=2 - ax).abs().max()))
    if grad * scale > 0.5:
        scale = 0.5 / grad
    return [(c, s, amp * scale) for (c, s, amp) in bumps], u * scale


def _invert(bumps, shape, tol=1e-5, max_iter=200, device=None):
    """w with w(y) = -u_gt(y + w(y)), by fixed-point iteration."""
    x, y, z = _grid(shape, device)
    w = -_bump_field(bumps, x, y, z)
    for _ in range(max_iter):
        nw = -_bump_field(bumps, x + w[0], y + w[1], z + w[2])
        delta = float((nw - w).abs().max())
        w = nw
        if delta < tol:
            break
    return w


# --------------------------------------------------------------------------- #
# CBCT-like corruption of the moving image (pelvis)
# --------------------------------------------------------------------------- #
def _bias_field(rng, shape):
    """Smooth random field in [-1, 1] from the lowest three cosine modes per axis."""
    x, y, z = (t.numpy() for t in _grid(shape))
    nz, ny, nx = shape
    b = np.zeros(shape, dtype=np.float64)
    for kx in range(3):
        for ky in range(3):
            for kz in range(3):
                if kx + ky + kz == 0:
                    continue
                a = rng.normal()
                phase = rng.uniform(0, 2 * math.pi)
                b += a * np.cos(math.pi * (kx * x / max(nx, 1) + ky * y / max(ny, 1)
                                           + kz * z / max(nz, 1)) + phase)
    return b / max(float(np.abs(b).max()), 1e-12)


def _bias_field_device(rng, shape, device):
    """``_bias_field`` evaluated with torch on ``device`` (the same draws)."""
    x, y, z = _grid(shape, device)
    nz, ny, nx = shape
    b = torch.zeros(shape, dtype=torch.float64, device=device)
    for kx in range(3):
        for ky in range(3):
            for kz in range(3):
                if kx + ky + kz == 0:
                    continue
                a = rng.normal()
                phase = rng.uniform(0, 2 * math.pi)
                b += a * torch.cos(math.pi * (kx * x / max(nx, 1) + ky * y / max(ny, 1)
                                              + kz * z / max(nz, 1)) + phase)
    return b / max(float(b.abs().max()), 1e-12)


def _streaks(rng, shape, n_lines=6, amp=60.0):
    nz, ny, nx = shape
    yy, xx = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64),
                         indexing="ij")
    cx, cy = 0.5 * (nx - 1), 0.5 * (ny - 1)
    r = np.sqrt((xx - cx) ** 2 + (yy - cy) ** 2)
    s = np.zeros((ny, nx))
    for _ in range(n_lines):
        th = rng.uniform(0, math.pi)
        d = np.abs((xx - cx) * math.sin(th) - (yy - cy) * math.cos(th))
        s += rng.choice([-1.0, 1.0]) * amp * np.exp(-0.5 * d * d) * np.exp(-r / (0.5 * nx))
    return np.broadcast_to(s, shape)


# --------------------------------------------------------------------------- #
# public entry points
# --------------------------------------------------------------------------- #
def _cache_path(name, index, shape, masks):
    import hashlib
    import os
    root = os.environ.get("CGDIR_PHANTOM_CACHE",
                          os.path.join(os.path.dirname(os.path.dirname(
                              os.path.abspath(__file__))), ".phantom_cache"))
    key = hashlib.sha1(repr((name, index, tuple(shape), tuple(masks or ()),
                             _GENERATOR_VERSION)).encode()).hexdigest()[:16]
    return os.path.join(root, f"{name}_{index}_{key}.npz")


_GENERATOR_VERSION = 1


def make_case(name: str, index: int = 0, shape: Optional[Tuple[int, int, int]] = None,
              masks: Optional[Sequence[str]] = None, cache: bool = True) -> Case:
    """Build (or load from the on-disk cache) one seeded case; see ``_generate``."""
    import os
    cfg = CONFIGS[name]
    shape = tuple(int(s) for s in (shape or cfg.shape))
    big = int(np.prod(shape)) >= (1 << 20)
    path = _cache_path(name, index, shape, masks) if (cache and big) else None
    if path and os.path.exists(path):
        d = np.load(path, allow_pickle=False)
        names = [str(s) for s in d["mask_names"]]
        return Case(name=name, seed=int(d["seed"]), static=d["static"], moving=d["moving"],
                    static_masks=d["static_masks"], moving_masks=d["moving_masks"],
                    u_gt=d["u_gt"], body=d["body"], signs=[int(s) for s in d["signs"]],
                    mask_names=names, spacing_mm=cfg.spacing_mm, levels=cfg.levels,
                    iters=tuple(cfg.iters), lam=[cfg.lam] * len(names))
    case = _generate(name, index, shape, masks)
    if path:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp.npz"
        np.savez(tmp, seed=case.seed, static=case.static, moving=case.moving,
                 static_masks=case.static_masks, moving_masks=case.moving_masks,
                 u_gt=case.u_gt, body=case.body, signs=np.array(case.signs),
                 mask_names=np.array(case.mask_names))
        os.replace(tmp, path)
    return case


def _generate(name: str, index: int = 0, shape: Optional[Tuple[int, int, int]] = None,
              masks: Optional[Sequence[str]] = None) -> Case:
    """Build one seeded case of config ``name``.

    ``shape`` (nz, ny, nx) overrides the volume size; structures are defined in
    fractions of the extent and the displacement cap scales with the volume, so
    a smaller shape gives the same anatomy at lower resolution.  ``masks``
    selects a subset of the config's structures."""
    cfg = CONFIGS[name]
    shape = tuple(int(s) for s in (shape or cfg.shape))
    seed = 1000 * cfg.number + int(index)
    rng = np.random.Generator(np.random.PCG64(seed))
    ratio = min(shape[a] / cfg.shape[a] for a in range(3))
    cap = max(cfg.cap * ratio, 1.0)

    bumps = _make_bumps(rng, cfg, shape, cap)
    bumps, u_gt = _scale_bumps(bumps, shape, cap)
    w = _invert(bumps, shape)

    x, y, z = _grid(shape)
    static = _paint(cfg.layers, x, y, z, shape).numpy()
    mx, my, mz = x + w[0], y + w[1], z + w[2]
    moving = _paint(cfg.layers, mx, my, mz, shape).numpy()
    u_gt = u_gt.numpy()

    layers = {l.name: l for l in cfg.layers}
    mask_names = list(masks) if masks is not None else list(cfg.masks)
    smasks = np.zeros((len(mask_names),) + shape, dtype=np.uint8)
    mmasks = np.zeros_like(smasks)
    signs = []
    for i, m in enumerate(mask_names):
        L = layers[m]
        smasks[i] = (_layer_occupancy(L, x, y, z, shape) >= 0.5).numpy()
        mmasks[i] = (_layer_occupancy(L, mx, my, mz, shape) >= 0.5).numpy()
        signs.append(1 if L.hu >= _surround_hu(cfg, L) else -1)
    body = (_layer_occupancy(layers[cfg.body], x, y, z, shape) >= 0.5).numpy().astype(np.uint8)

    if cfg.cbct:
        moving = moving * (1.0 + 0.05 * _bias_field(rng, shape)) + _streaks(rng, shape)
    static = static + rng.normal(0.0, cfg.noise_static, size=shape)
    moving = moving + rng.normal(0.0, cfg.noise_moving, size=shape)
    return Case(name=name, seed=seed,
                static=np.ascontiguousarray(static, dtype=np.float32),
                moving=np.ascontiguousarray(moving, dtype=np.float32),
                static_masks=smasks, moving_masks=mmasks,
                u_gt=np.ascontiguousarray(u_gt, dtype=np.float32), body=body,
                signs=signs, mask_names=mask_names, spacing_mm=cfg.spacing_mm,
                levels=cfg.levels, iters=tuple(cfg.iters),
                lam=[cfg.lam] * len(mask_names))


def make_case_device(name: str, index: int = 0, shape: Optional[Tuple[int, int, int]] = None,
                     masks: Optional[Sequence[str]] = None, device="cuda") -> Case:
    """``make_case`` evaluated with torch on ``device``: the same anatomy,
    bumps (the same NumPy draws) and deformation model, for volumes too large
    to build on the host in reasonable time.  The image noise comes from
    torch's generator seeded with the case seed, so the images are not the
    host case's bit for bit.  Fields are device tensors: static / moving
    float32 [nz,ny,nx], masks uint8 [k,nz,ny,nx], u_gt float32 [3,...]."""
    cfg = CONFIGS[name]
    shape = tuple(int(s) for s in (shape or cfg.shape))
    seed = 1000 * cfg.number + int(index)
    rng = np.random.Generator(np.random.PCG64(seed))
    ratio = min(shape[a] / cfg.shape[a] for a in range(3))
    cap = max(cfg.cap * ratio, 1.0)
    bumps = _make_bumps(rng, cfg, shape, cap)
    bumps, u_gt = _scale_bumps(bumps, shape, cap, device)
    w = _invert(bumps, shape, device=device)
    x, y, z = _grid(shape, device)
    mx, my, mz = x + w[0], y + w[1], z + w[2]
    del w
    static = _paint(cfg.layers, x, y, z, shape)
    moving = _paint(cfg.layers, mx, my, mz, shape)
    layers = {l.name: l for l in cfg.layers}
    mask_names = list(masks) if masks is not None else list(cfg.masks)
    k = len(mask_names)
    smasks = torch.empty((k,) + shape, dtype=torch.uint8, device=device)
    mmasks = torch.empty_like(smasks)
    signs = []
    for i, m in enumerate(mask_names):
        L = layers[m]
        smasks[i] = (_layer_occupancy(L, x, y, z, shape) >= 0.5)
        mmasks[i] = (_layer_occupancy(L, mx, my, mz, shape) >= 0.5)
        signs.append(1 if L.hu >= _surround_hu(cfg, L) else -1)
    body = (_layer_occupancy(layers[cfg.body], x, y, z, shape) >= 0.5).to(torch.uint8)
    del mx, my, mz, x, y, z
    if cfg.cbct:
        moving = moving * (1.0 + 0.05 * _bias_field_device(rng, shape, device)) + \
            torch.from_numpy(np.ascontiguousarray(_streaks(rng, shape))).to(device)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    static = static + cfg.noise_static * torch.randn(shape, generator=g, dtype=torch.float64, device=device)
    moving = moving + cfg.noise_moving * torch.randn(shape, generator=g, dtype=torch.float64, device=device)
    return Case(name=name, seed=seed, static=static.float().contiguous(), moving=moving.float().contiguous(),
                static_masks=smasks, moving_masks=mmasks, u_gt=u_gt.float().contiguous(), body=body,
                signs=signs, mask_names=mask_names, spacing_mm=cfg.spacing_mm,
                levels=cfg.levels, iters=tuple(cfg.iters), lam=[cfg.lam] * k)


def batch_mix_specs(n: int = 32, seed: int = 4000, scale: float = 1.0):
    """The draws of ``batch_mix_cases`` without building the cases: a list of
    (template, index, shape, mask names)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        shp = BATCH_SHAPES[int(rng.integers(len(BATCH_SHAPES)))]
        shp = tuple(max(4, int(round(s * scale))) for s in shp)
        tmpl = "headneck256" if rng.integers(2) == 0 else "pelvis512"
        names = CONFIGS[tmpl].masks
        k = int(rng.integers(2, 9))
        out.append((tmpl, 100 + i, shp, [names[j % len(names)] for j in range(k)]))
    return out


def _surround_hu(cfg: Config, layer: Layer) -> float:
    """HU of the tissue a structure is embedded in (the last painted layer
    before it whose name marks a body tissue)."""
    hu = AIR
    for l in cfg.layers:
        if l is layer:
            break
        if l.painted and l.shell == 0 and l.name in ("body", "tissue", "fat"):
            hu = l.hu
    if not layer.painted:
        return hu - 1.0
    return hu


def batch_mix_cases(n: int = 32, seed: int = 4000, scale: float = 1.0) -> List[Case]:
    """The uneven-size mix: sizes uniform over four CT shapes, 2-8 masks each
    (structures drawn from the head-and-neck and pelvic templates), bumps
    <= 10 voxels.  ``scale`` < 1 shrinks every shape (for tests)."""
    out = []
    for i, (tmpl, index, shp, chosen) in enumerate(batch_mix_specs(n, seed, scale)):
        c = make_case(tmpl, index=index, shape=shp, masks=chosen)
        c.name = f"batch{i}:{tmpl}"
        out.append(c)
    return out


def voxel_iters(shape: Tuple[int, int, int], levels: int, iters: Sequence[int]) -> int:
    """Sum over pyramid levels of voxels x iterations (coarse -> fine); level
    sizes halve with rounding up."""
    sizes = [tuple(shape)]
    for _ in range(levels - 1):
        sizes.append(tuple((s + 1) // 2 for s in sizes[-1]))
    sizes = sizes[::-1]
    return int(sum(int(np.prod(sz)) * int(it) for sz, it in zip(sizes, iters)))
