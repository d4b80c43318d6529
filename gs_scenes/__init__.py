"""Seeded synthetic inputs for the Top-K feature render.

This module only draws random numbers and lays them out: Gaussian parameter sets,
pinhole cameras, target maps and upstream gradients.  It contains none of the
rendering arithmetic (projection, blending, selection), so both the CUDA path and
the FP64 oracle can take their inputs from here without sharing any of the method.

The scene shapes follow the paper's workloads:
  * Gaussians carry colour, mean, covariance, opacity and a unit-norm language
    feature (Sec. 3.1, Sec. 3.2: features are directions in language space);
  * map sizes of ~200k Gaussians mirror the Replica maps of Tab. 6;
  * D = 512 mirrors the LSeg feature width used by the 512-D comparison of Tab. 2;
  * surface-concentrated placement (Gaussians on planes) mirrors the
    surface-aligned maps the method builds.
Replica / TUM-RGBD frames are not available, so these scenes stand in for them.

Covariances are drawn the usual way for random SPD matrices, R diag(s^2) R^T from
a random unit quaternion and log-normal scales, and handed over as 6 floats
(xx, xy, xz, yy, yz, zz); the renderer consumes the covariance itself, as the
paper parameterises each Gaussian by its covariance.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

__all__ = [
    "Camera", "Scene", "CONFIGS", "make_config", "random_scene_box",
    "planes_scene", "pinhole", "look_at", "orbit_cameras", "voronoi_targets",
    "upstream_grads", "crop_scene",
]


@dataclasses.dataclass
class Camera:
    """Pinhole camera. viewmat is the 4x4 row-major world->camera transform
    (camera looks along +z, x right, y down); pixel (i, j) is sampled at its
    centre (i + 0.5, j + 0.5)."""
    viewmat: np.ndarray          # (4, 4) float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.2

    @property
    def n_pix(self) -> int:
        return self.width * self.height


@dataclasses.dataclass
class Scene:
    mean3d: np.ndarray      # (N, 3) float32
    cov3d: np.ndarray       # (N, 6) float32: xx, xy, xz, yy, yz, zz
    opacity: np.ndarray     # (N,)   float32
    rgb: np.ndarray         # (N, 3) float32
    feats: np.ndarray       # (N, D) float32, unit-norm rows

    @property
    def n(self) -> int:
        return int(self.mean3d.shape[0])

    @property
    def d(self) -> int:
        return int(self.feats.shape[1])

    def subset(self, idx) -> "Scene":
        return Scene(self.mean3d[idx].copy(), self.cov3d[idx].copy(),
                     self.opacity[idx].copy(), self.rgb[idx].copy(),
                     self.feats[idx].copy())


def _unit_rows(rng, n, d, dtype=np.float64):
    v = rng.standard_normal((n, d), dtype=dtype)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def _random_cov6(rng, n, log_scale_mu=-3.0, log_scale_sigma=0.5, squash=None):
    """Random SPD covariances: R diag(s^2) R^T, unit quaternion ~ normalised N(0, I4),
    log-scales ~ N(mu, sigma) per axis.  Returned as (xx, xy, xz, yy, yz, zz)."""
    ls = rng.normal(log_scale_mu, log_scale_sigma, size=(n, 3))
    if squash is not None:
        ls[:, 2] += np.log(squash)
    s2 = np.exp(2.0 * ls)
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    S = np.einsum("nij,nj,nkj->nik", R, s2, R)
    return np.stack([S[:, 0, 0], S[:, 0, 1], S[:, 0, 2],
                     S[:, 1, 1], S[:, 1, 2], S[:, 2, 2]], axis=1)


def _attrs(rng, n, d, feat_dtype=np.float64):
    opac = 1.0 / (1.0 + np.exp(-rng.standard_normal(n)))
    rgb = rng.uniform(0.0, 1.0, size=(n, 3))
    feats = _unit_rows(rng, n, d, feat_dtype)
    return opac, rgb, feats


def _pack(mean, cov, opac, rgb, feats) -> Scene:
    f32 = np.float32
    return Scene(np.ascontiguousarray(mean, f32), np.ascontiguousarray(cov, f32),
                 np.ascontiguousarray(opac, f32), np.ascontiguousarray(rgb, f32),
                 np.ascontiguousarray(feats, f32))


BOX = ((-1.0, 1.0), (-1.0, 1.0), (1.0, 5.0))


def random_scene_box(seed: int, n: int, d: int, box=BOX,
                     log_scale_mu=-3.0, log_scale_sigma=0.5) -> Scene:
    """n Gaussians uniform in an axis-aligned box (default: the 2x2x4 m box 1-5 m in
    front of an identity camera)."""
    rng = np.random.default_rng(seed)
    lo = np.array([b[0] for b in box])
    hi = np.array([b[1] for b in box])
    mean = rng.uniform(lo, hi, size=(n, 3))
    cov = _random_cov6(rng, n, log_scale_mu, log_scale_sigma)
    opac, rgb, feats = _attrs(rng, n, d)
    return _pack(mean, cov, opac, rgb, feats)


def planes_scene(seed: int, n: int, d: int, n_planes=5, frac_on_planes=0.8,
                 box=BOX, patch=2.0, boxes_frac=0.0, feat_dtype=np.float64) -> Scene:
    """Surface-concentrated scene: frac_on_planes of the Gaussians lie uniformly on
    n_planes seeded 2x2 m planar patches (random normal, centre uniform in the box);
    a fraction boxes_frac of the patches are replaced by the six faces of a small
    axis-aligned box; the rest is uniform clutter in the box.  feat_dtype: precision in
    which the feature vectors are drawn (float32 keeps a multi-GB draw in memory)."""
    rng = np.random.default_rng(seed)
    lo = np.array([b[0] for b in box])
    hi = np.array([b[1] for b in box])
    n_on = int(round(n * frac_on_planes))
    n_clutter = n - n_on
    centres = rng.uniform(lo, hi, size=(n_planes, 3))
    normals = _unit_rows(rng, n_planes, 3)
    is_box = rng.uniform(size=n_planes) < boxes_frac
    which = rng.integers(0, n_planes, size=n_on)
    a = rng.uniform(-patch / 2, patch / 2, size=n_on)
    b = rng.uniform(-patch / 2, patch / 2, size=n_on)
    pts = np.empty((n_on, 3))
    for k in range(n_planes):
        sel = which == k
        nk = normals[k]
        helper = np.array([1.0, 0.0, 0.0]) if abs(nk[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
        u1 = np.cross(nk, helper)
        u1 /= np.linalg.norm(u1)
        u2 = np.cross(nk, u1)
        if is_box[k]:
            # six faces of a cube of edge patch/2 centred at centres[k]
            h = patch / 4
            face = rng.integers(0, 6, size=int(sel.sum()))
            s = rng.uniform(-h, h, size=(int(sel.sum()), 3))
            ax = face // 2
            s[np.arange(s.shape[0]), ax] = np.where(face % 2 == 0, -h, h)
            pts[sel] = centres[k] + s
        else:
            pts[sel] = centres[k] + a[sel, None] * u1 + b[sel, None] * u2
    clutter = rng.uniform(lo, hi, size=(n_clutter, 3))
    mean = np.concatenate([pts, clutter], axis=0)
    perm = rng.permutation(n)
    mean = mean[perm]
    cov = _random_cov6(rng, n)
    opac, rgb, feats = _attrs(rng, n, d, feat_dtype)
    return _pack(mean, cov, opac, rgb, feats)


def pinhole(width, height, fx, fy=None, cx=None, cy=None, viewmat=None, near=0.2) -> Camera:
    fy = fx if fy is None else fy
    cx = width / 2.0 if cx is None else cx
    cy = height / 2.0 if cy is None else cy
    vm = np.eye(4, dtype=np.float32) if viewmat is None else np.asarray(viewmat, np.float32)
    return Camera(vm, float(fx), float(fy), float(cx), float(cy), int(width), int(height), float(near))


def look_at(eye, target, up=(0.0, -1.0, 0.0)) -> np.ndarray:
    """World->camera 4x4 (row-major) for a camera at eye looking at target, with
    camera +z forward, +x right and +y down."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    upv = np.asarray(up, np.float64)
    right = np.cross(upv, fwd)
    if np.linalg.norm(right) < 1e-9:
        right = np.cross(np.array([1.0, 0.0, 0.0]), fwd)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], axis=0)
    vm = np.eye(4)
    vm[:3, :3] = R
    vm[:3, 3] = -R @ eye
    return vm.astype(np.float32)


def orbit_cameras(seed, sizes, radius=3.0, centre=(0.0, 0.0, 3.0)) -> List[Camera]:
    """Cameras at seeded random angles on a horizontal orbit of the given radius
    around centre, looking at it.  sizes: list of (W, H, fx)."""
    rng = np.random.default_rng(seed)
    cams = []
    c = np.asarray(centre)
    for (w, h, f) in sizes:
        th = rng.uniform(0, 2 * np.pi)
        el = rng.uniform(-0.3, 0.3)
        eye = c + radius * np.array([np.sin(th) * np.cos(el), np.sin(el), -np.cos(th) * np.cos(el)])
        cams.append(pinhole(w, h, f, viewmat=look_at(eye, c)))
    return cams


def voronoi_targets(seed, cams: List[Camera], d: int, n_sites=12):
    """Loss targets for each camera: piecewise-constant maps over n_sites seeded
    Voronoi cells in the image; each cell has a random unit D-vector, an RGB in
    U[0,1] and a depth in U[1,5].  Returned dense, pixel-major, cameras concatenated."""
    rng = np.random.default_rng(seed)
    F, C, Dp = [], [], []
    for cam in cams:
        sites = rng.uniform([0, 0], [cam.width, cam.height], size=(n_sites, 2))
        fv = _unit_rows(rng, n_sites, d)
        cv = rng.uniform(0, 1, size=(n_sites, 3))
        dv = rng.uniform(1, 5, size=n_sites)
        ys, xs = np.mgrid[0:cam.height, 0:cam.width]
        px = np.stack([xs.ravel() + 0.5, ys.ravel() + 0.5], axis=1)
        lab = np.argmin(((px[:, None, :] - sites[None]) ** 2).sum(-1), axis=1)
        F.append(fv[lab])
        C.append(cv[lab])
        Dp.append(dv[lab])
    f32 = np.float32
    return (np.ascontiguousarray(np.concatenate(F), f32),
            np.ascontiguousarray(np.concatenate(C), f32),
            np.ascontiguousarray(np.concatenate(Dp), f32))


def voronoi_sites(seed, cams: List[Camera], d: int, n_sites=12):
    """The same targets as voronoi_targets in factored form, for large frames: per-pixel
    cell labels (int32, pixel-major, cameras concatenated, with each camera's cells
    numbered after the previous camera's) and the per-cell values (unit D-vectors,
    RGB, depth).  Expand with values[labels]."""
    rng = np.random.default_rng(seed)
    labs, F, C, Dp = [], [], [], []
    base = 0
    for cam in cams:
        sites = rng.uniform([0, 0], [cam.width, cam.height], size=(n_sites, 2))
        fv = _unit_rows(rng, n_sites, d)
        cv = rng.uniform(0, 1, size=(n_sites, 3))
        dv = rng.uniform(1, 5, size=n_sites)
        ys, xs = np.mgrid[0:cam.height, 0:cam.width]
        px = np.stack([xs.ravel() + 0.5, ys.ravel() + 0.5], axis=1)
        lab = np.argmin(((px[:, None, :] - sites[None]) ** 2).sum(-1), axis=1)
        labs.append(lab + base)
        base += n_sites
        F.append(fv); C.append(cv); Dp.append(dv)
    f32 = np.float32
    return (np.concatenate(labs).astype(np.int32), np.concatenate(F).astype(f32),
            np.concatenate(C).astype(f32), np.concatenate(Dp).astype(f32))


def upstream_grads(seed, n_pix: int, d: int, scale=1.0):
    """Seeded upstream gradients dL/dF (P, D), dL/dC (P, 3), dL/dD (P,)."""
    rng = np.random.default_rng(seed)
    f32 = np.float32
    return (np.ascontiguousarray(rng.standard_normal((n_pix, d)) * scale, f32),
            np.ascontiguousarray(rng.standard_normal((n_pix, 3)) * scale, f32),
            np.ascontiguousarray(rng.standard_normal(n_pix) * scale, f32))


def crop_scene(scene: Scene, cam: Camera, n_keep=1000):
    """The n_keep Gaussians whose means lie closest to the camera's optical axis
    (the ray through the principal point), for small gradient checks."""
    vm = cam.viewmat.astype(np.float64)
    p = scene.mean3d.astype(np.float64) @ vm[:3, :3].T + vm[:3, 3]
    r = np.hypot(p[:, 0], p[:, 1]) / np.maximum(p[:, 2], 1e-6)
    r[p[:, 2] <= cam.near] = np.inf
    idx = np.sort(np.argsort(r)[:n_keep])
    return scene.subset(idx)


# --------------------------------------------------------------------------------------
# Named workloads.  Each returns (scene, cameras, K, tile (w, h), feature dtype).
# --------------------------------------------------------------------------------------

CONFIGS = {
    "small": "2,000 Gaussians in the 2x2x4 m box, 128x96, fx=fy=100, D=16, K=4, FP32, forward",
    "frame": "200k Gaussians (80% on 5 planes + 20% clutter), 640x480, fx=fy=525, D=512, K=8, FP32, fwd+bwd",
    "frame_1m_bf16": "1M Gaussians as 'frame', 640x480, D=512 BF16 rows, K=8, fwd+bwd",
    "batched": "1M Gaussians, D=512 BF16, 8 orbit keyframes 3x640x480 + 3x1200x680 + 2x320x240, K=8, fwd+bwd",
    "mapping": "3M Gaussians (70% on 20 planes/boxes + 30% clutter), 8 keyframes 1200x680, D=768 BF16, K=16, fwd+bwd",
}


def make_config(name: str, seed: int = 0, n_override: Optional[int] = None):
    if name == "small":
        sc = random_scene_box(seed, n_override or 2000, 16)
        return sc, [pinhole(128, 96, 100.0)], 4, (16, 16), "f32"
    if name == "frame":
        sc = planes_scene(seed, n_override or 200_000, 512)
        return sc, [pinhole(640, 480, 525.0)], 8, (16, 16), "f32"
    if name == "frame_1m_bf16":
        sc = planes_scene(seed, n_override or 1_000_000, 512)
        return sc, [pinhole(640, 480, 525.0)], 8, (16, 16), "bf16"
    if name == "batched":
        sc = planes_scene(seed, n_override or 1_000_000, 512)
        sizes = [(640, 480, 525.0)] * 3 + [(1200, 680, 600.0)] * 3 + [(320, 240, 262.5)] * 2
        return sc, orbit_cameras(seed + 1000, sizes), 8, (16, 16), "bf16"
    if name == "mapping":
        sc = planes_scene(seed, n_override or 3_000_000, 768, n_planes=20,
                          frac_on_planes=0.7, boxes_frac=0.3, feat_dtype=np.float32)
        sizes = [(1200, 680, 600.0)] * 8
        return sc, orbit_cameras(seed + 2000, sizes), 16, (16, 16), "bf16"
    raise KeyError(name)
