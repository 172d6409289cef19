"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and the benchmark.

This module only draws random numbers and lays out arrays: scenes of 3D Gaussians (means,
unnormalised quaternions (w, x, y, z), physical scales, opacities, RGB), pinhole cameras
(camera-to-world rotation, centre, intrinsics) and upstream gradients.  It contains none of
the rendering arithmetic; both the oracle and the CUDA path compute everything else
themselves.

The paper (RaySplats, arXiv 2501.19196) evaluates on Mip-NeRF360, Tanks&Temples and Deep
Blending scenes (Sec. 4, Table 1).  Those datasets and trained scenes are not available, so
these synthetic scenes stand in for them with the shapes, sizes and value distributions
listed per workload below.

Camera convention: world = R_wc @ cam + pos, camera axes x right, y down, z forward
(OpenCV).  fx = fy = W / (2 tan(fov/2)), principal point at the image centre.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Opacities are kept strictly inside (0, 1): the transmittance never reaches exactly 0.
OPACITY_CLIP = (1e-4, 1.0 - 1e-4)


@dataclasses.dataclass
class Scene:
    means: np.ndarray      # (N, 3) float32
    quats: np.ndarray      # (N, 4) float32, (w, x, y, z), unnormalised allowed
    scales: np.ndarray     # (N, 3) float32, physical (> 0)
    opacities: np.ndarray  # (N,)   float32 in (0, 1)
    rgb: np.ndarray        # (N, 3) float32

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx].copy(), self.quats[idx].copy(), self.scales[idx].copy(),
                     self.opacities[idx].copy(), self.rgb[idx].copy())


@dataclasses.dataclass
class Cameras:
    R_wc: np.ndarray   # (C, 3, 3) float32
    pos: np.ndarray    # (C, 3) float32
    fx: np.ndarray     # (C,) float32
    fy: np.ndarray
    cx: np.ndarray
    cy: np.ndarray
    width: np.ndarray  # (C,) int32
    height: np.ndarray

    @property
    def count(self) -> int:
        return int(self.pos.shape[0])

    def n_pixels(self) -> np.ndarray:
        return self.width.astype(np.int64) * self.height.astype(np.int64)

    def total_rays(self) -> int:
        return int(self.n_pixels().sum())

    def select(self, idx) -> "Cameras":
        idx = np.atleast_1d(np.asarray(idx))
        return Cameras(self.R_wc[idx].copy(), self.pos[idx].copy(), self.fx[idx].copy(),
                       self.fy[idx].copy(), self.cx[idx].copy(), self.cy[idx].copy(),
                       self.width[idx].copy(), self.height[idx].copy())

    def pack(self) -> np.ndarray:
        """(C, 20) float32/int32 records: R_wc[9], pos[3], fx, fy, cx, cy, width, height
        (the last two as int32 bit patterns) -- the plain camera struct layout."""
        rec = np.zeros((self.count, 18), dtype=np.float32)
        rec[:, 0:9] = self.R_wc.reshape(-1, 9)
        rec[:, 9:12] = self.pos
        rec[:, 12] = self.fx
        rec[:, 13] = self.fy
        rec[:, 14] = self.cx
        rec[:, 15] = self.cy
        wh = np.stack([self.width, self.height], axis=1).astype(np.int32).view(np.float32)
        rec[:, 16:18] = wh
        return rec


def look_at_camera(pos, target, width, height, fov_deg, up=(0.0, 1.0, 0.0)) -> Cameras:
    """One pinhole camera at `pos` looking at `target`; `fov_deg` is the horizontal field of view."""
    pos = np.asarray(pos, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - pos
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, dtype=np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], axis=1)  # columns: camera x, y, z in world
    f = width / (2.0 * math.tan(math.radians(fov_deg) / 2.0))
    return Cameras(R.astype(np.float32)[None], pos.astype(np.float32)[None],
                   np.array([f], np.float32), np.array([f], np.float32),
                   np.array([width / 2.0], np.float32), np.array([height / 2.0], np.float32),
                   np.array([width], np.int32), np.array([height], np.int32))


def concat_cameras(cams) -> Cameras:
    return Cameras(*[np.concatenate([getattr(c, f.name) for c in cams])
                     for f in dataclasses.fields(Cameras)])


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _flatten(rng, log_s, frac):
    """A fraction `frac` of the Gaussians get one uniformly chosen axis scaled by 0.01."""
    n = log_s.shape[0]
    flat = rng.random(n) < frac
    axis = rng.integers(0, 3, n)
    log_s[flat, axis[flat]] += math.log(0.01)
    return log_s


def _finish(means, quats, log_s, opac, rgb) -> Scene:
    opac = np.clip(opac, *OPACITY_CLIP)
    return Scene(means.astype(np.float32), quats.astype(np.float32),
                 np.exp(log_s).astype(np.float32), opac.astype(np.float32),
                 rgb.astype(np.float32))


def scene_uniform_cube(n=1000, seed=0, log_mu=-3.0, log_sigma=0.5) -> Scene:
    """1,000 Gaussians, means U[-1,1]^3, log-scales N(-3, 0.5), unit quaternions,
    opacity U(0.05, 0.95), RGB U(0, 1)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, (n, 3))
    quats = _unit_quats(rng, n)
    log_s = rng.normal(log_mu, log_sigma, (n, 3))
    opac = rng.uniform(0.05, 0.95, n)
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    return _finish(means, quats, log_s, opac, rgb)


def scene_object_shell(n=200_000, seed=0) -> Scene:
    """Object-scale scene: directions uniform on S^2, radius N(0.8, 0.1), log-scales
    N(-4.5, 0.6), 20 % flattened, opacity Beta(2, 2), RGB U(0, 1)."""
    rng = np.random.default_rng(seed)
    dirs = rng.standard_normal((n, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    means = dirs * rng.normal(0.8, 0.1, (n, 1))
    quats = _unit_quats(rng, n)
    log_s = _flatten(rng, rng.normal(-4.5, 0.6, (n, 3)), 0.2)
    opac = rng.beta(2.0, 2.0, n)
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    return _finish(means, quats, log_s, opac, rgb)


def scene_unbounded(n=1_000_000, seed=0, n_clusters=64) -> Scene:
    """Unbounded-scene scale: 90 % of the means from 64 anisotropic Gaussian clusters
    (centres U[-8,8]^3, random rotation, per-axis std U(0.2, 2.0), uniform assignment),
    10 % on a background shell (uniform direction, radius 20 + N(0, 0.5)); log-scales
    N(-4, 1) clipped at -1, 30 % flattened, opacity Beta(0.8, 0.8), RGB U(0, 1)."""
    rng = np.random.default_rng(seed)
    n_shell = n // 10
    n_cl = n - n_shell
    centres = rng.uniform(-8.0, 8.0, (n_clusters, 3))
    rots = np.linalg.qr(rng.standard_normal((n_clusters, 3, 3)))[0]
    stds = rng.uniform(0.2, 2.0, (n_clusters, 3))
    which = rng.integers(0, n_clusters, n_cl)
    local = rng.standard_normal((n_cl, 3)) * stds[which]
    pts = centres[which] + np.einsum("nij,nj->ni", rots[which], local)
    dirs = rng.standard_normal((n_shell, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    shell = dirs * (20.0 + rng.normal(0.0, 0.5, (n_shell, 1)))
    means = np.concatenate([pts, shell])
    perm = rng.permutation(n)
    means = means[perm]
    quats = _unit_quats(rng, n)
    log_s = _flatten(rng, np.minimum(rng.normal(-4.0, 1.0, (n, 3)), -1.0), 0.3)
    opac = rng.beta(0.8, 0.8, n)
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    return _finish(means, quats, log_s, opac, rgb)


def ring_cameras(n=16, radius=12.0, height=2.0, fov_deg=60.0) -> Cameras:
    """16 cameras on a ring looking at the origin: 8 at 1280x832, 4 at 960x640 and
    4 at 640x416, interleaved (even: 1280x832, i%4==1: 960x640, i%4==3: 640x416)."""
    cams = []
    for i in range(n):
        th = 2.0 * math.pi * i / n
        pos = (radius * math.cos(th), height, radius * math.sin(th))
        if i % 2 == 0:
            w, h = 1280, 832
        elif i % 4 == 1:
            w, h = 960, 640
        else:
            w, h = 640, 416
        cams.append(look_at_camera(pos, (0.0, 0.0, 0.0), w, h, fov_deg))
    return concat_cameras(cams)


def default_Q() -> float:
    """0.99 quantile of chi^2(3) (the confidence level the workloads use)."""
    return 11.344866730144373


@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    cams: Cameras
    Q: float
    eps1: float
    k_max: int
    background: tuple
    backward: bool


def workload(cfg: int, seed: int = 0) -> Workload:
    """The four rendering workloads by number (1: 1k / 64x64, 2: 200k / 800x800,
    3: 1M / 1280x832, 4: 1M / 16 ring cameras)."""
    K_UNBOUNDED = 2 ** 31 - 1
    if cfg == 1:
        return Workload("1k_gaussians_64x64", scene_uniform_cube(1000, seed),
                        look_at_camera((0.0, 0.0, -4.0), (0, 0, 0), 64, 64, 50.0),
                        default_Q(), 1e-4, K_UNBOUNDED, (0.0, 0.0, 0.0), False)
    if cfg == 2:
        return Workload("200k_gaussians_shell_800x800", scene_object_shell(200_000, seed),
                        look_at_camera((0.0, 0.0, -4.0), (0, 0, 0), 800, 800, 50.0),
                        default_Q(), 1e-4, K_UNBOUNDED, (1.0, 1.0, 1.0), True)
    if cfg == 3:
        return Workload("1m_gaussians_1280x832", scene_unbounded(1_000_000, seed),
                        ring_cameras().select([0]), default_Q(), 1e-4, K_UNBOUNDED,
                        (0.0, 0.0, 0.0), True)
    if cfg == 4:
        return Workload("1m_gaussians_16cams_mixed_res", scene_unbounded(1_000_000, seed),
                        ring_cameras(), default_Q(), 1e-4, K_UNBOUNDED, (0.0, 0.0, 0.0), True)
    raise ValueError(f"unknown workload {cfg}")


def upstream_grad(n_pixels: int, seed: int = 1):
    """dL/dRGB (n_pixels, 3) and dL/dalpha (n_pixels,) ~ N(0, 1), float32."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n_pixels, 3)).astype(np.float32),
            rng.standard_normal(n_pixels).astype(np.float32))


def random_tiny_scene(seed: int, n: int = 48, spread: float = 0.8, log_mu: float = -1.8,
                      log_sigma: float = 0.4, flat_frac: float = 0.0) -> Scene:
    """Small random scenes (a few dozen Gaussians around the origin) for many-seed tests."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-spread, spread, (n, 3))
    quats = rng.standard_normal((n, 4)) * rng.uniform(0.5, 2.0, (n, 1))  # unnormalised
    log_s = _flatten(rng, rng.normal(log_mu, log_sigma, (n, 3)), flat_frac)
    opac = rng.uniform(0.05, 0.95, n)
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    return _finish(means, quats, log_s, opac, rgb)


def pixel_grid(cams: Cameras, cam_subset=None, stride: int = 1, crop=None):
    """Ray list (cam, px, py) int32 arrays: every `stride`-th pixel in x and y of each camera,
    or a crop (x0, y0, w, h) of each camera."""
    cs, xs, ys = [], [], []
    ids = range(cams.count) if cam_subset is None else cam_subset
    for c in ids:
        W, H = int(cams.width[c]), int(cams.height[c])
        if crop is not None:
            x0, y0, w, h = crop
            gx, gy = np.meshgrid(np.arange(x0, min(x0 + w, W)), np.arange(y0, min(y0 + h, H)))
        else:
            gx, gy = np.meshgrid(np.arange(0, W, stride), np.arange(0, H, stride))
        cs.append(np.full(gx.size, c, np.int32))
        xs.append(gx.ravel().astype(np.int32))
        ys.append(gy.ravel().astype(np.int32))
    return np.concatenate(cs), np.concatenate(xs), np.concatenate(ys)


# ------------------------------------------------------------------------------------------
# Triangle meshes for the mirror / shadow scenes (geometry only; no rendering arithmetic)
# ------------------------------------------------------------------------------------------
def uv_sphere(radius=3.0, slices=200, stacks=126, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Triangles (T, 3, 3) float32 of a UV sphere: slices x (stacks - 2) quads as two triangles
    plus a triangle fan at each pole (200 x 126 gives 50,000 triangles), outward winding."""
    c = np.asarray(center, np.float64)
    th = np.linspace(0.0, np.pi, stacks + 1)          # polar angle, stacks bands
    ph = np.linspace(0.0, 2.0 * np.pi, slices + 1)    # azimuth
    P = np.stack([np.sin(th)[:, None] * np.cos(ph)[None, :], np.cos(th)[:, None] * np.ones_like(ph)[None, :],
                  np.sin(th)[:, None] * np.sin(ph)[None, :]], -1) * radius + c
    tris = []
    for i in range(stacks):
        for j in range(slices):
            a, b, cc, d = P[i, j], P[i, j + 1], P[i + 1, j], P[i + 1, j + 1]
            if i == 0:
                tris.append((a, d, cc))
            elif i == stacks - 1:
                tris.append((a, b, cc))
            else:
                tris.append((a, b, d))
                tris.append((a, d, cc))
    return np.asarray(tris, np.float32)


def ground_plane(y=-4.0, half=40.0) -> np.ndarray:
    """Two triangles (2, 3, 3) float32 spanning [-half, half]^2 at height y, facing up."""
    v = np.array([[-half, y, -half], [half, y, -half], [half, y, half], [-half, y, half]], np.float32)
    return np.stack([v[[0, 2, 1]], v[[0, 3, 2]]]).astype(np.float32)


def mirror_scene_mesh(slices=200, stacks=126, radius=3.0, plane_y=-4.0, plane_half=40.0,
                      light=(10.0, 15.0, -10.0), albedo=0.8, max_bounces=2, eps_off=1e-3) -> dict:
    """A mirror UV sphere at the origin and a diffuse grey ground plane lit by one point light."""
    sph = uv_sphere(radius, slices, stacks)
    gp = ground_plane(plane_y, plane_half)
    verts = np.concatenate([sph, gp])
    mat = np.concatenate([np.zeros(len(sph), np.int32), np.ones(len(gp), np.int32)])
    alb = np.zeros((len(verts), 3), np.float32)
    alb[len(sph):] = albedo
    return {"verts": verts, "mat": mat, "albedo": alb, "light": tuple(float(x) for x in light),
            "max_bounces": int(max_bounces), "eps_off": float(eps_off)}


def workload_mirror(seed: int = 0, n: int = 2_000_000, slices=200, stacks=126):
    """Secondary rays: 2M Gaussians of the unbounded distribution, a 50,000-triangle mirror
    sphere (radius 3) and a diffuse ground plane (y = -4, grey 0.8) lit from (10, 15, -10);
    one 1280 x 832 camera of the ring, up to two mirror bounces and one shadow ray."""
    return (scene_unbounded(n, seed), mirror_scene_mesh(slices, stacks), ring_cameras().select([0]))
