"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This module only draws random numbers and lays out cameras. It holds none of
the rasterizer's arithmetic (no covariance, no line integral, no spherical
harmonics evaluation), so the oracle and the CUDA path can both consume its
output without sharing any of the method.

Generators follow the workloads the paper trains on (view synthesis scenes of
1.5M-5.3M Gaussians, Supp. E; tomography scenes of 58-71K Gaussians, Sec. 6.2):
every array is float32 and laid out structure-of-arrays:

    mu     [N, 3]   Gaussian means (world)
    scale  [N, 3]   per-axis standard deviations s (positive)
    quat   [N, 4]   unit quaternions (w, x, y, z)
    kappa  [N]      densities (the kappa of Eq. 3)
    sh     [N, K, 3] spherical-harmonic colour coefficients, K = (deg+1)^2

Cameras use OpenCV axes (x right, y down, z forward); a world point x maps to
camera coordinates R x + t.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Scene", "Camera", "Beam", "look_at", "fibonacci_cameras", "random_unit_quats",
    "uniform_scene", "cluster_scene", "tomo_scene", "random_image",
    "config1", "config2", "config3", "config4", "config5", "small_views",
]


@dataclass
class Scene:
    mu: np.ndarray
    scale: np.ndarray
    quat: np.ndarray
    kappa: np.ndarray
    sh: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.mu.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.mu[idx].copy(), self.scale[idx].copy(), self.quat[idx].copy(),
                     self.kappa[idx].copy(), self.sh[idx].copy(), self.sh_degree)


@dataclass
class Camera:
    R: np.ndarray          # [3,3] float32, world -> camera rotation (rows = camera axes)
    t: np.ndarray          # [3] float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int


@dataclass
class Beam:
    """Parallel-beam tomography geometry: rotation axis is world z."""
    angles: np.ndarray     # [A] float32 radians
    det_w: int
    det_h: int
    pitch_u: float
    pitch_v: float
    u0: float              # detector coordinate of the left edge of column 0
    v0: float              # detector coordinate of the top edge of row 0


def _f32(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float32))


def look_at(eye, target, width, height, hfov_deg=60.0, down=(0.0, 1.0, 0.0)) -> Camera:
    """Pinhole camera at `eye` looking at `target`; horizontal field of view `hfov_deg`."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    dn = np.asarray(down, np.float64)
    if abs(float(np.dot(dn, fwd))) > 0.99:
        dn = np.array([0.0, 0.0, -1.0]) if abs(fwd[2]) < 0.9 else np.array([0.0, 1.0, 0.0])
    right = np.cross(dn, fwd)
    right /= np.linalg.norm(right)
    down_axis = np.cross(fwd, right)
    R = np.stack([right, down_axis, fwd])
    t = -R @ eye
    f = (width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)
    return Camera(_f32(R), _f32(t), float(f), float(f), width / 2.0, height / 2.0, int(width), int(height))


def fibonacci_cameras(n, radius, sizes, hfov_deg=60.0):
    """n cameras on a Fibonacci sphere of `radius`, all looking at the origin.

    `sizes` is a list of (width, height), one per camera."""
    cams = []
    golden = math.pi * (3.0 - math.sqrt(5.0))
    for i in range(n):
        y = 1.0 - 2.0 * (i + 0.5) / n
        r = math.sqrt(max(0.0, 1.0 - y * y))
        phi = golden * i
        eye = radius * np.array([math.cos(phi) * r, y, math.sin(phi) * r])
        w, h = sizes[i]
        cams.append(look_at(eye, (0.0, 0.0, 0.0), w, h, hfov_deg))
    return cams


def random_unit_quats(rng, n):
    """Uniform random rotations: normalised 4-D standard normal samples (Muller/Marsaglia)."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return _f32(q)


def _log_uniform(rng, lo, hi, n):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), n))


def _flatten(rng, scale, frac):
    n = scale.shape[0]
    sel = rng.random(n) < frac
    axis = rng.integers(0, 3, n)
    scale = scale.copy()
    scale[sel, axis[sel]] /= 100.0
    return scale


def _dc_colour_coeffs(rng, n):
    # DC coefficients uniform in [-sqrt(pi), sqrt(pi)]: with the degree-0 basis value
    # 1/(2 sqrt(pi)) and the +0.5 offset this is an RGB colour uniform in [0, 1].
    return rng.uniform(-math.sqrt(math.pi), math.sqrt(math.pi), (n, 1, 3))


def uniform_scene(n, seed, log_scale=(-4.0, -2.0), kappa=(0.5, 50.0), sh_degree=0,
                  sh_std=0.2, flatten_frac=0.0, extent=1.0) -> Scene:
    """Means uniform in [-extent, extent]^3, log-scales uniform, log-uniform densities."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mu = rng.uniform(-extent, extent, (n, 3))
    scale = np.exp(rng.uniform(log_scale[0], log_scale[1], (n, 3)))
    quat = random_unit_quats(rng, n)
    kap = _log_uniform(rng, kappa[0], kappa[1], n)
    K = (sh_degree + 1) ** 2
    if sh_degree == 0:
        sh = _dc_colour_coeffs(rng, n)
    else:
        sh = rng.normal(0.0, sh_std, (n, K, 3))
    scale = _flatten(rng, scale, flatten_frac)
    return Scene(_f32(mu), _f32(scale), quat, _f32(kap), _f32(sh), sh_degree)


def cluster_scene(n, seed, n_clusters=64, log_scale=(-6.0, -4.0), kappa=(0.1, 100.0),
                  sh_degree=3, sh_std=0.2, flatten_frac=0.2) -> Scene:
    """Means from a mixture of anisotropic clusters, clipped to [-1, 1]^3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.uniform(-0.8, 0.8, (n_clusters, 3))
    sig = rng.uniform(0.05, 0.25, (n_clusters, 3))
    rot = rng.standard_normal((n_clusters, 3, 3))
    rot, _ = np.linalg.qr(rot)                      # random orthonormal frames
    lab = rng.integers(0, n_clusters, n)
    z = rng.standard_normal((n, 3)) * sig[lab]
    mu = centres[lab] + np.einsum("nij,nj->ni", rot[lab], z)
    mu = np.clip(mu, -1.0, 1.0)
    scale = np.exp(rng.uniform(log_scale[0], log_scale[1], (n, 3)))
    quat = random_unit_quats(rng, n)
    kap = _log_uniform(rng, kappa[0], kappa[1], n)
    K = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, sh_std, (n, K, 3)) if sh_degree > 0 else _dc_colour_coeffs(rng, n)
    scale = _flatten(rng, scale, flatten_frac)
    return Scene(_f32(mu), _f32(scale), quat, _f32(kap), _f32(sh), sh_degree)


def tomo_scene(n, seed, log_scale=(-5.0, -3.0), kappa=(0.1, 10.0)) -> Scene:
    """Density-only Gaussians with means uniform in the unit ball."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = rng.random(n) ** (1.0 / 3.0)
    mu = v * r[:, None]
    scale = np.exp(rng.uniform(log_scale[0], log_scale[1], (n, 3)))
    quat = random_unit_quats(rng, n)
    kap = _log_uniform(rng, kappa[0], kappa[1], n)
    sh = np.zeros((n, 1, 3))
    return Scene(_f32(mu), _f32(scale), quat, _f32(kap), _f32(sh), 0)


def random_image(seed, shape):
    rng = np.random.Generator(np.random.PCG64(seed))
    return _f32(rng.random(shape))


def parallel_beam(n_angles, det=512, extent=2.0, angles=None) -> Beam:
    """Parallel beam: angles k*pi/n_angles, a det x det detector covering [-extent/2, extent/2]^2."""
    if angles is None:
        angles = np.arange(n_angles, dtype=np.float64) * math.pi / n_angles
    pitch = float(np.float32(extent / det))       # geometry is handed to the kernels as float32
    u0 = float(np.float32(-extent / 2.0))
    return Beam(_f32(angles), det, det, pitch, pitch, u0, u0)


# --------------------------------------------------------------------------------------------
# The five workloads. `frac` shrinks the Gaussian count (and view count for the batched ones)
# so that the same generator yields small parity cases.

def config1(frac=1.0):
    """2,000 Gaussians, SH degree 0, one 128x128 camera at distance 4, 60 deg FOV."""
    n = max(1, int(round(2000 * frac)))
    scene = uniform_scene(n, 1001)
    cam = look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 128, 128, 60.0)
    return scene, [cam]


def config2(frac=1.0, width=1280, height=832):
    """1,000,000 Gaussians from 64 clusters, 20% flattened, SH degree 3, one 1280x832 camera."""
    n = max(1, int(round(1_000_000 * frac)))
    scene = cluster_scene(n, 1002)
    cam = look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), width, height, 60.0)
    target = random_image(2002, (height, width, 3))
    return scene, [cam], target


def _batched_sizes(n_views, lo=(640, 416), hi=(1920, 1080)):
    sizes = []
    for i in range(n_views):
        f = i / max(1, n_views - 1)
        w = int(round((lo[0] + f * (hi[0] - lo[0])) / 16.0)) * 16
        h = int(round((lo[1] + f * (hi[1] - lo[1])) / 16.0)) * 16
        sizes.append((w, h))
    sizes[-1] = hi
    return sizes


def config3(frac=1.0, n_views=16):
    """3,000,000 Gaussians (cluster generator, 40% flattened), 16 views 640x416..1920x1080."""
    n = max(1, int(round(3_000_000 * frac)))
    scene = cluster_scene(n, 1003, flatten_frac=0.4)
    cams = fibonacci_cameras(n_views, 4.0, _batched_sizes(n_views))
    return scene, cams


def config4(frac=1.0, n_angles=256, det=512):
    """Tomography: 200,000 Gaussians, 256 parallel-beam angles over 180 deg, 512^2 detector;
    target from 50,000 ground-truth Gaussians."""
    n = max(1, int(round(200_000 * frac)))
    scene = tomo_scene(n, 1004)
    gt = tomo_scene(max(1, int(round(50_000 * frac))), 2004)
    return scene, parallel_beam(n_angles, det), gt


def cone_beam(n_angles, det=512, source_dist=4.0, cover=1.1):
    """Cone-beam geometry: n_angles X-ray sources on a circle of radius source_dist about the z
    axis (angles 2 pi k / n_angles), each a det x det pinhole camera looking at the origin with
    a field of view that covers a sphere of radius `cover`."""
    fov = math.degrees(2.0 * math.atan(cover / source_dist))
    cams = []
    for k in range(n_angles):
        a = 2.0 * math.pi * k / n_angles
        cams.append(look_at((source_dist * math.cos(a), source_dist * math.sin(a), 0.0), (0.0, 0.0, 0.0),
                            det, det, fov, down=(0.0, 0.0, -1.0)))
    return cams


def config5(frac=1.0, n_views=8, width=1920, height=1080):
    """6,000,000 Gaussians (cluster generator), SH degree 3, 8 views of 1920x1080."""
    n = max(1, int(round(6_000_000 * frac)))
    scene = cluster_scene(n, 1005)
    cams = fibonacci_cameras(n_views, 4.0, [(width, height)] * n_views)
    return scene, cams


def small_views(n_views, seed, sizes):
    """A few cameras on a sphere of radius 4 for multi-view parity cases."""
    return fibonacci_cameras(n_views, 4.0, sizes)
