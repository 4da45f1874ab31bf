"""FP64 CPU oracle for the volumetrically consistent Gaussian rasterizer (arXiv 2412.03378).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow reference the CUDA library is
checked against.  Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline legs of
`bench.py` may import it; the product package never does and shares no code with it.

The arithmetic lives in `vg_oracle.c` (plain C, FP64, OpenMP over pixels); this module
compiles it with gcc on first use (no floating-point contraction, so the FP32 key
function is reproducible) and wraps it for numpy inputs produced by `synth`.

Passages followed: Sec. 3.1-3.2 (Eq. 1-4), Sec. 4.1-4.2 (Eq. 8-19), Supp. B (the 1D
Gaussian along the ray), Sec. 6.2 (Eq. 21, tomography), Sec. 7 ("per-tile sorting"), and for
the 3DGS comparison mode Sec. 3.2 (Eq. 5-7: alpha = o G'(p), Sigma' = J W Sigma W^T J^T).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vg_oracle.c")
_HDR = os.path.join(_HERE, "vg_oracle.h")
_SO = os.path.join(_HERE, "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

#: exact mode: no alpha skip, no clamp, no early stop; footprint truncated at tau_cut.
#: density_theta: the density array holds Eq. 20's theta in [0, 1] instead of kappa;
#: softplus_beta > 0: colour activation softplus(beta) instead of the clamp at 0 (Supp. D).
#: splat: the 3DGS comparison mode (Eq. 5-7), where the density array holds the peak opacity o
#: and alpha = o G'(p) with G' the projected 2D Gaussian (covariance + splat_dilation I).
EXACT = dict(alpha_min=0.0, tau_cut=1e-6, tau_max=math.inf, T_stop=0.0, bg=(0.0, 0.0, 0.0), z_near=0.2,
             density_theta=False, softplus_beta=0.0, splat=False, splat_dilation=0.0)
#: compat mode: the 3DGS thresholds (alpha >= 1/255 blended, alpha <= 0.99, stop at T < 1e-4).
COMPAT = dict(alpha_min=1.0 / 255.0, tau_cut=-math.log1p(-1.0 / 255.0), tau_max=math.log(100.0),
              T_stop=1e-4, bg=(0.0, 0.0, 0.0), z_near=0.2, density_theta=False, softplus_beta=0.0,
              splat=False, splat_dilation=0.0)
#: the 3DGS rasterizer's own settings in splat mode: its thresholds, footprint cut at alpha 1/255
#: and a 0.3 px^2 dilation of the 2D covariance.
SPLAT_3DGS = dict(COMPAT, tau_cut=1.0 / 255.0, splat=True, splat_dilation=0.3)


# ------------------------------------------------------------------------------ Eq. 20
def kappa_from_theta(theta, scale):
    """Eq. 20: kappa = -ln(1 - 0.99 theta) (1/s_x + 1/s_y + 1/s_z) / 3, in FP64."""
    theta = np.asarray(theta, np.float64)
    s = np.asarray(scale, np.float64)
    return -np.log1p(-0.99 * theta) * (1.0 / s).sum(-1) / 3.0


def kappa_from_theta_grad(theta, scale, d_kappa):
    """Chain dL/dkappa through Eq. 20: returns (dL/dtheta, dL/dscale)."""
    theta = np.asarray(theta, np.float64)
    s = np.asarray(scale, np.float64)
    m = (1.0 / s).sum(-1) / 3.0
    lnv = -np.log1p(-0.99 * theta)
    d_theta = d_kappa * 0.99 / (1.0 - 0.99 * theta) * m
    d_scale = (d_kappa * lnv)[:, None] * (-1.0 / (3.0 * s * s))
    return d_theta, d_scale


def kappa_key_bound(theta, scale):
    """The FP32 upper bound of Eq. 20's kappa that sizes the footprint, with the GPU's operation
    order and only correctly rounded operations (no libm): with x = 0.99 theta and
    1 - x = m 2^-e (m in [0.5, 1)), -ln(1 - x) <= min(x / (1 - x), (e + 1) ln 2)."""
    f = np.float32
    th = np.asarray(theta, f)
    s = np.asarray(scale, f)
    x = f(0.99) * th
    om = f(1.0) - x
    b1 = x / om
    _, e = np.frexp(om)
    b2 = (f(1.0) - e.astype(f)) * f(0.6931472)
    lnb = np.minimum(b1, b2)
    m = ((f(1.0) / s[:, 0] + f(1.0) / s[:, 1]) + f(1.0) / s[:, 2]) * f(1.0 / 3.0)
    with np.errstate(invalid="ignore", divide="ignore"):
        out = lnb * m
    return np.where((th > 0) & (th <= 1), out, f(0.0)).astype(f)


def _density(scene, o, key=False):
    """The density each oracle function receives: kappa itself, or (density_theta) Eq. 20's
    kappa in FP64, or for the FP32 key function its upper bound."""
    if not (o or {}).get("density_theta"):
        return scene.kappa
    return kappa_key_bound(scene.kappa, scene.scale) if key else kappa_from_theta(scene.kappa, scene.scale)


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, FP64, OpenMP, no FP contraction)."""
    with _LOCK:
        stale = (not os.path.exists(_SO) or
                 os.path.getmtime(_SO) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
        if force or stale:
            tmp = _SO + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                   "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _SO)
    return _SO


def lib():
    global _LIB
    if _LIB is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        i32, i64, f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float
        L.orc_keys.restype = i64
        L.orc_keys.argtypes = [i32, P, P, P, P, i32, P, P, i32, i32, f32, f32, P, P, P]
        L.orc_tomo_keys.restype = i64
        L.orc_tomo_keys.argtypes = [i32, P, P, P, P, i32, P, i32, i32, f32, f32, f32, f32, i32, i32, f32, P, P]
        L.orc_keys_splat.restype = i64
        L.orc_keys_splat.argtypes = [i32, P, P, P, P, i32, P, P, i32, i32, f32, f32, f32, P, P, P]
        L.orc_splat2d.restype = None
        L.orc_splat2d.argtypes = [P, P, P, P, P, ctypes.c_double, P]
        L.orc_bin.restype = i64
        L.orc_bin.argtypes = [i32, i32, P, P, P, P, i64, i64, P, P]
        L.orc_sh_basis.restype = None
        L.orc_sh_basis.argtypes = [i32, P, P]
        L.orc_tau.restype = None
        L.orc_tau.argtypes = [P, P, P, ctypes.c_double, P, P, P]
        L.orc_render.restype = None
        L.orc_render.argtypes = [i32, P, P, P, P, P, i32, i32, P, P, i32, i32, P, P, P, P, i32, P, P, P, P, P, P, P,
                                 P, P]
        L.orc_render_grad.restype = None
        L.orc_render_grad.argtypes = [i32, P, P, P, P, P, i32, i32, P, P, i32, i32, P, P, P, P, P, P, P, P, P,
                                      P, P, P, P, P]
        L.orc_tomo.restype = None
        L.orc_tomo.argtypes = [i32, P, P, P, P, i32, P, i32, i32, f32, f32, f32, f32, i32, i32, P, P, P, i32, P, P, P]
        L.orc_tomo_grad.restype = None
        L.orc_tomo_grad.argtypes = [i32, P, P, P, P, i32, P, i32, i32, f32, f32, f32, f32, i32, i32, P, P, P, P, P,
                                    P, P, P, P]
        L.orc_cone.restype = None
        L.orc_cone.argtypes = [i32, P, P, P, P, i32, P, P, i32, i32, P, P, P, P, i32, P, P, P, P]
        L.orc_cone_grad.restype = None
        L.orc_cone_grad.argtypes = [i32, P, P, P, P, i32, P, P, i32, i32, P, P, P, P, P, P, P, P, P, P, P]
        L.orc_ray_march.restype = None
        L.orc_ray_march.argtypes = [i32, P, P, P, P, P, i32, i32, P, P, P, P, ctypes.c_double, ctypes.c_double,
                                    i32, P, P, P, P]
        L.orc_voxel_boxes.restype = i64
        L.orc_voxel_boxes.argtypes = [i32, P, P, P, P, P, P, P, f32, P]
        L.orc_voxel_density.restype = None
        L.orc_voxel_density.argtypes = [i32, P, P, P, P, P, i32, P, P, P, P, P]
        L.orc_num_threads.restype = i32
        L.orc_set_threads.restype = i32
        L.orc_set_threads.argtypes = [i32]
        _LIB = L
    return _LIB


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> int:
    """OpenMP threads of the oracle's later calls (n < 1: all cores); returns the count in use."""
    return int(lib().orc_set_threads(int(n)))


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _scene_arrays(scene, dt=np.float32):
    """FP32 for the key functions (the values the GPU sees), FP64 for everything else."""
    return (_c(scene.mu, dt), _c(scene.scale, dt), _c(scene.quat, dt), _c(scene.kappa, dt), _c(scene.sh, dt))


def cam_arrays(cams):
    cf = np.zeros((len(cams), 16), np.float32)
    wh = np.zeros((len(cams), 2), np.int32)
    for v, c in enumerate(cams):
        cf[v, :9] = np.asarray(c.R, np.float32).reshape(9)
        cf[v, 9:12] = np.asarray(c.t, np.float32)
        cf[v, 12:16] = [c.fx, c.fy, c.cx, c.cy]
        wh[v] = [c.width, c.height]
    return cf, wh


def tile_layout(cams, tile=(16, 16)):
    tx = np.array([(c.width + tile[0] - 1) // tile[0] for c in cams], np.int32)
    ty = np.array([(c.height + tile[1] - 1) // tile[1] for c in cams], np.int32)
    base = np.zeros(len(cams), np.int32)
    if len(cams) > 1:
        base[1:] = np.cumsum(tx * ty)[:-1]
    return tx, ty, base, int((tx * ty).sum())


def pix_bases(cams):
    sizes = np.array([c.width * c.height for c in cams], np.int64)
    base = np.zeros(len(cams), np.int64)
    if len(cams) > 1:
        base[1:] = np.cumsum(sizes)[:-1]
    return base, int(sizes.sum())


def _opts_arr(opts):
    o = dict(EXACT)
    o.update(opts or {})
    bg = o["bg"]
    return np.array([o["alpha_min"], o["tau_cut"], o["tau_max"], o["T_stop"], bg[0], bg[1], bg[2],
                     o["z_near"], o.get("softplus_beta", 0.0), 1.0 if o.get("splat") else 0.0,
                     o.get("splat_dilation", 0.0)], np.float64), o


# ------------------------------------------------------------------------------------------
def keys(scene, cams, opts=None, tile=(16, 16), with_pixels=False):
    """FP32 key function: depth key bits [V, N] (0xFFFFFFFF = invalid or behind z_near),
    tile rectangles [V, N, 4] = (tx0, ty0, tx1, ty1) inclusive, -1 when culled, and (with
    with_pixels) the pixel footprint rectangles [V, N, 4] = (x0, y0, x1, y1) inclusive."""
    _, o = _opts_arr(opts)
    mu, sc, q, _k, _sh = _scene_arrays(scene)
    k = _c(_density(scene, o, key=True), np.float32)
    cf, wh = cam_arrays(cams)
    V, N = len(cams), scene.n
    depth = np.zeros((V, N), np.uint32)
    rect = np.zeros((V, N, 4), np.int32)
    prect = np.zeros((V, N, 4), np.int32)
    if o.get("splat"):
        lib().orc_keys_splat(N, _p(mu), _p(sc), _p(q), _p(k), V, _p(cf), _p(wh), tile[0], tile[1],
                             np.float32(o["z_near"]), np.float32(o["tau_cut"]), np.float32(o["splat_dilation"]),
                             _p(depth), _p(rect), _p(prect))
    else:
        lib().orc_keys(N, _p(mu), _p(sc), _p(q), _p(k), V, _p(cf), _p(wh), tile[0], tile[1],
                       np.float32(o["z_near"]), np.float32(o["tau_cut"]), _p(depth), _p(rect), _p(prect))
    return (depth, rect, prect) if with_pixels else (depth, rect)


def bin(scene_n, n_views, depth, rect, tiles_x, tile_base, n_tiles):
    """Stable per-tile lists sorted by (tile, depth key, Gaussian index)."""
    rect = _c(rect, np.int32)
    dep = None if depth is None else _c(depth, np.uint32)
    tiles_x = _c(tiles_x, np.int32)
    tile_base = _c(tile_base, np.int32)
    ts = np.zeros(n_tiles + 1, np.int64)
    r = rect.reshape(-1, 4)
    vis = r[:, 0] >= 0
    total = int(((r[vis, 2] - r[vis, 0] + 1).astype(np.int64) * (r[vis, 3] - r[vis, 1] + 1)).sum())
    sg = np.zeros(max(total, 1), np.int32)
    got = lib().orc_bin(scene_n, n_views, _p(dep), _p(rect), _p(tiles_x), _p(tile_base), n_tiles, total,
                        _p(ts), _p(sg))
    assert got == total
    return ts, sg[:total]


def lists(scene, cams, opts=None, tile=(16, 16)):
    depth, rect, prect = keys(scene, cams, opts, tile, with_pixels=True)
    tx, ty, base, nt = tile_layout(cams, tile)
    ts, sg = bin(scene.n, len(cams), depth, rect, tx, base, nt)
    return dict(depth=depth, rect=rect, prect=prect, tile_start=ts, sorted_g=sg, tiles_x=tx, tiles_y=ty,
                tile_base=base, n_tiles=nt, tile=tile)


def render(scene, cams, opts=None, L=None, brute=False, mask=None, tile=(16, 16), diag=False):
    """Blend every pixel (Eq. 14 with the Eq. 19 alpha).  Returns per-view lists of
    rgb [H, W, 3] and T_final [H, W] (float64) and the blended-Gaussian count.  With diag=True a
    fourth item holds flat per-pixel arrays (views concatenated): "last" = position + 1, within the
    pixel's tile list, of the last blended pair (0 when none), "S" = sum of the blended tau, and
    "m_skip" / "m_clamp" / "m_stop" = the relative distance of the pixel's closest alpha_min,
    tau_max and T_stop decision to its threshold (inf when it met none)."""
    oa, o = _opts_arr(opts)
    if L is None:
        L = lists(scene, cams, o, tile)
    mu, sc, q, _k, sh = _scene_arrays(scene, np.float64)
    k = _c(_density(scene, o), np.float64)
    cf, wh = cam_arrays(cams)
    pb, P = pix_bases(cams)
    rgb = np.zeros((P, 3), np.float64)
    T = np.zeros(P, np.float64)
    nb = np.zeros(P, np.int32)
    last = np.zeros(P, np.int64) if diag else None
    dg = np.zeros((P, 4), np.float64) if diag else None
    m = None if mask is None else _c(mask, np.int32)
    lib().orc_render(scene.n, _p(mu), _p(sc), _p(q), _p(k), _p(sh), scene.sh_degree, len(cams), _p(cf), _p(wh),
                     L["tile"][0], L["tile"][1], _p(oa), _p(L["tile_start"]), _p(L["sorted_g"]),
                     _p(_c(L["tile_base"], np.int32)), int(brute), _p(_c(L["depth"], np.uint32)),
                     _p(_c(L["prect"], np.int32)), _p(pb), _p(m), _p(rgb), _p(T), _p(nb), _p(last), _p(dg))
    out_rgb, out_T, out_n = [], [], []
    for v, c in enumerate(cams):
        s = slice(pb[v], pb[v] + c.width * c.height)
        out_rgb.append(rgb[s].reshape(c.height, c.width, 3))
        out_T.append(T[s].reshape(c.height, c.width))
        out_n.append(nb[s].reshape(c.height, c.width))
    if diag:
        return out_rgb, out_T, out_n, dict(last=last, S=dg[:, 0], m_skip=dg[:, 1], m_clamp=dg[:, 2],
                                           m_stop=dg[:, 3])
    return out_rgb, out_T, out_n


def render_grad(scene, cams, opts, L, dL_drgb, dL_dT=None, mask=None):
    """Analytic FP64 gradient of sum(dL_drgb * rgb) + sum(dL_dT * T_final) with the tile
    lists `L` held fixed.  dL_drgb / dL_dT are per-view lists (or flat arrays)."""
    oa, o = _opts_arr(opts)
    mu, sc, q, _k, sh = _scene_arrays(scene, np.float64)
    k = _c(_density(scene, o), np.float64)
    cf, wh = cam_arrays(cams)
    pb, P = pix_bases(cams)
    g_rgb = _c(np.concatenate([np.asarray(a, np.float64).reshape(-1, 3) for a in dL_drgb])
               if isinstance(dL_drgb, (list, tuple)) else np.asarray(dL_drgb).reshape(-1, 3), np.float64)
    g_T = None
    if dL_dT is not None:
        g_T = _c(np.concatenate([np.asarray(a, np.float64).reshape(-1) for a in dL_dT])
                 if isinstance(dL_dT, (list, tuple)) else np.asarray(dL_dT).reshape(-1), np.float64)
    N, K = scene.n, (scene.sh_degree + 1) ** 2
    out = dict(mu=np.zeros((N, 3)), scale=np.zeros((N, 3)), quat=np.zeros((N, 4)), kappa=np.zeros(N),
               sh=np.zeros((N, K, 3)))
    m = None if mask is None else _c(mask, np.int32)
    lib().orc_render_grad(N, _p(mu), _p(sc), _p(q), _p(k), _p(sh), scene.sh_degree, len(cams), _p(cf), _p(wh),
                          L["tile"][0], L["tile"][1], _p(oa), _p(L["tile_start"]), _p(L["sorted_g"]),
                          _p(_c(L["tile_base"], np.int32)), _p(_c(L["prect"], np.int32)), _p(pb), _p(g_rgb),
                          _p(g_T), _p(m),
                          _p(out["mu"]), _p(out["scale"]), _p(out["quat"]), _p(out["kappa"]), _p(out["sh"]))
    if o.get("density_theta"):   # chain dL/dkappa through Eq. 20: "kappa" becomes dL/dtheta
        d_theta, d_scale = kappa_from_theta_grad(scene.kappa, scene.scale, out["kappa"])
        out["kappa"] = d_theta
        out["scale"] = out["scale"] + d_scale
    return out


def ray_march(scene, cams, opts=None, t_near=0.2, t_far=10.0, n_samples=256, mask=None, depth=None):
    """Supp. A's ray-marching reference: NeRF's quadrature of Eq. 1 with sigma = sum kappa G and
    c = sum c kappa G / sigma at n_samples midpoints of [t_near, t_far] along each pixel's unit
    ray, over every Gaussian with a valid depth key (no lists, no order, no overlap assumption).
    Returns per-view lists of rgb [H, W, 3] and T [H, W] (float64)."""
    oa, o = _opts_arr(opts)
    if depth is None:
        depth, _ = keys(scene, cams, o)
    mu, sc, q, _k, sh = _scene_arrays(scene, np.float64)
    k = _c(_density(scene, o), np.float64)
    cf, wh = cam_arrays(cams)
    pb, P = pix_bases(cams)
    rgb = np.zeros((P, 3), np.float64)
    T = np.zeros(P, np.float64)
    m = None if mask is None else _c(mask, np.int32)
    lib().orc_ray_march(scene.n, _p(mu), _p(sc), _p(q), _p(k), _p(sh), scene.sh_degree, len(cams), _p(cf), _p(wh),
                        _p(oa), _p(_c(depth, np.uint32)), float(t_near), float(t_far), int(n_samples), _p(pb), _p(m),
                        _p(rgb), _p(T))
    out_rgb, out_T = [], []
    for v, c in enumerate(cams):
        s_ = slice(pb[v], pb[v] + c.width * c.height)
        out_rgb.append(rgb[s_].reshape(c.height, c.width, 3))
        out_T.append(T[s_].reshape(c.height, c.width))
    return out_rgb, out_T


def tau(scene, g, o, d):
    """Closed-form line integral of Gaussian g along o + t d (d unit) and the Supp. B
    quantities: dict(tau, a, b, c, gamma, beta, gmax)."""
    out = np.zeros(7, np.float64)
    mu = _c(scene.mu[g], np.float64)
    sc = _c(scene.scale[g], np.float64)
    q = _c(scene.quat[g], np.float64)
    lib().orc_tau(_p(mu), _p(sc), _p(q), float(scene.kappa[g]), _p(_c(o, np.float64)),
                  _p(_c(d, np.float64)), _p(out))
    return dict(zip(("tau", "a", "b", "c", "gamma", "beta", "gmax"), out.tolist()))


def splat2d(scene, g, cam, dilation=0.0):
    """The projected 2D Gaussian of Gaussian g (Eq. 7, FP64): (mu' [2], Sigma' [2, 2]) in pixel index
    coordinates (pixel x has its centre at x), or None when it is not in front of the camera."""
    out = np.zeros(6, np.float64)
    cf, wh = cam_arrays([cam])
    lib().orc_splat2d(_p(_c(scene.mu[g], np.float64)), _p(_c(scene.scale[g], np.float64)),
                      _p(_c(scene.quat[g], np.float64)), _p(cf), _p(wh), float(dilation), _p(out))
    if out[5] == 0:
        return None
    return out[:2].copy(), np.array([[out[2], out[3]], [out[3], out[4]]])


def sh_basis(degree, direction):
    out = np.zeros(16, np.float64)
    lib().orc_sh_basis(degree, _p(_c(direction, np.float64)), _p(out))
    return out[: (degree + 1) ** 2]


# ------------------------------------------------------------------------------ tomography
def tomo_keys(scene, beam, tau_cut=1e-6, tile=(16, 16), with_pixels=False, density_theta=False):
    mu, sc, q, _k, _ = _scene_arrays(scene)
    k = _c(_density(scene, dict(density_theta=density_theta), key=True), np.float32)
    A, N = len(beam.angles), scene.n
    rect = np.zeros((A, N, 4), np.int32)
    prect = np.zeros((A, N, 4), np.int32)
    lib().orc_tomo_keys(N, _p(mu), _p(sc), _p(q), _p(k), A, _p(_c(beam.angles, np.float32)), beam.det_w,
                        beam.det_h, beam.pitch_u, beam.pitch_v, beam.u0, beam.v0, tile[0], tile[1],
                        np.float32(tau_cut), _p(rect), _p(prect))
    return (rect, prect) if with_pixels else rect


def tomo_lists(scene, beam, tau_cut=1e-6, tile=(16, 16), density_theta=False):
    rect, prect = tomo_keys(scene, beam, tau_cut, tile, with_pixels=True, density_theta=density_theta)
    A = len(beam.angles)
    tx = (beam.det_w + tile[0] - 1) // tile[0]
    ty = (beam.det_h + tile[1] - 1) // tile[1]
    txs = np.full(A, tx, np.int32)
    base = (np.arange(A) * tx * ty).astype(np.int32)
    ts, sg = bin(scene.n, A, None, rect, txs, base, A * tx * ty)
    return dict(rect=rect, prect=prect, tile_start=ts, sorted_g=sg, tiles_x=tx, tiles_y=ty, n_tiles=A * tx * ty,
                tile=tile)


def tomo(scene, beam, L=None, brute=False, mask=None, tau_cut=1e-6, tile=(16, 16), density_theta=False):
    """Parallel-beam projection: returns (line_sum, proj = exp(-line_sum)), each [A, H, W]."""
    if L is None and not brute:
        L = tomo_lists(scene, beam, tau_cut, tile, density_theta)
    mu, sc, q, _k, _ = _scene_arrays(scene, np.float64)
    k = _c(_density(scene, dict(density_theta=density_theta)), np.float64)
    A = len(beam.angles)
    ls = np.zeros((A, beam.det_h, beam.det_w))
    proj_out = np.zeros((A, beam.det_h, beam.det_w))
    ts = L["tile_start"] if L is not None else np.zeros(1, np.int64)
    sg = L["sorted_g"] if L is not None else np.zeros(1, np.int32)
    pr = _c(L["prect"], np.int32) if L is not None else None
    tl = L["tile"] if L is not None else tile
    m = None if mask is None else _c(mask, np.int32)
    lib().orc_tomo(scene.n, _p(mu), _p(sc), _p(q), _p(k), A, _p(_c(beam.angles, np.float32)), beam.det_w,
                   beam.det_h, beam.pitch_u, beam.pitch_v, beam.u0, beam.v0, tl[0], tl[1], _p(ts), _p(sg),
                   _p(pr), int(brute), _p(m), _p(ls), _p(proj_out))
    return ls, proj_out


def tomo_grad(scene, beam, L, dL_dproj, mask=None, density_theta=False):
    mu, sc, q, _k, _ = _scene_arrays(scene, np.float64)
    k = _c(_density(scene, dict(density_theta=density_theta)), np.float64)
    A, N = len(beam.angles), scene.n
    out = dict(mu=np.zeros((N, 3)), scale=np.zeros((N, 3)), quat=np.zeros((N, 4)), kappa=np.zeros(N))
    m = None if mask is None else _c(mask, np.int32)
    lib().orc_tomo_grad(N, _p(mu), _p(sc), _p(q), _p(k), A, _p(_c(beam.angles, np.float32)), beam.det_w,
                        beam.det_h, beam.pitch_u, beam.pitch_v, beam.u0, beam.v0, L["tile"][0], L["tile"][1],
                        _p(L["tile_start"]), _p(L["sorted_g"]), _p(_c(L["prect"], np.int32)),
                        _p(_c(dL_dproj, np.float64)), _p(m),
                        _p(out["mu"]), _p(out["scale"]), _p(out["quat"]), _p(out["kappa"]))
    if density_theta:
        d_theta, d_scale = kappa_from_theta_grad(scene.kappa, scene.scale, out["kappa"])
        out["kappa"] = d_theta
        out["scale"] = out["scale"] + d_scale
    return out


# ------------------------------------------------------------------------------ cone beam
def cone(scene, cams, opts=None, L=None, brute=False, mask=None, tile=(16, 16)):
    """Cone-beam projection (Eq. 21 with diverging rays): the source at each camera's centre and
    the detector its image plane.  Returns per-view lists of (line_sum, proj = exp(-line_sum)),
    each [H, W].  Tiled evaluation uses the perspective key function's lists and pixel
    rectangles (opts' tau_cut); brute force sums every valid Gaussian."""
    _, o = _opts_arr(opts)
    if L is None and not brute:
        L = lists(scene, cams, o, tile)
    mu, sc, q, _k, _ = _scene_arrays(scene, np.float64)
    k = _c(_density(scene, o), np.float64)
    cf, wh = cam_arrays(cams)
    pb, P = pix_bases(cams)
    ls = np.zeros(P)
    pr = np.zeros(P)
    m = None if mask is None else _c(mask, np.int32)
    tl = L["tile"] if L is not None else tile
    ts = L["tile_start"] if L is not None else np.zeros(1, np.int64)
    sg = L["sorted_g"] if L is not None else np.zeros(1, np.int32)
    tb = _c(L["tile_base"], np.int32) if L is not None else np.zeros(len(cams), np.int32)
    prc = _c(L["prect"], np.int32) if L is not None else None
    lib().orc_cone(scene.n, _p(mu), _p(sc), _p(q), _p(k), len(cams), _p(cf), _p(wh), tl[0], tl[1], _p(ts), _p(sg),
                   _p(tb), _p(prc), int(brute), _p(pb), _p(m), _p(ls), _p(pr))
    out = []
    for v, c in enumerate(cams):
        sl = slice(pb[v], pb[v] + c.width * c.height)
        out.append((ls[sl].reshape(c.height, c.width), pr[sl].reshape(c.height, c.width)))
    return out


def cone_grad(scene, cams, opts, L, dL_dproj, mask=None):
    """Analytic FP64 gradient of sum(dL_dproj * proj) for the cone beam (lists held fixed)."""
    _, o = _opts_arr(opts)
    mu, sc, q, _k, _ = _scene_arrays(scene, np.float64)
    k = _c(_density(scene, o), np.float64)
    cf, wh = cam_arrays(cams)
    pb, P = pix_bases(cams)
    g = _c(np.concatenate([np.asarray(a, np.float64).reshape(-1) for a in dL_dproj])
           if isinstance(dL_dproj, (list, tuple)) else np.asarray(dL_dproj).reshape(-1), np.float64)
    N = scene.n
    out = dict(mu=np.zeros((N, 3)), scale=np.zeros((N, 3)), quat=np.zeros((N, 4)), kappa=np.zeros(N))
    m = None if mask is None else _c(mask, np.int32)
    lib().orc_cone_grad(N, _p(mu), _p(sc), _p(q), _p(k), len(cams), _p(cf), _p(wh), L["tile"][0], L["tile"][1],
                        _p(L["tile_start"]), _p(L["sorted_g"]), _p(_c(L["tile_base"], np.int32)),
                        _p(_c(L["prect"], np.int32)), _p(pb), _p(g), _p(m),
                        _p(out["mu"]), _p(out["scale"]), _p(out["quat"]), _p(out["kappa"]))
    if o.get("density_theta"):
        d_theta, d_scale = kappa_from_theta_grad(scene.kappa, scene.scale, out["kappa"])
        out["kappa"] = d_theta
        out["scale"] = out["scale"] + d_scale
    return out


# ------------------------------------------------------------------------------ voxel density
def voxel_boxes(scene, origin, voxel, dims, sigma_cut=1e-6, density_theta=False):
    """Per-Gaussian truncation boxes [N, 6] = (x0, y0, z0, x1, y1, z1) inclusive voxel indices
    (-1 when empty), FP32 with the GPU's operation order; returns (boxes, total voxel pairs)."""
    mu, sc, q, _k, _ = _scene_arrays(scene)
    k = _c(_density(scene, dict(density_theta=density_theta), key=True), np.float32)
    box = np.zeros((scene.n, 6), np.int32)
    tot = lib().orc_voxel_boxes(scene.n, _p(mu), _p(sc), _p(q), _p(k), _p(_c(origin, np.float32)),
                                _p(_c(voxel, np.float32)), _p(_c(dims, np.int32)), np.float32(sigma_cut), _p(box))
    return box, int(tot)


def voxel_density(scene, origin, voxel, dims, sigma_cut=1e-6, brute=False, mask=None, density_theta=False):
    """sigma(x) = sum_g kappa_g G_g(x) at the voxel centres, [nz, ny, nx] (float64)."""
    box, _ = voxel_boxes(scene, origin, voxel, dims, sigma_cut, density_theta)
    mu, sc, q, _k, _ = _scene_arrays(scene, np.float64)
    k = _c(_density(scene, dict(density_theta=density_theta)), np.float64)
    nx, ny, nz = (int(d) for d in dims)
    out = np.zeros(nx * ny * nz)
    m = None if mask is None else _c(np.asarray(mask).reshape(-1), np.int32)
    lib().orc_voxel_density(scene.n, _p(mu), _p(sc), _p(q), _p(k), _p(box), int(brute),
                            _p(_c(origin, np.float32)), _p(_c(voxel, np.float32)), _p(_c(dims, np.int32)), _p(m),
                            _p(out))
    return out.reshape(nz, ny, nx)
