"""The ray-marching reference of Supp. A (NeRF quadrature of Eq. 1 with sigma = sum kappa G) on the
GPU against the FP64 oracle's march, and its overlap-error map against the rasterizer.

Scenes use Gaussians at least 0.02 wide along every axis, so that the 1D Gaussian along each ray
spans several samples: a march of sub-sample Gaussians is dominated by where the samples fall,
which FP32 and FP64 place differently."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev_scene, flat, run_forward

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4


def _march(vg, ws, P, t0, t1, n, raster=None):
    import torch
    dev = torch.device("cuda:0")
    rgb = torch.full((P, 3), float("nan"), device=dev)
    T = torch.full((P,), float("nan"), device=dev)
    err = None
    r = None
    if raster is not None:
        r = torch.as_tensor(np.ascontiguousarray(raster, np.float32)).to(dev)
        err = torch.full((P,), float("nan"), device=dev)
    ws.ray_march(t0, t1, n, rgb, T, r, err)
    torch.cuda.synchronize()
    out = [rgb.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64)]
    if err is not None:
        out.append(err.cpu().numpy().astype(np.float64))
    return out


def _scene(n, seed):
    sc = synth.uniform_scene(n, seed, log_scale=(-3.9, -2.3), kappa=(0.5, 20.0), sh_degree=1, sh_std=0.3,
                             extent=0.8)
    return sc


@pytest.mark.parametrize("theta,tile", [(False, (0, 0)), (True, (0, 0)), (False, (32, 16)), (False, (16, 8))])
def test_ray_march_matches_oracle(gpu_lib, theta, tile):
    """The march over each tile shape's lists (one CTA per tile, one pixel per thread)."""
    vg = gpu_lib
    sc = _scene(300, 61)
    o = dict(oracle.EXACT, bg=(0.2, 0.1, 0.4))
    if theta:
        sc.kappa = np.random.default_rng(62).uniform(0.05, 0.95, sc.n).astype(np.float32)
        o["density_theta"] = True
    cams = [synth.look_at((0.3, -0.4, -4.0), (0, 0, 0), 53, 37, 50.0),
            synth.look_at((-3.5, 0.5, 1.0), (0, 0, 0), 40, 30, 45.0)]
    ws, g, raster, _ = run_forward(vg, sc, cams, o, tile=tile)
    P = raster.shape[0]
    rgb, T, err = _march(vg, ws, P, 1.5, 7.0, 300, raster)
    ref_rgb, ref_T = oracle.ray_march(sc, cams, o, 1.5, 7.0, 300)
    assert np.max(np.abs(rgb - flat(ref_rgb))) < IMG_TOL
    assert np.max(np.abs(T - flat(ref_T))) < IMG_TOL
    want = np.max(np.abs(rgb.astype(np.float32) - raster.astype(np.float32)), axis=1)
    assert np.max(np.abs(err - want)) < 1e-6


def test_overlap_error_map_localises_overlap(gpu_lib):
    """Supp. A rows 1-3: Gaussians far apart along the rays match the blend to quadrature accuracy;
    two heavily overlapping ones do not, and the error map marks the overlap."""
    vg = gpu_lib
    def one(mu, s, q, k, c):
        return synth.Scene(np.array([mu], np.float32), np.array([s], np.float32), np.array([q], np.float32),
                           np.array([k], np.float32), np.array([[c]], np.float32), 0)

    def cat(*ss):
        return synth.Scene(*(np.concatenate([getattr(s, f) for s in ss]) for f in ("mu", "scale", "quat", "kappa", "sh")), 0)

    q = synth.random_unit_quats(np.random.default_rng(7), 4)
    sep = cat(one((0.01, 0.0, -1.0), (0.08, 0.06, 0.1), q[0], 3.0, (1.0, -0.5, 0.2)),
              one((-0.02, 0.01, 0.0), (0.07, 0.09, 0.05), q[1], 6.0, (-0.4, 0.9, 0.3)),
              one((0.0, -0.01, 1.0), (0.1, 0.08, 0.09), q[2], 1.5, (0.3, 0.3, -0.8)))
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 48, 40, 8.0)
    o = oracle.EXACT
    ws, _, raster, _ = run_forward(vg, sep, [cam], o)
    _, _, err = _march(vg, ws, raster.shape[0], 1.0, 7.0, 20000, raster)
    assert err.max() < 2e-4
    # two overlapping Gaussians at x = -0.2 and a lone one at x = +0.2 (columns ~10 and ~37)
    cam2 = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 48, 40, 10.0)
    ovl = cat(one((-0.2, 0.0, 0.0), (0.06, 0.06, 0.06), q[0], 6.0, (1.0, -0.5, 0.2)),
              one((-0.2, 0.0, 0.012), (0.06, 0.06, 0.06), q[1], 6.0, (-0.4, 0.9, 0.3)),
              one((0.2, 0.0, 0.0), (0.05, 0.05, 0.05), q[3], 6.0, (0.2, 0.2, 0.2)))
    ws2, _, raster2, _ = run_forward(vg, ovl, [cam2], o)
    _, _, err2 = _march(vg, ws2, raster2.shape[0], 1.0, 7.0, 20000, raster2)
    e = err2.reshape(cam2.height, cam2.width)
    fx = float(np.float32(cam2.fx))
    col_pair, col_lone = int(cam2.cx - 0.5 - fx * 0.05), int(cam2.cx - 0.5 + fx * 0.05)
    assert e[cam2.height // 2, col_pair] > 1e-2               # where the two overlap
    assert e[:, col_lone - 3:col_lone + 4].max() < 2e-4       # around the lone Gaussian


def test_ray_march_rejections(gpu_lib):
    vg = gpu_lib
    import torch
    sc = _scene(20, 63)
    cam = synth.look_at((0.0, 0.0, -4.0), (0, 0, 0), 16, 16, 50.0)
    ws = vg.Workspace()
    out = torch.zeros(256, 3, device="cuda:0")
    with pytest.raises(RuntimeError):
        ws.ray_march(1.0, 5.0, 64, out)          # nothing binned yet
    ws, g, _, _ = run_forward(vg, sc, [cam], oracle.EXACT, ws=ws)
    for t0, t1, n in [(5.0, 1.0, 64), (1.0, 5.0, 0), (-1.0, 5.0, 64)]:
        with pytest.raises(RuntimeError):
            ws.ray_march(t0, t1, n, out)
    with pytest.raises(RuntimeError):
        ws.ray_march(1.0, 5.0, 64, out, None, None, torch.zeros(256, device="cuda:0"))   # error map, no raster
    ws2, _, _, _ = run_forward(vg, sc, [cam], dict(oracle.EXACT, splat=True))
    with pytest.raises(RuntimeError):
        ws2.ray_march(1.0, 5.0, 64, out)
