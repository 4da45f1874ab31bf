"""Voxel density query (sigma = sum kappa G of Eq. 3-4 on a grid) on the GPU against the FP64 oracle.

A large sigma_cut makes the truncation boxes visible in the values (a voxel that one side
includes and the other leaves out differs by at least sigma_cut), so those cases also check
that the GPU's boxes equal the oracle's FP32 boxes exactly."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev_scene, vg_opts

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4   # of the largest |sigma| on the grid


def _query(vg, scene, origin, voxel, dims, sigma_cut, theta=False, ws=None, g=None):
    import torch
    g = g or dev_scene(vg, scene)
    ws = ws or vg.Workspace()
    nx, ny, nz = dims
    out = torch.full((nz, ny, nx), float("nan"), device="cuda:0")
    o = dict(oracle.EXACT, tau_cut=sigma_cut, density_theta=theta)
    ws.query_density(g, origin, voxel, dims, vg_opts(vg, o), out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def _check(got, ref):
    assert np.all(np.isfinite(got))
    scale = max(np.max(np.abs(ref)), 1e-30)
    err = np.max(np.abs(got - ref))
    assert err <= REL_TOL * scale, (err, scale)


@pytest.mark.parametrize("sigma_cut", [1e-6, 0.3])
@pytest.mark.parametrize("theta", [False, True])
def test_voxel_density_small(gpu_lib, sigma_cut, theta):
    """300 Gaussians in the unit ball, a 37 x 29 x 21 grid (ragged 8^3 bricks) over [-1.1, 1.1]^3."""
    vg = gpu_lib
    scene = synth.tomo_scene(300, 97, log_scale=(-3.5, -1.5))
    if theta:
        scene.kappa = np.random.default_rng(98).uniform(0.0, 1.0, scene.n).astype(np.float32)
    dims = (37, 29, 21)
    origin = (-1.1, -1.1, -1.1)
    voxel = (2.2 / 37, 2.2 / 29, 2.2 / 21)
    got = _query(vg, scene, origin, voxel, dims, sigma_cut, theta)
    ref = oracle.voxel_density(scene, origin, voxel, dims, sigma_cut=sigma_cut, density_theta=theta)
    _check(got, ref)


def test_voxel_density_partial_grid_and_outside(gpu_lib):
    """A grid covering one octant: Gaussians straddling the grid's faces are clipped, those
    entirely outside contribute nothing; a second query on the same workspace reuses its buffers."""
    vg = gpu_lib
    scene = synth.tomo_scene(500, 99, log_scale=(-3.0, -1.8))
    ws = vg.Workspace()
    g = dev_scene(vg, scene)
    for dims, origin, voxel in [((24, 17, 9), (0.0, 0.1, -0.2), (0.04, 0.05, 0.07)),
                                ((8, 8, 8), (5.0, 5.0, 5.0), (0.1, 0.1, 0.1)),
                                ((1, 1, 1), (-0.01, -0.01, -0.01), (0.02, 0.02, 0.02))]:
        got = _query(vg, scene, origin, voxel, dims, 0.05, ws=ws, g=g)
        ref = oracle.voxel_density(scene, origin, voxel, dims, sigma_cut=0.05)
        if np.max(np.abs(ref)) == 0.0:
            assert np.all(got == 0.0)
        else:
            _check(got, ref)


def test_voxel_density_empty_scene(gpu_lib):
    vg = gpu_lib
    scene = synth.tomo_scene(1, 100)
    scene.kappa[:] = 0.0   # no density: nothing to bin
    got = _query(vg, scene, (-1, -1, -1), (0.25, 0.25, 0.25), (8, 9, 10), 1e-6)
    assert np.all(got == 0.0)


def test_voxel_density_rejects_bad_grid(gpu_lib):
    vg = gpu_lib
    import torch
    scene = synth.tomo_scene(10, 101)
    g = dev_scene(vg, scene)
    ws = vg.Workspace()
    out = torch.zeros(8, device="cuda:0")
    o = vg_opts(vg, dict(oracle.EXACT, tau_cut=1e-6))
    for origin, voxel, dims in [((0, 0, 0), (0.1, 0.0, 0.1), (2, 2, 2)),
                                ((0, 0, 0), (0.1, 0.1, 0.1), (2, 0, 2)),
                                ((0, 0, float("nan")), (0.1, 0.1, 0.1), (2, 2, 2)),
                                ((0, 0, 0), (0.1, 0.1, 0.1), (40000, 2, 2))]:
        with pytest.raises(RuntimeError):
            ws.query_density(g, origin, voxel, dims, o, out)


def test_voxel_density_full_size_sampled(gpu_lib):
    """The 200,000-Gaussian tomography scene on a 256^3 grid over [-1, 1]^3 (the reconstruction
    grid of a volumetric comparison), checked on 2,000 sampled voxels."""
    vg = gpu_lib
    scene, _, _ = synth.config4(1.0)
    dims = (256, 256, 256)
    origin = (-1.0, -1.0, -1.0)
    voxel = (2.0 / 256,) * 3
    got = _query(vg, scene, origin, voxel, dims, 1e-6)
    rng = np.random.default_rng(102)
    pick = rng.choice(256 ** 3, 2000, replace=False)
    mask = np.zeros(256 ** 3, np.int32)
    mask[pick] = 1
    ref = oracle.voxel_density(scene, origin, voxel, dims, sigma_cut=1e-6, mask=mask).reshape(-1)
    g_s, r_s = got.reshape(-1)[pick], ref[pick]
    scale = np.max(np.abs(r_s))
    assert scale > 0
    assert np.max(np.abs(g_s - r_s)) <= REL_TOL * scale
