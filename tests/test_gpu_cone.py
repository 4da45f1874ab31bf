"""Cone-beam tomography (Eq. 21 with diverging rays) on the GPU against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import check_grads, dev_scene, vg_opts

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4
GRAD_TOL = 1e-3


def _run(vg, scene, cams, o, dL=None, ws=None, g=None, tile=(0, 0)):
    import torch
    dev = torch.device("cuda:0")
    g = g or dev_scene(vg, scene)
    ws = ws or vg.Workspace()
    P = sum(c.width * c.height for c in cams)
    proj = torch.full((P,), float("nan"), device=dev)
    grads = None
    if dL is not None:
        grads = [torch.zeros(scene.n, 3, device=dev), torch.zeros(scene.n, 3, device=dev),
                 torch.zeros(scene.n, 4, device=dev), torch.zeros(scene.n, device=dev)]
        ws.project_cone(g, cams, vg_opts(vg, o, tile=tile), proj,
                        torch.as_tensor(np.ascontiguousarray(dL, np.float32)).to(dev), *grads)
    else:
        ws.project_cone(g, cams, vg_opts(vg, o, tile=tile), proj)
    torch.cuda.synchronize()
    out = proj.cpu().numpy().astype(np.float64)
    if grads is not None:
        grads = {k: t.cpu().numpy().astype(np.float64) for k, t in zip(("mu", "scale", "quat", "kappa"), grads)}
    return ws, out, grads


@pytest.mark.parametrize("theta,tile", [(False, (0, 0)), (True, (0, 0)), (False, (16, 8)), (True, (32, 16))])
def test_cone_projection_and_gradient(gpu_lib, theta, tile):
    vg = gpu_lib
    scene = synth.tomo_scene(400, 95, log_scale=(-4.0, -2.5))
    o = dict(oracle.EXACT, density_theta=theta)
    rng = np.random.default_rng(96)
    if theta:
        scene.kappa = rng.uniform(0.0, 1.0, scene.n).astype(np.float32)
    cams = synth.cone_beam(3, det=48) + [synth.look_at((0.5, -3.0, 1.0), (0, 0, 0), 37, 29, 45.0)]
    P = sum(c.width * c.height for c in cams)
    dL = rng.normal(size=P)
    ws, proj, gg = _run(vg, scene, cams, o, dL, tile=tile)
    L = oracle.lists(scene, cams, o, tile=tile if tile[0] else (16, 16))
    depth, rect = ws.read_keys()
    assert np.array_equal(depth, L["depth"].reshape(-1)) and np.array_equal(rect, L["rect"].reshape(-1, 4))
    ts, items = ws.read_bins()
    assert np.array_equal(ts, L["tile_start"]) and np.array_equal(items % scene.n, L["sorted_g"])
    ref = np.concatenate([pr.reshape(-1) for _, pr in oracle.cone(scene, cams, o, L)])
    assert np.max(np.abs(proj - ref)) < IMG_TOL
    split = np.cumsum([0] + [c.width * c.height for c in cams])
    refg = oracle.cone_grad(scene, cams, o, L, [dL[split[v]:split[v + 1]] for v in range(len(cams))])
    check_grads(gg, refg, scene, GRAD_TOL, keys=("mu", "scale", "quat", "kappa"))


def test_cone_full_size(gpu_lib):
    """Config 4's 200,000 Gaussians, 64 sources on a circle, 512^2 detectors; sources 0 and 40
    at sampled pixels against the oracle, projection and gradient."""
    vg = gpu_lib
    scene, _, _ = synth.config4(1.0)
    cams = synth.cone_beam(64, det=512)
    o = dict(oracle.EXACT)
    P = sum(c.width * c.height for c in cams)
    rng = np.random.default_rng(97)
    pick = [0, 40]
    masks = []
    for v in pick:
        m = np.zeros(512 * 512, np.int32)
        m[rng.choice(512 * 512, size=3000, replace=False)] = 1
        masks.append(m)
    dL = np.zeros(P)
    for v, m in zip(pick, masks):
        dL[v * 512 * 512:(v + 1) * 512 * 512] = rng.normal(size=512 * 512) * m
    _, proj, gg = _run(vg, scene, cams, o, dL)
    sub = [cams[v] for v in pick]
    L = oracle.lists(scene, sub, o)
    mask = np.concatenate(masks)
    ref = oracle.cone(scene, sub, o, L, mask=mask)
    for i, v in enumerate(pick):
        sel = masks[i].astype(bool)
        got = proj[v * 512 * 512:(v + 1) * 512 * 512][sel]
        assert np.max(np.abs(got - ref[i][1].reshape(-1)[sel])) < IMG_TOL, v
    refg = oracle.cone_grad(scene, sub, o, L, [dL[v * 512 * 512:(v + 1) * 512 * 512] for v in pick], mask=mask)
    check_grads(gg, refg, scene, GRAD_TOL, keys=("mu", "scale", "quat", "kappa"))
