"""The allocation-free backward (vg_render_bwd_noalloc) against the regular backward.

Callers whose device memory belongs to another allocator or a fixed budget, or that must
not stall on the device-wide synchronisation cudaMalloc/cudaFree can cause, use
vg_render_bwd_noalloc: it keeps its gradient accumulator in a fixed array inside the library
instead of the workspace.  This test runs it twice in a row after one forward and compares
both results with vg_render_bwd's, within the gradient tolerance of the parity tests.  The
file is named to be collected last, and the test runs the same way alone in a fresh process.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import grad_rel_err, run_backward, run_forward

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3


def _grads(vg, ws, g, wr, wT, noalloc):
    import torch

    dev = torch.device("cuda:0")
    out = dict(mu=torch.zeros(g.n, 3, device=dev), scale=torch.zeros(g.n, 3, device=dev),
               quat=torch.zeros(g.n, 4, device=dev), kappa=torch.zeros(g.n, device=dev),
               sh=torch.zeros(tuple(g.sh.shape), device=dev))
    gr = torch.as_tensor(np.ascontiguousarray(wr, dtype=np.float32)).to(dev)
    gt = torch.as_tensor(np.ascontiguousarray(wT, dtype=np.float32)).to(dev)
    args = (gr, gt, out["mu"], out["scale"], out["quat"], out["kappa"], out["sh"])
    if noalloc:
        ws.render_bwd_noalloc(*args)
    else:
        ws.render_bwd(*args)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}


def test_noalloc_backward_matches_regular_backward(gpu_lib):
    vg = gpu_lib
    scene = synth.uniform_scene(400, 4243, log_scale=(-3.5, -2.2), sh_degree=3, sh_std=0.25, flatten_frac=0.2,
                                extent=0.9)
    cams = synth.small_views(2, 0, [(48, 32), (37, 29)])
    o = dict(oracle.EXACT, bg=(0.2, 0.4, 0.6))
    ws, g, rgb, T = run_forward(vg, scene, cams, o)
    rng = np.random.default_rng(3)
    wr = rng.normal(size=(rgb.shape[0], 3))
    wT = rng.normal(size=rgb.shape[0])
    ref = _grads(vg, ws, g, wr, wT, noalloc=False)
    for call in range(2):                  # the shared array keeps the previous call's sums
        got = _grads(vg, ws, g, wr, wT, noalloc=True)
        for k in ref:
            assert np.max(np.abs(ref[k])) > 0, k
            e = grad_rel_err(got[k], ref[k])
            assert e < GRAD_TOL, (call, k, e)


def test_noalloc_backward_allocates_nothing_on_a_fresh_workspace(gpu_lib):
    """On a workspace that never ran vg_render_bwd (so it holds no gradient accumulator) the
    allocation-free backward runs first; after one warm-up call (which loads the kernels), a
    second call leaves the device's free memory unchanged, and its result matches the regular
    backward run afterwards."""
    import torch

    vg = gpu_lib
    scene = synth.uniform_scene(350, 4244, log_scale=(-3.5, -2.2), sh_degree=2, sh_std=0.25, flatten_frac=0.2,
                                extent=0.9)
    cams = synth.small_views(2, 1, [(40, 32), (29, 37)])
    o = dict(oracle.EXACT, bg=(0.1, 0.3, 0.5))
    ws, g, rgb, T = run_forward(vg, scene, cams, o)
    rng = np.random.default_rng(5)
    wr = rng.normal(size=(rgb.shape[0], 3))
    wT = rng.normal(size=rgb.shape[0])
    dev = torch.device("cuda:0")
    out = dict(mu=torch.zeros(g.n, 3, device=dev), scale=torch.zeros(g.n, 3, device=dev),
               quat=torch.zeros(g.n, 4, device=dev), kappa=torch.zeros(g.n, device=dev),
               sh=torch.zeros(tuple(g.sh.shape), device=dev))
    gr = torch.as_tensor(np.ascontiguousarray(wr, dtype=np.float32)).to(dev)
    gt = torch.as_tensor(np.ascontiguousarray(wT, dtype=np.float32)).to(dev)
    args = (gr, gt, out["mu"], out["scale"], out["quat"], out["kappa"], out["sh"])
    ws.render_bwd_noalloc(*args)                    # warm-up: loads the kernels
    torch.cuda.synchronize()
    for t in out.values():
        t.zero_()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ws.render_bwd_noalloc(*args)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}
    ref = _grads(vg, ws, g, wr, wT, noalloc=False)
    for k in ref:
        assert np.max(np.abs(ref[k])) > 0, k
        e = grad_rel_err(got[k], ref[k])
        assert e < GRAD_TOL, (k, e)


def test_noalloc_backward_rejects_sizes_beyond_its_limit(gpu_lib):
    vg = gpu_lib
    n = 70000                              # views x Gaussians > VG_NOALLOC_MAX_ITEMS = 65536
    scene = synth.uniform_scene(n, 5, log_scale=(-6.0, -5.0))
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 32, 32, 60.0)
    ws, g, rgb, T = run_forward(vg, scene, [cam], oracle.COMPAT)
    with pytest.raises(vg.VGError) as ei:
        _grads(vg, ws, g, np.zeros((rgb.shape[0], 3)), np.zeros(rgb.shape[0]), noalloc=True)
    assert ei.value.status == 1 and "VG_NOALLOC_MAX_ITEMS" in str(ei.value)
