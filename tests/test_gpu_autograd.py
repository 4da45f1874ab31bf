"""The differentiable wrappers (torch.autograd.Function around the C ABI): gradients that reach
the leaf tensors through loss.backward() against the FP64 oracle's analytic gradients."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import check_grads, grad_rel_err

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3


def _leaves(scene, with_sh=True):
    import torch
    t = lambda a: torch.tensor(np.ascontiguousarray(a, np.float32), device="cuda:0", requires_grad=True)
    out = [t(scene.mu), t(scene.scale), t(scene.quat), t(scene.kappa)]
    if with_sh:
        out.append(t(scene.sh))
    return out


def test_rasterizer_autograd_matches_oracle(gpu_lib):
    import torch
    vg = gpu_lib
    scene = synth.uniform_scene(120, 4244, log_scale=(-3.2, -2.2), sh_degree=2, sh_std=0.25, flatten_frac=0.2,
                                extent=0.9)
    cams = synth.small_views(2, 3, [(40, 24), (31, 29)])
    o = dict(oracle.EXACT, bg=(0.2, 0.4, 0.1))
    opts = vg.Opts(alpha_min=0.0, tau_cut=o["tau_cut"], tau_max=float("inf"), T_stop=0.0, bg=o["bg"])
    r = vg.Rasterizer(opts)
    mu, sc, q, k, sh = _leaves(scene)
    rgb, T = r.render(mu, sc, q, k, sh, cams)
    rng = np.random.default_rng(12)
    wr = rng.normal(size=tuple(rgb.shape))
    wT = rng.normal(size=tuple(T.shape))
    loss = (rgb * torch.as_tensor(wr, dtype=torch.float32, device="cuda:0")).sum() + \
           (T * torch.as_tensor(wT, dtype=torch.float32, device="cuda:0")).sum()
    loss.backward()
    L = oracle.lists(scene, cams, o)
    ref = oracle.render_grad(scene, cams, o, L, wr, wT)
    gg = {n: t.grad.cpu().numpy().astype(np.float64) for n, t in zip(("mu", "scale", "quat", "kappa", "sh"),
                                                                    (mu, sc, q, k, sh))}
    check_grads(gg, ref, scene, GRAD_TOL)
    # a second forward on the same rasterizer invalidates the first graph's backward
    rgb2, _ = r.render(mu, sc, q, k, sh, cams)
    rgb3, _ = r.render(mu, sc, q, k, sh, cams)
    with pytest.raises(RuntimeError):
        rgb2.sum().backward()
    rgb3.sum().backward()


def test_projector_parallel_autograd_matches_oracle(gpu_lib):
    import torch
    vg = gpu_lib
    # config 4's Gaussians and detector pitch (2/512): means shrunk into a ball of radius 0.12 that
    # a 64 x 64 detector of extent 0.25 covers (sub-pixel Gaussians make cancelling per-pixel terms)
    scene, _, _ = synth.config4(frac=0.002)
    scene.mu = (scene.mu * 0.12).astype(np.float32)
    beam = synth.parallel_beam(4, det=64, extent=0.25)
    p = vg.Projector(vg.Opts(tau_cut=1e-6))
    mu, sc, q, k = _leaves(scene, with_sh=False)
    proj = p.parallel(mu, sc, q, k, beam)
    w = np.random.default_rng(13).normal(size=tuple(proj.shape))
    (proj * torch.as_tensor(w, dtype=torch.float32, device="cuda:0")).sum().backward()
    L = oracle.tomo_lists(scene, beam, 1e-6)
    _, ref_proj = oracle.tomo(scene, beam, L)
    assert np.max(np.abs(proj.detach().cpu().numpy() - ref_proj)) < 1e-4
    ref = oracle.tomo_grad(scene, beam, L, w)
    for name, t in zip(("mu", "scale", "quat", "kappa"), (mu, sc, q, k)):
        e = grad_rel_err(t.grad.cpu().numpy().astype(np.float64), ref[name])
        assert e < GRAD_TOL, (name, e)


def test_projector_cone_autograd_matches_oracle(gpu_lib):
    import torch
    vg = gpu_lib
    scene = synth.tomo_scene(300, 95, log_scale=(-4.0, -2.5))
    cams = synth.cone_beam(2, det=40)
    p = vg.Projector(vg.Opts(tau_cut=1e-6))
    mu, sc, q, k = _leaves(scene, with_sh=False)
    proj = p.cone(mu, sc, q, k, cams)
    w = np.random.default_rng(14).normal(size=tuple(proj.shape))
    (proj * torch.as_tensor(w, dtype=torch.float32, device="cuda:0")).sum().backward()
    o = dict(oracle.EXACT)
    L = oracle.lists(scene, cams, o)
    ref_proj = np.concatenate([pr.reshape(-1) for _, pr in oracle.cone(scene, cams, o, L)])
    assert np.max(np.abs(proj.detach().cpu().numpy() - ref_proj)) < 1e-4
    split = np.cumsum([0] + [c.width * c.height for c in cams])
    ref = oracle.cone_grad(scene, cams, o, L, [w[split[v]:split[v + 1]] for v in range(len(cams))])
    gg = {n: t.grad.cpu().numpy().astype(np.float64) for n, t in zip(("mu", "scale", "quat", "kappa"), (mu, sc, q, k))}
    check_grads(gg, ref, scene, GRAD_TOL, keys=("mu", "scale", "quat", "kappa"))
