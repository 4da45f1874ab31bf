"""Helpers for the GPU parity tests: run the CUDA path through the C ABI on synth inputs."""
import numpy as np
import torch

import oracle


def dev_scene(vg, scene, rec_dtype=torch.float32, sh_dtype=torch.float32):
    d = torch.device("cuda:0")
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).to(d, dt).contiguous()
    return vg.Gaussians(t(scene.mu, rec_dtype), t(scene.scale, rec_dtype), t(scene.quat, rec_dtype),
                        t(scene.kappa, rec_dtype), t(scene.sh, sh_dtype), scene.sh_degree)


def vg_opts(vg, o, flags=0):
    return vg.Opts(alpha_min=o["alpha_min"], tau_cut=o["tau_cut"], tau_max=o["tau_max"], T_stop=o["T_stop"],
                   bg=tuple(o["bg"]), z_near=o["z_near"], flags=flags)


def run_forward(vg, scene, cams, o, ws=None, flags=0, g=None):
    ws = ws or vg.Workspace()
    g = g or dev_scene(vg, scene)
    P = sum(c.width * c.height for c in cams)
    rgb = torch.full((P, 3), float("nan"), device="cuda:0")
    T = torch.full((P,), float("nan"), device="cuda:0")
    ws.preprocess(g, cams, vg_opts(vg, o, flags))
    ws.bin_sort()
    ws.render_fwd(rgb, T)
    torch.cuda.synchronize()
    return ws, g, rgb.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64)


def run_backward(vg, ws, g, dL_drgb, dL_dT=None):
    dev = torch.device("cuda:0")
    grads = dict(mu=torch.zeros(g.n, 3, device=dev), scale=torch.zeros(g.n, 3, device=dev),
                 quat=torch.zeros(g.n, 4, device=dev), kappa=torch.zeros(g.n, device=dev),
                 sh=torch.zeros(tuple(g.sh.shape), device=dev))
    gr = torch.as_tensor(np.ascontiguousarray(dL_drgb, dtype=np.float32)).to(dev)
    gt = None if dL_dT is None else torch.as_tensor(np.ascontiguousarray(dL_dT, dtype=np.float32)).to(dev)
    ws.render_bwd(gr, gt, grads["mu"], grads["scale"], grads["quat"], grads["kappa"], grads["sh"])
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}


def flat(per_view):
    return np.concatenate([np.asarray(a).reshape(-1, *np.asarray(a).shape[2:]) for a in per_view])


def grad_rel_err(g_gpu, g_ref):
    """max |g - g_ref| / max(|g_ref|, 1e-3 max|g_ref|) over one parameter type."""
    floor = 1e-3 * max(float(np.max(np.abs(g_ref))), 1e-30)
    return float(np.max(np.abs(g_gpu - g_ref) / np.maximum(np.abs(g_ref), floor)))


def oracle_lists_from_gpu_order(L):
    return L
