"""Helpers for the GPU parity tests: run the CUDA path through the C ABI on synth inputs."""
import numpy as np
import torch

import oracle


def dev_scene(vg, scene, rec_dtype=torch.float32, sh_dtype=torch.float32, mu_dtype=None):
    d = torch.device("cuda:0")
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).to(d, dt).contiguous()
    return vg.Gaussians(t(scene.mu, mu_dtype or rec_dtype), t(scene.scale, rec_dtype), t(scene.quat, rec_dtype),
                        t(scene.kappa, rec_dtype), t(scene.sh, sh_dtype), scene.sh_degree)


def vg_opts(vg, o, flags=0, ppt=0, chunk=0, tile=(0, 0)):
    if o.get("density_theta"):
        flags |= vg.FLAG_DENSITY_THETA
    if o.get("splat"):
        flags |= vg.FLAG_SPLAT
    return vg.Opts(alpha_min=o["alpha_min"], tau_cut=o["tau_cut"], tau_max=o["tau_max"], T_stop=o["T_stop"],
                   bg=tuple(o["bg"]), z_near=o["z_near"], flags=flags, pixels_per_thread=ppt,
                   softplus_beta=o.get("softplus_beta", 0.0), splat_dilation=o.get("splat_dilation", 0.0),
                   chunk=chunk, tile_w=tile[0], tile_h=tile[1])


def run_forward(vg, scene, cams, o, ws=None, flags=0, g=None, ppt=0, chunk=0, tile=(0, 0)):
    ws = ws or vg.Workspace()
    g = g or dev_scene(vg, scene)
    P = sum(c.width * c.height for c in cams)
    rgb = torch.full((P, 3), float("nan"), device="cuda:0")
    T = torch.full((P,), float("nan"), device="cuda:0")
    ws.preprocess(g, cams, vg_opts(vg, o, flags, ppt, chunk, tile))
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


def grad_block_err(g_gpu, g_ref, n):
    """Per-Gaussian relative error of one parameter block (vector norm over its components),
    floored at 1e-3 of the largest block norm of that parameter type."""
    g = np.asarray(g_gpu, np.float64).reshape(n, -1)
    r = np.asarray(g_ref, np.float64).reshape(n, -1)
    nr = np.linalg.norm(r, axis=1)
    floor = 1e-3 * max(float(nr.max()), 1e-30)
    return np.linalg.norm(g - r, axis=1) / np.maximum(nr, floor)


FLAT_ANISO = 20.0     # Gaussians with s_max / s_min above this count as flattened
FLAT_TOL = 5e-3       # FP32 conditioning of thin Gaussians: error ~ eps * distance / s_min


def check_grads(gg, ref, scene, tol, keys=("mu", "scale", "quat", "kappa", "sh"), flat_tol=None, label=""):
    """Non-flattened Gaussians within tol, flattened ones within FLAT_TOL (or flat_tol, a dict
    by parameter or a number), by the per-Gaussian block metric; returns the worst as
    {param: (block error non-flattened, block error flattened, element-wise error)} and prints it.
    The element-wise error (grad_rel_err: floor 1e-3 of the largest element) is reported beside
    the block metric, not asserted: tiny components of large gradients fail it by design."""
    aniso = scene.scale.max(1) / scene.scale.min(1)
    flat_ = aniso > FLAT_ANISO
    worst = {}
    for k in keys:
        e = grad_block_err(gg[k], ref[k], scene.n)
        assert np.max(np.abs(ref[k])) > 0, k
        worst[k] = (float(e[~flat_].max()) if (~flat_).any() else 0.0, float(e[flat_].max()) if flat_.any() else 0.0,
                    grad_rel_err(gg[k], ref[k]))
    print(f"gradient errors {label}(block, block flattened, element-wise):",
          {k: tuple(f"{x:.2e}" for x in v) for k, v in worst.items()})
    for k in keys:
        assert worst[k][0] < tol, (k, worst[k])
        ft = flat_tol.get(k, FLAT_TOL) if isinstance(flat_tol, dict) else (flat_tol or FLAT_TOL)
        assert worst[k][1] < ft, (k, worst[k])
    return worst


#: a flipped skip decision changes S = sum tau by at least tau_skip; half of it separates flips
#: from the FP32 rounding of S
NEAR_THRESHOLD = 1e-3   # a decision this close (relative) to its threshold may go either way in FP32
CLAMP_AMBIGUOUS = 1e-4  # pairs this close to tau_max: clamped on one side, not on the other


def threshold_flips(ws, diag, tau_skip, pixels=None, state=None):
    """Pixels where the GPU and the FP64 oracle took a threshold decision (alpha_min skip, T_stop
    early stop) differently, from the GPU's replay state (S, last blended position) against the
    oracle's; restricted to `pixels` (a boolean mask) when given.  Returns (flip mask, the largest
    relative threshold distance among flipped pixels): a flip is explained by rounding only when
    that distance is small."""
    S, last = ws.read_pixel_state() if state is None else state
    flip = (last.astype(np.int64) != diag["last"]) | (np.abs(S.astype(np.float64) - diag["S"]) > 0.5 * tau_skip)
    if pixels is not None:
        flip &= pixels
    near = np.minimum(diag["m_skip"], diag["m_stop"])
    worst = float(near[flip].max()) if flip.any() else 0.0
    return flip, worst


def tau_skip_of(o):
    a = float(o["alpha_min"])
    return -np.log1p(-a) if a > 0 else 0.0


IMG_TOL = 1e-4


def compat_check(ws, scene, cams, o, rgb, T=None, L=None, mask=None, state=None, label=""):
    """Image parity with thresholds (alpha_min skip, tau_max clamp, T_stop early stop): within 1e-4
    of the FP64 oracle at every pixel whose threshold decisions agree with the oracle's, and few
    flipped pixels, each explained by a decision within NEAR_THRESHOLD of its threshold (a culling
    bug that drops a blending Gaussian flips a pixel far from any threshold).  rgb / T: the GPU's
    images of `cams` (flat, float64); mask: the pixels to check (all when None); state: the GPU's
    (S, last) of these pixels (read from ws when None).  Returns (keep, L, flips): keep marks the
    checked pixels with no flip and no pair within CLAMP_AMBIGUOUS of tau_max, the pixels a
    gradient comparison may weight."""
    if L is None:
        L = oracle.lists(scene, cams, o)
    ref_rgb, ref_T, _, dg = oracle.render(scene, cams, o, L=L, mask=mask, diag=True)
    P = sum(c.width * c.height for c in cams)
    sel = np.ones(P, bool) if mask is None else np.asarray(mask).reshape(-1).astype(bool)
    flip, worst = threshold_flips(ws, dg, tau_skip_of(o), sel, state)
    ok = sel & ~flip
    err = np.max(np.abs(rgb - flat(ref_rgb)), axis=1)
    max_err = float(err[ok].max()) if ok.any() else 0.0
    print(f"compat image {label}: max abs err {max_err:.2e} over {int(ok.sum())} pixels; "
          f"{int(flip.sum())} of {int(sel.sum())} pixels flipped a threshold decision "
          f"(largest relative distance to the threshold among them {worst:.1e})")
    assert max_err < IMG_TOL, max_err
    if T is not None:
        assert np.max(np.abs(T - flat(ref_T))[ok], initial=0.0) < IMG_TOL
    assert flip.sum() <= max(2, 1e-3 * sel.sum()), int(flip.sum())
    assert worst < NEAR_THRESHOLD, worst
    keep = ok & (dg["m_clamp"] >= CLAMP_AMBIGUOUS)
    return keep, L, flip
