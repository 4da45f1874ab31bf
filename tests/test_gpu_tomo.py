"""GPU parity of the tomography mode (Sec. 6.2, Eq. 21) against the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import check_grads, grad_rel_err

pytestmark = pytest.mark.gpu

TAU_CUT = 1e-6
IMG_TOL = 1e-4
GRAD_TOL = 1e-3


def _run(vg, scene, beam, dL=None, ws=None):
    import torch

    from gpu_util import dev_scene

    ws = ws or vg.Workspace()
    g = dev_scene(vg, scene)
    A = len(beam.angles)
    proj = torch.full((A, beam.det_h, beam.det_w), float("nan"), device="cuda:0")
    grads = None
    if dL is not None:
        grads = [torch.zeros(scene.n, 3, device="cuda:0"), torch.zeros(scene.n, 3, device="cuda:0"),
                 torch.zeros(scene.n, 4, device="cuda:0"), torch.zeros(scene.n, device="cuda:0")]
        dLt = torch.as_tensor(np.ascontiguousarray(dL, dtype=np.float32)).to("cuda:0")
        ws.project_tomo(g, beam, vg.Opts(tau_cut=TAU_CUT), proj, dLt, *grads)
    else:
        ws.project_tomo(g, beam, vg.Opts(tau_cut=TAU_CUT), proj)
    torch.cuda.synchronize()
    out = proj.cpu().numpy().astype(np.float64)
    if grads is not None:
        grads = dict(zip(("mu", "scale", "quat", "kappa"), (t.cpu().numpy().astype(np.float64) for t in grads)))
    return ws, out, grads


def _case(frac=0.005, n_angles=5, det=72):
    scene, beam, _ = synth.config4(frac=frac, n_angles=n_angles, det=det)
    return scene, beam


def test_tomo_keys_bins_bit_exact(gpu_lib):
    vg = gpu_lib
    scene, beam = _case()
    ws, _, _ = _run(vg, scene, beam)
    _, rect = ws.read_keys()
    L = oracle.tomo_lists(scene, beam, TAU_CUT)
    assert np.array_equal(rect, L["rect"].reshape(-1, 4))
    ts, items = ws.read_bins()
    assert np.array_equal(ts, L["tile_start"])
    assert np.array_equal(items % scene.n, L["sorted_g"])


@pytest.mark.parametrize("det", [72, 64])
def test_tomo_projection(gpu_lib, det):
    vg = gpu_lib
    scene, beam = _case(det=det)
    _, proj, _ = _run(vg, scene, beam)
    L = oracle.tomo_lists(scene, beam, TAU_CUT)
    _, ref = oracle.tomo(scene, beam, L)
    assert np.max(np.abs(proj - ref)) < IMG_TOL
    assert proj.min() < 0.5          # the case is not trivially transparent


def _cfg4_sampling_case(n_angles=4, det=64):
    """Config-4 Gaussians and detector pitch (2/512) on a small detector: means shrunk
    into a ball of radius 0.12 so that they land on a 64 x 64 detector of extent 0.25."""
    scene, _, _ = synth.config4(frac=0.002)
    scene.mu = (scene.mu * 0.12).astype(np.float32)
    return scene, synth.parallel_beam(n_angles, det=det, extent=0.25)


def test_tomo_gradient(gpu_lib):
    vg = gpu_lib
    scene, beam = _cfg4_sampling_case()
    rng = np.random.default_rng(2)
    dL = rng.normal(size=(len(beam.angles), beam.det_h, beam.det_w))
    _, proj, gg = _run(vg, scene, beam, dL)
    L = oracle.tomo_lists(scene, beam, TAU_CUT)
    _, ref_proj = oracle.tomo(scene, beam, L)
    assert np.max(np.abs(proj - ref_proj)) < IMG_TOL
    ref = oracle.tomo_grad(scene, beam, L, dL)
    for k in ("mu", "scale", "quat", "kappa"):
        e = grad_rel_err(gg[k], ref[k])
        assert e < GRAD_TOL, (k, e)


def test_tomo_gradient_subpixel_gaussians(gpu_lib):
    """Gaussians narrower than a detector pixel (sigma 0.16-1.2 px): the position gradient is
    a sum of large per-pixel terms that cancel, so FP32 leaves an error of a few 1e-5 of each
    Gaussian's own gradient; against the floor of 1e-3 of the largest gradient the bound is 5e-3."""
    vg = gpu_lib
    scene, beam = _case(frac=0.002, n_angles=4, det=48)
    rng = np.random.default_rng(2)
    dL = rng.normal(size=(len(beam.angles), beam.det_h, beam.det_w))
    _, proj, gg = _run(vg, scene, beam, dL)
    L = oracle.tomo_lists(scene, beam, TAU_CUT)
    ref = oracle.tomo_grad(scene, beam, L, dL)
    for k in ("mu", "scale", "quat", "kappa"):
        e = grad_rel_err(gg[k], ref[k])
        assert e < 5e-3, (k, e)
        own = np.abs(gg[k] - ref[k]).reshape(scene.n, -1).max(1) / np.maximum(
            np.abs(ref[k]).reshape(scene.n, -1).max(1), 1e-3 * np.abs(ref[k]).max())
        assert own.max() < 1e-3, (k, own.max())


def test_tomo_many_angles_in_batches(gpu_lib):
    """More (angle, Gaussian) items than one batch holds: angles are processed in several
    batches; sampled angles on both sides of a batch boundary match the oracle."""
    vg = gpu_lib
    scene, beam, _ = synth.config4(frac=0.1, n_angles=256, det=40)       # 20,000 x 256 > 4M items
    _, proj, _ = _run(vg, scene, beam)
    batch = (1 << 22) // scene.n
    pick = [0, batch - 1, batch, 255]
    mask = np.zeros((256, beam.det_h, beam.det_w), np.int32)
    mask[pick] = 1
    _, ref = oracle.tomo(scene, beam, brute=True, mask=mask)
    # brute force over all Gaussians differs from the truncated footprints by < tau_cut each
    assert np.max(np.abs(proj[pick] - ref[pick])) < IMG_TOL + scene.n * TAU_CUT


def test_tomo_edge_cases(gpu_lib):
    vg = gpu_lib
    beam = synth.parallel_beam(3, det=37, extent=2.0)
    empty = synth.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), np.zeros((0, 4), np.float32),
                        np.zeros(0, np.float32), np.zeros((0, 1, 3), np.float32), 0)
    _, proj, _ = _run(vg, empty, beam)
    assert np.all(proj == 1.0)
    sc = synth.tomo_scene(60, 8, log_scale=(-3.0, -2.0))
    sc.kappa[0] = np.nan
    sc.scale[1, 0] = 0.0
    sc.quat[2] = 0.0
    _, proj, _ = _run(vg, sc, beam)
    _, ref = oracle.tomo(sc, beam)
    assert np.max(np.abs(proj - ref)) < IMG_TOL


def test_tomo_density_reparam(gpu_lib):
    """Tomography with Eq. 20's theta as the density input."""
    import torch

    from gpu_util import check_grads, dev_scene
    vg = gpu_lib
    scene, beam = _cfg4_sampling_case()
    rng = np.random.default_rng(19)
    scene.kappa = rng.uniform(0.02, 1.0, scene.n).astype(np.float32)
    A = len(beam.angles)
    dL = rng.normal(size=(A, beam.det_h, beam.det_w))
    g = dev_scene(vg, scene)
    dev = torch.device("cuda:0")
    proj = torch.empty(A, beam.det_h, beam.det_w, device=dev)
    grads = [torch.zeros(scene.n, 3, device=dev), torch.zeros(scene.n, 3, device=dev),
             torch.zeros(scene.n, 4, device=dev), torch.zeros(scene.n, device=dev)]
    ws = vg.Workspace()
    ws.project_tomo(g, beam, vg.Opts(tau_cut=TAU_CUT, flags=vg.FLAG_DENSITY_THETA), proj,
                    torch.as_tensor(dL.astype(np.float32)).to(dev), *grads)
    torch.cuda.synchronize()
    L = oracle.tomo_lists(scene, beam, TAU_CUT, density_theta=True)
    _, rect = ws.read_keys()
    assert np.array_equal(rect, L["rect"].reshape(-1, 4))
    _, ref_proj = oracle.tomo(scene, beam, L, density_theta=True)
    assert np.max(np.abs(proj.cpu().numpy() - ref_proj)) < IMG_TOL
    ref = oracle.tomo_grad(scene, beam, L, dL, density_theta=True)
    gg = {k: t.cpu().numpy().astype(np.float64) for k, t in zip(("mu", "scale", "quat", "kappa"), grads)}
    check_grads(gg, ref, scene, GRAD_TOL, keys=("mu", "scale", "quat", "kappa"))


def test_tomo_fused_l2_step_and_given_projection(gpu_lib):
    """vg_tomo_l2_step equals the two-call form (project; L2 loss; project with dL/dproj), and a
    backward call with VG_FLAG_PROJ_GIVEN (projection reused, not recomputed) gives the same
    gradients."""
    import torch
    from gpu_util import dev_scene
    vg = gpu_lib
    scene, beam = _cfg4_sampling_case(n_angles=7)
    gt, _ = _cfg4_sampling_case(n_angles=7)
    gt.mu = gt.mu[::-1].copy()
    dev = torch.device("cuda:0")
    g, gg = dev_scene(vg, scene), dev_scene(vg, gt)
    A = len(beam.angles)
    ws = vg.Workspace()
    tgt = torch.empty(A, beam.det_h, beam.det_w, device=dev)
    ws.project_tomo(gg, beam, vg.Opts(tau_cut=TAU_CUT), tgt)
    scale = 1.0 / tgt.numel()
    mk = lambda: [torch.zeros(scene.n, 3, device=dev), torch.zeros(scene.n, 3, device=dev),
                  torch.zeros(scene.n, 4, device=dev), torch.zeros(scene.n, device=dev)]
    # fused
    p1, l1, g1 = torch.empty_like(tgt), torch.zeros(1, device=dev), mk()
    ws.tomo_l2_step(g, beam, vg.Opts(tau_cut=TAU_CUT, flags=vg.FLAG_GRAD_ZERO), tgt, scale, p1, l1, *g1)
    # two calls, the second recomputing the projection
    p2, l2, dl, g2 = torch.empty_like(tgt), torch.zeros(1, device=dev), torch.empty_like(tgt), mk()
    ws.project_tomo(g, beam, vg.Opts(tau_cut=TAU_CUT), p2)
    ws.l2_loss(p2, tgt, scale, l2, dl)
    ws.project_tomo(g, beam, vg.Opts(tau_cut=TAU_CUT), p2, dl, *g2)
    # two calls, the second reusing the given projection
    g3 = mk()
    p3 = p2.clone()
    ws.project_tomo(g, beam, vg.Opts(tau_cut=TAU_CUT, flags=vg.FLAG_PROJ_GIVEN), p3, dl, *g3)
    torch.cuda.synchronize()
    assert torch.equal(p1, p2) and torch.equal(p3, p2)
    assert abs(float(l1) - float(l2)) <= 1e-6 * abs(float(l2))
    for a, b, c in zip(g1, g2, g3):   # atomics: equal up to the summation order
        tol = 1e-6 * float(b.abs().max())
        assert torch.allclose(b, c, rtol=1e-5, atol=tol) and torch.allclose(a, b, rtol=1e-5, atol=tol)
    # against the oracle: loss and gradient of the L2 loss
    L = oracle.tomo_lists(scene, beam, TAU_CUT)
    _, ref_proj = oracle.tomo(scene, beam, L)
    t_np = tgt.cpu().numpy().astype(np.float64)
    ref_loss = scale * np.sum((ref_proj - t_np) ** 2)
    assert abs(float(l1) - ref_loss) <= 1e-4 * ref_loss
    ref = oracle.tomo_grad(scene, beam, L, 2.0 * scale * (ref_proj - t_np))
    for k, t in zip(("mu", "scale", "quat", "kappa"), g1):
        e = grad_rel_err(t.cpu().numpy().astype(np.float64), ref[k])
        assert e < GRAD_TOL, (k, e)
