"""The 3DGS comparison mode (Eq. 5-7: alpha = o G'(p) of the splatted 2D Gaussian) on the GPU
against the FP64 oracle, through the C ABI: keys and lists bit-exact, images within 1e-4 (exact
thresholds), gradients within 1e-3 per Gaussian and parameter block (5e-3 flattened)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import check_grads, compat_check, dev_scene, flat, run_backward, run_forward, vg_opts

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4
GRAD_TOL = 1e-3


def _opac(scene, seed):
    scene.kappa = np.random.default_rng(seed).uniform(0.05, 0.99, scene.n).astype(np.float32)
    return scene


def _multi_view_scene():
    scene = synth.uniform_scene(300, 4243, log_scale=(-3.5, -2.2), sh_degree=3, sh_std=0.25, flatten_frac=0.2,
                                extent=0.9)
    cams = synth.small_views(3, 0, [(40, 24), (33, 17), (64, 48)])
    return _opac(scene, 1), cams


CASES = {
    "cfg1": lambda: (_opac(synth.config1()[0], 2), synth.config1()[1]),
    "cfg1_ragged": lambda: (_opac(synth.config1(0.5)[0], 3),
                            [synth.look_at((0.3, -0.2, -4.0), (0, 0, 0), 75, 53, 60.0)]),
    "multiview_sh3": _multi_view_scene,
}

MODES = {
    "exact": dict(oracle.EXACT, splat=True),
    "exact_dilated": dict(oracle.EXACT, splat=True, splat_dilation=0.3),
    "3dgs": dict(oracle.SPLAT_3DGS),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("mode", list(MODES))
def test_splat_keys_and_bins_bit_exact(gpu_lib, case, mode):
    vg = gpu_lib
    scene, cams = CASES[case]()
    o = MODES[mode]
    ws, g, _, _ = run_forward(vg, scene, cams, o)
    depth, rect = ws.read_keys()
    od, orc = oracle.keys(scene, cams, o)
    assert np.array_equal(depth, od.reshape(-1))
    assert np.array_equal(rect, orc.reshape(-1, 4))
    ts, items = ws.read_bins()
    L = oracle.lists(scene, cams, o)
    assert np.array_equal(ts, L["tile_start"])
    assert np.array_equal(items % scene.n, L["sorted_g"])


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("mode", ["exact", "exact_dilated"])
def test_splat_forward_exact(gpu_lib, case, mode):
    vg = gpu_lib
    scene, cams = CASES[case]()
    o = dict(MODES[mode], bg=(0.25, 0.5, 0.75))
    _, _, rgb, T = run_forward(vg, scene, cams, o)
    ref_rgb, ref_T, _ = oracle.render(scene, cams, o)
    assert np.max(np.abs(rgb - flat(ref_rgb))) < IMG_TOL
    assert np.max(np.abs(T - flat(ref_T))) < IMG_TOL


@pytest.mark.parametrize("case", list(CASES))
def test_splat_forward_3dgs_thresholds(gpu_lib, case):
    """alpha_min, the 0.99 clamp and T_stop may be decided differently by FP32 and FP64 at a few
    pixels (each near its threshold); every other pixel matches to 1e-4."""
    vg = gpu_lib
    scene, cams = CASES[case]()
    o = MODES["3dgs"]
    ws, _, rgb, T = run_forward(vg, scene, cams, o)
    compat_check(ws, scene, cams, o, rgb, T, label=f"splat {case}")


@pytest.mark.parametrize("ppt", [1, 2])
@pytest.mark.parametrize("case", ["cfg1", "multiview_sh3"])
def test_splat_backward_3dgs_thresholds(gpu_lib, case, ppt):
    """The splat mode's backward with the 3DGS rasterizer's own settings (thresholds, opacity
    cull, dilation) against the oracle's gradient, flipped pixels weighted zero on both sides."""
    vg = gpu_lib
    scene, cams = CASES[case]()
    o = dict(MODES["3dgs"], bg=(0.2, 0.3, 0.4))
    ws, g, rgb, T = run_forward(vg, scene, cams, o, ppt=ppt)
    keep, L, _ = compat_check(ws, scene, cams, o, rgb, T, label=f"splat {case} ppt {ppt}")
    rng = np.random.default_rng(20 + ppt)
    P = rgb.shape[0]
    wr = rng.normal(size=(P, 3)) * keep[:, None]
    wT = rng.normal(size=P) * keep
    gg = run_backward(vg, ws, g, wr, wT)
    ref = oracle.render_grad(scene, cams, o, L, wr, wT)
    check_grads(gg, ref, scene, GRAD_TOL, label=f"splat compat {case} ppt {ppt} ")


@pytest.mark.parametrize("case", ["cfg1", "multiview_sh3"])
@pytest.mark.parametrize("variant", ["exact", "dilated_clamped_bg"])
def test_splat_backward_matches_oracle_gradient(gpu_lib, case, variant):
    vg = gpu_lib
    scene, cams = CASES[case]()
    if case == "cfg1":
        scene = scene.subset(np.arange(0, scene.n, 4))
    o = dict(MODES["exact"])
    if variant == "dilated_clamped_bg":
        o.update(splat_dilation=0.3, tau_max=1.5, bg=(0.3, 0.6, 0.9), softplus_beta=10.0)
    ws, g, rgb, T = run_forward(vg, scene, cams, o)
    rng = np.random.default_rng(8)
    P = rgb.shape[0]
    wr = rng.normal(size=(P, 3))
    wT = rng.normal(size=P)
    gg = run_backward(vg, ws, g, wr, wT)
    L = oracle.lists(scene, cams, o)
    ref = oracle.render_grad(scene, cams, o, L, wr, wT)
    check_grads(gg, ref, scene, GRAD_TOL)


@pytest.mark.parametrize("ppt", [1, 2, 4])
def test_splat_pixels_per_thread_variants(gpu_lib, ppt):
    vg = gpu_lib
    scene, cams = CASES["multiview_sh3"]()
    o = MODES["exact_dilated"]
    ws, g, rgb, T = run_forward(vg, scene, cams, o, ppt=ppt)
    ref_rgb, _, _ = oracle.render(scene, cams, o)
    assert np.max(np.abs(rgb - flat(ref_rgb))) < IMG_TOL
    rng = np.random.default_rng(9)
    wr = rng.normal(size=(rgb.shape[0], 3))
    gg = run_backward(vg, ws, g, wr)
    ref = oracle.render_grad(scene, cams, o, oracle.lists(scene, cams, o), wr)
    check_grads(gg, ref, scene, GRAD_TOL)


def test_splat_edge_cases_and_rejections(gpu_lib):
    """Opaque splats (o = 1) at the clamp, invalid and behind-camera Gaussians; the options the
    splat mode does not combine with are rejected."""
    vg = gpu_lib
    import torch
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 37, 21, 60.0)
    sc = _opac(synth.uniform_scene(60, 10, log_scale=(-2.5, -1.5)), 4)
    sc.kappa[:5] = 1.0
    sc.kappa[5] = np.nan
    sc.scale[6, 2] = -1.0
    sc.mu[7] = (0.0, 0.0, -4.5)
    o = dict(MODES["exact"], bg=(0.1, 0.2, 0.3))
    _, _, rgb, T = run_forward(vg, sc, [cam], o)
    ref_rgb, ref_T, _ = oracle.render(sc, [cam], o)
    assert np.max(np.abs(rgb - flat(ref_rgb))) < IMG_TOL
    g = dev_scene(vg, sc)
    ws = vg.Workspace()
    bad = [vg_opts(vg, dict(o, density_theta=True)), vg_opts(vg, dict(o, splat_dilation=-1.0))]
    for b in bad:
        with pytest.raises(RuntimeError):
            ws.preprocess(g, [cam], b)
    proj = torch.zeros(cam.width * cam.height, device="cuda:0")
    with pytest.raises(RuntimeError):
        ws.project_cone(g, [cam], vg_opts(vg, o), proj)
