"""Edge cases of the rasterizer on the GPU against the FP64 oracle: the largest image width, a
footprint that covers the whole view, many tiny ragged views, Gaussians at the near plane and
degenerate parameters."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev_scene, flat, run_backward, run_forward, vg_opts

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4


def test_largest_image_width(gpu_lib):
    """A 32767 x 5 view (2048 x 1 tiles, ragged in both directions): keys and lists bit-exact,
    sampled pixels within 1e-4; 32768 pixels wide is rejected."""
    vg = gpu_lib
    import torch
    scene = synth.uniform_scene(400, 71, log_scale=(-4.5, -3.0), extent=1.0)
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 32767, 5, 60.0)
    o = dict(oracle.EXACT, bg=(0.1, 0.2, 0.3))
    ws, g, rgb, T = run_forward(vg, scene, [cam], o)
    depth, rect = ws.read_keys()
    od, orc = oracle.keys(scene, [cam], o)
    assert np.array_equal(depth, od.reshape(-1)) and np.array_equal(rect, orc.reshape(-1, 4))
    ts, items = ws.read_bins()
    L = oracle.lists(scene, [cam], o)
    assert np.array_equal(ts, L["tile_start"]) and np.array_equal(items, L["sorted_g"])
    rng = np.random.default_rng(3)
    mask = np.zeros(cam.width * cam.height, np.int32)
    mask[rng.choice(mask.size, 3000, replace=False)] = 1
    mask[-1] = mask[0] = 1
    ref_rgb, _, _ = oracle.render(scene, [cam], o, L=L, mask=mask)
    sel = mask.astype(bool)
    assert np.max(np.abs(rgb[sel] - flat(ref_rgb)[sel])) < IMG_TOL
    wide = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 32768, 2, 60.0)
    with pytest.raises(RuntimeError):
        ws.preprocess(g, [wide], vg_opts(vg, o))
    del torch


def test_whole_view_footprint_and_near_plane(gpu_lib):
    """A large Gaussian whose cut-off ellipsoid reaches the camera plane covers the whole view;
    Gaussians just in front of and behind z_near are kept and culled alike on both sides."""
    vg = gpu_lib
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 45, 29, 60.0)
    big = synth.Scene(np.array([[0.1, -0.2, -2.0]], np.float32), np.array([[1.5, 1.2, 2.5]], np.float32),
                      np.array([[0.9, 0.2, -0.3, 0.1]], np.float32), np.array([0.3], np.float32),
                      np.array([[[0.4, -0.2, 0.1]]], np.float32), 0)
    rest = synth.uniform_scene(200, 72, log_scale=(-3.5, -2.0), extent=0.8)
    near = synth.uniform_scene(4, 73, log_scale=(-3.0, -2.5), extent=0.1)
    near.mu[:, 2] = np.array([-3.8 + 1e-3, -3.8 - 1e-3, -3.8 + 0.05, -3.8 - 0.05], np.float32)  # z_near = 0.2
    scene = synth.Scene(*(np.concatenate([getattr(s, f) for s in (big, rest, near)])
                          for f in ("mu", "scale", "quat", "kappa", "sh")), 0)
    o = dict(oracle.EXACT, bg=(0.3, 0.3, 0.3))
    ws, g, rgb, T = run_forward(vg, scene, [cam], o)
    _, rect = ws.read_keys()
    od, orc, opr = oracle.keys(scene, [cam], o, with_pixels=True)
    assert np.array_equal(rect, orc.reshape(-1, 4))
    tx, ty = (cam.width + 15) // 16, (cam.height + 15) // 16
    assert list(orc[0, 0]) == [0, 0, tx - 1, ty - 1]                 # the whole view
    ref_rgb, ref_T, _ = oracle.render(scene, [cam], o)
    assert np.max(np.abs(rgb - flat(ref_rgb))) < IMG_TOL
    rng = np.random.default_rng(4)
    wr = rng.normal(size=rgb.shape)
    gg = run_backward(vg, ws, g, wr)
    ref = oracle.render_grad(scene, [cam], o, oracle.lists(scene, [cam], o), wr)
    for k in ("mu", "scale", "quat", "kappa", "sh"):
        assert np.all(np.isfinite(gg[k]))
        scale = np.max(np.abs(ref[k]))
        assert np.max(np.abs(gg[k] - ref[k])) <= 1e-3 * scale + 1e-6, k


def test_many_tiny_ragged_views(gpu_lib):
    """40 views of 1x1 to 17x3 pixels in one call: per-view tile bases and pixel offsets."""
    vg = gpu_lib
    scene = synth.uniform_scene(150, 74, log_scale=(-3.0, -1.8), sh_degree=1, sh_std=0.3, extent=0.7)
    rng = np.random.default_rng(5)
    sizes = [(int(rng.integers(1, 18)), int(rng.integers(1, 4))) for _ in range(40)]
    sizes[0] = (1, 1)
    cams = synth.small_views(40, 6, sizes)
    o = dict(oracle.EXACT, bg=(0.0, 0.5, 1.0))
    ws, g, rgb, T = run_forward(vg, scene, cams, o)
    ref_rgb, ref_T, _ = oracle.render(scene, cams, o)
    assert np.max(np.abs(rgb - flat(ref_rgb))) < IMG_TOL
    ts, items = ws.read_bins()
    L = oracle.lists(scene, cams, o)
    assert np.array_equal(ts, L["tile_start"]) and np.array_equal(items % scene.n, L["sorted_g"])


def test_degenerate_gaussians_stay_finite(gpu_lib):
    """Gaussians flattened 1000:1 and 10^4:1, tiny and huge densities, unnormalised quaternions of
    very different norms: finite images and gradients, within 1e-4 / 1e-3 of the oracle where the
    FP32 conditioning allows (flattening up to 1000:1)."""
    vg = gpu_lib
    rng = np.random.default_rng(7)
    sc = synth.uniform_scene(60, 75, log_scale=(-2.8, -2.0), extent=0.6)
    sc.scale[:20, 0] *= 1e-3
    sc.kappa[20:30] = 1e-4
    sc.kappa[30:40] = 500.0
    sc.quat[40:50] *= rng.uniform(1e-3, 1e3, (10, 1)).astype(np.float32)
    cam = synth.look_at((0.3, 0.2, -4.0), (0.0, 0.0, 0.0), 48, 40, 40.0)
    o = dict(oracle.EXACT)
    ws, g, rgb, T = run_forward(vg, sc, [cam], o)
    assert np.all(np.isfinite(rgb)) and np.all(np.isfinite(T))
    ref_rgb, _, _ = oracle.render(sc, [cam], o)
    assert np.max(np.abs(rgb - flat(ref_rgb))) < IMG_TOL
    wr = rng.normal(size=rgb.shape)
    gg = run_backward(vg, ws, g, wr)
    for k in gg:
        assert np.all(np.isfinite(gg[k])), k
    extreme = sc.subset(np.arange(20))
    extreme.scale[:, 0] *= 0.1                                      # 10^4 : 1
    _, _, rgb2, T2 = run_forward(vg, extreme, [cam], o)
    assert np.all(np.isfinite(rgb2)) and np.all((T2 >= 0) & (T2 <= 1))


def test_stage_profiler_mask(gpu_lib):
    """vg_profile_stages: with one stage selected only that stage is event-timed; the default
    (mask 0) records every stage of the step; the rendered image does not depend on either."""
    vg = gpu_lib
    import torch
    scene = synth.uniform_scene(300, 72, log_scale=(-3.5, -2.5), extent=1.0)
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 96, 64, 60.0)
    o = dict(oracle.EXACT)
    g = dev_scene(vg, scene)
    ws = vg.Workspace()
    P = cam.width * cam.height
    rgb, T = torch.empty(P, 3, device="cuda:0"), torch.empty(P, device="cuda:0")
    dl = torch.full((P, 3), 1e-3, device="cuda:0")
    grads = [torch.zeros(g.n, 3, device="cuda:0"), torch.zeros(g.n, 3, device="cuda:0"),
             torch.zeros(g.n, 4, device="cuda:0"), torch.zeros(g.n, device="cuda:0"),
             torch.zeros(tuple(g.sh.shape), device="cuda:0")]
    images = []
    for stages in (["render_bwd"], None):
        ws.profile_enable(True, stages=stages)
        for _ in range(2):
            ws.preprocess(g, [cam], vg_opts(vg, o))
            ws.bin_sort()
            ws.render_fwd(rgb, T)
            ws.render_bwd(dl, None, *grads)
        rec = ws.profile_read()
        ws.profile_enable(False)
        images.append(rgb.cpu().numpy().copy())
        if stages:
            assert set(rec) == {"render_bwd"} and rec["render_bwd"][0] == 2
        else:
            assert {"preprocess", "depth_sort", "scan", "duplicate", "tile_sort", "render_fwd", "render_bwd", "chain"} <= set(rec)
            assert all(c == 2 for c, _ in rec.values())
    assert np.array_equal(images[0], images[1])
    with pytest.raises(ValueError):
        ws.profile_enable(True, stages=["no_such_stage"])


def test_workspace_reuse_growing_and_shrinking_lists(gpu_lib):
    """One workspace bins three scenes in turn: a small one (the instance buffers are sized to
    it), a larger one (more instances than the buffers hold: the lists enqueued ahead of the
    count's readback are rebuilt after the buffers grow) and the small one again (enqueued ahead
    with spare capacity).  Every time the lists are bit-exact and the image matches the oracle."""
    vg = gpu_lib
    small = synth.uniform_scene(200, 73, log_scale=(-3.5, -2.5), extent=1.0)
    large = synth.uniform_scene(1500, 74, log_scale=(-3.0, -2.0), extent=1.0)
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 160, 112, 60.0)
    o = dict(oracle.EXACT)
    ws = vg.Workspace()
    counts = []
    for scene in (small, large, small):
        _, _, rgb, T = run_forward(vg, scene, [cam], o, ws=ws)
        L = oracle.lists(scene, [cam], o)
        ts, items = ws.read_bins()
        assert np.array_equal(ts, L["tile_start"]) and np.array_equal(items, L["sorted_g"])
        ref_rgb, ref_T, _ = oracle.render(scene, [cam], o, L=L)
        assert np.max(np.abs(rgb - flat(ref_rgb))) < IMG_TOL
        assert np.max(np.abs(T - flat(ref_T))) < IMG_TOL
        counts.append(ws.query()["n_instances"])
    assert counts[1] > counts[0] and counts[2] == counts[0]


def test_pipe_peak_microbenchmark(gpu_lib):
    """vg_pipe_peak's FP32 FMA rate cannot exceed 152 SMs x 128 lanes at the maximum SM clock and a
    healthy GPU reaches most of it; the ex2 rate is positive and below the FMA rate."""
    vg = gpu_lib
    ws = vg.Workspace()
    fma, ms = ws.pipe_peak("fma", 5.0)
    ex2, ms2 = ws.pipe_peak("ex2", 5.0)
    ceiling = 152 * 128 * 2.07e9
    print(f"FMA {fma / 1e12:.2f} T/s ({fma / ceiling:.3f} of 152 x 128 x 2070 MHz), ex2 {ex2 / 1e12:.2f} T/s")
    assert 0.3 * ceiling < fma <= 1.01 * ceiling
    assert 1e11 < ex2 < fma
    assert ms > 0 and ms2 > 0
    with pytest.raises(vg.VGError):
        ws.pipe_peak("fma", 0.0)
