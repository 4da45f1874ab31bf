"""Fixed-capacity binning (no host synchronisation) and a whole training step captured in a
CUDA graph, against the oracle and the eager path; failures reported by the device (capacity
overflow, a bounded wait that gave up) without a GPU fault."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import check_grads, dev_scene, flat, run_forward, vg_opts

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4
GRAD_TOL = 1e-3


def _scene():
    scene = synth.uniform_scene(700, 77, log_scale=(-3.5, -2.2), sh_degree=3, sh_std=0.25, flatten_frac=0.2,
                                extent=0.9)
    cams = synth.small_views(2, 3, [(64, 48), (45, 37)])
    return scene, cams


def _reserve(vg, ws, scene, cams, n_inst):
    P = sum(c.width * c.height for c in cams)
    tiles = sum(((c.width + 15) // 16) * ((c.height + 15) // 16) for c in cams)
    ws.reserve(scene.n * len(cams), n_inst, P, tiles)


def test_fixed_capacity_bins_match_oracle(gpu_lib):
    vg = gpu_lib
    scene, cams = _scene()
    o = dict(oracle.EXACT, bg=(0.2, 0.1, 0.3))
    L = oracle.lists(scene, cams, o)
    n_inst = int(L["tile_start"][-1])
    ws = vg.Workspace()
    _reserve(vg, ws, scene, cams, n_inst + 100)
    g = dev_scene(vg, scene)
    ws.preprocess(g, cams, vg_opts(vg, o, flags=vg.FLAG_FIXED_CAPACITY))
    ws.bin_sort()
    q = ws.query()
    assert q["n_instances"] == n_inst and q["instance_capacity"] >= n_inst
    ts, items = ws.read_bins()
    assert np.array_equal(ts, L["tile_start"])
    assert np.array_equal(items % scene.n, L["sorted_g"])
    import torch
    P = sum(c.width * c.height for c in cams)
    rgb = torch.empty(P, 3, device="cuda:0")
    ws.render_fwd(rgb)
    ref_rgb, _, _ = oracle.render(scene, cams, o)
    assert np.max(np.abs(rgb.cpu().numpy() - flat(ref_rgb))) < IMG_TOL


def test_fixed_capacity_overflow_is_latched(gpu_lib):
    vg = gpu_lib
    scene, cams = _scene()
    o = oracle.EXACT
    n_inst = int(oracle.lists(scene, cams, o)["tile_start"][-1])
    ws = vg.Workspace()
    _reserve(vg, ws, scene, cams, n_inst // 2)
    g = dev_scene(vg, scene)
    ws.preprocess(g, cams, vg_opts(vg, o, flags=vg.FLAG_FIXED_CAPACITY))
    ws.bin_sort()
    with pytest.raises(RuntimeError, match="capacity"):
        ws.query()
    # reported once: the workspace is usable again with enough capacity
    _reserve(vg, ws, scene, cams, n_inst)
    ws.preprocess(g, cams, vg_opts(vg, o, flags=vg.FLAG_FIXED_CAPACITY))
    ws.bin_sort()
    assert ws.query()["n_instances"] == n_inst


@pytest.mark.parametrize("mode", ["exact", "compat"])
def test_graph_captured_step_matches_eager(gpu_lib, mode):
    import torch
    vg = gpu_lib
    scene, cams = _scene()
    o = dict(oracle.EXACT if mode == "exact" else oracle.COMPAT, bg=(0.1, 0.2, 0.3))
    n_inst = int(oracle.lists(scene, cams, o)["tile_start"][-1])
    dev = torch.device("cuda:0")
    P = sum(c.width * c.height for c in cams)
    g = dev_scene(vg, scene)
    target = torch.as_tensor(synth.random_image(5, (P, 3)).astype(np.float32)).to(dev)
    opts = vg_opts(vg, o, flags=vg.FLAG_FIXED_CAPACITY | vg.FLAG_GRAD_ZERO)

    def buffers():
        return dict(rgb=torch.empty(P, 3, device=dev), T=torch.empty(P, device=dev),
                    dl=torch.empty(P, 3, device=dev), loss=torch.zeros(1, device=dev),
                    mu=torch.empty(g.n, 3, device=dev), scale=torch.empty(g.n, 3, device=dev),
                    quat=torch.empty(g.n, 4, device=dev), kappa=torch.empty(g.n, device=dev),
                    sh=torch.empty(tuple(g.sh.shape), device=dev))

    def step(ws, b):
        ws.preprocess(g, cams, opts)
        ws.bin_sort()
        ws.render_fwd(b["rgb"], b["T"])
        ws.l2_loss(b["rgb"], target, 1.0 / (3 * P), b["loss"], b["dl"])
        ws.render_bwd(b["dl"], None, b["mu"], b["scale"], b["quat"], b["kappa"], b["sh"])

    eager_ws, eb = vg.Workspace(), buffers()
    _reserve(vg, eager_ws, scene, cams, n_inst)
    step(eager_ws, eb)
    torch.cuda.synchronize()

    ws, b = vg.Workspace(), buffers()
    _reserve(vg, ws, scene, cams, n_inst)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step(ws, b)                      # warm-up: uploads the cameras
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step(ws, b)
    for v in b.values():
        v.fill_(float("nan"))
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(b["rgb"], eb["rgb"]) and torch.equal(b["T"], eb["T"])
    assert torch.allclose(b["loss"], eb["loss"], rtol=1e-6, atol=0)
    gg = {k: b[k].cpu().numpy().astype(np.float64) for k in ("mu", "scale", "quat", "kappa", "sh")}
    ge = {k: eb[k].cpu().numpy().astype(np.float64) for k in ("mu", "scale", "quat", "kappa", "sh")}
    check_grads(gg, ge, scene, 1e-4)
    assert ws.query()["n_instances"] == n_inst


@pytest.mark.parametrize("which", [0, 1, 2])
def test_bounded_wait_gives_up_and_is_reported(gpu_lib, which):
    """Failure detection of the bounded device waits, without a GPU fault: a binning look-back
    whose predecessor never publishes (which 0, 1) gives up after a few dozen polls, and the
    backward ring's wait on a full barrier no producer arrives on (which 2) after 48 us; each
    latches VG_ERR_TIMEOUT and returns; vg_query reports it once, and the workspace then renders
    as before (bit for bit)."""
    vg = gpu_lib
    scene, cams = synth.config1(0.25)
    o = oracle.EXACT
    ws, g, rgb0, T0 = run_forward(vg, scene, cams, o)
    ws.selftest_timeout(which, spin_limit=48)
    with pytest.raises(vg.VGError) as ei:
        ws.query()
    assert ei.value.status == 5 and "timed out" in str(ei.value)
    assert ws.query()["n_items"] == scene.n          # reported once, then cleared
    _, _, rgb1, T1 = run_forward(vg, scene, cams, o, ws=ws, g=g)
    assert np.array_equal(rgb0, rgb1) and np.array_equal(T0, T1)
    with pytest.raises(vg.VGError):
        ws.selftest_timeout(which, spin_limit=0)    # rejected on the host, nothing launched
