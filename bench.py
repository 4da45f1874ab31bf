"""Benchmark of the volumetric Gaussian rasterizer (arXiv 2412.03378) on GB300.

Workload (the view-synthesis configuration): 1,000,000 Gaussians from a mixture of 64
anisotropic clusters (20% flattened 100x), SH degree 3, densities log-uniform in
[0.1, 100], one 1280x832 camera; one step = preprocess + bin/sort + forward blend + L2
loss against a random target + backward (gradients w.r.t. means, scales, quaternions,
densities and SH), FP32, inputs resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  For N > 1 (torchrun, one rank per GPU) each rank renders its own
replica (a single view does not split; see the design notes), value = all ranks' steps
divided by the slowest rank's time.  `--impl reference` times the FP64 CPU oracle (the
reference implementation of this build) on a bounded sample of the same step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd steps/s & frames/s, 1M Gaussians @1280×832, vs plain FP32, % of pipe peak"
WORKLOAD = "1M Gaussians (64-cluster mixture, 20% flattened, SH deg 3), 1280x832, fwd+bwd, L2 loss, FP32"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
SMS = 152
# HBM-bound stages, algorithmic bytes per Gaussian of the FP32 workload (SH degree 3): parameters
# 236 B (mu 12, scale 12, quat 16, kappa 4, SH 192); the preprocess writes the 96 B blend record and
# 24 B of keys per item; the chain reads the parameters and the 64 B accumulator and writes 236 B of
# gradients
PARAM_BYTES = 236
PRE_WRITE_BYTES = 120
CHAIN_ACC_BYTES = 64
# Algorithmic FP32 work, FMA counted as 2 and each transcendental (rsqrt, exp2) as 1:
# evaluating the closed-form tau of one (pixel, Gaussian) pair (d' and o' x d' from the pixel
# offset, both squared norms, rsqrt, exponent, exp2), then for pairs with tau >= tau_skip the
# forward blend step, or the backward replay and gradient (colour, dL/dtau, the two moment
# matrices and dL/dln kappa).
FLOPS_EVAL_PAIR = 44
FLOPS_FWD_BLEND = 12
FLOPS_BWD_BLEND = 64
# of which transcendental-unit (MUFU) operations: rsqrt and ex2 per evaluated pair; the ex2 of
# alpha (and, in the backward, of the replayed transmittance) per blended pair
XU_EVAL_PAIR = 2
XU_FWD_BLEND = 1
XU_BWD_BLEND = 2
# the CPU baseline's bounded sample: the same seeded tiles in the GPU arm's cpu_baseline and in
# every step of --impl reference
CPU_SAMPLE_TILES = 64
CPU_SAMPLE_SEED = 5


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.idx)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [[x.strip() for x in l.split(",")] for l in self.lines if l]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, n in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- setup
def make_workload(frac):
    import synth

    scene, cams, target = synth.config2(frac)
    return scene, cams, target


TRAFFIC_SOURCES = ("render_bwd.cu", "blend.cuh", "geometry.cuh", "vg_internal.cuh")


def kernel_source_sha1():
    """sha1 over the sources the backward blend kernel is compiled from, in a fixed order."""
    h = hashlib.sha1()
    for name in TRAFFIC_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2412_03378_gb300", "csrc", name), "rb").read())
    return h.hexdigest()


def step_config(scene, cams, world, frac):
    """The workload of the headline line, the same for both arms."""
    return {"workload": WORKLOAD, "gaussians": scene.n, "width": cams[0].width, "height": cams[0].height,
            "sh_degree": scene.sh_degree, "mode": "alpha_min 1/255, tau_max ln100, T_stop 1e-4",
            "l2": "inputs larger than L2 (236 MB Gaussian parameters + 12.8 MB target per step)",
            "parallelism": f"replicas x{world}", "frac": frac}


def traffic_record():
    """DRAM bytes per launch of the backward blend kernel from the committed ncu summary,
    valid only while the kernel's sources are unchanged (null otherwise)."""
    p = os.path.join(ROOT, "profiles", "render_bwd_cfg2_traffic.txt")
    if not os.path.exists(p):
        return None
    kv = {}
    for line in open(p):
        if ":" in line:
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_sha1") != kernel_source_sha1():
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def peaks():
    try:
        return json.load(open(PEAKS_PATH))
    except Exception:
        return {}


# ----------------------------------------------------------------------------- pipe peaks
def measure_pipe_peaks(vg, gpu_id, min_ms=50.0):
    """Measured FP32 FMA and ex2 (MUFU) rates of this GPU (vg_pipe_peak) with the SM clock sampled
    during the measurement: the denominators of the blend kernels' roofline."""
    ws = vg.Workspace()
    clk = ClockSampler(gpu_id)
    clk.start()
    fma, fma_ms = ws.pipe_peak("fma", min_ms)
    ex2, ex2_ms = ws.pipe_peak("ex2", min_ms)
    fma2, _ = ws.pipe_peak("fma", min_ms)   # again, after the ex2 run: the clock may have moved
    c = clk.stop()
    fma = max(fma, fma2)
    out = {"fma_tflops": 2.0 * fma / 1e12, "ex2_tops": ex2 / 1e12, "fma_launch_ms": fma_ms, "ex2_launch_ms": ex2_ms,
           "clocks": c, "method": "vg_pipe_peak: 8 independent FMA (or ex2.approx) chains per thread, grid at the "
                                  "occupancy limit on every SM, fastest of 3 event-timed launches"}
    if c and c.get("sm_mhz"):
        mhz = c["sm_mhz"]
        out["fma_per_sm_per_clk"] = fma / (SMS * mhz * 1e6)
        out["ex2_per_sm_per_clk"] = ex2 / (SMS * mhz * 1e6)
    return out


# ----------------------------------------------------------------------------- cone beam
def run_cone(args):
    """Cone-beam tomography: config 4's Gaussians (200,000; --frac scales them) seen by 256 X-ray
    sources on a circle of radius 4, each with a 512^2 detector; one step = the projections of
    all sources, L2 loss against those of the 50,000 ground-truth Gaussians, and the backward."""
    import torch

    import paper_2412_03378_gb300 as vg
    import synth

    vg.load()
    dev = torch.device("cuda:0")
    scene, _, gt = synth.config4(args.frac)
    cams = synth.cone_beam(256, det=512)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev).contiguous()
    g = vg.Gaussians(t(scene.mu), t(scene.scale), t(scene.quat), t(scene.kappa), None, 0)
    gg = vg.Gaussians(t(gt.mu), t(gt.scale), t(gt.quat), t(gt.kappa), None, 0)
    P = sum(c.width * c.height for c in cams)
    ws = vg.Workspace()
    o = vg.Opts(tau_cut=1e-6, flags=vg.FLAG_GRAD_ZERO)
    tgt = torch.empty(P, device=dev)
    ws.project_cone(gg, cams, o, tgt)
    proj, dl, loss = torch.empty(P, device=dev), torch.empty(P, device=dev), torch.zeros(1, device=dev)
    grads = [torch.empty(g.n, 3, device=dev), torch.empty(g.n, 3, device=dev), torch.empty(g.n, 4, device=dev),
             torch.empty(g.n, device=dev)]

    def step():
        ws.project_cone(g, cams, o, proj)
        ws.l2_loss(proj, tgt, 1.0 / P, loss, dl)
        ws.project_cone(g, cams, o, proj, dl, *grads)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ws.profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    stages = ws.profile_read()
    q = ws.query()
    t_s = e0.elapsed_time(e1) / 1e3
    out = {"metric": "cone-beam tomography fwd+bwd steps/s", "value": args.steps / t_s, "unit": "steps/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_s * 1e3 / args.steps,
           "higher_is_better": True, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"cone-beam tomography, {g.n} Gaussians, {len(cams)} sources at radius 4, "
                                  "512x512 detectors", "frac": args.frac},
           "stages_ms_per_step": {k: round(v[1] / args.steps, 3) for k, v in stages.items()},
           "instances": q["n_instances"], "workspace_bytes": q["device_bytes"], "loss": float(loss.item())}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- voxel density query
def run_voxel(args):
    """Voxel density query: config 4's Gaussians (200,000; --frac scales them) evaluated on a
    256^3 grid over [-1, 1]^3; one step = one full query (truncation boxes, binning into 8^3
    bricks, per-brick sums)."""
    import torch

    import paper_2412_03378_gb300 as vg
    import synth

    vg.load()
    dev = torch.device("cuda:0")
    scene, _, _ = synth.config4(args.frac)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev).contiguous()
    g = vg.Gaussians(t(scene.mu), t(scene.scale), t(scene.quat), t(scene.kappa), None, 0)
    dims, origin, voxel = (256, 256, 256), (-1.0, -1.0, -1.0), (2.0 / 256,) * 3
    ws = vg.Workspace()
    o = vg.Opts(tau_cut=1e-6)
    out = torch.empty(dims[::-1], device=dev)

    def step():
        ws.query_density(g, origin, voxel, dims, o, out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ws.profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    stages = ws.profile_read()
    q = ws.query()
    t_s = e0.elapsed_time(e1) / 1e3
    nvox = dims[0] * dims[1] * dims[2]
    out_ = {"metric": "voxel density queries/s", "value": args.steps / t_s, "unit": "queries/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_s * 1e3 / args.steps,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"voxel density, {g.n} Gaussians, 256^3 grid", "frac": args.frac},
            "gvoxels_per_s": nvox * args.steps / t_s / 1e9,
            "stages_ms_per_step": {k: round(v[1] / args.steps, 3) for k, v in stages.items()},
            "instances": q["n_instances"], "sum": float(out.sum().item())}
    print(json.dumps(out_), flush=True)


# ----------------------------------------------------------------------------- ray-march reference
def run_march(args):
    """Supp. A at scale: config 1's scene (2,000 Gaussians, uniform in [-1, 1]^3, scales 0.018-0.135)
    seen by a 1280x832 camera, rasterized (exact mode) and ray-marched with 1,024 samples on
    [2.5, 5.5] (spacing 0.003, well below the smallest scale); one step = one march with the
    overlap-error map.  Also times the march on config 2's 1M Gaussians (512 samples), where the
    thinnest Gaussians are below the sample spacing (a timing, not a reference image)."""
    import torch

    import paper_2412_03378_gb300 as vg
    import synth

    vg.load()
    dev = torch.device("cuda:0")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev).contiguous()

    def setup(scene, cam):
        g = vg.Gaussians(t(scene.mu), t(scene.scale), t(scene.quat), t(scene.kappa), t(scene.sh), scene.sh_degree)
        ws = vg.Workspace()
        P = cam.width * cam.height
        raster, T = torch.empty(P, 3, device=dev), torch.empty(P, device=dev)
        ws.preprocess(g, [cam], vg.Opts.exact())
        ws.bin_sort()
        ws.render_fwd(raster, T)
        return g, ws, raster, P

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    scene, _ = synth.config1()
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 1280, 832, 60.0)
    g, ws, raster, P = setup(scene, cam)
    rgb, T, err = torch.empty(P, 3, device=dev), torch.empty(P, device=dev), torch.empty(P, device=dev)
    ms = timed(lambda: ws.ray_march(2.5, 5.5, 1024, rgb, T, raster, err), args.steps, args.warmup)
    e = err.cpu().numpy()
    q = ws.query()
    scene2, cams2, _ = synth.config2(args.frac)
    g2, ws2, raster2, P2 = setup(scene2, cams2[0])
    rgb2 = torch.empty(P2, 3, device=dev)
    ms2 = timed(lambda: ws2.ray_march(2.2, 5.8, 512, rgb2), max(1, args.steps // 4), 1)
    q2 = ws2.query()
    out = {"metric": "ray-march reference (Supp. A) marches/s", "value": 1e3 / ms, "unit": "marches/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": "config 1 scene (2,000 Gaussians) at 1280x832, 1,024 samples on [2.5, 5.5], "
                                  "overlap-error map against the exact-mode raster"},
           "instances": q["n_instances"],
           "overlap_error": {"mean": float(e.mean()), "p99": float(np.quantile(e, 0.99)), "max": float(e.max()),
                             "frac_above_1e-2": float((e > 1e-2).mean())},
           "config2_march_ms": ms2, "config2_instances": q2["n_instances"],
           "config2_note": "1M Gaussians, 1280x832, 512 samples on [2.2, 5.8]; the thinnest Gaussians are "
                           "narrower than the sample spacing, so this is a timing only"}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- batched graph path
def graph_step(vg, g, cams, steps, warmup, dev, target_seed=2102):
    """A whole training step over all `cams` (preprocess, bin/sort, forward with the L2 loss fused, backward)
    with fixed-capacity binning, autotuned pixels per thread, captured once as a CUDA graph and
    replayed `steps` times.  Returns the timing, the rendered images and the workspace."""
    import torch

    import synth

    P = sum(c.width * c.height for c in cams)
    tgt = torch.as_tensor(synth.random_image(target_seed, (P, 3))).to(dev)
    ws = vg.Workspace()
    # tune on one eager pass (tile shape, pixels per thread, chunk depth), then size the
    # instance capacity from the tuned binning (10% headroom)
    ws.preprocess(g, cams, vg.Opts.compat())
    ws.bin_sort()
    ppt = ws.autotune(reps=3)
    q0 = ws.query()
    n_inst = q0["n_instances"]
    ws.reserve(g.n * len(cams), int(n_inst * 1.10) + 4096, P, q0["n_tiles"])
    opts = vg.Opts.compat(flags=vg.FLAG_GRAD_ZERO | vg.FLAG_FIXED_CAPACITY)
    rgb, T, dl = torch.empty(P, 3, device=dev), torch.empty(P, device=dev), torch.empty(P, 3, device=dev)
    loss = torch.zeros(1, device=dev)
    grads = [torch.empty(g.n, 3, device=dev), torch.empty(g.n, 3, device=dev), torch.empty(g.n, 4, device=dev),
             torch.empty(g.n, device=dev), torch.empty(tuple(g.sh.shape), device=dev)]
    scale = 1.0 / float(rgb.numel())

    def step():
        ws.preprocess(g, cams, opts)
        ws.bin_sort()
        ws.render_fwd_l2(rgb, T, tgt, scale, loss, dl)
        ws.render_bwd(dl, None, *grads)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(max(1, warmup)):
            step()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for _ in range(max(1, warmup)):
        graph.replay()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    q = ws.query()   # raises if the fixed capacity overflowed during the run
    out = {"views": len(cams), "sizes": sorted({f"{c.width}x{c.height}" for c in cams}),
           "launch": "fixed-capacity binning, autotuned pixels per thread and chunk depth, whole step replayed as one "
                     "CUDA graph",
           "tile": f"{ppt[4]}x{ppt[5]}", "pixels_per_thread": {"fwd": ppt[0], "bwd": ppt[1]},
           "chunk": {"fwd": ppt[2], "bwd": ppt[3]},
           "steps_per_s": steps / t, "views_per_s": steps * len(cams) / t, "ms_per_step": t * 1e3 / steps,
           "instances": q["n_instances"], "instance_capacity": q["instance_capacity"],
           "workspace_bytes": q["device_bytes"]}
    return out, rgb, ws


def reduced_gaussians(vg, scene, dev, rec=None, sh=None, mu32=False):
    """Reduced-precision storage: scale/quat/kappa in `rec`, SH in `sh`, the means in `rec` or
    (mu32) in FP32."""
    import torch

    rec = rec or torch.bfloat16
    sh = sh or torch.float16
    cv = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(dev).to(dt).contiguous()
    return vg.Gaussians(cv(scene.mu, torch.float32 if mu32 else rec), cv(scene.scale, rec), cv(scene.quat, rec),
                        cv(scene.kappa, rec), cv(scene.sh, sh), scene.sh_degree)


def batched_graph(vg, scene, cam0, rgb_view0, n_views, steps, warmup, dev, with_oracle=True):
    """The headline scene with BF16 scales/rotations/densities, FP16 SH and FP32 means, rendered from
    n_views views of uneven resolution (the single-view camera first, then views stepping from
    640x416 to 1920x1080 as in the 16-view configuration), the step replayed as one CUDA graph.
    Reports throughput against the plain FP32 single view, the compute error per view against the
    oracle on the dequantised parameters (sampled pixels), and the quantisation error of view 0
    against the FP32-parameter image for this storage and for all-BF16 storage (means included)."""
    import torch

    import synth

    cams = [cam0] + synth.fibonacci_cameras(n_views - 1, 4.0, synth._batched_sizes(n_views - 1))
    g = reduced_gaussians(vg, scene, dev, mu32=True)
    out, rgb, _ = graph_step(vg, g, cams, steps, warmup, dev)
    out["storage"] = "fp32 mu, bf16 scale/quat/kappa, f16 SH (124 B per Gaussian against 236 B in FP32); " \
                     "FP32 records and arithmetic"
    out["pixels_per_s"] = out["steps_per_s"] * sum(c.width * c.height for c in cams)
    P0 = cam0.width * cam0.height

    def quant_err(img):
        err = (img[:P0] - rgb_view0).abs()
        return {"max_abs": float(err.max()), "mean_abs": float(err.mean()),
                "p99_abs": float(err.flatten().kthvalue(max(1, int(0.99 * err.numel()))).values)}

    out["view0_vs_fp32_params"] = quant_err(rgb)
    # the same view with every parameter in BF16 (means too), one eager forward
    gb = reduced_gaussians(vg, scene, dev, mu32=False)
    ws = vg.Workspace()
    rgb_b = torch.empty(P0, 3, device=dev)
    ws.preprocess(gb, [cam0], vg.Opts.compat())
    ws.bin_sort()
    ws.render_fwd(rgb_b)
    out["view0_vs_fp32_params_all_bf16"] = quant_err(rgb_b)
    out["quantisation_note"] = "difference from the FP32-parameter image: the rounding of the stored inputs"
    if with_oracle:
        import oracle

        rd = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a, np.float32)).to(dt).float().numpy()
        sq = synth.Scene(np.asarray(scene.mu, np.float32), rd(scene.scale, torch.bfloat16),
                         rd(scene.quat, torch.bfloat16), rd(scene.kappa, torch.bfloat16),
                         rd(scene.sh, torch.float16), scene.sh_degree)
        rng = np.random.default_rng(77)
        masks = []
        for c in cams:
            m = np.zeros(c.width * c.height, np.int32)
            m[rng.choice(c.width * c.height, size=2000, replace=False)] = 1
            masks.append(m)
        ref, _, _ = oracle.render(sq, cams, oracle.COMPAT, mask=np.concatenate(masks))
        got = rgb.cpu().numpy().astype(np.float64)
        per_view, o = [], 0
        for c, m, r in zip(cams, masks, ref):
            sel = m.astype(bool)
            e = np.abs(got[o:o + c.width * c.height][sel] - r.reshape(-1, 3)[sel]).max(axis=1)
            per_view.append({"size": f"{c.width}x{c.height}", "max_abs": float(e.max()),
                             "pixels_above_1e-4": int((e > 1e-4).sum()), "pixels": int(sel.sum())})
            o += c.width * c.height
        out["compute_error_vs_oracle"] = per_view
        out["compute_error_note"] = ("FP64 oracle on the dequantised parameters (the values the GPU reads), 2,000 "
                                     "seeded pixels per view, compat thresholds")
    return out


def run_batched_config(args):
    """--workload cfg3 / cfg5: the batched configurations, one JSON line each."""
    import torch

    import paper_2412_03378_gb300 as vg
    import synth

    vg.load()
    dev = torch.device("cuda:0")
    if args.workload == "cfg3":
        scene, cams = synth.config3(args.frac)
        g = reduced_gaussians(vg, scene, dev, torch.bfloat16, torch.float16)
        name = (f"{scene.n} Gaussians (cluster generator, 40% flattened, SH deg 3), BF16 parameters, FP16 SH, "
                f"{len(cams)} views 640x416..1920x1080")
    else:
        scene, cams = synth.config5(args.frac)
        g = reduced_gaussians(vg, scene, dev, torch.bfloat16, torch.float32)
        name = f"{scene.n} Gaussians (cluster generator, SH deg 3), BF16 parameters, {len(cams)} views 1920x1080"
    torch.cuda.reset_peak_memory_stats()
    out, _, ws = graph_step(vg, g, cams, args.steps, args.warmup, dev)
    res = {"metric": "fwd+bwd steps/s (all views per step)", "value": out["steps_per_s"], "unit": "steps/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": out["ms_per_step"],
           "higher_is_better": True, "dtype": "f32 arithmetic, bf16/f16 storage", "data": "synthetic",
           "config": {"workload": name, "frac": args.frac}, "views_per_s": out["views_per_s"],
           "detail": out, "peak_device_bytes": {"workspace": out["workspace_bytes"],
                                                "torch": int(torch.cuda.max_memory_allocated())}}
    print(json.dumps(res), flush=True)


# ----------------------------------------------------------------------------- GPU arm
def max_over_ranks(t_local, dev, world):
    """The timed region's duration of the slowest rank (every rank calls this after its own
    barrier-bracketed region): the job finishes when its last replica does."""
    if world <= 1:
        return t_local
    import torch
    import torch.distributed as dist

    tt = torch.tensor([t_local], dtype=torch.float64, device=dev)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_value(steps, world, t_max):
    """Whole-job throughput: the steps all ranks processed over the slowest rank's time."""
    return steps * world / t_max


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2412_03378_gb300 as vg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", torch.cuda.current_device())
    vg.load()

    scene, cams, target = make_workload(args.frac)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev).contiguous()
    g = vg.Gaussians(t(scene.mu), t(scene.scale), t(scene.quat), t(scene.kappa), t(scene.sh), scene.sh_degree)
    tgt = t(target.reshape(-1, 3))
    P = cams[0].width * cams[0].height
    ws = vg.Workspace()
    opts = vg.Opts.compat(flags=vg.FLAG_GRAD_ZERO)
    rgb = torch.empty(P, 3, device=dev)
    T = torch.empty(P, device=dev)
    dldrgb = torch.empty(P, 3, device=dev)
    loss = torch.zeros(1, device=dev)
    grads = [torch.zeros(g.n, 3, device=dev), torch.zeros(g.n, 3, device=dev), torch.zeros(g.n, 4, device=dev),
             torch.zeros(g.n, device=dev), torch.zeros(tuple(g.sh.shape), device=dev)]
    scale = 1.0 / float(rgb.numel())

    def step(gg=g, target_dev=None):
        ws.preprocess(gg, cams, opts)
        ws.bin_sort()
        ws.render_fwd_l2(rgb, T, tgt if target_dev is None else target_dev, scale, loss, dldrgb)
        ws.render_bwd(dldrgb, None, *grads)

    def fwd_only():
        ws.preprocess(g, cams, opts)
        ws.bin_sort()
        ws.render_fwd(rgb, T)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- one-time set-up: the autotuner picks the tile shape, pixels per thread and chunk depth
    # on this workload (kept as the workspace's defaults); the instance capacity is reserved
    # from that binning (10% headroom) and the steps bin with VG_FLAG_FIXED_CAPACITY, so no
    # step waits on a host readback (an overflow would be reported by the query after the
    # timed region).  Then warm-up and exactly K timed steps bracketed by barrier + synchronize.
    ws.preprocess(g, cams, opts)
    ws.bin_sort()
    tuned = ws.autotune(reps=3)
    q0 = ws.query()
    capacity = int(q0["n_instances"] * 1.10) + 4096
    ws.reserve(g.n * len(cams), capacity, P, q0["n_tiles"])
    opts = vg.Opts.compat(flags=vg.FLAG_GRAD_ZERO | vg.FLAG_FIXED_CAPACITY)
    for _ in range(args.warmup):
        step()
    barrier()
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [x for x in cvd.split(",") if x.strip()]
    gpu_id = ids[local] if local < len(ids) else (ids[0] if ids else str(local))
    clocks = ClockSampler(gpu_id)
    clocks.start()
    l0 = ws.query()["launches"]
    # inside the timed region only the dominant kernel is bracketed by events (its live launch
    # time for the roofline); the per-stage breakdown comes from a separate pass below
    ws.profile_enable(True, stages=["render_bwd"])
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    stages_timed = ws.profile_read()
    ws.profile_enable(False)
    launches = ws.query()["launches"] - l0
    ms = e0.elapsed_time(e1)
    t_local = ms / 1e3
    t_max = max_over_ranks(t_local, dev, world)
    value = job_value(args.steps, world, t_max)

    # ---- per-stage breakdown: every stage bracketed by events, outside the timed region
    ws.profile_enable(True)
    for _ in range(args.steps):
        step()
    barrier()
    stages = ws.profile_read()
    ws.profile_enable(False)

    # ---- forward-only frames/s (same protocol, not part of the headline value)
    for _ in range(2):
        fwd_only()
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        fwd_only()
    f1.record(stream)
    barrier()
    frames = args.steps * world / (f0.elapsed_time(f1) / 1e3)

    # ---- pair counts for the roofline (separate, counted launches outside the timed region)
    ws.preprocess(g, cams, vg.Opts.compat(flags=vg.FLAG_GRAD_ZERO | vg.FLAG_COUNT_PAIRS))
    ws.bin_sort()
    ws.render_fwd_l2(rgb, T, tgt, scale, loss, dldrgb)
    ws.render_bwd(dldrgb, None, *grads)
    q = ws.query()

    # ---- end to end through the public API, copies timed.  As in any training step the model
    # state (the Gaussians, 236 MB) stays resident in HBM; the step's input is the view: its
    # camera (passed by value to vg_preprocess) and its target image, copied every step from
    # pinned host memory, and its result (the loss) is read back to the host.  The loop is the
    # one a training script runs: the next step's target is copied on a second stream into the
    # other of two device buffers while the current step computes, and each step's loss is read
    # on the host once the following step has been issued.  The same loop with the copy on the
    # compute stream and a host synchronisation after every step is reported as e2e.serial.
    host = [torch.as_tensor(np.ascontiguousarray(target.reshape(-1, 3))).pin_memory()]
    h2d = sum(h.numel() * h.element_size() for h in host)
    main_stream = torch.cuda.current_stream()
    copy_stream = torch.cuda.Stream(device=dev)
    tbuf = [tgt, torch.empty_like(tgt)]
    ev_copy = [torch.cuda.Event(), torch.cuda.Event()]
    ev_done = [torch.cuda.Event(), torch.cuda.Event()]
    loss_h = [torch.zeros(1).pin_memory(), torch.zeros(1).pin_memory()]
    losses = []

    def issue_copy(k):   # step k's target into buffer k % 2, once step k - 2 is done with it
        b = k % 2
        copy_stream.wait_event(ev_done[b])
        with torch.cuda.stream(copy_stream):
            tbuf[b].copy_(host[0], non_blocking=True)
            ev_copy[b].record(copy_stream)

    def e2e_loop(k_steps):
        issue_copy(0)
        for k in range(k_steps):
            b = k % 2
            main_stream.wait_event(ev_copy[b])
            step(target_dev=tbuf[b])
            loss_h[b].copy_(loss, non_blocking=True)
            ev_done[b].record(main_stream)
            if k + 1 < k_steps:
                issue_copy(k + 1)
            if k >= 1:
                ev_done[(k - 1) % 2].synchronize()
                losses.append(float(loss_h[(k - 1) % 2][0]))
        ev_done[(k_steps - 1) % 2].synchronize()
        losses.append(float(loss_h[(k_steps - 1) % 2][0]))

    def e2e_serial_step():
        tgt.copy_(host[0], non_blocking=True)
        step()
        loss_h[0].copy_(loss, non_blocking=True)
        main_stream.synchronize()
        return float(loss_h[0][0])

    e2e_loop(2)
    barrier()
    w0 = time.perf_counter()
    e2e_loop(args.steps)
    barrier()
    e2e_t = max_over_ranks(time.perf_counter() - w0, dev, world)
    e2e_value = job_value(args.steps, world, e2e_t)
    if not all(np.isfinite(losses)):
        raise RuntimeError("non-finite loss in the end-to-end loop")
    for _ in range(2):
        e2e_serial_step()
    barrier()
    w0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_serial_step()
    barrier()
    e2e_serial_value = job_value(args.steps, world, max_over_ranks(time.perf_counter() - w0, dev, world))

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (the backward blend), measured live, against the
    # measured FMA and ex2 rates of this GPU
    calls_bwd, ms_bwd = stages_timed.get("render_bwd", (0, 0.0))
    per_launch_s = (ms_bwd / max(1, calls_bwd)) / 1e3
    pp = measure_pipe_peaks(vg, gpu_id)
    traffic = traffic_record()

    def alu_roofline(kernel, pairs, blended, f_blend, xu_blend, t_s):
        flops = pairs * FLOPS_EVAL_PAIR + blended * f_blend
        xu = pairs * XU_EVAL_PAIR + blended * xu_blend
        fma_flops = flops - xu               # FP32-pipe work: FMA = 2 flop, other FP32 operations 1
        ach = fma_flops / t_s / 1e12 if t_s > 0 else None
        xu_rate = xu / t_s / 1e12 if t_s > 0 else None
        return {"bound": "alu", "kernel": kernel, "achieved": ach, "peak": pp["fma_tflops"], "unit": "TFLOP/s",
                "frac": ach / pp["fma_tflops"] if ach else None,
                "peak_basis": "measured FP32 FMA rate x 2 flop (vg_pipe_peak, clocks in pipe_peaks)",
                "xu": {"achieved_tops": xu_rate, "peak_tops": pp["ex2_tops"],
                       "frac": xu_rate / pp["ex2_tops"] if xu_rate else None,
                       "basis": "rsqrt + ex2 per evaluated pair, ex2 per blended pair (x2 in the backward) "
                                "against the measured ex2 rate"},
                "pairs_per_launch": pairs, "blended_pairs_per_launch": blended, "flops_per_launch": flops,
                "fma_pipe_flops_per_launch": fma_flops, "xu_ops_per_launch": xu,
                "flops_basis": f"{FLOPS_EVAL_PAIR} per evaluated pair + {f_blend} per blended pair (FMA = 2, "
                               f"transcendental = 1; {XU_EVAL_PAIR} + {xu_blend} of them on the MUFU)",
                "launch_ms": t_s * 1e3}

    roofline = alu_roofline("k_render_bwd", q["n_pairs_bwd"], q["n_blend_bwd"], FLOPS_BWD_BLEND, XU_BWD_BLEND,
                            per_launch_s)
    roofline["traffic"] = traffic
    hbm_peak = float(peaks().get("hbm_gbs", 6788.6))

    def hbm_roofline(stage, nbytes):
        calls, ms_tot = stages.get(stage, (0, 0.0))
        if not calls or ms_tot <= 0:
            return None
        gbs = nbytes / (ms_tot / calls / 1e3) / 1e9
        return {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "bytes_per_launch": nbytes, "launch_ms": ms_tot / calls,
                "peak_basis": "MEASURED_PEAKS.json hbm_gbs (copy)"}

    roofline_hbm = {"k_preprocess": hbm_roofline("preprocess", g.n * (PARAM_BYTES + PRE_WRITE_BYTES)),
                    "k_chain": hbm_roofline("chain", g.n * (2 * PARAM_BYTES + CHAIN_ACC_BYTES))}

    stage_ms = {k: round(v[1] / max(1, v[0]), 4) for k, v in stages.items()}
    calls_f, ms_f = stages.get("render_fwd", (0, 0.0))
    fwd_roof = alu_roofline("k_render_fwd", q["n_pairs"], q["n_blend"], FLOPS_FWD_BLEND, XU_FWD_BLEND,
                            (ms_f / max(1, calls_f)) / 1e3)

    out = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": step_config(scene, cams, world, args.frac),
        "binning": f"fixed capacity: {capacity} instances reserved from one tuned eager binning + 10%",
        "tuned": {"tile": f"{tuned[4]}x{tuned[5]}", "pixels_per_thread": {"fwd": tuned[0], "bwd": tuned[1]},
                  "chunk": {"fwd": tuned[2], "bwd": tuned[3]}, "by": "vg_autotune, once before the warm-up"},
        "frames_per_s": frames,
        "stages_ms": stage_ms,
        "stages_basis": "event-timed per stage over a separate pass of the same steps; inside the timed "
                        "region only k_render_bwd is bracketed by events; the L2 loss is fused into the "
                        "forward (vg_render_fwd_l2), so render_fwd includes it",
        "roofline": roofline,
        "roofline_fwd": fwd_roof,
        "roofline_hbm": roofline_hbm,
        "pipe_peaks": pp,
        "counts": {"visible": q["n_visible"], "instances": q["n_instances"], "pairs_fwd": q["n_pairs"],
                   "blend_fwd": q["n_blend"], "pairs_bwd": q["n_pairs_bwd"], "blend_bwd": q["n_blend_bwd"],
                   "workspace_bytes": q["device_bytes"]},
        "e2e": {"value": e2e_value, "unit": "steps/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 4,
                "inputs": "per step: target image H2D from pinned memory, camera by value, loss D2H; "
                          "Gaussians resident in HBM as training state",
                "loop": "next step's target copied on a second stream into the other of two device buffers "
                        "while the current step computes; each loss read on the host after the next step is issued",
                "serial": {"value": e2e_serial_value, "unit": "steps/s",
                           "loop": "copy on the compute stream, host synchronisation after every step"}},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    try:   # the same FP32 single-view step replayed as one CUDA graph (fixed capacity, autotuned)
        gs, _, _ = graph_step(vg, g, cams, args.steps, args.warmup, dev)
        out["graph_single_view"] = {"steps_per_s": gs["steps_per_s"], "ms_per_step": gs["ms_per_step"],
                                    "pixels_per_thread": gs["pixels_per_thread"], "chunk": gs["chunk"],
                                    "launch": gs["launch"]}
    except Exception as e:  # a side measurement, never the headline
        out["graph_single_view"] = {"error": str(e)}
    if args.batch_views > 1:
        # the plain FP32 image of the view, rendered again (the timed loop left rgb of the last step)
        ws.preprocess(g, cams, opts)
        ws.bin_sort()
        ws.render_fwd(rgb, T)
        bg_ = batched_graph(vg, scene, cams[0], rgb.detach().clone(), args.batch_views, args.steps, args.warmup, dev,
                            with_oracle=not args.no_cpu_baseline)
        bg_["ratio_vs_plain_views_per_s"] = bg_["views_per_s"] / value * world
        bg_["ratio_vs_plain_pixels_per_s"] = bg_["pixels_per_s"] / (value / world * P)
        out["batched_graph"] = bg_
        try:   # the 16-view configuration (3M Gaussians, BF16/FP16 storage, 640x416..1920x1080)
            import synth
            s3, c3 = synth.config3(1.0)
            g3 = reduced_gaussians(vg, s3, dev, torch.bfloat16, torch.float16)
            o3, _, ws3 = graph_step(vg, g3, c3, min(args.steps, 10), max(3, min(args.warmup, 5)), dev)
            out["config3_graph"] = {"workload": f"{s3.n} Gaussians, BF16 parameters, FP16 SH, {len(c3)} views "
                                                "640x416..1920x1080", "steps_per_s": o3["steps_per_s"],
                                    "views_per_s": o3["views_per_s"], "ms_per_step": o3["ms_per_step"],
                                    "tile": o3["tile"], "instances": o3["instances"],
                                    "launch": o3["launch"]}
            del ws3, g3
        except Exception as e:  # a side measurement, never the headline
            out["config3_graph"] = {"error": str(e)}
    try:
        out["splat_ab"] = splat_ab(vg, scene, cams, tgt, args.steps, args.warmup, dev, t_max * 1e3 / args.steps,
                                   frames / world)
    except Exception as e:  # a side measurement, never the headline
        out["splat_ab"] = {"error": str(e)}
    if world == 1 and not args.no_cpu_baseline:
        try:
            out["cpu_baseline"] = cpu_baseline(scene, cams, target)
        except Exception as e:  # the baseline is reported, never the headline
            out["cpu_baseline"] = {"error": str(e)}
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- 3DGS A/B
def splat_ab(vg, scene, cams, tgt, steps, warmup, dev, vol_step_ms, vol_frames):
    """The same scene and step in the 3DGS comparison mode (Eq. 5-7: alpha = o G' of the
    splatted 2D Gaussian, the 3DGS rasterizer's thresholds, footprint cut at alpha 1/255 and a
    0.3 px^2 dilation), against the volumetric step measured above.  Each Gaussian's opacity is
    the volumetric mode's opacity along the ray through its centre at its geometric-mean scale,
    o = 1 - exp(-kappa sqrt(2 pi) s), so that both modes see comparably dense scenes."""
    import torch

    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev).contiguous()
    sgeo = np.exp(np.log(scene.scale.astype(np.float64)).mean(1))
    opac = (-np.expm1(-scene.kappa.astype(np.float64) * math.sqrt(2 * math.pi) * sgeo)).astype(np.float32)
    g = vg.Gaussians(t(scene.mu), t(scene.scale), t(scene.quat), t(opac), t(scene.sh), scene.sh_degree)
    opts = vg.Opts.compat(flags=vg.FLAG_GRAD_ZERO | vg.FLAG_SPLAT, tau_cut=1.0 / 255.0, splat_dilation=0.3)
    P = cams[0].width * cams[0].height
    ws = vg.Workspace()
    rgb, T = torch.empty(P, 3, device=dev), torch.empty(P, device=dev)
    dl, loss = torch.empty(P, 3, device=dev), torch.zeros(1, device=dev)
    grads = [torch.zeros(g.n, 3, device=dev), torch.zeros(g.n, 3, device=dev), torch.zeros(g.n, 4, device=dev),
             torch.zeros(g.n, device=dev), torch.zeros(tuple(g.sh.shape), device=dev)]

    def fwd():
        ws.preprocess(g, cams, opts)
        ws.bin_sort()
        ws.render_fwd(rgb, T)

    def step():
        ws.preprocess(g, cams, opts)
        ws.bin_sort()
        ws.render_fwd_l2(rgb, T, tgt, 1.0 / float(rgb.numel()), loss, dl)
        ws.render_bwd(dl, None, *grads)

    def timed(fn):
        for _ in range(max(3, warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    fwd_ms = timed(fwd)
    ws.profile_enable(True)
    step_ms = timed(step)
    stages = ws.profile_read()
    ws.profile_enable(False)
    opts.flags |= vg.FLAG_COUNT_PAIRS
    step()
    opts.flags &= ~vg.FLAG_COUNT_PAIRS
    torch.cuda.synchronize()
    q = ws.query()
    return {"mode": "3DGS splat alpha (Eq. 5-7), alpha_min 1/255, alpha <= 0.99, T_stop 1e-4, dilation 0.3 px^2",
            "opacity": "o = 1 - exp(-kappa sqrt(2 pi) s_geomean)",
            "splat_step_ms": step_ms, "vol_step_ms": vol_step_ms,
            "splat_frames_per_s": 1e3 / fwd_ms, "vol_frames_per_s": vol_frames,
            "vol_over_splat_frames": vol_frames * fwd_ms / 1e3,
            "vol_over_splat_steps": step_ms / vol_step_ms,
            "splat_instances": q["n_instances"],
            "splat_counts": {"pairs_fwd": q["n_pairs"], "blend_fwd": q["n_blend"], "pairs_bwd": q["n_pairs_bwd"],
                             "blend_bwd": q["n_blend_bwd"]},
            "splat_stages_ms": {k: round(v[1] / max(1, v[0]), 4) for k, v in stages.items()},
            "paper_ratio_frames": "Tab. 1 (Mip-NeRF360, RTX 3090 Ti): 136 / 159 FPS = 0.86"}


# ----------------------------------------------------------------------------- CPU oracle
def oracle_step(scene, cams, target, n_sample, seed, oracle):
    """One oracle step on a bounded sample: keys + binning of every Gaussian, then the
    forward blend and the analytic gradient on n_sample seeded random tiles.  Returns the
    per-step time extrapolated to all tiles."""
    o = dict(oracle.COMPAT)
    t0 = time.perf_counter()
    L = oracle.lists(scene, cams, o)
    t1 = time.perf_counter()
    cam = cams[0]
    ntx, nty = L["tiles_x"][0], L["tiles_y"][0]
    n_tiles = int(ntx * nty)
    rng = np.random.default_rng(seed)
    pick = rng.choice(n_tiles, size=min(n_sample, n_tiles), replace=False)
    tile_of_pix = ((np.arange(cam.height)[:, None] // 16) * ntx + (np.arange(cam.width)[None, :] // 16)).reshape(-1)
    mask = np.isin(tile_of_pix, pick).astype(np.int32)
    empty = np.zeros_like(mask)
    # fixed per-call set-up of the oracle (FP64 parameters, colours) measured separately
    s0 = time.perf_counter()
    oracle.render(scene, cams, o, L, mask=empty)
    s1 = time.perf_counter()
    rgb, _, _ = oracle.render(scene, cams, o, L, mask=mask)
    s2 = time.perf_counter()
    g = np.zeros_like(rgb[0].reshape(-1, 3))
    sel = mask.astype(bool)
    g[sel] = 2.0 * (rgb[0].reshape(-1, 3)[sel] - target.reshape(-1, 3)[sel]) / float(target.size)
    s3 = time.perf_counter()
    oracle.render_grad(scene, cams, o, L, g, None, mask=empty)
    s4 = time.perf_counter()
    oracle.render_grad(scene, cams, o, L, g, None, mask=mask)
    s5 = time.perf_counter()
    fixed = (t1 - t0) + (s1 - s0) + (s4 - s3)
    per_tile = ((s2 - s1) - (s1 - s0) + (s5 - s4) - (s4 - s3)) / len(pick)
    est = fixed + max(per_tile, 0.0) * n_tiles
    wall = (t1 - t0) + (s5 - s0)
    return est, wall, len(pick), n_tiles


def cpu_baseline(scene, cams, target, n_sample=CPU_SAMPLE_TILES):
    """The oracle on the fixed seeded tile sample, on all host cores and on one core."""
    import oracle

    cores = oracle.set_threads(0)
    est, wall, k, n_tiles = oracle_step(scene, cams, target, n_sample, CPU_SAMPLE_SEED, oracle)
    oracle.set_threads(1)
    est1, wall1, _, _ = oracle_step(scene, cams, target, n_sample, CPU_SAMPLE_SEED, oracle)
    oracle.set_threads(0)
    return {"value": 1.0 / est, "unit": "steps/s", "cores": cores, "kind": "oracle", "extrapolated": True,
            "sample": f"FP64 oracle: keys+binning of all {scene.n} Gaussians, forward+gradient on {k} of "
                      f"{n_tiles} tiles (seed {CPU_SAMPLE_SEED}, the sample of --impl reference), per-tile time "
                      f"extrapolated to the full frame; {wall:.1f} s wall for the sample",
            "single_core": {"value": 1.0 / est1, "unit": "steps/s", "cores": 1, "extrapolated": True,
                            "sample_wall_s": wall1}}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return
    import oracle

    oracle.build()
    cores = oracle.set_threads(0)
    scene, cams, target = make_workload(args.frac)
    for w in range(args.warmup):
        oracle_step(scene, cams, target, 8, 100 + w, oracle)
    ests = []
    t0 = time.perf_counter()
    for k in range(args.steps):
        est, _, n_pick, n_tiles = oracle_step(scene, cams, target, CPU_SAMPLE_TILES, CPU_SAMPLE_SEED, oracle)
        ests.append(est)
    wall = time.perf_counter() - t0
    value = args.steps / sum(ests)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(ests) / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": step_config(scene, cams, world, args.frac),
           "cpu_baseline": {"value": value, "unit": "steps/s", "cores": cores, "kind": "oracle",
                            "extrapolated": True,
                            "sample": f"each step: keys+binning of all {scene.n} Gaussians, forward+gradient "
                                      f"on the same {n_pick} tiles of {n_tiles} (seed {CPU_SAMPLE_SEED}, the GPU "
                                      f"arm's cpu_baseline sample), extrapolated to the full frame; ms_per_step is "
                                      f"that extrapolation; {wall:.1f} s wall for all {args.steps} sampled steps"},
           "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- tomography
def run_tomo(args):
    """Tomography (config 4: 200,000 Gaussians, 256 parallel-beam angles, 512^2 detector; --frac
    scales the Gaussian count): one step = projection, L2 loss against the projection of the
    50,000 ground-truth Gaussians, and the backward.  Prints one JSON line."""
    import torch

    import paper_2412_03378_gb300 as vg
    import synth

    vg.load()
    dev = torch.device("cuda:0")
    scene, beam, gt = synth.config4(args.frac)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev).contiguous()
    g = vg.Gaussians(t(scene.mu), t(scene.scale), t(scene.quat), t(scene.kappa), t(scene.sh), 0)
    gg = vg.Gaussians(t(gt.mu), t(gt.scale), t(gt.quat), t(gt.kappa), t(gt.sh), 0)
    A = len(beam.angles)
    ws = vg.Workspace()
    tgt = torch.empty(A, beam.det_h, beam.det_w, device=dev)
    ws.project_tomo(gg, beam, vg.Opts(tau_cut=1e-6), tgt)
    proj, dl = torch.empty_like(tgt), torch.empty_like(tgt)
    loss = torch.zeros(1, device=dev)
    grads = [torch.zeros(g.n, 3, device=dev), torch.zeros(g.n, 3, device=dev), torch.zeros(g.n, 4, device=dev),
             torch.zeros(g.n, device=dev)]
    o = vg.Opts(tau_cut=1e-6, flags=vg.FLAG_GRAD_ZERO)

    def step():   # fused: each angle batch is preprocessed, binned and projected once
        ws.tomo_l2_step(g, beam, o, tgt, 1.0 / proj.numel(), proj, loss, *grads)

    def step_two_calls():   # project; loss; project again with dL/dproj, reusing the projection
        ws.project_tomo(g, beam, o, proj)
        ws.l2_loss(proj, tgt, 1.0 / proj.numel(), loss, dl)
        ws.project_tomo(g, beam, o2, proj, dl, *grads)

    o2 = vg.Opts(tau_cut=1e-6, flags=vg.FLAG_GRAD_ZERO | vg.FLAG_PROJ_GIVEN)

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ws.profile_enable(True)
    t_s = timed(step, args.steps)
    stages = ws.profile_read()
    ws.profile_enable(False)
    n_prof = args.steps + args.warmup   # timed() repeats the warm-up inside the profiled region
    t2 = timed(step_two_calls, max(1, args.steps // 2)) / max(1, args.steps // 2)
    out = {"metric": "tomography fwd+bwd steps/s", "value": args.steps / t_s, "unit": "steps/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_s * 1e3 / args.steps,
           "higher_is_better": True, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"tomography, {g.n} Gaussians, {A} parallel-beam angles, "
                                  f"{beam.det_w}x{beam.det_h} detector", "frac": args.frac},
           "stages_ms_per_step": {k: round(v[1] / n_prof, 3) for k, v in stages.items()},
           "two_call_ms_per_step": t2 * 1e3,
           "step": "vg_tomo_l2_step (fused per angle batch); two_call: vg_project_tomo, vg_l2_loss, "
                   "vg_project_tomo with dL/dproj and VG_FLAG_PROJ_GIVEN",
           "loss": float(loss.item())}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--frac", type=float, default=1.0, help="scale the Gaussian count (parity/smoke use only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-views", type=int, default=4,
                    help="views of the BF16 / graph-replayed batched measurement (0: skip it)")
    ap.add_argument("--workload", choices=["render", "tomo", "cone", "voxel", "march", "cfg3", "cfg5"], default="render",
                    help="render: the headline training step; tomo: the tomography step (config 4); "
                         "cone: cone-beam tomography; voxel: the voxel density query; "
                         "march: the ray-marching reference and its overlap-error map; "
                         "cfg3 / cfg5: the batched BF16 configurations as one CUDA graph per step")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        log("note: fewer than 3 warm-up steps")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "tomo":
        run_tomo(args)
    elif args.workload == "cone":
        run_cone(args)
    elif args.workload == "voxel":
        run_voxel(args)
    elif args.workload == "march":
        run_march(args)
    elif args.workload in ("cfg3", "cfg5"):
        run_batched_config(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
