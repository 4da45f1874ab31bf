"""Volumetrically consistent 3D Gaussian rasterizer for NVIDIA GB300 (sm_103a).

Thin Python binding over the C ABI in `include/vg.h` (libvg.so, built in-tree by
`paper_2412_03378_gb300.build`).  Every step of the rasterizer runs in the library's
CUDA kernels; this module only marshals torch tensors (device memory, streams) into the
C calls and wraps forward/backward in a `torch.autograd.Function`.  There is no CPU or
PyTorch fallback: if the library is missing, `load()` raises.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field
from typing import Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvg.so")
_LIB = None

VG_F32, VG_BF16, VG_F16 = 0, 1, 2
FLAG_FIXED_CAPACITY = 1
FLAG_COUNT_PAIRS = 2
FLAG_GRAD_ZERO = 4
FLAG_DENSITY_THETA = 8
FLAG_SPLAT = 16
FLAG_PROJ_GIVEN = 32
# stage names of the event profiler, in the bit order of vg_profile_stages
STAGES = ("preprocess", "depth_sort", "scan", "duplicate", "tile_sort", "ranges", "render_fwd", "render_bwd",
          "chain", "l2_loss", "tomo_fwd", "tomo_bwd", "voxel_eval", "ray_march")
_STATUS = {0: "VG_OK", 1: "VG_ERR_INVALID_ARG", 2: "VG_ERR_CUDA", 3: "VG_ERR_OOM", 4: "VG_ERR_CAPACITY",
           5: "VG_ERR_TIMEOUT", 6: "VG_ERR_UNSUPPORTED", 7: "VG_ERR_STATE"}
TILE = 16


class VGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Gaussians(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_void_p), ("scale", ctypes.c_void_p), ("quat", ctypes.c_void_p),
                ("kappa", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("rec_dtype", ctypes.c_int32),
                ("sh_dtype", ctypes.c_int32), ("n", ctypes.c_int32), ("sh_degree", ctypes.c_int32),
                ("mu_f32", ctypes.c_int32)]


class _Camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class _Beam(ctypes.Structure):
    _fields_ = [("n_angles", ctypes.c_int32), ("angles", ctypes.c_void_p), ("det_w", ctypes.c_int32),
                ("det_h", ctypes.c_int32), ("pitch_u", ctypes.c_float), ("pitch_v", ctypes.c_float),
                ("u0", ctypes.c_float), ("v0", ctypes.c_float)]


class _Opts(ctypes.Structure):
    _fields_ = [("alpha_min", ctypes.c_float), ("tau_cut", ctypes.c_float), ("tau_max", ctypes.c_float),
                ("T_stop", ctypes.c_float), ("bg", ctypes.c_float * 3), ("z_near", ctypes.c_float),
                ("flags", ctypes.c_uint32), ("pixels_per_thread", ctypes.c_int32), ("softplus_beta", ctypes.c_float),
                ("splat_dilation", ctypes.c_float), ("chunk", ctypes.c_int32), ("tile_w", ctypes.c_int32),
                ("tile_h", ctypes.c_int32)]


class _Grid(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("voxel", ctypes.c_float * 3), ("nx", ctypes.c_int32),
                ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


class _StageTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("calls", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("n_items", "n_visible", "n_culled", "n_instances", "n_tiles",
                                              "n_pixels", "instance_capacity", "n_pairs", "launches",
                                              "device_bytes", "n_pairs_bwd", "n_blend", "n_blend_bwd")]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


#: every entry point of include/vg.h with its argument types
_SIGS = {
    "vg_workspace_create": [ctypes.c_void_p],
    "vg_workspace_destroy": [ctypes.c_void_p],
    "vg_workspace_reserve": [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64],
    "vg_autotune": [ctypes.c_void_p, ctypes.c_int32] + [ctypes.c_void_p] * 7,
    "vg_preprocess": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                      ctypes.c_void_p],
    "vg_bin_sort": [ctypes.c_void_p, ctypes.c_void_p],
    "vg_render_fwd": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "vg_render_fwd_l2": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float,
                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "vg_render_bwd": [ctypes.c_void_p] + [ctypes.c_void_p] * 7 + [ctypes.c_void_p],
    "vg_render_bwd_noalloc": [ctypes.c_void_p] + [ctypes.c_void_p] * 7 + [ctypes.c_void_p],
    "vg_project_tomo": [ctypes.c_void_p] * 11,
    "vg_project_cone": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32] + [ctypes.c_void_p] * 8,
    "vg_query_density": [ctypes.c_void_p] * 6,
    "vg_tomo_l2_step": [ctypes.c_void_p] * 5 + [ctypes.c_float] + [ctypes.c_void_p] * 7,
    "vg_ray_march": [ctypes.c_void_p, ctypes.c_float, ctypes.c_float, ctypes.c_int32] + [ctypes.c_void_p] * 5,
    "vg_l2_loss": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_float,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "vg_query": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "vg_read_keys": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "vg_profile_enable": [ctypes.c_void_p, ctypes.c_int32],
    "vg_profile_stages": [ctypes.c_void_p, ctypes.c_uint32],
    "vg_profile_read": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p],
    "vg_read_bins": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "vg_read_pixel_state": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "vg_selftest_timeout": [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p],
    "vg_pipe_peak": [ctypes.c_void_p, ctypes.c_int32, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p,
                     ctypes.c_void_p],
    "vg_read_bins_range": [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                           ctypes.c_int64, ctypes.c_void_p],
}


def load(path: str | None = None):
    """Load libvg.so (raises if it has not been built: there is no fallback path)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library {p} is missing; build it with paper_2412_03378_gb300.build.build()")
    L = ctypes.CDLL(p)
    for name, args in _SIGS.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.vg_last_error.argtypes = [ctypes.c_void_p]
    L.vg_last_error.restype = ctypes.c_char_p
    _LIB = L
    return L


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


_DT = {torch.float32: VG_F32, torch.bfloat16: VG_BF16, torch.float16: VG_F16}


@dataclass
class Opts:
    """Blend options (see vg_opts in include/vg.h)."""
    alpha_min: float = 0.0
    tau_cut: float = 1e-6
    tau_max: float = math.inf
    T_stop: float = 0.0
    bg: tuple = (0.0, 0.0, 0.0)
    z_near: float = 0.2
    flags: int = 0
    pixels_per_thread: int = 0
    softplus_beta: float = 0.0
    splat_dilation: float = 0.0
    chunk: int = 0
    tile_w: int = 0
    tile_h: int = 0

    @staticmethod
    def exact(**kw):
        """No skip, no clamp, no early stop; footprints truncated at tau = tau_cut."""
        return Opts(**kw)

    @staticmethod
    def compat(**kw):
        """The 3DGS thresholds: alpha >= 1/255 blended, alpha <= 0.99, stop at T < 1e-4."""
        d = dict(alpha_min=1.0 / 255.0, tau_cut=-math.log1p(-1.0 / 255.0), tau_max=math.log(100.0), T_stop=1e-4)
        d.update(kw)
        return Opts(**d)

    def c(self):
        o = _Opts()
        o.alpha_min, o.tau_cut, o.tau_max, o.T_stop = self.alpha_min, self.tau_cut, self.tau_max, self.T_stop
        for k in range(3):
            o.bg[k] = self.bg[k]
        o.z_near, o.flags, o.pixels_per_thread = self.z_near, self.flags, self.pixels_per_thread
        o.softplus_beta = self.softplus_beta
        o.splat_dilation = self.splat_dilation
        o.chunk = self.chunk
        o.tile_w, o.tile_h = self.tile_w, self.tile_h
        return o


@dataclass
class Gaussians:
    """Device tensors: mu [N,3], scale [N,3], quat [N,4] (w,x,y,z), kappa [N], sh [N,K,3]."""
    mu: torch.Tensor
    scale: torch.Tensor
    quat: torch.Tensor
    kappa: torch.Tensor
    sh: torch.Tensor | None
    sh_degree: int = 0

    @property
    def n(self):
        return int(self.mu.shape[0])

    def c(self):
        for t in (self.mu, self.scale, self.quat, self.kappa):
            if not (t.is_cuda and t.is_contiguous()):
                raise ValueError("Gaussian parameters must be contiguous CUDA tensors")
        g = _Gaussians()
        g.mu, g.scale, g.quat, g.kappa = (t.data_ptr() for t in (self.mu, self.scale, self.quat, self.kappa))
        g.sh = self.sh.data_ptr() if self.sh is not None else None
        # scale, quat and kappa share one dtype; mu has it too or is float32 (mixed storage)
        rec = _DT[self.scale.dtype]
        if self.quat.dtype != self.scale.dtype or self.kappa.dtype != self.scale.dtype:
            raise ValueError("scale, quat and kappa must share one dtype")
        if self.mu.dtype != self.scale.dtype and self.mu.dtype != torch.float32:
            raise ValueError("mu must have the dtype of scale/quat/kappa or be float32")
        g.rec_dtype = rec
        g.mu_f32 = 1 if self.mu.dtype == torch.float32 else 0
        g.sh_dtype = _DT[self.sh.dtype] if self.sh is not None else VG_F32
        g.n = self.n
        g.sh_degree = self.sh_degree
        return g


def camera_struct(cam):
    """Any object with R (3x3), t (3), fx, fy, cx, cy, width, height."""
    c = _Camera()
    R = [float(x) for row in cam.R for x in row]
    for k in range(9):
        c.R[k] = R[k]
    for k in range(3):
        c.t[k] = float(cam.t[k])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def _cams_array(cams):
    arr = (_Camera * len(cams))()
    for i, cam in enumerate(cams):
        arr[i] = camera_struct(cam)
    return arr


class Workspace:
    """A library workspace (device scratch owned by the C library)."""

    def __init__(self):
        self._L = load()
        h = ctypes.c_void_p()
        st = self._L.vg_workspace_create(ctypes.byref(h))
        if st != 0:
            raise VGError(st, "vg_workspace_create failed")
        self.h = h
        self.generation = 0

    def close(self):
        if getattr(self, "h", None):
            self._L.vg_workspace_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        if st != 0:
            raise VGError(st, self._L.vg_last_error(self.h).decode())

    # ---- raw entry points (same names as the C ABI) ----
    def reserve(self, n_items, n_instances, n_pixels, n_tiles):
        self._chk(self._L.vg_workspace_reserve(self.h, n_items, n_instances, n_pixels, n_tiles))

    def autotune(self, reps=3, stream=None):
        """Pick the tile shape, pixels per thread and the chunk depth of the blend kernels on the
        binned workload (left binned with the chosen shape); returns
        (ppt_fwd, ppt_bwd, chunk_fwd, chunk_bwd, tile_w, tile_h)."""
        v = [ctypes.c_int32(0) for _ in range(6)]
        self._chk(self._L.vg_autotune(self.h, int(reps), *(ctypes.byref(x) for x in v), _stream(stream)))
        return tuple(x.value for x in v)

    def preprocess(self, g: Gaussians, cams, opts: Opts, stream=None):
        self._keep = (g, _cams_array(cams), opts.c())
        self._chk(self._L.vg_preprocess(self.h, ctypes.byref(g.c()), self._keep[1], len(cams),
                                        ctypes.byref(self._keep[2]), _stream(stream)))
        self.generation += 1

    def bin_sort(self, stream=None):
        self._chk(self._L.vg_bin_sort(self.h, _stream(stream)))

    def render_fwd(self, rgb, T_final=None, stream=None):
        self._chk(self._L.vg_render_fwd(self.h, _ptr(rgb), _ptr(T_final), _stream(stream)))

    def render_fwd_l2(self, rgb, T_final, target, scale, loss, dL_drgb, stream=None):
        """vg_render_fwd_l2: the forward with the L2 loss against `target` fused into it."""
        self._chk(self._L.vg_render_fwd_l2(self.h, _ptr(rgb), _ptr(T_final), _ptr(target), float(scale), _ptr(loss),
                                           _ptr(dL_drgb), _stream(stream)))

    def render_bwd(self, dL_drgb, dL_dT, dmu, dscale, dquat, dkappa, dsh, stream=None):
        self._chk(self._L.vg_render_bwd(self.h, _ptr(dL_drgb), _ptr(dL_dT), _ptr(dmu), _ptr(dscale), _ptr(dquat),
                                        _ptr(dkappa), _ptr(dsh), _stream(stream)))

    def render_bwd_noalloc(self, dL_drgb, dL_dT, dmu, dscale, dquat, dkappa, dsh, stream=None):
        """vg_render_bwd_noalloc: the backward without any device allocation (see vg.h)."""
        self._chk(self._L.vg_render_bwd_noalloc(self.h, _ptr(dL_drgb), _ptr(dL_dT), _ptr(dmu), _ptr(dscale),
                                                _ptr(dquat), _ptr(dkappa), _ptr(dsh), _stream(stream)))

    def pipe_peak(self, pipe, min_ms=50.0, stream=None):
        """Measured peak of one pipe ("fma": FP32 FMA instructions/s, "ex2": ex2 instructions/s,
        per lane) and the duration of the timed launch in ms (see vg_pipe_peak)."""
        r, ms = ctypes.c_double(0.0), ctypes.c_float(0.0)
        self._chk(self._L.vg_pipe_peak(self.h, {"fma": 0, "ex2": 1}[pipe], float(min_ms), ctypes.byref(r),
                                       ctypes.byref(ms), _stream(stream)))
        return r.value, ms.value

    def selftest_timeout(self, which=0, spin_limit=64, stream=None):
        """Run one bounded look-back wait that must give up (see vg_selftest_timeout); the next
        query() raises VGError with VG_ERR_TIMEOUT."""
        self._chk(self._L.vg_selftest_timeout(self.h, int(which), int(spin_limit), _stream(stream)))

    def project_tomo(self, g: Gaussians, beam, opts: Opts, proj, dL_dproj=None, dmu=None, dscale=None, dquat=None,
                     dkappa=None, stream=None):
        ang = (ctypes.c_float * len(beam.angles))(*[float(a) for a in beam.angles])
        b = _Beam()
        b.n_angles, b.angles = len(beam.angles), ctypes.cast(ang, ctypes.c_void_p)
        b.det_w, b.det_h = int(beam.det_w), int(beam.det_h)
        b.pitch_u, b.pitch_v, b.u0, b.v0 = float(beam.pitch_u), float(beam.pitch_v), float(beam.u0), float(beam.v0)
        oc = opts.c()
        self._chk(self._L.vg_project_tomo(self.h, ctypes.byref(g.c()), ctypes.byref(b), ctypes.byref(oc), _ptr(proj),
                                          _ptr(dL_dproj), _ptr(dmu), _ptr(dscale), _ptr(dquat), _ptr(dkappa),
                                          _stream(stream)))

    def tomo_l2_step(self, g: Gaussians, beam, opts: Opts, target, scale, proj, loss, dmu, dscale, dquat, dkappa,
                     stream=None):
        """Fused tomography training step with the L2 loss (see vg_tomo_l2_step)."""
        ang = (ctypes.c_float * len(beam.angles))(*[float(a) for a in beam.angles])
        b = _Beam()
        b.n_angles, b.angles = len(beam.angles), ctypes.cast(ang, ctypes.c_void_p)
        b.det_w, b.det_h = int(beam.det_w), int(beam.det_h)
        b.pitch_u, b.pitch_v, b.u0, b.v0 = float(beam.pitch_u), float(beam.pitch_v), float(beam.u0), float(beam.v0)
        oc = opts.c()
        self._chk(self._L.vg_tomo_l2_step(self.h, ctypes.byref(g.c()), ctypes.byref(b), ctypes.byref(oc), _ptr(target),
                                          float(scale), _ptr(proj), _ptr(loss), _ptr(dmu), _ptr(dscale), _ptr(dquat),
                                          _ptr(dkappa), _stream(stream)))

    def project_cone(self, g: Gaussians, cams, opts: Opts, proj, dL_dproj=None, dmu=None, dscale=None, dquat=None,
                     dkappa=None, stream=None):
        """Cone-beam projection exp(-sum tau) per detector pixel, the source at each camera's
        centre; with dL_dproj also the gradients (see vg_project_cone)."""
        self._keep = (g, _cams_array(cams), opts.c())
        self._chk(self._L.vg_project_cone(self.h, ctypes.byref(g.c()), self._keep[1], len(cams),
                                          ctypes.byref(self._keep[2]), _ptr(proj), _ptr(dL_dproj), _ptr(dmu),
                                          _ptr(dscale), _ptr(dquat), _ptr(dkappa), _stream(stream)))
        self.generation += 1

    def query_density(self, g: Gaussians, origin, voxel, dims, opts: Opts, out, stream=None):
        """sigma = sum kappa G at the voxel centres of the grid, out [nz, ny, nx] float32 (see vg_query_density)."""
        gr = _Grid()
        for a in range(3):
            gr.origin[a], gr.voxel[a] = float(origin[a]), float(voxel[a])
        gr.nx, gr.ny, gr.nz = (int(d) for d in dims)
        oc = opts.c()
        self._chk(self._L.vg_query_density(self.h, ctypes.byref(g.c()), ctypes.byref(gr), ctypes.byref(oc), _ptr(out),
                                           _stream(stream)))

    def ray_march(self, t_near, t_far, n_samples, rgb=None, T=None, raster_rgb=None, err_map=None, stream=None):
        """Ray-marching reference of the binned views (see vg_ray_march): rgb [P, 3], T [P] and the
        overlap-error map err_map [P] (needs raster_rgb, the vg_render_fwd image)."""
        self._chk(self._L.vg_ray_march(self.h, float(t_near), float(t_far), int(n_samples), _ptr(raster_rgb), _ptr(rgb),
                                       _ptr(T), _ptr(err_map), _stream(stream)))

    def l2_loss(self, x, y, scale, loss, grad, stream=None):
        self._chk(self._L.vg_l2_loss(self.h, _ptr(x), _ptr(y), x.numel(), float(scale), _ptr(loss), _ptr(grad),
                                     _stream(stream)))

    def query(self, stream=None) -> dict:
        s = Stats()
        self._chk(self._L.vg_query(self.h, ctypes.byref(s), _stream(stream)))
        return s.as_dict()

    def profile_enable(self, on=True, stages=None):
        """Per-stage event timing on (clearing earlier records) or off; `stages` (names from
        STAGES) restricts the recorded stages, None records all."""
        mask = 0
        for name in stages or ():
            mask |= 1 << STAGES.index(name)
        self._chk(self._L.vg_profile_stages(self.h, mask))
        self._chk(self._L.vg_profile_enable(self.h, 1 if on else 0))

    def profile_read(self) -> dict:
        """{stage: (calls, total_ms)} of the event-timed stages since profile_enable."""
        arr = (_StageTime * 32)()
        n = ctypes.c_int32()
        self._chk(self._L.vg_profile_read(self.h, arr, 32, ctypes.byref(n)))
        return {arr[i].name.decode(): (int(arr[i].calls), float(arr[i].total_ms)) for i in range(n.value)}

    def read_keys(self):
        import numpy as np
        n = self.query()["n_items"]
        depth = np.zeros(n, np.uint32)
        rect = np.zeros((n, 4), np.int32)
        self._chk(self._L.vg_read_keys(self.h, depth.ctypes.data_as(ctypes.c_void_p),
                                       rect.ctypes.data_as(ctypes.c_void_p)))
        return depth, rect

    def read_bins(self):
        import numpy as np
        q = self.query()
        ts = np.zeros(q["n_tiles"] + 1, np.int64)
        si = np.zeros(max(1, q["n_instances"]), np.int32)
        self._chk(self._L.vg_read_bins(self.h, ts.ctypes.data_as(ctypes.c_void_p),
                                       si.ctypes.data_as(ctypes.c_void_p)))
        return ts, si[: q["n_instances"]]

    def read_pixel_state(self):
        """(S [n_pixels] float32, last [n_pixels] uint32) of the last forward (see vg_read_pixel_state)."""
        import numpy as np
        n = self.query()["n_pixels"]
        S = np.zeros(max(1, n), np.float32)
        last = np.zeros(max(1, n), np.uint32)
        self._chk(self._L.vg_read_pixel_state(self.h, S.ctypes.data_as(ctypes.c_void_p),
                                              last.ctypes.data_as(ctypes.c_void_p)))
        return S[:n], last[:n]

    def read_bins_range(self, tile0, tile1, cap):
        """Lists of tiles [tile0, tile1): (counts [tile1 - tile0], items concatenated)."""
        import numpy as np
        counts = np.zeros(max(1, tile1 - tile0), np.int64)
        items = np.zeros(max(1, cap), np.int32)
        n = ctypes.c_int64(0)
        self._chk(self._L.vg_read_bins_range(self.h, int(tile0), int(tile1), counts.ctypes.data_as(ctypes.c_void_p),
                                             items.ctypes.data_as(ctypes.c_void_p), int(cap), ctypes.byref(n)))
        return counts[: tile1 - tile0], items[: n.value]


def n_pixels(cams):
    return sum(int(c.width) * int(c.height) for c in cams)


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, ws, cams, opts, sh_degree, mu, scale, quat, kappa, sh):
        g = Gaussians(mu.detach().contiguous(), scale.detach().contiguous(), quat.detach().contiguous(),
                      kappa.detach().contiguous(), sh.detach().contiguous(), sh_degree)
        P = n_pixels(cams)
        rgb = torch.empty((P, 3), device=mu.device, dtype=torch.float32)
        T = torch.empty((P,), device=mu.device, dtype=torch.float32)
        ws.preprocess(g, cams, opts)
        ws.bin_sort()
        ws.render_fwd(rgb, T)
        ctx.ws, ctx.gen, ctx.g = ws, ws.generation, g
        return rgb, T

    @staticmethod
    def backward(ctx, g_rgb, g_T):
        ws, g = ctx.ws, ctx.g
        if ws.generation != ctx.gen:
            raise RuntimeError("the workspace was reused by another forward before this backward")
        dmu = torch.zeros_like(g.mu, dtype=torch.float32)
        dscale = torch.zeros_like(g.scale, dtype=torch.float32)
        dquat = torch.zeros_like(g.quat, dtype=torch.float32)
        dkappa = torch.zeros_like(g.kappa, dtype=torch.float32)
        dsh = torch.zeros_like(g.sh, dtype=torch.float32)
        g_rgb = (g_rgb if g_rgb is not None else torch.zeros((n_pixels_ws(ws), 3), device=g.mu.device)).contiguous()
        g_T = g_T.contiguous() if g_T is not None else None
        ws.render_bwd(g_rgb.float(), None if g_T is None else g_T.float(), dmu, dscale, dquat, dkappa, dsh)
        return (None, None, None, None, dmu.to(g.mu.dtype), dscale.to(g.scale.dtype), dquat.to(g.quat.dtype),
                dkappa.to(g.kappa.dtype), dsh.to(g.sh.dtype))


class _TomoFn(torch.autograd.Function):
    """proj = exp(-sum tau) of a parallel beam (vg_project_tomo); the backward calls it again
    with dL/dproj, which recomputes the projection and accumulates the gradients."""

    @staticmethod
    def forward(ctx, ws, beam, opts, mu, scale, quat, kappa):
        g = Gaussians(mu.detach().contiguous(), scale.detach().contiguous(), quat.detach().contiguous(),
                      kappa.detach().contiguous(), None, 0)
        proj = torch.empty((len(beam.angles), int(beam.det_h), int(beam.det_w)), device=mu.device,
                           dtype=torch.float32)
        ws.project_tomo(g, beam, opts, proj)
        ctx.ws, ctx.beam, ctx.opts, ctx.g = ws, beam, opts, g
        return proj

    @staticmethod
    def backward(ctx, g_proj):
        g = ctx.g
        grads = [torch.zeros_like(t, dtype=torch.float32) for t in (g.mu, g.scale, g.quat, g.kappa)]
        proj = torch.empty_like(g_proj, dtype=torch.float32)
        ctx.ws.project_tomo(g, ctx.beam, ctx.opts, proj, g_proj.contiguous().float(), *grads)
        return (None, None, None) + tuple(d.to(t.dtype) for d, t in zip(grads, (g.mu, g.scale, g.quat, g.kappa)))


class _ConeFn(torch.autograd.Function):
    """Cone-beam projection (vg_project_cone) with the same recompute-in-backward scheme."""

    @staticmethod
    def forward(ctx, ws, cams, opts, mu, scale, quat, kappa):
        g = Gaussians(mu.detach().contiguous(), scale.detach().contiguous(), quat.detach().contiguous(),
                      kappa.detach().contiguous(), None, 0)
        proj = torch.empty((n_pixels(cams),), device=mu.device, dtype=torch.float32)
        ws.project_cone(g, cams, opts, proj)
        ctx.ws, ctx.cams, ctx.opts, ctx.g = ws, cams, opts, g
        return proj

    @staticmethod
    def backward(ctx, g_proj):
        g = ctx.g
        grads = [torch.zeros_like(t, dtype=torch.float32) for t in (g.mu, g.scale, g.quat, g.kappa)]
        proj = torch.empty_like(g_proj, dtype=torch.float32)
        ctx.ws.project_cone(g, ctx.cams, ctx.opts, proj, g_proj.contiguous().float(), *grads)
        return (None, None, None) + tuple(d.to(t.dtype) for d, t in zip(grads, (g.mu, g.scale, g.quat, g.kappa)))


class Projector:
    """Differentiable tomography bound to one workspace (Sec. 6.2, Eq. 21): `parallel` for a
    parallel beam, `cone` for point sources (density only; colour coefficients unused)."""

    def __init__(self, opts: Opts | None = None):
        self.ws = Workspace()
        self.opts = opts or Opts(tau_cut=1e-6)

    def parallel(self, mu, scale, quat, kappa, beam):
        """proj [A, det_h, det_w] = exp(-sum of the line integrals)."""
        return _TomoFn.apply(self.ws, beam, self.opts, mu, scale, quat, kappa)

    def cone(self, mu, scale, quat, kappa, cams: Sequence):
        """proj [sum H*W] over the cameras' detectors."""
        return _ConeFn.apply(self.ws, list(cams), self.opts, mu, scale, quat, kappa)


def n_pixels_ws(ws):
    return ws.query()["n_pixels"]


class Rasterizer:
    """Differentiable renderer bound to one workspace.  One forward may be outstanding per
    rasterizer: a second forward before the first backward invalidates the first."""

    def __init__(self, opts: Opts | None = None):
        self.ws = Workspace()
        self.opts = opts or Opts.compat()

    def render(self, mu, scale, quat, kappa, sh, cams: Sequence, sh_degree: int | None = None):
        """Returns (rgb [sum H*W, 3], T_final [sum H*W]) for the concatenated views."""
        if sh_degree is None:
            sh_degree = int(round(math.sqrt(sh.shape[1]))) - 1
        return _RenderFn.apply(self.ws, list(cams), self.opts, sh_degree, mu, scale, quat, kappa, sh)

    def split(self, flat, cams):
        """Split a concatenated per-pixel buffer into per-view [H, W, ...] tensors."""
        out, o = [], 0
        for c in cams:
            n = int(c.width) * int(c.height)
            out.append(flat[o:o + n].reshape(int(c.height), int(c.width), *flat.shape[1:]))
            o += n
        return out
