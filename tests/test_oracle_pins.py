"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each check uses an independent route (numerical quadrature, a library rotation,
brute force, closed forms) so that a dropped term, a wrong sign or a transposed
operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.spatial.transform import Rotation

import oracle
import synth


# ----------------------------------------------------------------------------- helpers
def rot(q):
    w, x, y, z = np.asarray(q, np.float64)
    return Rotation.from_quat([x, y, z, w]).as_matrix()      # scipy is scalar-last


def cov_world(scene, g):
    R = rot(scene.quat[g])
    return R @ np.diag(np.asarray(scene.scale[g], np.float64) ** 2) @ R.T


def mahal(x, mu, Sig):
    d = np.asarray(x, np.float64) - mu
    return float(d @ np.linalg.solve(Sig, d))


def pixel_rays(cam):
    """Unit world directions through pixel centres (the camera model, written out)."""
    R = np.asarray(cam.R, np.float64)
    t = np.asarray(cam.t, np.float64)
    fx, fy, cx, cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))   # stored as float32
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    dc = np.stack([(xs + 0.5 - cx) / fx, (ys + 0.5 - cy) / fy, np.ones_like(xs, float)], -1)
    d = dc @ R          # R^T dc for row vectors
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    return -R.T @ t, d


def one_gaussian(mu, scale, quat, kappa, sh0=(0.0, 0.0, 0.0)):
    return synth.Scene(np.array([mu], np.float32), np.array([scale], np.float32), np.array([quat], np.float32),
                       np.array([kappa], np.float32), np.array([[sh0]], np.float32), 0)


def concat(*scenes):
    return synth.Scene(*(np.concatenate([getattr(s, f) for s in scenes]) for f in ("mu", "scale", "quat", "kappa", "sh")),
                       scenes[0].sh_degree)


def tau_all_pixels(scene, cam):
    """Test-side closed form for every (pixel, Gaussian): kappa sqrt(2pi/a) exp(-(c-b^2/a)/2)."""
    o, d = pixel_rays(cam)
    out = np.zeros((scene.n,) + d.shape[:2])
    for g in range(scene.n):
        P = np.linalg.inv(cov_world(scene, g))
        p = o - scene.mu[g].astype(np.float64)
        a = np.einsum("hwi,ij,hwj->hw", d, P, d)
        b = d @ (P @ p)
        c = p @ P @ p
        out[g] = scene.kappa[g] * np.sqrt(2 * np.pi / a) * np.exp(-0.5 * (c - b * b / a))
    return out


# ------------------------------------------------------------------ Eq. 19 and Supp. B
@pytest.mark.parametrize("seed", range(8))
def test_tau_closed_form_equals_line_integral(seed):
    """Eq. 19 is the integral of kappa G(o + t d) over the whole line (Sec. 4.2, Supp. B)."""
    rng = np.random.default_rng(seed)
    scene = synth.uniform_scene(6, 700 + seed, log_scale=(-3.0, -1.0), flatten_frac=0.5)
    for g in range(scene.n):
        mu = scene.mu[g].astype(np.float64)
        Sig = cov_world(scene, g)
        o = mu + rng.normal(size=3) * 2.0 + np.array([0, 0, -3.0])
        target = mu + rng.normal(size=3) * float(scene.scale[g].max())
        d = (target - o) / np.linalg.norm(target - o)
        # -log G along the ray is exactly quadratic in t: fit it from three points.
        q = [mahal(o + t * d, mu, Sig) for t in (-1.0, 0.0, 1.0)]
        A = 0.5 * (q[0] + q[2]) - q[1]
        B = 0.5 * (q[2] - q[0])
        t_star = -B / (2 * A)
        beta_star = 1.0 / math.sqrt(A)
        kap = float(scene.kappa[g])
        f = lambda t: kap * math.exp(-0.5 * mahal(o + t * d, mu, Sig))
        val, err = integrate.quad(f, t_star - 40 * beta_star, t_star + 40 * beta_star, points=[t_star],
                                  epsabs=0.0, epsrel=1e-13, limit=400)
        res = oracle.tau(scene, g, o, d)
        assert res["tau"] == pytest.approx(val, rel=1e-10)
        # Supp. B: the maximiser gamma, the width beta and the peak value G(o + gamma d)
        assert res["gamma"] == pytest.approx(t_star, rel=1e-9, abs=1e-12)
        assert res["beta"] == pytest.approx(beta_star, rel=1e-9)
        assert res["gmax"] == pytest.approx(math.exp(-0.5 * mahal(o + t_star * d, mu, Sig)), rel=1e-9, abs=1e-300)


def test_isotropic_alpha_is_analytic():
    """Sigma = s^2 I: alpha = 1 - exp(-kappa sqrt(2 pi) s exp(-r^2 / 2 s^2)), r = ray-to-mean distance."""
    s, kap = 0.1, 7.0
    mu = np.array([0.05, -0.03, 0.2])
    q = synth.random_unit_quats(np.random.default_rng(3), 1)[0]
    for bg in [(0.0, 0.0, 0.0), (0.2, 0.7, 0.1)]:
        scene = one_gaussian(mu, (s, s, s), q, kap, sh0=(0.0, 0.0, 0.0))
        cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 32, 32, 20.0)
        opts = dict(oracle.EXACT, bg=bg)
        rgb, T, _ = oracle.render(scene, [cam], opts, brute=True)
        o, d = pixel_rays(cam)
        m32 = scene.mu[0].astype(np.float64)
        pm = m32 - o
        r2 = np.sum(pm * pm) - (d @ pm) ** 2
        s32 = float(scene.scale[0, 0])                      # the stored (float32) scale
        alpha = 1.0 - np.exp(-kap * math.sqrt(2 * math.pi) * s32 * np.exp(-r2 / (2 * s32 * s32)))
        assert np.max(np.abs((1.0 - T[0]) - alpha)) < 1e-12
        # a single Gaussian: C = c alpha + (1 - alpha) bg with c = 0.5 for zero SH coefficients
        for ch in range(3):
            assert np.max(np.abs(rgb[0][..., ch] - (0.5 * alpha + (1 - alpha) * bg[ch]))) < 1e-12


# ------------------------------------------------------------------ Eq. 14 vs Eq. 1
def _ray_march(scene, cam, t_lo, t_hi, n):
    """Supp. A: march Eq. 1 with sigma(x) = sum kappa_i G_i, c(x) = sum kappa_i c_i G_i / sigma."""
    o, d = pixel_rays(cam)
    d = d.reshape(-1, 3)
    dt = (t_hi - t_lo) / n
    ts = t_lo + (np.arange(n) + 0.5) * dt
    Y00 = oracle.sh_basis(0, np.array([0.0, 0.0, 1.0]))[0]
    col = np.clip(scene.sh[:, 0, :].astype(np.float64) * Y00 + 0.5, 0, None)
    out = np.zeros((d.shape[0], 3))
    for r in range(d.shape[0]):
        x = o[None, :] + ts[:, None] * d[r][None, :]
        sig = np.zeros(n)
        csum = np.zeros((n, 3))
        for g in range(scene.n):
            P = np.linalg.inv(cov_world(scene, g))
            dx = x - scene.mu[g].astype(np.float64)
            Gv = scene.kappa[g] * np.exp(-0.5 * np.einsum("ni,ij,nj->n", dx, P, dx))
            sig += Gv
            csum += Gv[:, None] * col[g][None, :]
        cx = csum / np.maximum(sig, 1e-300)[:, None]
        tau = sig * dt
        T = np.exp(-np.concatenate([[0.0], np.cumsum(tau)[:-1]]))
        out[r] = np.sum((T * (1.0 - np.exp(-tau)))[:, None] * cx, axis=0)
    return out.reshape(cam.height, cam.width, 3)


def test_blend_equals_volume_rendering_without_overlap():
    """Sorted, non-overlapping Gaussians: the Eq. 14 blend equals the ray-marched Eq. 1
    (Supp. A, rows 1-2); with heavy overlap it does not (row 3)."""
    q = synth.random_unit_quats(np.random.default_rng(5), 3)
    sep = concat(one_gaussian((0.01, 0.0, -1.0), (0.08, 0.06, 0.1), q[0], 3.0, (1.0, -0.5, 0.2)),
                 one_gaussian((-0.02, 0.01, 0.0), (0.07, 0.09, 0.05), q[1], 6.0, (-0.4, 0.9, 0.3)),
                 one_gaussian((0.0, -0.01, 1.0), (0.1, 0.08, 0.09), q[2], 1.5, (0.3, 0.3, -0.8)))
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 6, 6, 4.0)
    rgb, _, _ = oracle.render(sep, [cam], oracle.EXACT, brute=True)
    ref = _ray_march(sep, cam, 1.0, 7.0, 120000)
    assert np.max(np.abs(rgb[0] - ref)) < 2e-6
    ovl = concat(one_gaussian((0.0, 0.0, 0.0), (0.1, 0.1, 0.1), q[0], 4.0, (1.0, -0.5, 0.2)),
                 one_gaussian((0.0, 0.0, 0.02), (0.1, 0.1, 0.1), q[1], 4.0, (-0.4, 0.9, 0.3)))
    rgb2, _, _ = oracle.render(ovl, [cam], oracle.EXACT, brute=True)
    ref2 = _ray_march(ovl, cam, 2.0, 6.0, 60000)
    assert np.max(np.abs(rgb2[0] - ref2)) > 1e-2


def test_transmittance_is_monotone_and_bounded():
    scene, cams = synth.config1(0.25)
    rgb, T, _ = oracle.render(scene, cams, oracle.EXACT, brute=True)
    assert np.all(T[0] >= 0) and np.all(T[0] <= 1)
    # removing Gaussians can only raise the transmittance (each one multiplies T by e^-tau <= 1)
    sub = scene.subset(np.arange(0, scene.n, 2))
    _, Ts, _ = oracle.render(sub, cams, oracle.EXACT, brute=True)
    assert np.all(T[0] <= Ts[0] * (1 + 1e-12))
    assert np.all(rgb[0] >= 0)


# ------------------------------------------------------------------ footprint and sort
@pytest.mark.parametrize("mode", ["compat", "exact"])
def test_footprint_is_conservative(mode):
    """Every (pixel, Gaussian) pair with tau >= tau_cut lies in the pixel's tile list
    (brute force over all pairs of the 2,000-Gaussian 128x128 scene)."""
    opts = oracle.COMPAT if mode == "compat" else oracle.EXACT
    scene, cams = synth.config1()
    cam = cams[0]
    L = oracle.lists(scene, cams, opts)
    tau = tau_all_pixels(scene, cam)
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    tile = (ys // 16) * L["tiles_x"][0] + xs // 16
    member = np.zeros((scene.n, L["n_tiles"]), bool)
    for t in range(L["n_tiles"]):
        member[L["sorted_g"][L["tile_start"][t]:L["tile_start"][t + 1]], t] = True
    zc = (scene.mu.astype(np.float64) @ np.asarray(cam.R, np.float64).T + cam.t)[:, 2]
    need = (tau >= opts["tau_cut"]) & (zc > opts["z_near"])[:, None, None]
    g_idx, py, px = np.nonzero(need)
    assert g_idx.size > 1000
    missing = ~member[g_idx, tile[py, px]]
    assert missing.sum() == 0
    # ... and inside the Gaussian's pixel footprint rectangle
    pr = L["prect"][0]
    inside = (px >= pr[g_idx, 0]) & (px <= pr[g_idx, 2]) & (py >= pr[g_idx, 1]) & (py <= pr[g_idx, 3])
    assert inside.all()
    # the rectangle lies within the tile rectangle
    ok = L["rect"][0, :, 0] >= 0
    assert np.all(pr[ok, 0] // 16 == L["rect"][0, ok, 0]) and np.all(pr[ok, 3] // 16 == L["rect"][0, ok, 3])
    # and the blend over tile lists equals the blend over all Gaussians up to truncation
    rgb, T, _ = oracle.render(scene, cams, opts, L)
    rgbb, Tb, _ = oracle.render(scene, cams, opts, L, brute=True)
    bound = 0.0 if mode == "compat" else opts["tau_cut"] * scene.n
    assert np.max(np.abs(rgb[0] - rgbb[0])) <= bound + 1e-15


def test_sort_order_and_depth_keys():
    scene, cams = synth.config1(0.5)
    cams = cams + synth.small_views(2, 0, [(40, 24), (33, 17)])
    L = oracle.lists(scene, cams, oracle.COMPAT)
    inst = []
    for v in range(len(cams)):
        for g in range(scene.n):
            r = L["rect"][v, g]
            if r[0] < 0:
                continue
            for ty in range(r[1], r[3] + 1):
                for tx in range(r[0], r[2] + 1):
                    inst.append((int(L["tile_base"][v] + ty * L["tiles_x"][v] + tx), int(L["depth"][v, g]), g))
    inst.sort()
    assert np.array_equal(np.array([i[2] for i in inst], np.int32), L["sorted_g"])
    counts = np.bincount(np.array([i[0] for i in inst]), minlength=L["n_tiles"])
    assert np.array_equal(np.diff(L["tile_start"]), counts)
    # depth key = FP32 view-space z of the mean, within one ulp of the FP64 value
    for v, cam in enumerate(cams):
        z = (scene.mu.astype(np.float64) @ np.asarray(cam.R, np.float64).T + cam.t.astype(np.float64))[:, 2]
        ok = L["depth"][v] != 0xFFFFFFFF
        zf = L["depth"][v][ok].view(np.float32).astype(np.float64)
        assert np.all(np.abs(zf - z[ok]) <= 2 * np.spacing(np.float32(z[ok]).astype(np.float32)))
        assert np.all(z[~ok] <= 0.2 + 1e-6)


def test_invalid_and_behind_camera_are_culled():
    q = [1.0, 0.0, 0.0, 0.0]
    bad = [one_gaussian((0, 0, 0), (0.1, 0.1, 0.1), q, float("nan")),
           one_gaussian((0, 0, 0), (0.1, -0.1, 0.1), q, 1.0),
           one_gaussian((0, 0, 0), (0.1, 0.1, 0.1), [0, 0, 0, 0], 1.0),
           one_gaussian((0, 0, 0), (0.1, 0.1, 0.1), q, 0.0),
           one_gaussian((0, 0, -4.1), (0.1, 0.1, 0.1), q, 1.0),         # behind the camera
           one_gaussian((0, 0, float("inf")), (0.1, 0.1, 0.1), q, 1.0)]
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 16, 16, 60.0)
    for sc in bad:
        depth, rect = oracle.keys(sc, [cam], oracle.COMPAT)
        assert rect[0, 0, 0] == -1
    # an empty scene renders the background with T = 1
    empty = synth.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), np.zeros((0, 4), np.float32),
                        np.zeros(0, np.float32), np.zeros((0, 1, 3), np.float32), 0)
    rgb, T, _ = oracle.render(empty, [cam], dict(oracle.EXACT, bg=(0.1, 0.2, 0.3)))
    assert np.all(T[0] == 1.0) and np.allclose(rgb[0], [0.1, 0.2, 0.3])


# ------------------------------------------------------------------ Fig. 2 properties
def test_opacity_grows_with_density_and_depth_scale():
    """Sec. 4.3 / Fig. 2: alpha rises with kappa and with the scale along the ray; tau is
    linear in kappa."""
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 8, 8, 10.0)
    o, d = pixel_rays(cam)
    centre = d[4, 4]
    prev = -1.0
    for kap in [0.5, 1.0, 2.0, 4.0, 8.0]:
        sc = one_gaussian((0, 0, 0), (0.05, 0.05, 0.05), [1, 0, 0, 0], kap)
        t1 = oracle.tau(sc, 0, o, centre)["tau"]
        assert t1 > prev
        t2 = oracle.tau(one_gaussian((0, 0, 0), (0.05, 0.05, 0.05), [1, 0, 0, 0], 2 * kap), 0, o, centre)["tau"]
        assert t2 == pytest.approx(2 * t1, rel=1e-14)
        prev = t1
    prev = -1.0
    for sz in [0.01, 0.03, 0.1, 0.3]:                     # scale along the optical axis (world z)
        sc = one_gaussian((0, 0, 0), (0.05, 0.05, sz), [1, 0, 0, 0], 3.0)
        a = 1 - math.exp(-oracle.tau(sc, 0, o, centre)["tau"])
        assert a > prev
        prev = a


def test_sh_basis_is_orthonormal():
    """Real spherical harmonics to degree 3: Gram matrix over the sphere is the identity
    (Gauss-Legendre in cos(theta) times a uniform grid in phi, exact for these degrees)."""
    xg, wg = np.polynomial.legendre.leggauss(12)
    phis = np.arange(24) * 2 * np.pi / 24
    Gm = np.zeros((16, 16))
    for zc, w in zip(xg, wg):
        r = math.sqrt(1 - zc * zc)
        for ph in phis:
            Y = oracle.sh_basis(3, np.array([r * math.cos(ph), r * math.sin(ph), zc]))
            Gm += w * (2 * np.pi / 24) * np.outer(Y, Y)
    assert np.max(np.abs(Gm - np.eye(16))) < 1e-12
    # the degree-1 block is proportional to (-y, z, -x)
    Y = oracle.sh_basis(1, np.array([0.0, 0.0, 1.0]))
    assert Y[2] > 0 and abs(Y[1]) < 1e-15 and abs(Y[3]) < 1e-15
    Y = oracle.sh_basis(1, np.array([1.0, 0.0, 0.0]))
    assert Y[3] < 0


def _real_sh_scipy(l, m, d):
    """Real SH of degree l, order m at unit direction d, from scipy's complex spherical harmonics
    (which carry the Condon-Shortley phase): sqrt2 Re Y_l^m for m > 0, Y_l^0, sqrt2 Im Y_l^|m| for
    m < 0 -- the basis whose degree-1 block is proportional to (-y, z, -x)."""
    import scipy.special as sp
    theta = math.acos(max(-1.0, min(1.0, d[2])))
    phi = math.atan2(d[1], d[0])
    if hasattr(sp, "sph_harm_y"):
        Y = complex(sp.sph_harm_y(l, abs(m), theta, phi))
    else:   # older scipy: sph_harm(order, degree, azimuth, polar)
        Y = complex(sp.sph_harm(abs(m), l, phi, theta))
    if m > 0:
        return math.sqrt(2.0) * Y.real
    if m < 0:
        return math.sqrt(2.0) * Y.imag
    return Y.real


def test_sh_basis_matches_associated_legendre_definition():
    """Every function of degree 0-3 (graphics ordering k = l^2 + l + m) equals the real SH built
    from scipy's associated-Legendre spherical harmonics at fixed and random directions: a swapped
    pair, a wrong constant or sign of any degree-2 or degree-3 function fails here."""
    rng = np.random.default_rng(31)
    dirs = [np.array(v, np.float64) for v in ((0, 0, 1), (1, 0, 0), (0, 1, 0), (0.6, -0.48, 0.64), (-0.3, 0.4, -0.866))]
    dirs += [v / np.linalg.norm(v) for v in rng.normal(size=(12, 3))]
    for d in dirs:
        d = d / np.linalg.norm(d)
        Y = oracle.sh_basis(3, d)
        for l in range(4):
            for m in range(-l, l + 1):
                assert abs(Y[l * l + l + m] - _real_sh_scipy(l, m, d)) < 1e-12, (l, m, d)


# ------------------------------------------------------------------ thresholds (reading 8)
def _on_axis_scene(taus, colours, s=0.1):
    """Isotropic Gaussians of scale s centred on the optical axis of _axis_camera, front to back;
    along that ray each has tau = kappa sqrt(2 pi) s exactly (Eq. 19 with the ray through the mean)."""
    y00 = 0.5 / math.sqrt(math.pi)
    gs = [one_gaussian((0.0, 0.0, -1.0 + 0.5 * i), (s, s, s), (1.0, 0.0, 0.0, 0.0), t / (math.sqrt(2 * math.pi) * s),
                       sh0=tuple((np.asarray(c) - 0.5) / y00)) for i, (t, c) in enumerate(zip(taus, colours))]
    return concat(*gs)


def _stored_taus_colours(scene):
    """tau along the axis and the colour of each Gaussian from the stored (float32) parameters."""
    y00 = 0.5 / math.sqrt(math.pi)
    taus = [float(scene.kappa[i]) * math.sqrt(2 * math.pi) * float(scene.scale[i, 0]) for i in range(scene.n)]
    cols = [np.maximum(scene.sh[i, 0].astype(np.float64) * y00 + 0.5, 0.0) for i in range(scene.n)]
    return taus, cols


def _axis_camera():
    """One pixel whose centre ray is the optical axis (0, 0, 1) from the centre (0, 0, -4)."""
    return synth.Camera(np.eye(3, dtype=np.float32), np.array([0.0, 0.0, 4.0], np.float32), 100.0, 100.0, 0.5, 0.5,
                        1, 1)


def _blend_reading8(taus, colours, o, slip=None):
    """Eq. 14 with the thresholds as read (reading 8), written independently of the oracle: clamp tau
    at tau_max, skip when the clamped tau < -ln(1 - alpha_min), blend, then stop once T < T_stop.
    `slip` plants one plausible mistake."""
    tau_skip = -math.log1p(-o["alpha_min"]) if o["alpha_min"] > 0 else 0.0
    T, C, n = 1.0, np.zeros(3), 0
    for t, c in zip(taus, colours):
        if slip != "no_clamp" and slip != "skip_before_clamp":
            t = min(t, o["tau_max"])
        if slip != "no_skip" and t < tau_skip:
            continue
        if slip == "skip_before_clamp":
            t = min(t, o["tau_max"])
        if slip == "stop_before_blend" and T * math.exp(-t) < o["T_stop"]:
            break
        C = C + np.asarray(c) * (-math.expm1(-t)) * T
        T *= math.exp(-t)
        n += 1
        if slip != "no_stop" and T < o["T_stop"]:
            break
    return C + T * np.asarray(o["bg"]), T, n


def test_volumetric_thresholds_follow_reading_8():
    """The compat thresholds on one ray through six Gaussians where each rule changes the result:
    tau 0.002 (skipped: below -ln(1 - 1/255)), 6 (clamped to ln 100), 0.003 (skipped), 3, 2 (blended;
    T crosses 1e-4 here, so the pixel stops after it), 1.5 (never reached).  The oracle equals the
    independent blend to 1e-12, and every planted slip of the blend moves the result."""
    taus = [0.002, 6.0, 0.003, 3.0, 2.0, 1.5]
    cols = [(0.9, 0.1, 0.1), (0.1, 0.8, 0.2), (0.2, 0.2, 0.9), (0.7, 0.7, 0.1), (0.3, 0.9, 0.6), (0.95, 0.4, 0.05)]
    o = dict(oracle.COMPAT, tau_cut=1e-6, bg=(0.25, 0.5, 0.75))   # footprints keep even the skipped pairs
    scene, cam = _on_axis_scene(taus, cols), _axis_camera()
    taus, cols = _stored_taus_colours(scene)
    rgb, T, nb = oracle.render(scene, [cam], o)
    C, Tw, n = _blend_reading8(taus, cols, o)
    assert n == 3 and nb[0][0, 0] == 3
    assert np.max(np.abs(rgb[0][0, 0] - C)) < 1e-12 and abs(T[0][0, 0] - Tw) < 1e-15
    for slip in ("no_clamp", "no_skip", "stop_before_blend", "no_stop"):
        Cs, Ts, _ = _blend_reading8(taus, cols, o, slip)
        assert np.max(np.abs(Cs - C)) > 1e-6 or abs(Ts - Tw) > 1e-9, slip
    # clamp, then skip: with tau_max below the skip threshold every clamped pair is skipped
    o2 = dict(o, tau_max=0.003)
    rgb2, T2, nb2 = oracle.render(scene, [cam], o2)
    C2, T2w, n2 = _blend_reading8(taus, cols, o2)
    assert n2 == 0 and nb2[0][0, 0] == 0 and T2[0][0, 0] == 1.0
    assert np.max(np.abs(rgb2[0][0, 0] - C2)) < 1e-12
    Cs, _, ns = _blend_reading8(taus, cols, o2, "skip_before_clamp")
    assert ns > 0 and np.max(np.abs(Cs - C2)) > 1e-6


def test_early_stop_is_strict():
    """T_stop ends a pixel only once T < T_stop (strictly): with T_stop set to the oracle's own T
    after two blends the pixel goes on to blend the third (whose T is below it) and stops there; one
    ulp above it, it stops after those two."""
    taus = [1.0, 2.0, 0.5, 0.7]
    cols = [(0.9, 0.1, 0.1), (0.1, 0.8, 0.2), (0.2, 0.2, 0.9), (0.7, 0.7, 0.1)]
    scene, cam = _on_axis_scene(taus, cols), _axis_camera()
    o = dict(oracle.EXACT, tau_cut=1e-6)
    _, T2, _ = oracle.render(scene.subset([0, 1]), [cam], o)
    t2 = float(T2[0][0, 0])
    _, _, nb = oracle.render(scene, [cam], dict(o, T_stop=t2))
    assert nb[0][0, 0] == 3
    _, T, nb = oracle.render(scene, [cam], dict(o, T_stop=float(np.nextafter(t2, 1.0))))
    assert nb[0][0, 0] == 2 and T[0][0, 0] == t2


# ------------------------------------------------------------------ gradients
def _fd_check(f, x, g_an, idx, h_rel=1e-5, rtol=1e-6):
    scale = max(1e-300, float(np.max(np.abs(g_an))))
    for i in idx:
        x0 = x.flat[i]
        h = h_rel * max(1.0, abs(x0))
        x.flat[i] = x0 + h
        fp = f()
        x.flat[i] = x0 - h
        fm = f()
        x.flat[i] = x0
        fd = (fp - fm) / (2 * h)
        den = max(abs(fd), 1e-3 * scale)
        assert abs(fd - g_an.flat[i]) / den < rtol, (i, fd, g_an.flat[i])


@pytest.mark.parametrize("variant", ["exact", "clamped", "theta_softplus"])
def test_render_gradient_matches_finite_differences(variant):
    """Analytic FP64 gradient of the blend (tile lists held fixed) vs central differences."""
    rng = np.random.default_rng(11)
    scene = synth.uniform_scene(9, 321, log_scale=(-2.5, -1.5), kappa=(0.5, 6.0), sh_degree=3, sh_std=0.3,
                                flatten_frac=0.3, extent=0.4)
    scene = synth.Scene(*(np.asarray(getattr(scene, f), np.float64) for f in ("mu", "scale", "quat", "kappa", "sh")),
                        3)
    scene.quat = scene.quat * rng.uniform(0.7, 1.3, (scene.n, 1))   # unnormalised input quaternions
    cams = synth.small_views(2, 0, [(20, 18), (17, 23)])
    opts = dict(oracle.EXACT, bg=(0.3, 0.1, 0.6))
    if variant == "clamped":
        opts["tau_max"] = 1.2
    if variant == "theta_softplus":   # Eq. 20 density (kappa holds theta) and softplus colour
        opts.update(density_theta=True, softplus_beta=10.0)
        scene.kappa = rng.uniform(0.05, 0.95, scene.n)
    L = oracle.lists(scene, cams, opts)
    wr = [rng.normal(size=(c.height, c.width, 3)) for c in cams]
    wT = [rng.normal(size=(c.height, c.width)) for c in cams]

    def loss():
        rgb, T, _ = oracle.render(scene, cams, opts, L)
        return sum(float(np.sum(a * b)) for a, b in zip(rgb, wr)) + sum(float(np.sum(a * b)) for a, b in zip(T, wT))

    g = oracle.render_grad(scene, cams, opts, L, wr, wT)
    for name, arr in (("mu", scene.mu), ("scale", scene.scale), ("quat", scene.quat), ("kappa", scene.kappa),
                      ("sh", scene.sh)):
        idx = range(arr.size) if arr.size <= 40 else rng.choice(arr.size, 40, replace=False)
        assert np.max(np.abs(g[name])) > 0, name
        _fd_check(loss, arr, g[name], idx, rtol=2e-6)


# ------------------------------------------------------------------ tomography (Eq. 21)
def test_tomography_detector_integral_and_marginal():
    """Parallel beam: the detector integral of the line integrals of one Gaussian is
    kappa (2 pi)^(3/2) sqrt(det Sigma); each pixel equals the 2D marginal Gaussian."""
    q = synth.random_unit_quats(np.random.default_rng(9), 1)[0]
    s = np.array([0.06, 0.045, 0.07])
    kap = 3.0
    g = one_gaussian((0.03, -0.02, 0.05), s, q, kap)
    beam = synth.parallel_beam(3, det=96, extent=2.0, angles=np.array([0.0, 0.7, 2.9]))
    ls, proj = oracle.tomo(g, beam, brute=True)
    want = kap * (2 * np.pi) ** 1.5 * float(np.prod(g.scale[0].astype(np.float64)))
    Sig = cov_world(g, 0)
    mu = g.mu[0].astype(np.float64)
    for a, th in enumerate(beam.angles.astype(np.float64)):
        assert float(ls[a].sum()) * beam.pitch_u * beam.pitch_v == pytest.approx(want, rel=1e-9)
        assert np.allclose(proj[a], np.exp(-ls[a]), rtol=1e-15, atol=0)
        E = np.array([[-math.sin(th), 0.0], [math.cos(th), 0.0], [0.0, 1.0]])
        S2 = E.T @ Sig @ E
        u = beam.u0 + (np.arange(beam.det_w) + 0.5) * beam.pitch_u
        v = beam.v0 + (np.arange(beam.det_h) + 0.5) * beam.pitch_v
        D = np.stack(np.meshgrid(u, v), -1) - (E.T @ mu)
        amp = want / (2 * np.pi * math.sqrt(np.linalg.det(S2)))
        ref = amp * np.exp(-0.5 * np.einsum("hwi,ij,hwj->hw", D, np.linalg.inv(S2), D))
        assert np.max(np.abs(ls[a] - ref)) <= 1e-10 * ref.max()


def test_tomography_order_independent_and_tiled():
    scene, beam, _ = synth.config4(frac=0.002, n_angles=3, det=64)
    L = oracle.tomo_lists(scene, beam)
    ls, _ = oracle.tomo(scene, beam, L)
    perm = np.random.default_rng(1).permutation(scene.n)
    ls2, _ = oracle.tomo(scene.subset(perm), beam)
    assert np.max(np.abs(ls - ls2)) <= 1e-12 * max(1.0, ls.max())
    lsb, _ = oracle.tomo(scene, beam, brute=True)
    assert np.max(np.abs(ls - lsb)) <= 1e-6 * scene.n


@pytest.mark.parametrize("theta", [False, True])
def test_tomography_gradient_matches_finite_differences(theta):
    rng = np.random.default_rng(4)
    scene = synth.tomo_scene(7, 77, log_scale=(-2.5, -1.8))
    scene = synth.Scene(*(np.asarray(getattr(scene, f), np.float64) for f in ("mu", "scale", "quat", "kappa", "sh")), 0)
    if theta:   # Eq. 20: the density array holds theta
        scene.kappa = rng.uniform(0.05, 0.95, scene.n)
    beam = synth.parallel_beam(2, det=24, extent=2.4)
    L = oracle.tomo_lists(scene, beam, density_theta=theta)
    w = rng.normal(size=(2, 24, 24))

    def loss():
        _, pr = oracle.tomo(scene, beam, L, density_theta=theta)
        return float(np.sum(pr * w))

    g = oracle.tomo_grad(scene, beam, L, w, density_theta=theta)
    for name, arr in (("mu", scene.mu), ("scale", scene.scale), ("quat", scene.quat), ("kappa", scene.kappa)):
        assert np.max(np.abs(g[name])) > 0
        _fd_check(loss, arr, g[name], range(arr.size), rtol=2e-6)


# ------------------------------------------------------------------ Eq. 20 and the softplus colour
@pytest.mark.parametrize("theta", [0.0, 0.3, 0.9, 1.0])
def test_density_reparam_centre_opacity_is_scale_independent(theta):
    """Eq. 20 with an isotropic Gaussian: kappa = -ln(1 - 0.99 theta) / s, so the ray through
    the mean sees tau = kappa sqrt(2 pi) s = -sqrt(2 pi) ln(1 - 0.99 theta) whatever the scale:
    alpha = 1 - (1 - 0.99 theta)^sqrt(2 pi) (the reparameterisation's purpose, Sec. 5)."""
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 33, 33, 30.0)   # a pixel centre on the axis
    th = float(np.float32(theta))                                              # theta as stored
    want = 1.0 - (1.0 - 0.99 * th) ** math.sqrt(2.0 * math.pi)
    q = synth.random_unit_quats(np.random.default_rng(5), 1)[0]
    got = []
    for s in (0.03, 0.1, 0.3):
        scene = one_gaussian((0.0, 0.0, 0.0), (s, s, s), q, theta)
        opts = dict(oracle.EXACT, density_theta=True)
        _, T, _ = oracle.render(scene, [cam], opts, brute=True)
        got.append(1.0 - T[0][16, 16])
    assert np.max(np.abs(np.array(got) - want)) < 1e-12, (got, want)


def test_density_key_bound_is_conservative():
    """The FP32 bound that sizes footprints under Eq. 20 is never below the density and at most
    ~1.6x above it, over theta in [0, 1] and scales over three decades."""
    rng = np.random.default_rng(6)
    theta = np.concatenate([[0.0, 1e-7, 1e-3, 0.5, 0.55, 0.6, 0.99, 1.0], rng.uniform(0, 1, 20000)]).astype(np.float32)
    scale = np.exp(rng.uniform(-7, 0, (theta.size, 3))).astype(np.float32)
    bound = oracle.kappa_key_bound(theta, scale).astype(np.float64)
    exact = oracle.kappa_from_theta(theta.astype(np.float64), scale.astype(np.float64))
    pos = theta > 0
    assert np.all(bound[~pos] == 0)
    assert np.all(bound[pos] >= exact[pos] * (1 - 1e-6))
    assert np.max(bound[pos] / exact[pos]) < 1.6


def test_softplus_colour_tends_to_the_clamp():
    """softplus_beta(x) = ln(1 + e^(beta x)) / beta lies within ln 2 / beta of max(x, 0)."""
    scene = synth.uniform_scene(40, 61, log_scale=(-2.5, -1.5), sh_degree=2, sh_std=0.6)
    cams = [synth.look_at((0.2, 0.1, -4.0), (0.0, 0.0, 0.0), 24, 20, 40.0)]
    base = dict(oracle.EXACT, bg=(0.1, 0.2, 0.3))
    ref, _, _ = oracle.render(scene, cams, base)
    for beta in (1e3, 1e5):
        got, _, _ = oracle.render(scene, cams, dict(base, softplus_beta=beta))
        err = np.max(np.abs(got[0] - ref[0]))
        assert 0 < err <= math.log(2.0) / beta + 1e-12, (beta, err)


# ------------------------------------------------------------------ cone-beam tomography
def _far_cone_camera(beam, D):
    """A pinhole camera on the -x axis at distance D looking along +x, whose pixel rays cross
    the plane x = 0 at the parallel beam's (angle 0) detector pixel centres."""
    R = np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 1.0], [1.0, 0.0, 0.0]], np.float32)   # rows: u, v, forward
    t = np.array([0.0, 0.0, D], np.float32)                                          # t = -R o, o = (-D, 0, 0)
    f = D / beam.pitch_u
    cx = -beam.u0 / beam.pitch_u
    cy = -beam.v0 / beam.pitch_v
    return synth.Camera(R, t, float(f), float(D / beam.pitch_v), float(cx), float(cy), beam.det_w, beam.det_h)


def test_cone_beam_far_source_is_the_parallel_beam():
    """With the source 1e8 away the cone's rays are parallel to within 1e-8 rad: the cone-beam
    projection equals the (pinned) parallel-beam projection at angle 0."""
    scene = synth.tomo_scene(30, 91, log_scale=(-3.0, -2.0))
    beam = synth.parallel_beam(1, det=40, extent=2.2)
    cam = _far_cone_camera(beam, 1e8)
    ref_ls, _ = oracle.tomo(scene, beam, brute=True)
    (ls, pr), = oracle.cone(scene, [cam], brute=True)
    assert np.max(np.abs(ls - ref_ls[0])) < 1e-5 * max(1.0, float(np.max(ref_ls)))
    assert np.allclose(pr, np.exp(-ls), rtol=0, atol=1e-15)


def test_cone_beam_isotropic_sum_and_order():
    """One isotropic Gaussian: the line sum through each pixel is kappa sqrt(2 pi) s exp(-r^2/2s^2)
    (r the ray-to-mean distance, computed here from the camera model); permuting a scene's
    Gaussians leaves the projection unchanged; tiled evaluation equals brute force within the
    truncation bound."""
    s, kap = 0.08, 3.0
    scene = one_gaussian((0.1, -0.05, 0.2), (s, s, s), (0.9, 0.1, -0.3, 0.2), kap)
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 30, 26, 25.0)
    (ls, _), = oracle.cone(scene, [cam], brute=True)
    o, d = pixel_rays(cam)
    pm = scene.mu[0].astype(np.float64) - o
    r2 = np.sum(pm * pm) - (d @ pm) ** 2
    s32 = float(scene.scale[0, 0])
    want = kap * math.sqrt(2 * math.pi) * s32 * np.exp(-r2 / (2 * s32 * s32))
    assert np.max(np.abs(ls - want)) < 1e-12
    many = synth.tomo_scene(60, 92, log_scale=(-3.0, -2.0))
    perm = many.subset(np.random.default_rng(1).permutation(many.n))
    o_ = dict(oracle.EXACT)
    (a, _), = oracle.cone(many, [cam], o_)
    (b, _), = oracle.cone(perm, [cam], o_)
    (c, _), = oracle.cone(many, [cam], o_, brute=True)
    assert np.max(np.abs(a - b)) < 1e-12
    assert np.max(np.abs(a - c)) < many.n * o_["tau_cut"]


@pytest.mark.parametrize("theta", [False, True])
def test_cone_beam_gradient_matches_finite_differences(theta):
    rng = np.random.default_rng(8)
    scene = synth.tomo_scene(7, 93, log_scale=(-2.5, -1.8))
    scene = synth.Scene(*(np.asarray(getattr(scene, f), np.float64) for f in ("mu", "scale", "quat", "kappa", "sh")), 0)
    opts = dict(oracle.EXACT, density_theta=theta)
    if theta:
        scene.kappa = rng.uniform(0.05, 0.95, scene.n)
    cams = synth.small_views(2, 4, [(22, 18), (19, 21)])
    L = oracle.lists(scene, cams, opts)
    w = [rng.normal(size=(c.height, c.width)) for c in cams]

    def loss():
        return sum(float(np.sum(pr * ww)) for (_, pr), ww in zip(oracle.cone(scene, cams, opts, L), w))

    g = oracle.cone_grad(scene, cams, opts, L, w)
    for name, arr in (("mu", scene.mu), ("scale", scene.scale), ("quat", scene.quat), ("kappa", scene.kappa)):
        assert np.max(np.abs(g[name])) > 0
        _fd_check(loss, arr, g[name], range(arr.size), rtol=2e-6)


# ------------------------------------------------------------------ voxel density
def test_voxel_density_integral_and_values():
    """One rotated anisotropic Gaussian on a grid finer than its scales: the voxel sum of sigma
    times the voxel volume is kappa (2 pi)^(3/2) sqrt(det Sigma) (a smooth integrand, spectrally
    accurate midpoint rule), and each voxel's value is kappa exp(-d' Sigma^-1 d / 2) with Sigma
    formed here from a library rotation."""
    q = synth.random_unit_quats(np.random.default_rng(21), 1)[0]
    s = (0.09, 0.05, 0.13)
    kap = 2.5
    scene = one_gaussian((0.013, -0.021, 0.008), s, q, kap)
    dims = (64, 64, 64)
    vox = np.full(3, 2.0 / 64, np.float32)
    org = np.full(3, -1.0, np.float32)
    sig = oracle.voxel_density(scene, org, vox, dims, brute=True)
    S = cov_world(scene, 0)
    integral = sig.sum() * float(np.prod(vox.astype(np.float64)))
    assert abs(integral / (kap * (2 * np.pi) ** 1.5 * math.sqrt(np.linalg.det(S))) - 1.0) < 1e-9
    rng = np.random.default_rng(22)
    Sinv = np.linalg.inv(S)
    for _ in range(200):
        i, j, k = (int(v) for v in rng.integers(0, 64, 3))
        x = org.astype(np.float64) + (np.array([i, j, k]) + 0.5) * vox.astype(np.float64)
        d = x - scene.mu[0].astype(np.float64)
        assert abs(sig[k, j, i] - kap * math.exp(-0.5 * d @ Sinv @ d)) < 1e-12


def test_voxel_boxes_are_conservative():
    """Boxed sums equal brute force within the truncation bound: a Gaussian outside its box
    contributes less than sigma_cut at the voxel."""
    scene = synth.tomo_scene(300, 23, log_scale=(-3.5, -2.0))
    dims = (40, 36, 44)
    vox = np.array([0.05, 0.055, 0.045], np.float32)
    org = np.array([-1.0, -1.0, -1.0], np.float32)
    cut = 1e-4
    a = oracle.voxel_density(scene, org, vox, dims, sigma_cut=cut)
    b = oracle.voxel_density(scene, org, vox, dims, sigma_cut=cut, brute=True)
    assert np.all(b - a >= -1e-12)
    assert np.max(b - a) < scene.n * cut
    assert np.max(b - a) > 0            # truncation happens


# ------------------------------------------------------------------ 3DGS splat mode (Eq. 5-7)
def _project(cam, x):
    """Pinhole projection of a world point to pixel index coordinates (pixel x has its centre
    at x + 1/2 in the continuous image plane), written out from the camera model."""
    R = np.asarray(cam.R, np.float64)
    t = np.asarray(cam.t, np.float64)
    fx, fy, cx, cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    X, Y, Z = R @ np.asarray(x, np.float64) + t
    return np.array([fx * X / Z + cx - 0.5, fy * Y / Z + cy - 0.5]), Z


def _splat_alpha_all(scene, cam, dil):
    """o G'(p) of every (Gaussian, pixel) from the oracle's 2D Gaussians, evaluated here."""
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    out = np.zeros((scene.n, cam.height, cam.width))
    for g in range(scene.n):
        sp = oracle.splat2d(scene, g, cam, dil)
        if sp is None:
            continue
        m, S = sp
        Q = np.linalg.inv(S)
        wx, wy = xs - m[0], ys - m[1]
        q = Q[0, 0] * wx * wx + 2 * Q[0, 1] * wx * wy + Q[1, 1] * wy * wy
        out[g] = float(scene.kappa[g]) * np.exp(-0.5 * q)
    return out


@pytest.mark.parametrize("dil", [0.0, 0.3])
def test_splat_isotropic_on_axis_is_the_scaled_disc(dil):
    """A sphere of radius s on the optical axis at distance z projects to an isotropic 2D Gaussian
    of standard deviation f s / z (plus the dilation) centred at the principal point:
    alpha = o exp(-r^2 / (2 ((f s / z)^2 + dil))) at every pixel (brute force, black background)."""
    mu, s, o = (0.2, -0.1, 0.3), 0.07, 0.8
    eye = np.array([0.2, -0.1, 0.3]) + np.array([0.5, -0.3, -3.5])
    cam = synth.look_at(eye, mu, 41, 33, 50.0)
    scene = one_gaussian(mu, (s, s, s), (0.7, 0.2, -0.5, 0.1), o)
    opts = dict(oracle.EXACT, splat=True, splat_dilation=dil)
    L = oracle.lists(scene, [cam], opts)
    _, T, _ = oracle.render(scene, [cam], opts, L, brute=True)
    c, z = _project(cam, np.asarray(scene.mu[0], np.float64))
    f = float(np.float32(cam.fx))
    sig2 = (f * float(scene.scale[0, 0]) / z) ** 2 + dil
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    want = float(np.float32(o)) * np.exp(-((xs - c[0]) ** 2 + (ys - c[1]) ** 2) / (2 * sig2))
    # the FP32 camera rotation is orthonormal to ~6e-8, which moves alpha by ~1e-8
    assert np.max(np.abs((1.0 - T[0]) - want)) < 1e-7


def test_splat_covariance_is_the_projection_jacobian():
    """Off-axis anisotropic Gaussians: the oracle's mu' is the pinhole projection of mu and its
    Sigma' equals J_fd Sigma J_fd^T with J_fd the central-difference Jacobian of that projection
    (Eq. 7); a tiny Gaussian's projected samples have that covariance (the affine approximation)."""
    rng = np.random.default_rng(31)
    cam = synth.look_at((0.7, -1.2, -3.4), (0.1, 0.2, 0.0), 64, 48, 70.0)
    for g_seed in range(6):
        r = np.random.default_rng(100 + g_seed)
        mu = r.uniform(-0.6, 0.6, 3)
        sc = np.exp(r.uniform(-3.5, -1.5, 3))
        q = r.normal(size=4)
        scene = one_gaussian(mu, sc, q, 0.5)
        m, S = oracle.splat2d(scene, 0, cam, 0.0)
        x0 = np.asarray(scene.mu[0], np.float64)
        c, _ = _project(cam, x0)
        assert np.max(np.abs(m - c)) < 1e-9
        J = np.zeros((2, 3))
        for k in range(3):
            h = 1e-5
            e = np.zeros(3)
            e[k] = h
            J[:, k] = (_project(cam, x0 + e)[0] - _project(cam, x0 - e)[0]) / (2 * h)
        Sfd = J @ cov_world(scene, 0) @ J.T
        assert np.max(np.abs(S - Sfd)) < 1e-6 * np.max(np.abs(S)), (S, Sfd)
    # sampling: 400,000 points of a Gaussian 1000x smaller than its distance
    scene = one_gaussian((0.3, -0.2, 0.1), (0.004, 0.002, 0.001), (0.3, 0.8, -0.2, 0.4), 0.5)
    m, S = oracle.splat2d(scene, 0, cam, 0.0)
    x = rng.multivariate_normal(np.asarray(scene.mu[0], np.float64), cov_world(scene, 0), size=400_000)
    R = np.asarray(cam.R, np.float64)
    t = np.asarray(cam.t, np.float64)
    Xc = x @ R.T + t
    fx, fy = float(np.float32(cam.fx)), float(np.float32(cam.fy))
    px = np.stack([fx * Xc[:, 0] / Xc[:, 2], fy * Xc[:, 1] / Xc[:, 2]], 1)
    Ss = np.cov(px.T)
    assert np.max(np.abs(Ss - S)) < 0.02 * np.max(np.abs(S))


@pytest.mark.parametrize("mode", ["exact", "3dgs"])
def test_splat_footprint_is_conservative(mode):
    """Every (pixel, Gaussian) pair with o G' >= alpha_cut lies in the Gaussian's footprint
    rectangle and tile lists (brute force over the 2,000-Gaussian 128x128 scene), and the tiled
    blend equals the brute-force blend up to the truncation."""
    opts = dict(oracle.EXACT, splat=True) if mode == "exact" else dict(oracle.SPLAT_3DGS)
    scene, cams = synth.config1()
    scene.kappa = np.random.default_rng(5).uniform(0.02, 1.0, scene.n).astype(np.float32)
    cam = cams[0]
    L = oracle.lists(scene, cams, opts)
    al = _splat_alpha_all(scene, cam, opts["splat_dilation"])
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    tile = (ys // 16) * L["tiles_x"][0] + xs // 16
    member = np.zeros((scene.n, L["n_tiles"]), bool)
    for t in range(L["n_tiles"]):
        member[L["sorted_g"][L["tile_start"][t]:L["tile_start"][t + 1]], t] = True
    zc = (scene.mu.astype(np.float64) @ np.asarray(cam.R, np.float64).T + cam.t)[:, 2]
    need = (al >= opts["tau_cut"]) & (zc > opts["z_near"])[:, None, None]
    g_idx, py, px = np.nonzero(need)
    assert g_idx.size > 1000
    assert member[g_idx, tile[py, px]].all()
    pr = L["prect"][0]
    assert ((px >= pr[g_idx, 0]) & (px <= pr[g_idx, 2]) & (py >= pr[g_idx, 1]) & (py <= pr[g_idx, 3])).all()
    rgb, T, _ = oracle.render(scene, cams, opts, L)
    rgbb, Tb, _ = oracle.render(scene, cams, opts, L, brute=True)
    bound = 0.0 if mode == "3dgs" else 2 * opts["tau_cut"] * scene.n
    assert np.max(np.abs(rgb[0] - rgbb[0])) <= bound + 1e-15


def test_splat_3dgs_thresholds():
    """3DGS conventions in splat mode: alpha = min(o G', 0.99), pairs with alpha < 1/255 skipped:
    one opaque Gaussian (o = 1) leaves T = 1 - min(G', 0.99) where G' >= 1/255, else T = 1."""
    mu = (0.0, 0.0, 0.0)
    cam = synth.look_at((0.0, 0.0, -4.0), mu, 33, 31, 40.0)
    scene = one_gaussian(mu, (0.12, 0.08, 0.1), (0.9, 0.1, 0.3, -0.2), 1.0)
    opts = dict(oracle.SPLAT_3DGS)
    L = oracle.lists(scene, [cam], opts)
    _, T, _ = oracle.render(scene, [cam], opts, L)
    al = _splat_alpha_all(scene, cam, 0.3)[0]
    want = np.where(al >= 1.0 / 255.0, 1.0 - np.minimum(al, 0.99), 1.0)
    assert np.max(np.abs(T[0] - want)) < 1e-12
    assert np.isclose(T[0].min(), 0.01) and (T[0] == 1.0).any()


@pytest.mark.parametrize("variant", ["exact", "dilated_clamped"])
def test_splat_gradient_matches_finite_differences(variant):
    """Analytic FP64 gradient of the splat-mode blend (lists held fixed) vs central differences."""
    rng = np.random.default_rng(12)
    scene = synth.uniform_scene(9, 322, log_scale=(-2.5, -1.5), kappa=(0.5, 6.0), sh_degree=2, sh_std=0.3,
                                flatten_frac=0.3, extent=0.4)
    scene = synth.Scene(*(np.asarray(getattr(scene, f), np.float64) for f in ("mu", "scale", "quat", "kappa", "sh")),
                        2)
    scene.quat = scene.quat * rng.uniform(0.7, 1.3, (scene.n, 1))
    scene.kappa = rng.uniform(0.1, 0.95, scene.n)
    cams = synth.small_views(2, 1, [(20, 18), (17, 23)])
    opts = dict(oracle.EXACT, splat=True, bg=(0.3, 0.1, 0.6))
    if variant == "dilated_clamped":
        opts.update(splat_dilation=0.3, tau_max=1.0, softplus_beta=10.0)
        scene.kappa[:3] = 0.99
    L = oracle.lists(scene, cams, opts)
    wr = [rng.normal(size=(c.height, c.width, 3)) for c in cams]
    wT = [rng.normal(size=(c.height, c.width)) for c in cams]

    def loss():
        rgb, T, _ = oracle.render(scene, cams, opts, L)
        return sum(float(np.sum(a * b)) for a, b in zip(rgb, wr)) + sum(float(np.sum(a * b)) for a, b in zip(T, wT))

    g = oracle.render_grad(scene, cams, opts, L, wr, wT)
    for name, arr in (("mu", scene.mu), ("scale", scene.scale), ("quat", scene.quat), ("kappa", scene.kappa),
                      ("sh", scene.sh)):
        idx = range(arr.size) if arr.size <= 40 else rng.choice(arr.size, 40, replace=False)
        assert np.max(np.abs(g[name])) > 0, name
        _fd_check(loss, arr, g[name], idx, rtol=2e-6)


# ------------------------------------------------------------------ ray-marching reference (Supp. A)
def test_ray_march_single_gaussian_is_the_closed_form():
    """One Gaussian: the marched transmittance is exp(-tau) with tau the closed form of Eq. 19 up to
    the midpoint rule's O(delta^2) error, and the colour is c (1 - T) (constant c(x))."""
    scene = one_gaussian((0.05, -0.03, 0.1), (0.12, 0.07, 0.1), (0.8, 0.3, -0.2, 0.4), 5.0, (0.6, -0.3, 0.9))
    cam = synth.look_at((0.3, 0.2, -4.0), (0.0, 0.0, 0.0), 9, 7, 8.0)
    rgb, T = oracle.ray_march(scene, [cam], oracle.EXACT, 2.0, 6.0, 20000)
    o, d = pixel_rays(cam)
    want = np.zeros((cam.height, cam.width))
    for yy in range(cam.height):
        for xx in range(cam.width):
            want[yy, xx] = oracle.tau(scene, 0, o, d[yy, xx])["tau"]
    assert want.max() > 0.5
    assert np.max(np.abs(T[0] - np.exp(-want))) < 1e-7
    c = np.clip(scene.sh[0, 0].astype(np.float64) * oracle.sh_basis(0, np.array([0.0, 0.0, 1.0]))[0] + 0.5, 0, None)
    assert np.max(np.abs(rgb[0] - c[None, None, :] * (1.0 - T[0])[..., None])) < 1e-12
    # starting the march at the maximiser gamma of the 1D Gaussian along a ray integrates its
    # second half: T = exp(-tau / 2) (this fixes the sample positions at the interval midpoints)
    yy, xx = cam.height // 2, cam.width // 2
    info = oracle.tau(scene, 0, o, d[yy, xx])
    _, Th = oracle.ray_march(scene, [cam], oracle.EXACT, info["gamma"], info["gamma"] + 3.0, 2000)
    assert abs(Th[0][yy, xx] - math.exp(-0.5 * info["tau"])) < 1e-7


def test_ray_march_matches_an_independent_march_and_the_blend_without_overlap():
    """The oracle's march equals the test-side march (same quadrature, written independently) on a
    random scene; without overlap it equals the Eq. 14 blend; with heavy overlap it does not."""
    sc = synth.uniform_scene(12, 77, log_scale=(-2.5, -1.8), kappa=(0.5, 8.0), extent=0.5)
    cam = synth.look_at((0.2, -0.1, -3.0), (0.0, 0.0, 0.0), 8, 6, 30.0)
    rgb, _ = oracle.ray_march(sc, [cam], oracle.EXACT, 1.5, 4.5, 3000)
    ref = _ray_march(sc, cam, 1.5, 4.5, 3000)
    assert np.max(np.abs(rgb[0] - ref)) < 1e-10
    q = synth.random_unit_quats(np.random.default_rng(6), 3)
    sep = concat(one_gaussian((0.01, 0.0, -1.0), (0.08, 0.06, 0.1), q[0], 3.0, (1.0, -0.5, 0.2)),
                 one_gaussian((-0.02, 0.01, 0.0), (0.07, 0.09, 0.05), q[1], 6.0, (-0.4, 0.9, 0.3)),
                 one_gaussian((0.0, -0.01, 1.0), (0.1, 0.08, 0.09), q[2], 1.5, (0.3, 0.3, -0.8)))
    cam2 = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 6, 6, 4.0)
    blend, _, _ = oracle.render(sep, [cam2], oracle.EXACT, brute=True)
    march, _ = oracle.ray_march(sep, [cam2], oracle.EXACT, 1.0, 7.0, 120000)
    assert np.max(np.abs(blend[0] - march[0])) < 2e-6
    ovl = concat(one_gaussian((0.0, 0.0, 0.0), (0.1, 0.1, 0.1), q[0], 4.0, (1.0, -0.5, 0.2)),
                 one_gaussian((0.0, 0.0, 0.02), (0.1, 0.1, 0.1), q[1], 4.0, (-0.4, 0.9, 0.3)))
    blend2, _, _ = oracle.render(ovl, [cam2], oracle.EXACT, brute=True)
    march2, _ = oracle.ray_march(ovl, [cam2], oracle.EXACT, 2.0, 6.0, 60000)
    assert np.max(np.abs(blend2[0] - march2[0])) > 1e-2


# ------------------------------------------------------------------ values printed by the paper
def _paper_values():
    import os
    out = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")):
        if line.strip() and not line.startswith("#"):
            name, value = line.split()[:2]
            out[name] = float(value)
    return out


def test_eq20_constant_from_the_paper():
    """Eq. 20 with the printed constant: theta = 1 gives kappa = -ln(1 - 0.99) times the mean
    inverse scale; the oracle's kappa_from_theta follows it at every theta."""
    c = _paper_values()["eq20_theta_scale"]
    s = np.array([[0.1, 0.2, 0.4], [0.05, 0.05, 0.05]])
    th = np.array([1.0, 0.37])
    want = -np.log(1.0 - c * th) * (1.0 / s).sum(1) / 3.0
    assert np.allclose(oracle.kappa_from_theta(th, s), want, rtol=1e-15, atol=0)
    assert abs(oracle.kappa_from_theta(np.array([1.0]), np.array([[1.0, 1.0, 1.0]]))[0] - math.log(100.0)) < 1e-12
