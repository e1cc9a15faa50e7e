"""Pins of the FP64 oracle against what the mathematics fixes independently of
the oracle's own code: closed forms, invariants, brute force and central finite
differences.  CPU only."""
import math

import numpy as np
import pytest

from paper_2401_05345_gb300 import scenes as S


def _scene(mean, scale, quat, opacity, feat, sh_degree=-1):
    f32 = lambda a: np.asarray(a, np.float32)
    return S.Scene(f32(mean), f32(scale), f32(quat), f32(opacity), sh_degree, f32(feat))


def _cam(W=33, H=33, dist=4.0, fov=60.0):
    return S.front_camera(W, H, dist, fov)


# ----------------------------------------------------------------------------
# spherical harmonics
# ----------------------------------------------------------------------------

def test_sh_basis_orthonormal(orc):
    """Real SH basis of degree <= 3 is orthonormal on the unit sphere
    (Gauss-Legendre in cos(theta) x uniform phi, exact for degree <= 6)."""
    xg, wg = np.polynomial.legendre.leggauss(8)
    nphi = 16
    gram = np.zeros((16, 16))
    for ct, w in zip(xg, wg):
        st = math.sqrt(1 - ct * ct)
        for k in range(nphi):
            ph = 2 * math.pi * k / nphi
            d = np.array([st * math.cos(ph), st * math.sin(ph), ct])
            y = orc.sh_basis(3, d)
            gram += w * (2 * math.pi / nphi) * np.outer(y, y)
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)


def test_sh_basis_low_orders_closed_form(orc):
    d = np.array([0.36, -0.48, 0.8])
    y = orc.sh_basis(1, d)
    c0 = 0.5 / math.sqrt(math.pi)
    c1 = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(y, [c0, -c1 * d[1], c1 * d[2], -c1 * d[0]], rtol=1e-14)


def test_sh_basis_signs_from_the_complex_harmonics(orc):
    """Every basis function of degree <= 3, sign included, against the
    complex spherical harmonics of scipy.special (Condon-Shortley phase).
    The standard real form is sqrt(2) (-1)^m Im Y_l^|m| for m < 0, Y_l^0,
    and sqrt(2) (-1)^m Re Y_l^m for m > 0; the rasterizer's basis (the 3DGS
    convention) is that times (-1)^m, at index l^2 + l + m."""
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy.special.sph_harm_y not available")
    rng = np.random.default_rng(11)
    for _ in range(20):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])  # polar, azimuth
        ref = np.zeros(16)
        for l in range(4):
            for m in range(-l, l + 1):
                y = complex(sp.sph_harm_y(l, abs(m), theta, phi))
                real = y.real if m == 0 else math.sqrt(2) * (-1) ** m * (y.imag if m < 0 else y.real)
                ref[l * l + l + m] = (-1) ** m * real
        np.testing.assert_allclose(orc.sh_basis(3, d), ref, rtol=1e-12, atol=1e-14)


def test_sh_basis_gradient_fd(orc):
    rng = np.random.default_rng(3)
    for _ in range(5):
        d = rng.normal(size=3)
        g = orc.sh_basis_grad(3, d)
        h = 1e-6
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            fd = (orc.sh_basis(3, d + e) - orc.sh_basis(3, d - e)) / (2 * h)
            np.testing.assert_allclose(g[:, a], fd, rtol=1e-7, atol=1e-8)


# ----------------------------------------------------------------------------
# projection / covariance closed forms
# ----------------------------------------------------------------------------

def test_point_projection_closed_form(orc):
    cam = _cam(65, 49)
    means = np.array([[0.0, 0.0, 0.0], [0.3, -0.2, 0.5], [-0.7, 0.4, -1.0]])
    sc = _scene(means, np.full((3, 3), 0.01), np.tile([1, 0, 0, 0], (3, 1)), [0.5] * 3,
                np.full((3, 3), 0.5))
    pp = orc.preprocess(sc, cam)
    m = sc.mean.astype(np.float64)
    z = m[:, 2] + 4.0
    u = cam.fx * m[:, 0] / z + cam.cx
    v = cam.fy * m[:, 1] / z + cam.cy
    np.testing.assert_allclose(pp["uv"][:, 0], u, rtol=1e-13)
    np.testing.assert_allclose(pp["uv"][:, 1], v, rtol=1e-13)
    np.testing.assert_allclose(pp["depth"], z, rtol=1e-13)


@pytest.mark.parametrize("s", [0.01, 0.05, 0.2])
def test_isotropic_conic_on_axis(orc, s):
    """Isotropic Gaussian on the optical axis: Sigma2 = (s f / z)^2 I + 0.3 I."""
    cam = _cam(33, 33)
    sc = _scene([[0, 0, 0]], [[s, s, s]], [[0.3, 0.1, -0.5, 0.7]], [0.5], [[0.2, 0.4, 0.6]])
    pp = orc.preprocess(sc, cam)
    z = 4.0
    var = (np.float64(np.float32(s)) * cam.fx / z) ** 2 + float(np.float32(0.3))
    np.testing.assert_allclose(pp["conic"][0], [1 / var, 0.0, 1 / var], rtol=1e-12, atol=1e-14)
    assert pp["radius"][0] == math.ceil(3 * math.sqrt(var + math.sqrt(float(np.float32(0.1)))))


def test_rotated_anisotropic_conic_on_axis(orc):
    """Rotation by theta about the optical axis, q = (cos t/2, 0, 0, sin t/2):
    Sigma2 = k^2 [[a c^2 + b s^2, (a-b) c s], [(a-b) c s, a s^2 + b c^2]] + 0.3 I."""
    cam = _cam(33, 33)
    th = 0.7
    sx, sy, sz = 0.08, 0.02, 0.05
    q = [math.cos(th / 2), 0, 0, math.sin(th / 2)]
    sc = _scene([[0, 0, 0]], [[sx, sy, sz]], [q], [0.5], [[0.2, 0.4, 0.6]])
    pp = orc.preprocess(sc, cam)
    sx, sy = float(np.float32(sx)), float(np.float32(sy))
    qq = np.asarray(np.float32(q), np.float64)
    qq /= np.linalg.norm(qq)
    th = 2 * math.atan2(qq[3], qq[0])
    c, s_ = math.cos(th), math.sin(th)
    k = cam.fx / 4.0
    dil = float(np.float32(0.3))
    S2 = k * k * np.array([[sx**2 * c * c + sy**2 * s_ * s_, (sx**2 - sy**2) * c * s_],
                           [(sx**2 - sy**2) * c * s_, sx**2 * s_ * s_ + sy**2 * c * c]]) + dil * np.eye(2)
    inv = np.linalg.inv(S2)
    np.testing.assert_allclose(pp["conic"][0], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-10)


def _rotated_sigma2(cam, sx, sy, th):
    """Closed-form screen covariance of a Gaussian on the optical axis rotated
    by th about it (scales sx, sy across the axis): k^2 R diag(sx^2, sy^2) R^T
    + 0.3 I with k = f / z."""
    k = cam.fx / 4.0
    c, s_ = math.cos(th), math.sin(th)
    sx, sy = float(np.float32(sx)), float(np.float32(sy))
    S2 = k * k * np.array([[sx**2 * c * c + sy**2 * s_ * s_, (sx**2 - sy**2) * c * s_],
                           [(sx**2 - sy**2) * c * s_, sx**2 * s_ * s_ + sy**2 * c * c]])
    return S2 + float(np.float32(0.3)) * np.eye(2)


def test_radius_is_three_sigma_of_the_larger_eigenvalue(orc):
    """Strongly anisotropic splat (eigenvalue gap far above the 0.1 floor):
    radius = ceil(3 sqrt(lambda_max)) with lambda_max from a library
    eigensolver of the closed-form screen covariance; the smaller eigenvalue
    would give 4 instead of 14."""
    cam = _cam(257, 257)
    th, sx, sy = 0.7, 0.08, 0.02
    q = [math.cos(th / 2), 0, 0, math.sin(th / 2)]
    pp = orc.preprocess(_scene([[0, 0, 0]], [[sx, sy, 0.05]], [q], [0.5], [[0.2, 0.4, 0.6]]), cam)
    ev = np.linalg.eigvalsh(_rotated_sigma2(cam, sx, sy, th))
    assert ((ev[1] - ev[0]) / 2) ** 2 > 10.0
    assert pp["pp_ambig"][0] == 0
    assert pp["radius"][0] == math.ceil(3 * math.sqrt(ev[1])) == 14
    assert math.ceil(3 * math.sqrt(ev[0])) != 14


def test_radius_floor_of_the_eigenvalue_gap(orc):
    """Nearly isotropic splat whose squared half eigenvalue gap (0.022) lies
    below the 0.1 floor: the extent uses mean eigenvalue + sqrt(0.1), which
    here rounds up to 4 where the larger eigenvalue itself gives 3."""
    cam = _cam(97, 97)
    th, sx, sy = 0.4, 0.0375, 0.027
    q = [math.cos(th / 2), 0, 0, math.sin(th / 2)]
    pp = orc.preprocess(_scene([[0, 0, 0]], [[sx, sy, 0.05]], [q], [0.5], [[0.2, 0.4, 0.6]]), cam)
    ev = np.linalg.eigvalsh(_rotated_sigma2(cam, sx, sy, th))
    gap2 = ((ev[1] - ev[0]) / 2) ** 2
    assert 0.0 < gap2 < 0.1
    assert pp["pp_ambig"][0] == 0
    floor = float(np.float32(0.1))
    assert pp["radius"][0] == math.ceil(3 * math.sqrt(ev.mean() + math.sqrt(floor))) == 4
    assert math.ceil(3 * math.sqrt(ev[1])) == 3


def test_identity_quaternion_covariance_is_diag_scale(orc):
    """Identity rotation: Sigma3 = diag(s^2); on the axis Sigma2 = diag((f/z)^2 sx^2, (f/z)^2 sy^2) + 0.3."""
    cam = _cam(33, 33)
    sx, sy, sz = 0.03, 0.07, 0.11
    sc = _scene([[0, 0, 0]], [[sx, sy, sz]], [[2.0, 0, 0, 0]], [0.5], [[0.2, 0.4, 0.6]])
    pp = orc.preprocess(sc, cam)
    k = cam.fx / 4.0
    dil = float(np.float32(0.3))
    a = k * k * float(np.float32(sx)) ** 2 + dil
    b = k * k * float(np.float32(sy)) ** 2 + dil
    np.testing.assert_allclose(pp["conic"][0], [1 / a, 0, 1 / b], rtol=1e-12, atol=1e-15)


def test_ewa_jacobian_matches_numeric_projection_derivative(orc):
    """Off-axis Gaussian: Sigma2 = J W Sigma3 W^T J^T + 0.3 I with J the
    derivative of the pixel position w.r.t. the camera-space mean.  J is taken
    here by central differences of the oracle's own (u, v) output."""
    cam = S.look_at_camera((1.0, -0.5, -3.5), (0.2, 0.1, 0.3), 64, 48)
    rng = np.random.default_rng(11)
    m0 = np.array([0.3, -0.2, 0.4])
    sc = _scene([m0], [[0.05, 0.02, 0.08]], [rng.normal(size=4)], [0.5], [[0.2, 0.4, 0.6]])
    pp = orc.preprocess(sc, cam)
    # numeric d(u,v)/d(mean) (world) from shifted means
    h = 1e-6
    Jw = np.zeros((2, 3))
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        up = orc.preprocess(_scene([m0 + e], sc.scale, sc.quat, sc.opacity, sc.feat), cam)["uv"][0]
        dn = orc.preprocess(_scene([m0 - e], sc.scale, sc.quat, sc.opacity, sc.feat), cam)["uv"][0]
        # float32 rounding of the shifted means: use the stored values for the step
        mp = np.float64(np.float32(m0 + e))[a]
        mm = np.float64(np.float32(m0 - e))[a]
        Jw[:, a] = (up - dn) / (mp - mm)
    q = sc.quat[0].astype(np.float64)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    # R must be a proper rotation
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
    Sg = R @ np.diag(sc.scale[0].astype(np.float64) ** 2) @ R.T
    S2 = Jw @ Sg @ Jw.T + float(np.float32(0.3)) * np.eye(2)
    inv = np.linalg.inv(S2)
    np.testing.assert_allclose(pp["conic"][0], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=2e-6)


def test_near_plane_cull(orc):
    cam = _cam(33, 33)
    sc = _scene([[0, 0, -3.85], [0, 0, -3.75]], np.full((2, 3), 0.05), [[1, 0, 0, 0]] * 2,
                [0.5, 0.5], np.full((2, 3), 0.5))
    pp = orc.preprocess(sc, cam)
    assert pp["radius"][0] == 0 and pp["radius"][1] > 0


# ----------------------------------------------------------------------------
# compositing closed forms and invariants
# ----------------------------------------------------------------------------

def _render_2d(orc, W, H, uv, conic, opac, rgb, bg, g=None, tile=(16, 16), radius=None, depth=None):
    uv = np.asarray(uv, np.float64)
    n = len(uv)
    if radius is None:
        radius = np.full(n, 40, np.int32)
    if depth is None:
        depth = np.arange(1, n + 1, dtype=np.float64)
    keys, pl, ranges = orc.bin_sort(uv, depth, radius, W, H, tile)
    return orc.render(W, H, ranges, pl, uv, conic, opac, rgb, bg, g, tile)


def test_single_isotropic_splat_pixel_values(orc):
    """One isotropic splat on a pixel centre: out = o c + (1 - o) bg there, and
    alpha = o exp(-|d|^2 / (2 var)) at offset d."""
    W = H = 32
    var = 6.0
    o, c, bg = 0.7, np.array([0.2, 0.5, 0.9]), np.array([0.1, 0.3, 0.05])
    out = _render_2d(orc, W, H, [[12.0, 17.0]], [[1 / var, 0, 1 / var]], [o], [c], bg)
    img = out["image"]
    np.testing.assert_allclose(img[:, 17, 12], o * c + (1 - o) * bg, rtol=1e-14)
    for (dx, dy) in [(1, 0), (2, 3), (-4, 1), (0, -5)]:
        a = o * math.exp(-(dx * dx + dy * dy) / (2 * var))
        exp_val = (a * c + (1 - a) * bg) if a >= 1 / 255 else bg
        np.testing.assert_allclose(img[:, 17 + dy, 12 + dx], exp_val, rtol=1e-13)


def test_alpha_cap(orc):
    out = _render_2d(orc, 16, 16, [[5.0, 5.0]], [[0.5, 0, 0.5]], [0.9999], [[1.0, 1.0, 1.0]], [0, 0, 0])
    assert abs(out["image"][0, 5, 5] - float(np.float32(0.99))) < 1e-15


def test_transmittance_telescopes(orc):
    """Sum_j alpha_j T_j + T_final = 1: white splats over a white background
    render exactly 1, and over black render 1 - T_final."""
    rng = np.random.default_rng(5)
    n, W, H = 60, 40, 36
    uv = rng.uniform(0, [W, H], size=(n, 2))
    L = rng.normal(size=(n, 2, 2)) * 0.6
    cov = L @ L.transpose(0, 2, 1) + 2.0 * np.eye(2)
    inv = np.linalg.inv(cov)
    conic = np.stack([inv[:, 0, 0], inv[:, 0, 1], inv[:, 1, 1]], 1)
    opac = rng.uniform(0.3, 0.99, size=n)
    ones = np.ones((n, 3))
    out1 = _render_2d(orc, W, H, uv, conic, opac, ones, [1, 1, 1], radius=np.full(n, 12, np.int32))
    np.testing.assert_allclose(out1["image"], 1.0, atol=1e-13)
    out0 = _render_2d(orc, W, H, uv, conic, opac, ones, [0, 0, 0], radius=np.full(n, 12, np.int32))
    np.testing.assert_allclose(out0["image"][0], 1.0 - out0["final_T"], atol=1e-13)
    assert (out0["final_T"] < 1).any() and (out0["final_T"] > 1e-4 * 0.5).all()


def test_single_splat_gradient_closed_form(orc):
    """out = c a + (1 - a) bg: dL/dc = a g, dL/do = G (c - bg).g, and the
    position gradient points along the conic-weighted offset."""
    W = H = 16
    var, o = 5.0, 0.6
    c, bg = np.array([0.3, 0.8, 0.4]), np.array([0.2, 0.1, 0.7])
    g = np.zeros((3, H, W), np.float32)
    g[:, 7, 9] = [1.0, -1.0, 1.0]
    u, v = 8.25, 6.5
    out = _render_2d(orc, W, H, [[u, v]], [[1 / var, 0, 1 / var]], [o], [c], bg, g)
    dx, dy = u - 9, v - 7
    G = math.exp(-(dx * dx + dy * dy) / (2 * var))
    a = o * G
    gv = g[:, 7, 9].astype(np.float64)
    gr = out["grad2d"][0]
    np.testing.assert_allclose(gr[6:9], a * gv, rtol=1e-13)
    dalpha = float(np.dot(c - bg, gv))
    np.testing.assert_allclose(gr[5], G * dalpha, rtol=1e-12)
    dsig = -o * G * dalpha
    np.testing.assert_allclose(gr[0:2], [dx / var * dsig, dy / var * dsig], rtol=1e-12)
    np.testing.assert_allclose(gr[2:5], [0.5 * dx * dx * dsig, dx * dy * dsig, 0.5 * dy * dy * dsig],
                               rtol=1e-12)


def test_two_stacked_splats_closed_form(orc):
    """out = c1 a1 + c2 a2 (1-a1) + bg (1-a1)(1-a2):
    dL/da1 = (c1 - c2 a2 - bg (1 - a2)).g, dL/da2 = (1-a1)(c2 - bg).g."""
    W = H = 16
    c1, c2, bg = np.array([0.9, 0.1, 0.3]), np.array([0.2, 0.6, 0.5]), np.array([0.05, 0.2, 0.9])
    o1, o2 = 0.55, 0.8
    g = np.zeros((3, H, W), np.float32)
    g[:, 4, 4] = [1.0, 1.0, -1.0]
    out = _render_2d(orc, W, H, [[4.0, 4.0], [4.0, 4.0]], [[0.2, 0, 0.2]] * 2, [o1, o2], [c1, c2], bg,
                     g, depth=np.array([1.0, 2.0]))
    gv = g[:, 4, 4].astype(np.float64)
    np.testing.assert_allclose(out["image"][:, 4, 4],
                               c1 * o1 + c2 * o2 * (1 - o1) + bg * (1 - o1) * (1 - o2), rtol=1e-14)
    gr = out["grad2d"]
    np.testing.assert_allclose(gr[0, 5], np.dot(c1 - c2 * o2 - bg * (1 - o2), gv), rtol=1e-12)
    np.testing.assert_allclose(gr[1, 5], (1 - o1) * np.dot(c2 - bg, gv), rtol=1e-12)
    np.testing.assert_allclose(gr[1, 6:9], o2 * (1 - o1) * gv, rtol=1e-13)


def test_occluded_splat_has_zero_gradient(orc):
    """Splats behind an opaque pair (T (1 - alpha) < 1e-4) get exactly zero."""
    W = H = 16
    n = 5
    uv = np.full((n, 2), 8.0)
    conic = np.tile([0.02, 0.0, 0.02], (n, 1))
    opac = np.array([1.0, 1.0, 0.5, 0.7, 0.9])
    rng = np.random.default_rng(2)
    rgb = rng.uniform(size=(n, 3))
    g = np.zeros((3, H, W), np.float32)
    g[:, 8, 8] = 1.0   # only the pixel where the front pair is opaque
    out = _render_2d(orc, W, H, uv, conic, opac, rgb, [0.3, 0.3, 0.3], g,
                     depth=np.arange(1.0, n + 1))
    gr = out["grad2d"]
    assert np.all(gr[1:] == 0.0)
    assert np.any(gr[0] != 0.0)
    assert out["n_contrib"][8, 8] == 1


def test_ambiguous_alpha_floor_gets_allowance(orc):
    """alpha within FP32 rounding of 1/255: the oracle flags the decision and
    the image allowance equals the contribution of either outcome."""
    W = H = 16
    amin = float(np.float32(1.0) / np.float32(255.0))
    o = amin * (1 + 1e-9)
    out = _render_2d(orc, W, H, [[8.0, 8.0]], [[0.5, 0, 0.5]], [o], [[1.0, 0.5, 0.25]], [0, 0, 0],
                     np.ones((3, H, W), np.float32))
    assert out["pix_ambig"][8, 8] >= 1
    np.testing.assert_allclose(out["iallow"][:, 8, 8], o * np.array([1.0, 0.5, 0.25]), rtol=1e-12)
    assert out["gallow"][0, 6] > 0


def _center_pixel_grad(W, H):
    g = np.zeros((3, H, W), np.float32)
    g[:, 8, 8] = 1.0  # upstream gradient at the one pixel where a decision is ambiguous
    return g


def test_ambiguous_sigma_sign_gets_allowance(orc):
    """A splat centred 2^-20 px from a pixel centre: sigma ~ 2e-13 is within
    the FP32 rounding of the offset's products, so FP32 may find it negative
    and skip the splat there.  The allowance is that pixel's whole
    contribution (alpha c over a black background) and the splat's whole
    single-splat gradient there: dL/dc = alpha g, dL/do = G c.g."""
    W = H = 16
    u, o, c = 8.0 + 2.0 ** -20, 0.6, np.array([1.0, 0.5, 0.25])
    out = _render_2d(orc, W, H, [[u, 8.0]], [[0.5, 0, 0.5]], [o], [c], [0, 0, 0], _center_pixel_grad(W, H))
    assert out["pix_ambig"][8, 8] == 1 and out["pix_ambig"].sum() == 1
    G = math.exp(-0.25 * (u - 8.0) ** 2)
    np.testing.assert_allclose(out["iallow"][:, 8, 8], o * G * c, rtol=1e-12)
    np.testing.assert_allclose(out["gallow"][0, 6:9], [o * G] * 3, rtol=1e-12)
    np.testing.assert_allclose(out["gallow"][0, 5], G * c.sum(), rtol=1e-12)
    np.testing.assert_allclose(out["gallow"][0], np.abs(out["grad2d"][0]), rtol=1e-12)


def test_ambiguous_alpha_cap_gets_allowance(orc):
    """o G = 0.99 (1 + 1e-7) at the splat's centre: FP32 may leave alpha
    uncapped.  Capped, dL/do is 0; uncapped, dL/do = G dL/dalpha = c.g (single
    splat, black background, G = 1); the image differs by (o - 0.99) c."""
    W = H = 16
    cap = float(np.float32(0.99))
    o, c = cap * (1 + 1e-7), np.array([1.0, 0.5, 0.25])
    out = _render_2d(orc, W, H, [[8.0, 8.0]], [[0.5, 0, 0.5]], [o], [c], [0, 0, 0], _center_pixel_grad(W, H))
    assert out["pix_ambig"][8, 8] == 1 and out["pix_ambig"].sum() == 1
    assert out["grad2d"][0, 5] == 0.0  # capped: no opacity gradient
    np.testing.assert_allclose(out["iallow"][:, 8, 8], (o - cap) * c, rtol=1e-9)
    np.testing.assert_allclose(out["gallow"][0, 5], c.sum(), rtol=1e-12)
    np.testing.assert_allclose(out["gallow"][0, 6:9], [o - cap] * 3, rtol=1e-9)
    assert np.all(out["gallow"][0, 0:5] == 0.0)  # at the centre the conic and position terms vanish


def test_ambiguous_transmittance_stop_gets_allowance(orc):
    """Three stacked splats at a pixel centre with the third leaving
    T = 1e-4 (1 + 1e-8): FP32 may stop before it.  Then n_contrib is 2, the
    image differs by alpha_3 T_3 (c_3 - bg), the third splat loses its whole
    gradient and the two in front change dL/dalpha by
    alpha_3 T_3 (c_3 - bg).g / (1 - alpha_j)."""
    W = H = 16
    tmin = float(np.float32(1e-4))
    o01 = 0.95
    T3 = (1 - o01) * (1 - o01)
    o3 = 1 - tmin * (1 + 1e-8) / T3
    cs = np.array([[0.9, 0.1, 0.3], [0.2, 0.6, 0.5], [0.7, 0.3, 0.8]])
    bg = np.array([0.05, 0.2, 0.1])
    out = _render_2d(orc, W, H, [[8.0, 8.0]] * 3, [[0.5, 0, 0.5]] * 3, [o01, o01, o3], cs, bg,
                     _center_pixel_grad(W, H))
    assert out["pix_ambig"][8, 8] == 1
    assert out["n_contrib"][8, 8] == 3 and out["nc_alt"][8, 8] == 2
    d3 = o3 * T3 * (cs[2] - bg)
    np.testing.assert_allclose(out["iallow"][:, 8, 8], np.abs(d3), rtol=1e-9)
    np.testing.assert_allclose(out["gallow"][0:2, 5], [abs(d3.sum()) / (1 - o01)] * 2, rtol=1e-9)
    np.testing.assert_allclose(out["gallow"][2, 6:9], [o3 * T3] * 3, rtol=1e-9)
    np.testing.assert_allclose(out["gallow"][2, 5], T3 * (cs[2] - bg).sum(), rtol=1e-9)


def test_widening_covers_fp32_alpha_error_in_front(orc):
    """The per-pixel widening of the gradient scale must cover the FP32
    error of alpha in front of a pixel, amplified by 1 / (1 - alpha) in
    every transmittance behind it, without being orders of magnitude larger.
    Measured on the oracle itself: the change of every gradient when the
    front splat's alpha (0.98) moves by k ulp.  A 40-ulp move stays inside
    the widened bound; a 5-ulp move already comes near the unwidened one
    (so the widening is needed) and uses more than 1/128 of the widened one
    (so it is not inflated)."""
    W = H = 16
    eps32 = 2.0 ** -24
    off = (0.1, 0.1)
    o0 = 0.98 / math.exp(-0.25 * (off[0] ** 2 + off[1] ** 2))
    cs = np.array([[0.9, 0.1, 0.3], [0.2, 0.6, 0.5]])
    bg = [0.3, 0.2, 0.1]
    g = _center_pixel_grad(W, H)

    def run(o):
        return _render_2d(orc, W, H, [[8.0 + off[0], 8.0 + off[1]], [8.0, 8.0]], [[0.5, 0, 0.5]] * 2,
                          [o, 0.5], cs, bg, g)
    ref = run(o0)
    assert ref["pix_ambig"][8, 8] == 0 and ref["pix_widen"][8, 8] > 1.0

    def effect(k):
        return np.maximum(*[np.abs(run(o0 * (1 + s * k * eps32))["grad2d"] - ref["grad2d"]) for s in (-1, 1)])
    widened = lambda d: float((d / (1e-5 * ref["gscale"] + 1e-7)).max())
    literal = lambda d: float((d / (1e-5 * ref["glit"] + 1e-7)).max())
    assert widened(effect(40)) <= 1.0
    d5 = effect(5)
    assert literal(d5) > 0.5
    assert widened(d5) > 1.0 / 128


# ----------------------------------------------------------------------------
# binning: brute force
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 16)])
def test_binning_matches_brute_force(orc, tile):
    """Tile t = (tx, ty) holds Gaussian i iff floor(u)-r <= tw*tx + tw-1 and
    floor(u)+r >= tw*tx + 1 (same in y): the 3DGS bounding-box rule stated as
    interval overlap; lists ordered by (tile, depth, id)."""
    rng = np.random.default_rng(7)
    W, H, n = 77, 53, 300
    uv = np.asarray(rng.uniform(-20, [W + 20, H + 20], size=(n, 2)), np.float32).astype(np.float64)
    radius = rng.integers(0, 25, size=n).astype(np.int32)
    depth = rng.uniform(0.5, 5, size=n).astype(np.float32).astype(np.float64)
    depth[::7] = depth[3]  # equal depths: ties broken by id
    keys, pl, ranges = orc.bin_sort(uv, depth, radius, W, H, tile)
    tw, th = tile
    gx, gy = -(-W // tw), -(-H // th)
    entries = []
    for i in range(n):
        if radius[i] <= 0:
            continue
        fu, fv = math.floor(uv[i, 0]), math.floor(uv[i, 1])
        r = int(radius[i])
        for ty in range(gy):
            if not (fv - r <= th * ty + th - 1 and fv + r >= th * ty + 1):
                continue
            for tx in range(gx):
                if fu - r <= tw * tx + tw - 1 and fu + r >= tw * tx + 1:
                    entries.append((ty * gx + tx, float(np.float32(depth[i])), i))
    entries.sort()
    assert len(entries) == len(pl)
    assert [e[2] for e in entries] == [int(x) for x in pl]
    exp_ranges = np.zeros((gx * gy, 2), np.int64)
    for k, e in enumerate(entries):
        t = e[0]
        if k == 0 or entries[k - 1][0] != t:
            exp_ranges[t, 0] = k
        exp_ranges[t, 1] = k + 1
    np.testing.assert_array_equal(ranges, exp_ranges)
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    np.testing.assert_array_equal(tiles, [e[0] for e in entries])


# ----------------------------------------------------------------------------
# finite differences
# ----------------------------------------------------------------------------

def _random_2d(rng, n, W, H):
    uv = rng.uniform(2, [W - 2, H - 2], size=(n, 2))
    L = rng.normal(size=(n, 2, 2)) * 0.8
    cov = L @ L.transpose(0, 2, 1) + 1.5 * np.eye(2)
    inv = np.linalg.inv(cov)
    conic = np.stack([inv[:, 0, 0], inv[:, 0, 1], inv[:, 1, 1]], 1)
    opac = rng.uniform(0.2, 0.95, size=n)
    rgb = rng.uniform(size=(n, 3))
    return uv, conic, opac, rgb


def test_render_gradient_matches_central_differences(orc):
    """grad2d of L = sum(g * image) against central differences of the FP64
    forward for every 2D parameter of every splat."""
    rng = np.random.default_rng(21)
    W, H, n = 24, 20, 14
    uv, conic, opac, rgb = _random_2d(rng, n, W, H)
    bg = np.array([0.2, 0.4, 0.1])
    g = rng.normal(size=(3, H, W)).astype(np.float32)
    radius = np.full(n, 12, np.int32)
    depth = rng.uniform(1, 3, size=n)
    base = _render_2d(orc, W, H, uv, conic, opac, rgb, bg, g, radius=radius, depth=depth)
    gr = base["grad2d"]
    gd = g.astype(np.float64)

    def L(uv_, conic_, opac_, rgb_):
        o = _render_2d(orc, W, H, uv_, conic_, opac_, rgb_, bg, None, radius=radius, depth=depth)
        return float(np.sum(gd * o["image"]))

    h = 1e-6
    for i in range(n):
        for p in range(9):
            args = [uv.copy(), conic.copy(), opac.copy(), rgb.copy()]
            if p < 2:
                arr, idx = 0, (i, p)
            elif p < 5:
                arr, idx = 1, (i, p - 2)
            elif p == 5:
                arr, idx = 2, (i,)
            else:
                arr, idx = 3, (i, p - 6)
            args[arr][idx] += h
            lp = L(*args)
            args[arr][idx] -= 2 * h
            lm = L(*args)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gr[i, p]) <= 1e-6 * (abs(gr[i, p]) + 1e-3), (i, p, fd, gr[i, p])


def _fd_backproject_check(orc, sc, cam, rng, n_check=None):
    pp0 = orc.preprocess(sc, cam)
    vis = pp0["radius"] > 0
    lam = rng.normal(size=(sc.n, 9))

    def L(scene):
        pp = orc.preprocess(scene, cam)
        v = np.concatenate([pp["uv"], pp["conic"], pp["opacity"][:, None], pp["rgb"]], 1)
        return float(np.sum(lam[vis] * v[vis]))

    bp = orc.backproject(sc, cam, lam)
    fields = [("mean", "dmean"), ("scale", "dscale"), ("quat", "dquat"), ("opacity", "dopacity"),
              ("feat", "dfeat")]
    checked = 0
    for i in np.nonzero(vis)[0][:n_check]:
        for fname, gname in fields:
            arr = getattr(sc, fname)
            flat_idx = list(np.ndindex(arr[i].shape)) if arr[i].shape else [()]
            for j in flat_idx:
                x0 = float(arr[(i,) + j])
                h = 1e-3 * max(abs(x0), 1e-2)
                # the parameters are float32: step between representable values
                xp, xm = np.float32(x0 + h), np.float32(x0 - h)
                arr[(i,) + j] = xp
                lp = L(sc)
                arr[(i,) + j] = xm
                lm = L(sc)
                arr[(i,) + j] = x0
                fd = (lp - lm) / (float(xp) - float(xm))
                an = bp[gname][(i,) + j]
                tol = 2e-5 * (abs(an) + np.abs(bp[gname][i]).max() + 1e-6)
                assert abs(fd - an) <= tol, (i, fname, j, fd, an)
                checked += 1
    return checked


@pytest.mark.parametrize("sh_degree", [-1, 0, 1, 3])
def test_backproject_matches_central_differences(orc, sh_degree):
    """Backward projection of an arbitrary linear functional of the 2D outputs
    (u, v, A, B, C, o, rgb) against central differences of the FP64 preprocess
    w.r.t. mean, scale, unnormalised quaternion, opacity and SH/colour."""
    rng = np.random.default_rng(100 + sh_degree)
    n = 6
    cam = S.look_at_camera((0.6, -0.4, -3.6), (0.0, 0.1, 0.2), 96, 72)
    mean = rng.uniform(-0.6, 0.6, size=(n, 3))
    scale = np.exp(rng.normal(-2.5, 0.4, size=(n, 3)))
    quat = rng.normal(size=(n, 4))
    opac = rng.uniform(0.2, 0.9, size=n)
    if sh_degree < 0:
        feat = rng.uniform(size=(n, 3))
    else:
        k = (sh_degree + 1) ** 2
        feat = rng.normal(0, 0.3, size=(n, k, 3))
        feat[:, 0] = rng.uniform(0.5, 1.5, size=(n, 3))
    sc = _scene(mean, scale, quat, opac, feat, sh_degree)
    assert _fd_backproject_check(orc, sc, cam, rng) > 0


def test_backproject_frustum_clamp_branch(orc):
    """Gaussian beyond 1.3 tan(fov/2) in x (clamped Jacobian) but large enough
    to reach the screen: the exact derivative of the clamped projection."""
    rng = np.random.default_rng(9)
    cam = S.front_camera(64, 64)
    sc = _scene([[3.4, 0.1, 0.0]], [[0.9, 0.5, 0.6]], [rng.normal(size=4)], [0.6],
                [[0.3, 0.5, 0.7]], -1)
    pp = orc.preprocess(sc, cam)
    assert pp["radius"][0] > 0
    assert abs(3.4 / 4.0) > 1.3 * cam.tan_fovx
    assert _fd_backproject_check(orc, sc, cam, rng) > 0


def test_end_to_end_gradient_matches_central_differences(orc):
    """Full FP64 pipeline (preprocess -> bin -> render): d sum(g*image) / d theta
    by the oracle's backward (render then backproject) against central
    differences of the forward, on a tiny SH-degree-1 scene."""
    rng = np.random.default_rng(4)
    n, W, H = 8, 40, 32
    cam = S.front_camera(W, H)
    mean = rng.uniform(-0.5, 0.5, size=(n, 3))
    scale = np.exp(rng.normal(-2.2, 0.3, size=(n, 3)))
    feat = rng.normal(0, 0.2, size=(n, 4, 3))
    feat[:, 0] = rng.uniform(0.5, 1.5, size=(n, 3))
    sc = _scene(mean, scale, rng.normal(size=(n, 4)), rng.uniform(0.3, 0.9, size=n), feat, 1)
    g = rng.normal(size=(3, H, W)).astype(np.float32)
    gd = g.astype(np.float64)
    bg = (0.1, 0.2, 0.3)
    out = orc.render_scene(sc, cam, bg, g)
    bp = orc.backproject(sc, cam, out["grad2d"])

    def L():
        return float(np.sum(gd * orc.render_scene(sc, cam, bg)["image"]))

    for i in range(n):
        for fname, gname in [("mean", "dmean"), ("scale", "dscale"), ("quat", "dquat"),
                             ("opacity", "dopacity"), ("feat", "dfeat")]:
            arr = getattr(sc, fname)
            for j in (list(np.ndindex(arr[i].shape)) if arr[i].shape else [()])[:6]:
                x0 = float(arr[(i,) + j])
                h = 1e-3 * max(abs(x0), 1e-2)
                xp, xm = np.float32(x0 + h), np.float32(x0 - h)
                arr[(i,) + j] = xp
                lp = L()
                arr[(i,) + j] = xm
                lm = L()
                arr[(i,) + j] = x0
                fd = (lp - lm) / (float(xp) - float(xm))
                an = bp[gname][(i,) + j]
                assert abs(fd - an) <= 1e-4 * (abs(an) + np.abs(bp[gname][i]).max() + 1e-4), \
                    (i, fname, j, fd, an)


# ----------------------------------------------------------------------------
# Adam
# ----------------------------------------------------------------------------

def test_adam_first_steps_closed_form(orc):
    """From zero moments with a constant gradient, every bias-corrected Adam
    step moves each parameter by -lr g / (|g| + eps)."""
    rng = np.random.default_rng(0)
    p0 = rng.normal(size=50)
    gr = rng.normal(size=50)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    lr, eps = 1e-2, 1e-8
    for step in (1, 2, 3):
        orc.adam(p, gr.copy(), m, v, lr, 0.9, 0.999, eps, step)
        np.testing.assert_allclose(p, p0 - step * lr * gr / (np.abs(gr) + eps), rtol=1e-9, atol=1e-12)


def test_scatter_add_definition_by_brute_force(orc):
    rng = np.random.default_rng(12)
    idx = rng.integers(0, 7, size=200)
    vals = rng.normal(size=(200, 9))
    got = orc.scatter_add9(idx, vals, 7)
    ref = np.zeros((7, 9))
    for i, d in enumerate(idx):
        for q in range(9):
            ref[d, q] += vals[i, q]
    np.testing.assert_allclose(got, ref, rtol=1e-14, atol=1e-14)


# ----------------------------------------------------------------------------
# cube-map texture sampling and its gradient (cube_oracle.c)
# ----------------------------------------------------------------------------

def _dirs(rng, n):
    d = rng.normal(size=(n, 3)).astype(np.float32)
    return d


def test_cube_face_is_the_major_axis(orc):
    """Face = axis of the largest |component| (ties: x, then y), positive for
    components >= 0: brute force over random and tied directions; all-zero
    directions (either sign) have no sample."""
    rng = np.random.default_rng(0)
    d = _dirs(rng, 4000)
    d[:200, 1] = d[:200, 0]                      # |x| == |y|
    d[200:400, 2] = -d[200:400, 1]               # |y| == |z|
    d[400:450] = [[0.0, -0.0, 0.0]] * 50         # no sample
    d[450:500] = [[-0.0, 0.0, 0.0]] * 50
    d[450:500, 0] = np.float32(-0.0)
    d[450:500, 2] = np.float32(0.0)
    face, texel, w = orc.cube_taps(d, 16)
    a = np.abs(d)
    for i, v in enumerate(d):
        if not (a[i].max() > 0):
            assert face[i] == -1
            continue
        if a[i, 0] >= a[i, 1] and a[i, 0] >= a[i, 2]:
            ax = 0
        elif a[i, 1] >= a[i, 2]:
            ax = 1
        else:
            ax = 2
        pos = not np.signbit(v[ax]) or v[ax] == 0.0
        assert face[i] == 2 * ax + (0 if pos else 1), (i, v, face[i])


def test_cube_axis_directions_hit_the_face_centre(orc):
    """Along each axis (s, t) = (1/2, 1/2): u = v = R/2 - 1/2, so the four
    centre texels of the face get 1/4 each."""
    R = 8
    d = np.float32([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]]) * 3.0
    face, texel, w = orc.cube_taps(d, R)
    for f in range(6):
        assert face[f] == f
        cols = sorted({int(t % R) for t in texel[f]})
        rows = sorted({int(t // R % R) for t in texel[f]})
        assert cols == [R // 2 - 1, R // 2] and rows == [R // 2 - 1, R // 2]
        np.testing.assert_allclose(w[f], 0.25, rtol=0, atol=0)


def test_cube_coordinates_are_the_projection_onto_the_face(orc):
    """On every face the texel coordinates are the central projection of d
    onto the face: sampling a texture that stores each texel's own column and
    row returns (u, v) = (s R - 1/2, t R - 1/2) with s - 1/2 and t - 1/2
    equal to +-1/2 times the two minor components over the major one, each
    coordinate on a different minor axis.  (Which sign each face uses is the
    OpenGL convention and is not pinned here.)"""
    R = 64
    tex = np.zeros((6, R, R, 4), np.float32)
    tex[..., 0] = np.arange(R, dtype=np.float32)[None, None, :]
    tex[..., 1] = np.arange(R, dtype=np.float32)[None, :, None]
    rng = np.random.default_rng(1)
    for f in range(6):
        ax, sgn = f // 2, (1.0 if f % 2 == 0 else -1.0)
        minor = [a for a in range(3) if a != ax]
        d = rng.uniform(-0.9, 0.9, size=(300, 3))
        d[:, ax] = sgn
        d = d.astype(np.float32)
        out, _ = orc.cube_forward(d, R, tex)
        face, _, _ = orc.cube_taps(d, R)
        assert np.all(face == f)
        s = (out[:, 0] + 0.5) / R - 0.5
        t = (out[:, 1] + 0.5) / R - 0.5
        ratios = d[:, minor].astype(np.float64) / np.abs(d[:, [ax]].astype(np.float64))
        for coord in (s, t):
            coef, *_ = np.linalg.lstsq(ratios, coord, rcond=None)
            assert sorted(np.round(np.abs(coef), 6)) == [0.0, 0.5], (f, coef)
        cs, *_ = np.linalg.lstsq(ratios, s, rcond=None)
        ct, *_ = np.linalg.lstsq(ratios, t, rcond=None)
        assert np.argmax(np.abs(cs)) != np.argmax(np.abs(ct))


def test_cube_constant_texture_samples_the_constant(orc):
    """Bilinear weights sum to 1, also where taps are clamped at face edges."""
    R = 5
    tex = np.full((6, R, R, 4), 0.375, np.float32)
    tex[..., 1] = 2.0
    tex[..., 2] = -1.5
    rng = np.random.default_rng(2)
    d = _dirs(rng, 3000)
    d[:100] = np.float32([1, 0.999, -0.9999])      # near corners: clamped taps
    out, _ = orc.cube_forward(d, R, tex)
    np.testing.assert_allclose(out, np.broadcast_to([0.375, 2.0, -1.5], out.shape), rtol=1e-15, atol=1e-15)


def test_cube_worked_example(orc):
    """d = (1, 0.25, -0.5), R = 4: face +x, s = (0.5 + 1)/2 = 0.75, t =
    (-0.25 + 1)/2 = 0.375, u = 2.5, v = 1.0: taps (2,1), (3,1) with 1/2 each,
    (2,2), (3,2) with 0."""
    face, texel, w = orc.cube_taps(np.float32([[1.0, 0.25, -0.5]]), 4)
    assert face[0] == 0
    assert [(int(t % 4), int(t // 4 % 4)) for t in texel[0]] == [(2, 1), (3, 1), (2, 2), (3, 2)]
    np.testing.assert_array_equal(w[0], [0.5, 0.5, 0.0, 0.0])


def test_cube_backward_is_the_derivative_of_the_forward(orc):
    """The sample is linear in the texture, so the central difference of
    L = sum(dL * sample) in one texel channel is exact (up to FP64 rounding)
    and must equal the backward's gradient of that texel channel."""
    R = 6
    rng = np.random.default_rng(3)
    d = _dirs(rng, 500)
    d[:20] = 0.0
    dL = rng.normal(size=(500, 3)).astype(np.float32)
    tex = (rng.integers(0, 64, size=(6, R, R, 4)) / 64.0).astype(np.float32)  # +-0.5 stays exact
    grad, _ = orc.cube_backward(d, dL, R)
    for _ in range(40):
        f, j, i, c = rng.integers(6), rng.integers(R), rng.integers(R), rng.integers(3)
        tp, tm = tex.copy(), tex.copy()
        tp[f, j, i, c] += 0.5
        tm[f, j, i, c] -= 0.5
        lp = float((orc.cube_forward(d, R, tp)[0] * dL).sum())
        lm = float((orc.cube_forward(d, R, tm)[0] * dL).sum())
        assert abs((lp - lm) - grad[f, j, i, c]) <= 1e-12 * (1 + abs(grad[f, j, i, c])), (f, j, i, c)


def test_cube_gradient_sum_rule(orc):
    """Weights sum to 1 per sample, so the texture gradient summed over all
    texels equals the upstream gradient summed over the samples."""
    rng = np.random.default_rng(4)
    d = _dirs(rng, 2000)
    d[::7] = 0.0
    dL = rng.normal(size=(2000, 3)).astype(np.float32)
    grad, _ = orc.cube_backward(d, dL, 9)
    act = np.abs(d).max(1) > 0
    np.testing.assert_allclose(grad.reshape(-1, 3).sum(0), dL[act].astype(np.float64).sum(0), rtol=1e-12)
