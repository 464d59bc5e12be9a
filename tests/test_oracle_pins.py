"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a closed form derived by
hand from Eq. Q_ray, a brute-force search, an independent library routine (scipy), or an
identity the paper proves (Props. A.1-A.5, App. A.1-A.4, Sec. 5).
"""
import math

import numpy as np
import pytest

from paper_2503_18682_gb300 import scenes

PMIN = 1.0 / 255.0


def single(mu_w, log_s, quat, logit, rgb, sh_degree=0):
    k = (sh_degree + 1) ** 2
    sh = np.zeros((1, k, 3), dtype=np.float32)
    sh[0, 0] = rgb
    return dict(means=np.array([mu_w], np.float32), log_scales=np.array([log_s], np.float32),
                quats=np.array([quat], np.float32), opacity_logits=np.array([logit], np.float32),
                sh=sh, sh_degree=sh_degree)


def rand_rot(rng):
    q = rng.standard_normal(4)
    return q / np.linalg.norm(q)


def sigma_inv(R, s):
    return R @ np.diag(1.0 / np.asarray(s) ** 2) @ R.T


# ---------------------------------------------------------------- closed forms

def test_closed_form_axis_aligned(oracle_lib):
    """R = I, mu = (0,0,z0), scales (sx,sy,sz), ray x = (X,Y,1).  From Eq. Q_ray by hand:
    n = z0/sz^2, d = X^2/sx^2 + Y^2/sy^2 + 1/sz^2, c^2 = z0^2/sz^2 and D = c^2 - n^2/d, i.e.
    D = z0^2 (X^2/sx^2 + Y^2/sy^2) / (sz^2 (X^2/sx^2 + Y^2/sy^2 + 1/sz^2))."""
    z0, s = 3.0, np.array([0.05, 0.02, 0.2])
    logit, rgb = 1.3, np.array([0.2, 0.7, 0.9])
    sc = single([0, 0, z0], np.log(s), [1, 0, 0, 0], logit, rgb)
    cam = scenes.make_camera(48, 40, 400.0, 380.0, 24.0, 20.0)
    out = oracle_lib.render(sc, cam)
    j, i = np.divmod(np.arange(48 * 40), 48)
    X = (i + 0.5 - np.float32(24.0)) / np.float32(400.0)
    Y = (j + 0.5 - np.float32(20.0)) / np.float32(380.0)
    sf = np.exp(np.log(s).astype(np.float32).astype(np.float64))
    u = X ** 2 / sf[0] ** 2 + Y ** 2 / sf[1] ** 2
    D = z0 ** 2 * u / (sf[2] ** 2 * (u + 1.0 / sf[2] ** 2))
    o = 1.0 / (1.0 + np.exp(-np.float64(np.float32(logit))))
    kappa = -2 * np.log(PMIN / o)
    om = np.where(D <= kappa, np.minimum(o * np.exp(-D / 2), 0.99), 0.0)
    rgbf = rgb.astype(np.float32).astype(np.float64)
    np.testing.assert_allclose(out["rgb"], om[:, None] * rgbf[None, :], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(out["T"], 1 - om, rtol=1e-12, atol=1e-15)
    # on the principal ray D = 0 and the pixel is min(o, 0.99) * rgb
    one = oracle_lib.render(sc, scenes.make_camera(1, 1, 400.0, 380.0, 0.5, 0.5))
    np.testing.assert_allclose(one["rgb"][0], min(o, 0.99) * rgbf, rtol=1e-12)


def test_closed_form_isotropic(oracle_lib):
    """Sigma = s^2 I: the ray maximum is the point of closest approach, so
    D = |mu x x^|^2 / s^2 (squared distance from the mean to the ray, over s^2)."""
    rng = np.random.default_rng(11)
    for _ in range(200):
        mu = rng.uniform(-1, 1, 3) + np.array([0, 0, 4.0])
        s = rng.uniform(0.01, 0.5)
        x = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), 1.0])
        D, tau = oracle_lib.D_ray(mu, np.eye(3) / s ** 2, x)
        xh = x / np.linalg.norm(x)
        assert D == pytest.approx(np.linalg.norm(np.cross(mu, xh)) ** 2 / s ** 2, rel=1e-10)
        assert tau * np.linalg.norm(x) == pytest.approx(np.dot(mu, xh), rel=1e-10)


def test_support_mask_isotropic_closed_form(oracle_lib):
    """Support mask over a pixel rectangle for Sigma = s^2 I: a pixel is in the support
    exactly when its ray passes within s sqrt(kappa) of the mean, in front of the camera
    (closest-approach distance, D = |mu x x^|^2 / s^2).  Includes a mean behind the camera
    plane, whose support must be empty."""
    cam = dict(fx=40.0, fy=50.0, cx=20.0, cy=12.0)
    for mu, s, kappa in (([0.1, -0.05, 1.0], 0.08, 9.0), ([-0.3, 0.2, 0.4], 0.05, 4.0),
                         ([0.0, 0.0, -1.0], 0.3, 9.0)):
        mu = np.array(mu)
        m = oracle_lib.support_mask(mu, np.eye(3) / s ** 2, kappa, cam, -3, -2, 47, 29)
        jj, ii = np.mgrid[-2:27, -3:44]
        X = np.stack([(ii + 0.5 - 20.0) / 40.0, (jj + 0.5 - 12.0) / 50.0, np.ones(ii.shape)], -1)
        Xh = X / np.linalg.norm(X, axis=-1, keepdims=True)
        dist2 = np.sum(np.cross(mu, Xh) ** 2, axis=-1)
        expect = (dist2 <= kappa * s ** 2) & (Xh @ mu > 0)
        assert np.array_equal(m, expect)
        assert m.any() == (mu[2] > 0)


def test_ray_march_bruteforce(oracle_lib):
    """Prop. A.1: tau(x) x is the density maximum along the ray.  Brute force: a dense march
    over t in (0, t_max] with three refinement levels finds the same minimum of the
    Mahalanobis distance."""
    rng = np.random.default_rng(5)
    for _ in range(40):
        R = oracle_lib.quat_to_rot(rand_rot(rng))
        s = np.exp(rng.uniform(np.log(0.01), np.log(0.3), 3))
        Si = sigma_inv(R, s)
        mu = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(2, 5)])
        x = mu / mu[2] + np.array([rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1), 0.0])
        D, tau = oracle_lib.D_ray(mu, Si, x)
        if not tau > 0:
            continue
        lo, hi = 1e-6, 10.0
        for _lvl in range(4):
            t = np.linspace(lo, hi, 20001)
            P = t[:, None] * x[None, :] - mu[None, :]
            f = np.einsum("ni,ij,nj->n", P, Si, P)
            k = int(np.argmin(f))
            step = t[1] - t[0]
            lo, hi = max(1e-9, t[k] - 2 * step), t[k] + 2 * step
        assert f[k] == pytest.approx(D, rel=1e-7, abs=1e-9)
        assert t[k] == pytest.approx(tau, rel=1e-6)


def test_render_pixel_matches_ray_march(oracle_lib):
    """Single anisotropic primitive: the oracle's pixel value equals o exp(-D/2) * rgb with
    D found by brute-force ray marching (the render's whitened evaluation path)."""
    rng = np.random.default_rng(9)
    q = rand_rot(rng)
    s = np.array([0.08, 0.03, 0.15])
    mu_w = np.array([0.1, -0.05, 2.5])
    sc = single(mu_w, np.log(s), q, 2.0, [1.0, 0.5, 0.25])
    cam = scenes.make_camera(24, 24, 60.0, 60.0, 12.0, 12.0)
    out = oracle_lib.render(sc, cam)
    R = oracle_lib.quat_to_rot(np.float32(q).astype(np.float64))
    sf = np.exp(np.log(s).astype(np.float32).astype(np.float64))
    Si = sigma_inv(R, sf)
    muf = mu_w.astype(np.float32).astype(np.float64)
    o = 1 / (1 + np.exp(-2.0))
    kappa = -2 * np.log(PMIN / o)
    t = np.linspace(1e-4, 8.0, 40001)
    for p in range(0, 24 * 24, 7):
        i, j = p % 24, p // 24
        x = np.array([(i + 0.5 - 12) / 60.0, (j + 0.5 - 12) / 60.0, 1.0])
        P = t[:, None] * x[None, :] - muf[None, :]
        k = int(np.argmin(np.einsum("ni,ij,nj->n", P, Si, P)))
        tt = np.linspace(t[max(k - 1, 0)], t[min(k + 1, len(t) - 1)], 20001)
        P = tt[:, None] * x[None, :] - muf[None, :]
        D = np.einsum("ni,ij,nj->n", P, Si, P).min()
        om = min(o * math.exp(-D / 2), 0.99) if D <= kappa else 0.0
        assert out["rgb"][p, 0] == pytest.approx(om, rel=1e-7, abs=1e-12)


# ------------------------------------------------------- propositions (App. A)

def _prim(rng, far=True):
    R = oracle_lib_global.quat_to_rot(rand_rot(rng))
    s = np.exp(rng.uniform(np.log(0.02), np.log(0.3), 3))
    mu = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(2, 5) if far else 0.0])
    return R, s, mu


oracle_lib_global = None


@pytest.fixture(autouse=True)
def _bind(oracle_lib):
    global oracle_lib_global
    oracle_lib_global = oracle_lib


def test_prop_full_support(oracle_lib):
    """Prop. A.2: if c^2 <= kappa, every ray is in the support (D <= kappa)."""
    rng = np.random.default_rng(21)
    for _ in range(50):
        R = oracle_lib.quat_to_rot(rand_rot(rng))
        s = np.exp(rng.uniform(np.log(0.5), np.log(2.0), 3))
        mu = rng.uniform(-0.2, 0.2, 3)
        Si = sigma_inv(R, s)
        c2 = mu @ Si @ mu
        kappa = c2 * rng.uniform(1.0, 3.0)
        for _r in range(20):
            x = rng.standard_normal(3)
            D, _ = oracle_lib.D_ray(mu, Si, x)
            assert D <= kappa * (1 + 1e-12)


def test_props_boundary_ellipse(oracle_lib):
    """Props. A.3-A.5 on the boundary set E, generated by Eq. invPhi:
    e = ((c^2 - kappa)/c) Q H(a u) for u on S^1.  On E: D = kappa, tau(e) = 1 and
    e^T Sigma^-1 e = e^T Sigma^-1 mu = c^2 - kappa; tau (mu^T Sigma^-1 x) >= c^2 - kappa > 0
    for rays inside the support."""
    rng = np.random.default_rng(22)
    for _ in range(60):
        R, s, mu = _prim(rng)
        Si = sigma_inv(R, s)
        c2 = mu @ Si @ mu
        kappa = rng.uniform(0.5, 12.0)
        if c2 <= kappa:
            continue
        qd = oracle_lib.quad(mu, R, s, kappa)
        assert qd["c2"] == pytest.approx(c2, rel=1e-12)
        c = math.sqrt(c2)
        for th in np.linspace(0, 2 * np.pi, 17):
            u = np.array([math.cos(th), math.sin(th)])
            e = (c2 - kappa) / c * qd["Q"] @ np.array([qd["a"] * u[0], qd["a"] * u[1], 1.0])
            D, tau = oracle_lib.D_ray(mu, Si, e)
            assert D == pytest.approx(kappa, rel=1e-9)
            assert tau == pytest.approx(1.0, rel=1e-10)
            assert e @ Si @ e == pytest.approx(c2 - kappa, rel=1e-9)
            assert e @ Si @ mu == pytest.approx(c2 - kappa, rel=1e-9)
            # a ray strictly inside the support: shrink u towards the ellipse centre
            x = (c2 - kappa) / c * qd["Q"] @ np.array([0.5 * qd["a"] * u[0], 0.5 * qd["a"] * u[1], 1.0])
            D2, tau2 = oracle_lib.D_ray(mu, Si, x)
            assert D2 < kappa
            assert tau2 * (mu @ Si @ x) >= (c2 - kappa) * (1 - 1e-12)


def test_rotation_align(oracle_lib):
    """App. A.1: R_{mu^<-v} is a rotation (orthonormal, det +1) mapping v = e_z to mu^, in
    both branches, including mu^ = +-v."""
    rng = np.random.default_rng(23)
    dirs = [np.array([0, 0, 1.0]), np.array([0, 0, -1.0]), np.array([1.0, 0, 0]),
            np.array([0, 1.0, 1e-300])]
    dirs += [v / np.linalg.norm(v) for v in rng.standard_normal((200, 3))]
    for mh in dirs:
        R = oracle_lib.rot_align(mh)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-13)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-12)
        np.testing.assert_allclose(R @ np.array([0, 0, 1.0]), mh, atol=1e-13)


def test_quad_geometry(oracle_lib):
    """Sec. 4.1 / App. A.2-A.4: the quad centre is mu; u1 maximises u^T B u over S^1 (dense
    sweep); U_ray is orthonormal with u0 = rot90(u1); for points V alpha of the quad the
    fragment formula 1/(c^-2 + |Z alpha|^-2) equals the definition (Eq. Q_ray)."""
    rng = np.random.default_rng(24)
    for _ in range(60):
        R, s, mu = _prim(rng)
        Si = sigma_inv(R, s)
        kappa = rng.uniform(0.5, 12.0)
        if mu @ Si @ mu <= kappa:
            continue
        qd = oracle_lib.quad(mu, R, s, kappa)
        V, Z, U = qd["V"], qd["Z"], qd["U"]
        np.testing.assert_allclose(V.mean(axis=1), mu, atol=1e-12)
        np.testing.assert_allclose(U.T @ U, np.eye(2), atol=1e-13)
        np.testing.assert_allclose(U[:, 0], [-U[1, 1], U[0, 1]], atol=1e-15)
        Q01 = qd["Q"][:, :2]
        B = Q01.T @ Q01
        th = np.linspace(0, np.pi, 100001)
        uu = np.stack([np.cos(th), np.sin(th)])
        vals = np.einsum("in,ij,jn->n", uu, B, uu)
        u1 = U[:, 1]
        assert u1 @ B @ u1 >= vals.max() * (1 - 1e-9)
        c2 = qd["c2"]
        for _k in range(20):
            al = rng.dirichlet(np.ones(4))
            x = V @ al
            D, _ = oracle_lib.D_ray(mu, Si, x)
            za = Z @ al
            nz2 = za @ za
            Dfrag = 1.0 / (1.0 / c2 + 1.0 / nz2) if nz2 > 0 else 0.0
            assert D == pytest.approx(Dfrag, rel=1e-8, abs=1e-12)


def test_quad_contains_support(oracle_lib):
    """Brute-force pixel sweep: every pixel whose ray meets the support (the oracle
    composites it) lies inside the projected quad (Eq. V_ray), and every pixel ray through
    the inscribed ellipse of the quad has D <= kappa."""
    rng = np.random.default_rng(25)
    W = H = 96
    f = 80.0
    checked = 0
    for trial in range(30):
        q = rand_rot(rng)
        s = np.exp(rng.uniform(np.log(0.02), np.log(0.25), 3))
        mu_w = np.array([rng.uniform(-0.6, 0.6), rng.uniform(-0.6, 0.6), rng.uniform(1.5, 4.0)])
        logit = rng.uniform(-1, 3)
        sc = single(mu_w, np.log(s), q, logit, [1, 1, 1])
        cam = scenes.make_camera(W, H, f, f, W / 2, H / 2)
        out = oracle_lib.render(sc, cam)
        info = oracle_lib.prepare(sc, cam)[0]
        if info[0] != 0:
            continue
        mu = info[2:5]
        Rc = info[14:23].reshape(3, 3)
        sf = info[11:14]
        qd = oracle_lib.quad(mu, Rc, sf, info[6])
        V = qd["V"]
        if np.any(V[2] <= 1e-9):
            continue
        P = np.stack([f * V[0] / V[2] + W / 2, f * V[1] / V[2] + H / 2], axis=1)
        inside_any = 0
        for p in np.nonzero(out["ncontrib"] > 0)[0]:
            px, py = p % W + 0.5, p // W + 0.5
            # convex polygon test (vertices in order around the quad)
            sgn = []
            for k in range(4):
                a, b = P[k], P[(k + 1) % 4]
                sgn.append((b[0] - a[0]) * (py - a[1]) - (b[1] - a[1]) * (px - a[0]))
            sgn = np.array(sgn)
            assert np.all(sgn >= -1e-9) or np.all(sgn <= 1e-9), (trial, p)
            inside_any += 1
        checked += inside_any
        # rays through the inscribed ellipse of the quad
        Si = sigma_inv(Rc, sf)
        T01 = qd["Q"][:, :2] @ qd["U"]
        zs = math.sqrt(info[6]) / qd["b"]
        for th in np.linspace(0, 2 * np.pi, 13):
            for r in (0.3, 0.7, 0.999):
                pt = mu + zs * r * (T01 @ np.array([math.cos(th), math.sin(th)]))
                D, tau = oracle_lib.D_ray(mu, Si, pt)
                assert D <= info[6] * (1 + 1e-12) and tau > 0
    assert checked > 500


# --------------------------------------------------------------- colour (SH)

def test_sh_basis_orthonormal_and_scipy(oracle_lib):
    """Real SH (no Condon-Shortley phase): orthonormal on the sphere (Gauss-Legendre x
    uniform quadrature), Y_00 = 1/(2 sqrt(pi)), and equal to scipy's complex harmonics
    combined into real ones: Y_lm = sqrt(2) (-1)^m Re/Im Y_l^|m| (scipy has the phase)."""
    sp = pytest.importorskip("scipy.special")
    xg, wg = np.polynomial.legendre.leggauss(24)
    nphi = 48
    phis = 2 * np.pi * np.arange(nphi) / nphi
    G = np.zeros((16, 16))
    for ct, w in zip(xg, wg):
        st = math.sqrt(1 - ct * ct)
        for ph in phis:
            Y = oracle_lib.sh_basis(3, [st * math.cos(ph), st * math.sin(ph), ct])
            G += np.outer(Y, Y) * w * (2 * np.pi / nphi)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)
    assert oracle_lib.sh_basis(0, [0, 0, 1])[0] == pytest.approx(0.5 / math.sqrt(math.pi), rel=1e-15)
    rng = np.random.default_rng(3)
    for _ in range(30):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        Y = oracle_lib.sh_basis(3, d)
        for l in range(4):
            for m in range(-l, l + 1):
                am = abs(m)
                if hasattr(sp, "sph_harm_y"):
                    Yc = sp.sph_harm_y(l, am, theta, phi)
                else:
                    Yc = sp.sph_harm(am, l, phi, theta)
                if m == 0:
                    ref = Yc.real
                elif m > 0:
                    ref = math.sqrt(2) * (-1) ** am * Yc.real
                else:
                    ref = math.sqrt(2) * (-1) ** am * Yc.imag
                assert Y[l * l + l + m] == pytest.approx(ref, abs=1e-12)


def test_quaternion_vs_scipy(oracle_lib):
    sp = pytest.importorskip("scipy.spatial.transform")
    rng = np.random.default_rng(4)
    for _ in range(50):
        q = rng.standard_normal(4) * rng.uniform(0.1, 3)
        R = oracle_lib.quat_to_rot(q)
        Rs = sp.Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        np.testing.assert_allclose(R, Rs, atol=1e-13)


def test_colour_direction_dependence(oracle_lib):
    """Degree-1 colour: rgb = k0 + Y_1m(d) k_1m with d from the camera centre to the mean;
    Y_10 = sqrt(3/(4 pi)) z (textbook), so a z-coefficient adds sqrt(3/4pi) d_z."""
    sc = single([0.0, 0.0, 2.0], np.log([0.05] * 3), [1, 0, 0, 0], 3.0, [0.3, 0.3, 0.3], sh_degree=1)
    sc["sh"][0, 2, :] = [0.1, 0.2, 0.4]          # index l*l+l+m = 2 is (l=1, m=0)
    cam = scenes.make_camera(16, 16, 20.0, 20.0)
    info = oracle_lib.prepare(sc, cam)[0]
    c = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(info[8:11], np.float32([0.3] * 3) + c * np.float32([0.1, 0.2, 0.4]), rtol=1e-7)


# ------------------------------------------------------------- compositing

def test_compositing_closed_form(oracle_lib):
    """k coincident primitives seen head-on (D = 0): omega = min(o, 0.99) each, so
    C = rgb (1 - (1 - omega)^k') with k' the count composited before T would drop below
    t_stop (textbook over-compositing)."""
    n = 60
    sc = dict(means=np.tile(np.float32([0, 0, 3.0]), (n, 1)),
              log_scales=np.full((n, 3), np.log(0.1), np.float32),
              quats=np.tile(np.float32([1, 0, 0, 0]), (n, 1)),
              opacity_logits=np.full(n, 0.4, np.float32),
              sh=np.tile(np.float32([[[0.9, 0.5, 0.1]]]), (n, 1, 1)), sh_degree=0)
    cam = scenes.make_camera(1, 1, 10.0, 10.0, 0.5, 0.5)
    out = oracle_lib.render(sc, cam)
    om = 1 / (1 + math.exp(-np.float64(np.float32(0.4))))
    k = 0
    while (1 - om) ** (k + 1) >= 1e-4 and k < n:
        k += 1
    assert out["ncontrib"][0] == k
    np.testing.assert_allclose(out["rgb"][0], np.float32([0.9, 0.5, 0.1]).astype(np.float64) * (1 - (1 - om) ** k), rtol=1e-12)
    assert out["T"][0] == pytest.approx((1 - om) ** k, rel=1e-12)


def test_depth_order_and_ties(oracle_lib):
    """Eq. rendering: ascending depth of the centres, ties by index.  The key is the float32
    depth within 2 ulp of the exact view-space depth."""
    rng = np.random.default_rng(8)
    sc = scenes.uniform_scene(300, seed=8)
    sc["means"][10] = sc["means"][20]               # an exact tie
    R, t = scenes.look_at([0.3, -0.2, -1.0], [0, 0, 3.0])
    cam = scenes.make_camera(32, 32, 30.0, 30.0, R=R, t=t)
    info = oracle_lib.prepare(sc, cam)
    keys = info[:, 1].astype(np.uint32)
    z = info[:, 2:5][:, 2]
    zf = keys.view(np.float32).astype(np.float64)
    ok = info[:, 0] == 0
    assert np.all(np.abs(zf[ok] - z[ok]) <= 2 * np.spacing(np.float32(zf[ok]).astype(np.float32)))
    assert keys[10] == keys[20]
    # a red primitive at index 0 and a blue one at index 1 at the same depth: red is in front
    two = single([0, 0, 2.0], np.log([0.3] * 3), [1, 0, 0, 0], 6.0, [1, 0, 0])
    for k in ("means", "log_scales", "quats", "opacity_logits"):
        two[k] = np.concatenate([two[k], two[k]])
    two["sh"] = np.concatenate([two["sh"], np.float32([[[0, 0, 1]]])])
    out = oracle_lib.render(two, scenes.make_camera(1, 1, 10, 10, 0.5, 0.5))
    assert out["rgb"][0, 0] > out["rgb"][0, 2]
    two["means"][1, 2] = np.nextafter(np.float32(2.0), np.float32(0))   # blue now nearer
    out = oracle_lib.render(two, scenes.make_camera(1, 1, 10, 10, 0.5, 0.5))
    assert out["rgb"][0, 2] > out["rgb"][0, 0]


def test_culling_rules(oracle_lib):
    """Near-plane cull (Sec. 4.1), kappa <= 0 skip (Sec. 3) and camera-inside skip
    (Sec. 3.2, Eq. c)."""
    cam = scenes.make_camera(8, 8, 10.0, 10.0)
    sc = single([0, 0, 0.005], np.log([0.01] * 3), [1, 0, 0, 0], 0.0, [1, 1, 1])
    assert oracle_lib.prepare(sc, cam)[0, 0] == 1
    sc = single([0, 0, 2.0], np.log([0.1] * 3), [1, 0, 0, 0], -6.0, [1, 1, 1])   # o < 1/255
    assert oracle_lib.prepare(sc, cam)[0, 0] == 2
    sc = single([0, 0, 0.3], np.log([1.0] * 3), [1, 0, 0, 0], 2.0, [1, 1, 1])    # camera inside
    assert oracle_lib.prepare(sc, cam)[0, 0] == 3
    assert oracle_lib.render(sc, cam)["rgb"].max() == 0.0


# ----------------------------------------------------------------------- MIP

def test_mip_limits(oracle_lib):
    """Sec. 5, Eq. mip.  sigma -> 0 reproduces the plain render; for an isotropic primitive
    (by hand: c^2 = |mu|^2/s^2, c^^2 = |mu|^2/(s^2+lam), |Sigma|/|Sigma^| = (s^2/(s^2+lam))^3)
    the modulated opacity is o s^2/(s^2 + lam) with lam = sigma^2 |mu|^2/(fx fy); the
    modulation never exceeds 1."""
    sc, cams = scenes.workload_small()
    cam = dict(cams[0])
    plain = oracle_lib.render(sc, cam)
    cam_m = dict(cam, mip=True)
    zero = oracle_lib.render(sc, cam_m, cfg=dict(mip_sigma2=0.0))
    np.testing.assert_array_equal(plain["rgb"], zero["rgb"])
    s = 0.02
    one = single([0.1, -0.2, 3.0], np.log([s] * 3), [1, 0, 0, 0], 1.0, [1, 1, 1])
    info = oracle_lib.prepare(one, dict(cam_m, fx=np.float32(64), fy=np.float32(64)))[0]
    sf = math.exp(float(np.float32(np.log(s))))
    mu = np.float32([0.1, -0.2, 3.0]).astype(np.float64)
    lam = 0.1 * (mu @ mu) / (64.0 * 64.0)
    o = 1 / (1 + math.exp(-1.0))
    assert info[7] == pytest.approx(o * sf ** 2 / (sf ** 2 + lam), rel=1e-12)
    np.testing.assert_allclose(info[11:14], math.sqrt(sf ** 2 + lam), rtol=1e-12)
    rng = np.random.default_rng(6)
    sc2 = scenes.blob_scene(2000, seed=6, sh_degree=0)
    cam2 = scenes.make_camera(64, 64, 64.0, 64.0, mip=True)
    i2 = oracle_lib.prepare(sc2, cam2, cfg=dict(mip_sigma2=2.0))
    i1 = oracle_lib.prepare(sc2, dict(cam2, mip=False))
    ok = (i2[:, 0] != 1) & (i2[:, 0] != 4)
    assert np.all(i2[ok, 7] <= i1[ok, 7] * (1 + 1e-12))
    assert np.any(i2[ok, 7] < 0.9 * i1[ok, 7])


def load_golden_small():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "small_uniform_64x64.txt")
    a = np.loadtxt(path, comments="#")
    return a[:, :2].astype(np.int32), a[:, 2:5], a[:, 5], a[:, 6].astype(np.int32)


def test_golden_small_scene_regression(oracle_lib):
    """The stored oracle image of the 64x64 scene (tests/golden, written by make_golden.py
    from the oracle alone) is reproduced: a regression guard on the oracle, not a pin."""
    from paper_2503_18682_gb300 import scenes
    pix, rgb, T, flags = load_golden_small()
    scene, cams = scenes.workload_small()
    out = oracle_lib.render(scene, cams[0], pixels=pix)
    np.testing.assert_allclose(out["rgb"], rgb, rtol=0, atol=1e-12)
    np.testing.assert_allclose(out["T"], T, rtol=0, atol=1e-12)
    assert np.array_equal(out["flags"].astype(np.int32), flags)


# ---------------------------------------------------------------- GS divergence (Sec. 3.1)

def _gs_single_T(o, D, kappa):
    om = np.where(D <= kappa, np.minimum(o * np.exp(-D / 2), 0.99), 0.0)
    return 1.0 - om


def test_gs_isotropic_on_axis(oracle_lib):
    """Sigma = s^2 I at mu = (0, 0, z0): J = diag(fx/z0, fy/z0) (third column zero), so by hand
    D_gs = (dx z0 / (fx s))^2 + (dy z0 / (fy s))^2 with (dx, dy) the offset of the pixel centre
    from the principal point.  fx != fy catches swapped Jacobian rows."""
    z0, s, logit = 2.5, 0.04, 0.7
    sc = single([0, 0, z0], np.log([s] * 3), [1, 0, 0, 0], logit, [1, 1, 1])
    cam = scenes.make_camera(40, 36, 300.0, 220.0, 20.0, 18.0)
    out = oracle_lib.render(sc, cam, cfg=dict(divergence=1))
    j, i = np.divmod(np.arange(40 * 36), 40)
    sf = math.exp(float(np.float32(np.log(s))))
    D = ((i + 0.5 - 20.0) * z0 / (300.0 * sf)) ** 2 + ((j + 0.5 - 18.0) * z0 / (220.0 * sf)) ** 2
    o = 1.0 / (1.0 + math.exp(-float(np.float32(logit))))
    kappa = -2 * math.log(PMIN / o)
    np.testing.assert_allclose(out["T"], _gs_single_T(o, D, kappa), rtol=1e-12, atol=1e-15)
    assert np.count_nonzero(out["ncontrib"]) > 100


def _project(p, f, c):
    return np.array([f[0] * p[0] / p[2] + c[0], f[1] * p[1] / p[2] + c[1]])


def test_gs_numeric_jacobian(oracle_lib):
    """Random rotated, anisotropic primitives seen by a rotated camera.  Independent
    restatement: Sigma from scipy's rotation of the quaternion, the camera-frame mean from
    the camera's R and t, J of the projection by central differences (exact to ~1e-10 for a
    rational map), Sigma_pi = J Sigma J^T and D by np.linalg.solve.  A transposed J, a dropped
    off-axis column or a wrong world-to-camera step fails it."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(21)
    R, t = scenes.look_at([0.3, -0.2, -4.0], [0.0, 0.1, 0.0])
    cam = scenes.make_camera(48, 40, 260.0, 240.0, 22.5, 21.0, R=R, t=t)
    Rf, tf = cam["R"].astype(np.float64), cam["t"].astype(np.float64)
    f, c = (260.0, 240.0), (22.5, 21.0)
    checked = 0
    for _ in range(12):
        mu_w = rng.uniform(-0.6, 0.6, 3).astype(np.float32)
        ls = np.log(rng.uniform(0.05, 0.3, 3)).astype(np.float32)
        q = rand_rot(rng).astype(np.float32)
        sc = single(mu_w, ls, q, 2.0, [1, 1, 1])
        out = oracle_lib.render(sc, cam, cfg=dict(divergence=1))
        mu = Rf @ mu_w.astype(np.float64) + tf
        Rq = Rot.from_quat(q.astype(np.float64)[[1, 2, 3, 0]]).as_matrix()
        Sw = Rq @ np.diag(np.exp(2 * ls.astype(np.float64))) @ Rq.T
        Sc = Rf @ Sw @ Rf.T
        J = np.zeros((2, 3))
        for k in range(3):
            h = 1e-6 * abs(mu[2])
            e = np.zeros(3); e[k] = h
            J[:, k] = (_project(mu + e, f, c) - _project(mu - e, f, c)) / (2 * h)
        Sp = J @ Sc @ J.T
        u = _project(mu, f, c)
        j, i = np.divmod(np.arange(48 * 40), 48)
        dlt = np.stack([i + 0.5 - u[0], j + 0.5 - u[1]])
        D = np.einsum("ip,ip->p", dlt, np.linalg.solve(Sp, dlt))
        o = 1.0 / (1.0 + math.exp(-float(np.float32(2.0))))
        kappa = -2 * math.log(PMIN / o)
        keep = np.abs(D - kappa) > 1e-6 * kappa
        np.testing.assert_allclose(out["T"][keep], _gs_single_T(o, D, kappa)[keep], rtol=1e-7, atol=1e-9)
        checked += np.count_nonzero(out["ncontrib"][keep])
    assert checked > 500


def test_gs_approaches_ray_for_small_far_primitives(oracle_lib):
    """Sec. 3.1 vs 3.2: the EWA linearisation is exact in the limit of a primitive that is
    small against its distance and near the principal ray, where D_gs and D_ray agree.  For an
    isotropic primitive on the axis, by hand, D_ray = D_gs / (1 + |x_n|^2) with x_n the
    normalised image coordinate, so the images differ by O(field of view^2)."""
    rng = np.random.default_rng(5)
    cam = scenes.make_camera(32, 32, 4000.0, 4000.0)
    for _ in range(6):
        mu = np.array([*rng.uniform(-0.02, 0.02, 2), 50.0], np.float32)
        sc = single(mu, np.log(rng.uniform(0.02, 0.05, 3)), rand_rot(rng), 1.5, [1, 1, 1])
        a = oracle_lib.render(sc, cam)
        b = oracle_lib.render(sc, cam, cfg=dict(divergence=1))
        assert np.count_nonzero(a["ncontrib"]) > 50
        both = (a["ncontrib"] > 0) == (b["ncontrib"] > 0)
        np.testing.assert_allclose(b["T"][both], a["T"][both], atol=1e-3)
        # where one support edge passes the pixel and the other does not, omega ~ p_min
        assert np.all(np.abs(b["T"] - a["T"])[~both] <= 1.05 * PMIN)
        assert np.count_nonzero(~both) <= 0.05 * np.count_nonzero(a["ncontrib"])


def test_gs_refuses_mip_and_skips_no_inside_camera(oracle_lib):
    """D_gs has no camera-inside skip: a primitive whose RayGS support holds the camera
    centre (c^2 <= kappa) is culled by RayGS but still splatted by GS.  Eq. mip is a RayGS
    term: a MIP camera with the GS divergence is refused."""
    sc = single([0, 0, 0.5], np.log([0.6] * 3), [1, 0, 0, 0], 3.0, [1, 1, 1])
    cam = scenes.make_camera(16, 16, 20.0, 20.0)
    assert np.all(oracle_lib.render(sc, cam)["ncontrib"] == 0)
    assert np.any(oracle_lib.render(sc, cam, cfg=dict(divergence=1))["ncontrib"] > 0)
    with pytest.raises(RuntimeError):
        oracle_lib.render(sc, dict(cam, mip=True), cfg=dict(divergence=1))


# ---------------------------------------------------------------- exact pixel-dependent MIP (Sec. 5)

def _single_T(om):
    return np.where(om >= PMIN, 1.0 - np.minimum(om, 0.99), 1.0)


def test_mip_exact_isotropic_closed_form(oracle_lib):
    """Sigma = s^2 I seen off-axis through a wide field of view.  By hand, for the unit ray
    xh: tau = mu . xh, lambda = sigma^2 cos^3(theta) tau^2 / (fx fy) with cos(theta) = 1/|x|,
    Sigma^_x = (s^2 + lambda) I, so D = |mu x xh|^2 / (s^2 + lambda) and the modulation is
    sqrt(s^6 s^-2 / ((s^2 + lambda)^3 (s^2 + lambda)^-1)) = s^2 / (s^2 + lambda)."""
    mu = np.array([0.3, -0.2, 2.0])
    s, logit, sig2 = 0.3, 1.0, 10.0
    sc = single(mu, np.log([s] * 3), [1, 0, 0, 0], logit, [1, 1, 1])
    cam = scenes.make_camera(48, 40, 22.0, 19.0, 24.0, 20.0, mip="exact")
    out = oracle_lib.render(sc, cam, cfg=dict(mip_sigma2=sig2))
    j, i = np.divmod(np.arange(48 * 40), 48)
    x = np.stack([(i + 0.5 - 24.0) / 22.0, (j + 0.5 - 20.0) / 19.0, np.ones(i.size)], axis=1)
    xn = np.linalg.norm(x, axis=1)
    xh = x / xn[:, None]
    muf = np.float32(mu).astype(np.float64)
    sf = math.exp(float(np.float32(np.log(s))))
    tau = xh @ muf
    lam = sig2 * xn ** -3 * tau ** 2 / (22.0 * 19.0)
    D = np.sum(np.cross(muf, xh) ** 2, axis=1) / (sf ** 2 + lam)
    o = 1.0 / (1.0 + math.exp(-float(np.float32(logit))))
    om = o * sf ** 2 / (sf ** 2 + lam) * np.exp(-D / 2)
    np.testing.assert_allclose(out["T"], _single_T(om), rtol=1e-12, atol=1e-14)
    assert np.count_nonzero(out["ncontrib"]) > 100
    assert (lam / sf ** 2).max() > 0.5  # the smoothing is not negligible here


def test_mip_exact_tangent_plane_restatement(oracle_lib):
    """The appendix's tangent-plane form, restated independently: an orthonormal F with
    F^T xh = 0 (numpy null space), A = F^T Sigma F, A^ = A + lambda I, D = (F^T mu)^T A^-1
    (F^T mu), modulation sqrt(det A / det A^), Sigma from scipy's rotation, tau from
    np.linalg.inv(Sigma).  It equals the oracle's eigenframe evaluation of D_ray(x; mu,
    Sigma^_x) and sqrt(|Sigma| x^T Sigma^-1 x / (|Sigma^_x| x^T Sigma^_x^-1 x))."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(31)
    cam = scenes.make_camera(40, 36, 30.0, 26.0, 19.5, 18.0, mip="exact")
    sig2 = 25.0
    checked = 0
    for _ in range(10):
        mu = np.float32(np.array([*rng.uniform(-0.3, 0.3, 2), rng.uniform(1.5, 3.0)]))
        ls = np.float32(np.log(rng.uniform(0.02, 0.2, 3)))
        q = np.float32(rand_rot(rng))
        sc = single(mu, ls, q, 1.5, [1, 1, 1])
        out = oracle_lib.render(sc, cam, cfg=dict(mip_sigma2=sig2))
        Rq = Rot.from_quat(q.astype(np.float64)[[1, 2, 3, 0]]).as_matrix()
        S = Rq @ np.diag(np.exp(2 * ls.astype(np.float64))) @ Rq.T
        Si = np.linalg.inv(S)
        m = mu.astype(np.float64)
        o = 1.0 / (1.0 + math.exp(-float(np.float32(1.5))))
        T = np.ones(40 * 36)
        for p in range(40 * 36):
            jj, ii = divmod(p, 40)
            x = np.array([(ii + 0.5 - 19.5) / 30.0, (jj + 0.5 - 18.0) / 26.0, 1.0])
            xh = x / np.linalg.norm(x)
            tau = (m @ Si @ xh) / (xh @ Si @ xh)
            if tau <= 0:
                continue
            lam = sig2 * (1.0 / np.linalg.norm(x)) ** 3 * tau ** 2 / (30.0 * 26.0)
            Sh = S + lam * np.eye(3)
            Shi = np.linalg.inv(Sh)
            if (m @ Shi @ xh) <= 0:
                continue
            F = np.linalg.svd(xh[None, :])[2][1:].T          # 3x2, orthonormal, F^T xh = 0
            A = F.T @ S @ F
            Ah = A + lam * np.eye(2)
            pp = F.T @ m
            D = pp @ np.linalg.solve(Ah, pp)
            om = o * math.sqrt(np.linalg.det(A) / np.linalg.det(Ah)) * math.exp(-D / 2)
            if abs(om - PMIN) < 1e-9:
                continue
            T[p] = _single_T(np.array(om))
        np.testing.assert_allclose(out["T"], T, rtol=1e-9, atol=1e-12)
        checked += np.count_nonzero(out["ncontrib"])
    assert checked > 500


def test_mip_exact_limits(oracle_lib):
    """sigma -> 0 gives the plain image; on the optical axis, at the pixel whose ray passes
    through the mean, the exact form equals the pixel-invariant Eq. mip (tau = |mu|,
    cos(theta) = 1, x ∝ mu so x^T Sigma^-1 x / x^T Sigma^^-1 x = c^2 / c^^2 and D = 0)."""
    sc, cams = scenes.workload_small()
    cam = dict(cams[0])
    plain = oracle_lib.render(sc, cam)
    zero = oracle_lib.render(sc, dict(cam, mip="exact"), cfg=dict(mip_sigma2=0.0))
    np.testing.assert_allclose(zero["rgb"], plain["rgb"], rtol=1e-10, atol=1e-13)
    np.testing.assert_array_equal(zero["ncontrib"], plain["ncontrib"])
    rng = np.random.default_rng(8)
    for _ in range(5):
        one = single([0.0, 0.0, rng.uniform(2, 4)], np.log(rng.uniform(0.002, 0.02, 3)), rand_rot(rng), 0.8,
                     [1, 1, 1])
        c1 = scenes.make_camera(1, 1, 64.0, 64.0, 0.5, 0.5)
        ex = oracle_lib.render(one, dict(c1, mip="exact"), cfg=dict(mip_sigma2=2.0))
        ap = oracle_lib.render(one, dict(c1, mip=True), cfg=dict(mip_sigma2=2.0))
        pl = oracle_lib.render(one, c1)
        assert ex["T"][0] == pytest.approx(ap["T"][0], rel=1e-12)
        assert ex["T"][0] > pl["T"][0]  # the smoothing lowers the peak opacity
