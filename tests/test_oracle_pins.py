"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: finite
differences (brute force), Hamilton's equations, closed forms of uniform media,
invariants of symmetric backgrounds with their third-order convergence, the
values the source profile takes (Sec. 3c), and exact algebraic consequences of
the saturation and projection formulas.  A plausible slip in the oracle (a
dropped metric term, a sign, a transposed flux index) fails one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2309_11257_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


# ------------------------------------------------------------------ helpers

def linear_background(grid, u0=5.0, du=(2e-5, -1e-5, 1e-3), v0=-2.0, dv=(-1e-5, 3e-5, -5e-4),
                      n20=4e-4, dn2=(1e-10, -2e-10, 1e-9), rho0=1.0, H=7000.0):
    x, y, z = synth.node_coords(grid)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    u = u0 + du[0] * X + du[1] * Y + du[2] * Z
    v = v0 + dv[0] * X + dv[1] * Y + dv[2] * Z
    n2 = n20 + dn2[0] * X + dn2[1] * Y + dn2[2] * Z
    rho = rho0 * np.exp(-Z / H)
    return u, v, n2, rho


def model(grid, params=None, bg=None):
    p = dict(synth.DEFAULT_PARAMS)
    if params:
        p.update(params)
    M = oracle.Model(grid, p)
    if bg is not None:
        M.set_background(*bg)
    return M


def fd(fun, x, h):
    return (fun(x + h) - fun(x - h)) / (2.0 * h)


# ------------------------------------------------------------------ dispersion relation (Eq. dispersion)

def _rand_wave(g):
    k, l, m = g.normal(size=3) * 10.0 ** g.uniform(-5.5, -3.5, 3)
    n2 = 10.0 ** g.uniform(-4.5, -3.3)
    f2 = n2 * g.uniform(0.0, 0.3) ** 2
    g2 = 10.0 ** g.uniform(-10, -7)
    return k, l, m, n2, g2, f2


def test_intrinsic_frequency_between_f_and_N():
    g = np.random.default_rng(11)
    for _ in range(500):
        k, l, m, n2, g2, f2 = _rand_wave(g)
        w = oracle.dispersion(k, l, m, n2, g2, f2)[0]
        assert f2 * (1 - 1e-13) <= w * w <= n2 * (1 + 1e-13)


def test_textbook_limits():
    # non-rotating, no scale-height correction: w = N |k_h| / |k|
    for (k, l, m) in [(1e-4, 0, -1e-3), (3e-5, 4e-5, -2e-4), (1e-3, -1e-3, 5e-4)]:
        w = oracle.dispersion(k, l, m, 4e-4, 0.0, 0.0)[0]
        assert w == pytest.approx(0.02 * math.hypot(k, l) / math.sqrt(k * k + l * l + m * m), rel=1e-14)
    # purely vertical wavevector: inertial oscillation w = |f|
    assert oracle.dispersion(0.0, 0.0, -1e-3, 4e-4, 0.0, 1e-8)[0] == pytest.approx(1e-4, rel=1e-14)
    # purely horizontal wavevector, Gamma = 0: buoyancy oscillation w = N
    assert oracle.dispersion(1e-4, 2e-4, 0.0, 4e-4, 0.0, 1e-8)[0] == pytest.approx(0.02, rel=1e-14)


def test_group_velocity_is_grad_k_of_frequency():
    g = np.random.default_rng(12)
    for _ in range(200):
        k, l, m, n2, g2, f2 = _rand_wave(g)
        ch = oracle.dispersion(k, l, m, n2, g2, f2)[1:4]
        scale = np.linalg.norm(ch) + 1e-30
        kk = np.array([k, l, m])
        hh = 1e-6 * np.linalg.norm(kk)
        for q in range(3):
            def w_of(t, q=q):
                v = kk.copy()
                v[q] = t
                return oracle.dispersion(v[0], v[1], v[2], n2, g2, f2)[0]
            assert abs(fd(w_of, kk[q], hh) - ch[q]) <= 1e-6 * scale


def test_frequency_homogeneity_and_euler_identity():
    # w(s k, s Gamma) = w(k, Gamma)  =>  k . grad_k w = -Gamma dw/dGamma = -2 Gamma^2 dw/d(Gamma^2)
    g = np.random.default_rng(13)
    for _ in range(200):
        k, l, m, n2, g2, f2 = _rand_wave(g)
        s = 10.0 ** g.uniform(-1, 1)
        w = oracle.dispersion(k, l, m, n2, g2, f2)
        ws = oracle.dispersion(s * k, s * l, s * m, n2, s * s * g2, f2)
        assert ws[0] == pytest.approx(w[0], rel=1e-13)
        kdotc = k * w[1] + l * w[2] + m * w[3]
        dw_dg2 = fd(lambda t: oracle.dispersion(k, l, m, n2, t, f2)[0], g2, 1e-4 * g2)
        assert kdotc == pytest.approx(-2.0 * g2 * dw_dg2, rel=1e-5, abs=1e-9 * abs(w[1]) + 1e-30)


# ------------------------------------------------------------------ refraction: Hamilton's equations

def test_cartesian_ray_equations_are_hamiltonian():
    grid = synth.fplane_grid(nx=32, ny=32, nz=40, dx=50e3, dy=37e3, dz=500.0)
    M = model(grid, bg=linear_background(grid))
    g = np.random.default_rng(21)
    for _ in range(20):
        X = (g.integers(8, 24) + g.uniform(0.6, 1.4)) * grid["dx"]
        Y = (g.integers(8, 24) + g.uniform(0.6, 1.4)) * grid["dy"]
        Z = (g.integers(8, 30) + g.uniform(0.6, 1.4)) * grid["dz"]
        k, l = (2 * math.pi / 3e5 * g.normal(size=2)).tolist()
        m = -2 * math.pi / 3e3
        F = M.rhs([X, Y, Z, k, l, m, 0.0, 0.0, 0.0])
        # xdot = dOmega/dk, kdot = -dOmega/dx
        pos = [X, Y, Z]
        wav = [k, l, m]
        for q in range(3):
            def om_k(t, q=q):
                w = list(wav); w[q] = t
                return M.omega(*pos, *w)
            def om_x(t, q=q):
                p = list(pos); p[q] = t
                return M.omega(*p, *wav)
            hk = 1e-6 * abs(m)
            hx = [1.0, 1.0, 0.1][q]
            assert F[q] == pytest.approx(fd(om_k, wav[q], hk), rel=1e-6, abs=1e-9)
            assert F[3 + q] == pytest.approx(-fd(om_x, pos[q], hx), rel=1e-5, abs=1e-14)
        assert np.all(F[6:] == 0.0)


def _sphere_bg(grid):
    u, v, n2, rho = synth.perturbed(synth.jet_background(grid), tag=5)
    return u, v, n2, rho


def _sphere_linear_bg(grid):
    """Linear in lambda, phi and z (exactly represented by the interpolated node gradients away
    from the periodic seam); density exp(-z sqrt(g0 + g1 phi)) so that Gamma^2 = (g0 + g1 phi)/4
    is linear in phi as well."""
    x, y, z = synth.node_coords(grid)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    u = 5.0 + 3.0 * X + 20.0 * Y + 1e-3 * Z
    v = -2.0 + 1.5 * X - 10.0 * Y - 5e-4 * Z
    n2 = 4e-4 + 1e-5 * X + 2e-5 * Y + 1e-9 * Z
    g0 = 1.0 / 7000.0 ** 2
    rho = 1.2 * np.exp(-Z * np.sqrt(g0 * (1.0 + 0.3 * Y)))
    return u, v, n2, rho


def _canonical(M, a):
    """Hamiltonian in canonical coordinates (lambda, phi, r, p_lambda = r cos(phi) k, p_phi = r l, p_r = m)."""
    def H(q):
        lam, phi, r, pl, pp, pr = q
        return M.omega(lam, phi, r - a, pl / (r * math.cos(phi)), pp / r, pr)
    return H


def _canonical_rates(M, a, q):
    """(lambda, phi, r, p)-rates from the oracle's ray equations (zero extents)."""
    lam, phi, r, pl, pp, pr = q
    k, l, m = pl / (r * math.cos(phi)), pp / r, pr
    F = M.rhs([lam, phi, r - a, k, l, m, 0.0, 0.0, 0.0])
    lamd, phid, zd, kd, ld, md = F[:6]
    pld = zd * math.cos(phi) * k - r * math.sin(phi) * phid * k + r * math.cos(phi) * kd
    ppd = zd * l + r * ld
    return np.array([lamd, phid, zd, pld, ppd, md])


def test_spherical_ray_equations_are_hamiltonian():
    """Eq. eikonal-sphere:1-3 with their metric terms equal Hamilton's equations in canonical
    momenta (r cos(phi) k_lambda, r k_phi, k_r), checked by finite differences of Omega."""
    grid = synth.sphere_grid(nx=64, ny=40, nz=30, dz=1000.0)
    M = model(grid, bg=_sphere_linear_bg(grid))
    a = grid["radius"]
    H = _canonical(M, a)
    g = np.random.default_rng(22)
    dlam, dphi = 2 * math.pi / 64, math.pi / 40
    for _ in range(20):
        lam = (g.integers(2, 60) + g.uniform(0.6, 1.4)) * dlam
        phi = -0.5 * math.pi + (g.integers(6, 32) + g.uniform(0.6, 1.4)) * dphi
        r = a + (g.integers(3, 25) + g.uniform(0.6, 1.4)) * 1000.0
        k, l = 2 * math.pi / 3e5 * g.normal(size=2)
        m = -2 * math.pi / 4e3
        q0 = np.array([lam, phi, r, r * math.cos(phi) * k, r * l, m])
        rates = _canonical_rates(M, a, q0)
        hs = [1e-7, 1e-7, 0.05, 1e-6 * abs(q0[3]) + 1e-12, 1e-6 * abs(q0[4]) + 1e-12, 1e-6 * abs(m)]
        grad = np.zeros(6)
        for c in range(6):
            def Hc(t, c=c):
                qq = q0.copy(); qq[c] = t
                return H(qq)
            grad[c] = fd(Hc, q0[c], hs[c])
        expect = np.concatenate([grad[3:], -grad[:3]])
        for c in range(6):
            sc = np.abs(expect[c]) + 1e-6 * np.abs(expect).max()
            assert abs(rates[c] - expect[c]) <= 1e-5 * sc, (c, rates[c], expect[c])


def test_phase_space_velocity_is_divergence_free():
    """Eq. vpvel_nondiv and, in Cartesian coordinates, per axis (Eq. vpvol_cons_cart)."""
    grid = synth.fplane_grid(nx=32, ny=32, nz=40, dz=500.0)
    M = model(grid, bg=linear_background(grid))
    y0 = np.array([15.7 * grid["dx"], 16.2 * grid["dy"], 20.3 * grid["dz"], 2e-5, -1.5e-5, -2e-3, 0, 0, 0])
    hs = [1.0, 1.0, 0.1, 1e-10, 1e-10, 1e-8]
    for ax in range(3):
        d_pos = fd(lambda t: M.rhs(np.r_[y0[:ax], t, y0[ax + 1:]])[ax], y0[ax], hs[ax])
        d_wav = fd(lambda t: M.rhs(np.r_[y0[:3 + ax], t, y0[4 + ax:]])[3 + ax], y0[3 + ax], hs[3 + ax])
        assert abs(d_pos + d_wav) <= 1e-6 * (abs(d_pos) + abs(d_wav)) + 1e-20
    # sphere, canonical coordinates
    gs = synth.sphere_grid(nx=64, ny=40, nz=30, dz=1000.0)
    Ms = model(gs, bg=_sphere_linear_bg(gs))
    a = gs["radius"]
    q0 = np.array([1.1, 0.4, a + 12345.0, 0.0, 0.0, -1.5e-3])
    q0[3] = q0[2] * math.cos(q0[1]) * 2e-5
    q0[4] = q0[2] * -1e-5
    hs = [1e-7, 1e-7, 0.05, 1e-6 * abs(q0[3]), 1e-6 * abs(q0[4]), 1e-6 * abs(q0[5])]
    div, mag = 0.0, 0.0
    for c in range(6):
        def rc(t, c=c):
            qq = q0.copy(); qq[c] = t
            return _canonical_rates(Ms, a, qq)[c]
        d = fd(rc, q0[c], hs[c])
        div += d
        mag += abs(d)
    assert abs(div) <= 1e-5 * mag


def test_face_difference_is_the_compression_rate():
    """For small ray volumes the face difference of the group velocity tends to dX * d(Xdot)/dX."""
    grid = synth.fplane_grid(nx=32, ny=32, nz=40, dx=50e3, dy=37e3, dz=500.0)
    M = model(grid, bg=linear_background(grid))
    y0 = np.array([15.7 * grid["dx"], 16.2 * grid["dy"], 20.3 * grid["dz"], 2e-5, -1.5e-5, -2e-3, 0, 0, 0])
    ext = [50.0, 50.0, 1.0]
    hs = [1.0, 1.0, 0.1]
    y = y0.copy()
    y[6:] = ext
    F = M.rhs(y)
    for ax in range(3):
        dv = fd(lambda t: M.rhs(np.r_[y0[:ax], t, y0[ax + 1:]])[ax], y0[ax], hs[ax])
        assert F[6 + ax] == pytest.approx(ext[ax] * dv, rel=1e-5, abs=1e-18)


def test_carrier_advance_is_mirror_symmetric():
    """The ray volume has no preferred side: mirroring the background about the carrier
    (x -> 2 x0 - x, U -> -U) and the wave (k -> -k) mirrors the carrier velocity and keeps the
    extent rates, for finite extents in a background varying along every axis."""
    grid = synth.fplane_grid(nx=32, ny=32, nz=40, dx=50e3, dy=37e3, dz=500.0)
    x, y, z = synth.node_coords(grid)
    x0 = x[16]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    shape = Z.shape
    n2a = 4e-4 + 3e-9 * (X - x0) + 1e-10 * (Y - y[16]) + 2e-9 * (Z - z[20])
    n2b = 4e-4 - 3e-9 * (X - x0) + 1e-10 * (Y - y[16]) + 2e-9 * (Z - z[20])
    ua = 2.0 + 4e-5 * (X - x0) + 1e-3 * (Z - z[20])
    ub = -(2.0 - 4e-5 * (X - x0) + 1e-3 * (Z - z[20]))
    rho = np.exp(-Z / 7e3)
    Ma = model(grid, None, (ua, np.zeros(shape), n2a, rho))
    Mb = model(grid, None, (ub, np.zeros(shape), n2b, rho))
    ya = np.array([x0, y[16] + 0.3 * 37e3, z[20] + 0.2 * 500.0, 2e-5, -1.5e-5, -2e-3, 40e3, 30e3, 400.0])
    yb = ya.copy()
    yb[3] = -ya[3]
    Fa, Fb = Ma.rhs(ya), Mb.rhs(yb)
    assert Fb[0] == pytest.approx(-Fa[0], rel=1e-12)
    for q in (1, 2, 6, 7, 8):
        assert Fb[q] == pytest.approx(Fa[q], rel=1e-12, abs=1e-300)
    assert Fa[6] != 0.0 and Fa[8] != 0.0


# ------------------------------------------------------------------ integrated ray paths

def test_uniform_background_straight_lines():
    """f-plane workload: uniform background, so k, N and the extents are constant and
    x(t) = x0 + c_g t with c_g = ch + U (the straight-line closed form), after 100 steps."""
    w = synth.workload("fplane")
    M = model(w["grid"], w["params"], w["background"])
    rays = w["rays"]
    M.add_rays(rays)
    r0 = M.rays()
    T = 0.0
    for _ in range(w["steps"]):
        M.step(w["dt"])
        T += w["dt"]
    r1 = M.rays()
    assert 0 < len(r1["id"]) <= len(r0["id"])
    src = {int(i): q for q, i in enumerate(r0["id"])}
    q0 = np.array([src[int(i)] for i in r1["id"]])
    G = w["grid"]
    Lx, Ly = G["nx"] * G["dx"], G["ny"] * G["dy"]
    U, V, N2 = 10.0, 0.0, 4e-4
    g2 = 0.25 / 7000.0 ** 2
    for name in ("n", "px", "py", "pz"):
        np.testing.assert_array_equal(r1[name], r0[name][q0])
    # Gamma^2 from finite differences of ln(rho) is constant only to rounding
    for name in ("k", "l", "m", "ex", "ey", "ez"):
        np.testing.assert_allclose(r1[name], r0[name][q0], rtol=1e-12)
    for q, j in enumerate(q0):
        d = oracle.dispersion(r0["k"][j], r0["l"][j], r0["m"][j], N2, g2, G["f0"] ** 2)
        xe = (r0["x"][j] + (d[1] + U) * T) % Lx
        ye = (r0["y"][j] + (d[2] + V) * T) % Ly
        ze = r0["z"][j] + d[3] * T
        dxp = (r1["x"][q] - xe + 0.5 * Lx) % Lx - 0.5 * Lx
        dyp = (r1["y"][q] - ye + 0.5 * Ly) % Ly - 0.5 * Ly
        assert abs(dxp) <= 1e-12 * Lx and abs(dyp) <= 1e-12 * Ly
        assert abs(r1["z"][q] - ze) <= 1e-12 * G["nz"] * G["dz"]
    st = M.stats()
    assert st["n_exited"] + st["n_live"] == 4096 and st["n_split_v"] == st["n_split_h"] == 0


def _cart(lam, phi, z, k, l, m, a):
    r = a + z
    er = np.array([math.cos(phi) * math.cos(lam), math.cos(phi) * math.sin(lam), math.sin(phi)])
    el = np.array([-math.sin(lam), math.cos(lam), 0.0])
    ep = np.array([-math.sin(phi) * math.cos(lam), -math.sin(phi) * math.sin(lam), math.cos(phi)])
    return r * er, k * el + l * ep + m * er


def _integrate(M, y, dt, T):
    y = np.array(y, dtype=float)
    for _ in range(int(round(T / dt))):
        y = M.rk3(y, dt)
    return y


def _order(errs):
    return [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]


def test_great_circles_in_a_uniform_atmosphere_at_rest():
    """Sec. 2a: with U = 0, f = 0 and N, Gamma functions of r only, the metric terms keep the
    ray on a great circle: L = r x k is conserved (to RK3 truncation, third order in dt)."""
    grid = synth.sphere_grid(nx=32, ny=16, nz=12, dz=10000.0, omega=0.0)
    shape = (12, 16, 32)
    bg = (np.zeros(shape), np.zeros(shape), np.full(shape, 4e-4), np.ones(shape))
    M = model(grid, dict(gamma_mode=0), bg)
    a = grid["radius"]
    y0 = [1.0, 0.3, 30e3, 2 * math.pi / 2e5, 2 * math.pi / 3e5, -2 * math.pi / 20e3, 0.0, 0.0, 0.0]
    L0 = np.cross(*_cart(*y0[:6], a))
    errs = []
    for dt in (1600.0, 800.0, 400.0):
        y = _integrate(M, y0, dt, 64000.0)
        L = np.cross(*_cart(*y[:6], a))
        errs.append(np.linalg.norm(L - L0) / np.linalg.norm(L0))
    assert errs[-1] < 1e-7
    for r in _order(errs):
        assert 6.0 < r < 10.0, errs
    # the ray actually travelled a good fraction of a radian
    assert abs(y[0] - y0[0]) > 0.05


def test_steady_background_conserves_frequency():
    """Steady background: the Hamiltonian Omega = k.U + w is constant along rays (third order)."""
    grid = synth.fplane_grid(nx=56, ny=56, nz=40, dz=500.0, f0=1e-4)
    M = model(grid, bg=linear_background(grid))
    y0 = [20.3 * grid["dx"], 19.6 * grid["dy"], 15.2 * grid["dz"], 2 * math.pi / 2e5, -2 * math.pi / 4e5,
          -2 * math.pi / 3e3, 0.0, 0.0, 0.0]
    O0 = M.omega(*y0[:6])
    errs = []
    for dt in (1200.0, 600.0, 300.0):
        y = _integrate(M, y0, dt, 24000.0)
        errs.append(abs(M.omega(*y[:6]) - O0) / abs(O0))
    assert errs[-1] < 1e-7
    for r in _order(errs):
        assert 7.0 < r < 9.0, errs


def test_zonal_symmetry_conserves_angular_momentum():
    """Zonally symmetric background: p_lambda = r cos(phi) k_lambda is conserved (third order)."""
    grid = synth.sphere_grid(nx=32, ny=64, nz=40, dz=1000.0)
    x, phi, z = synth.node_coords(grid)
    Z, P, _ = np.meshgrid(z, phi, x, indexing="ij")
    u = 10.0 + 20.0 * P + 5e-4 * Z
    v = np.zeros_like(u)
    n2 = 3.5e-4 + 2e-10 * Z + 2e-5 * P
    rho = 1.2 * np.exp(-Z / 7000.0)
    M = model(grid, None, (u, v, n2, rho))
    a = grid["radius"]
    y0 = [1.0, 0.5, 15e3, 2 * math.pi / 1.5e5, 2 * math.pi / 3e5, -2 * math.pi / 5e3, 0.0, 0.0, 0.0]
    p0 = (a + y0[2]) * math.cos(y0[1]) * y0[3]
    errs = []
    for dt in (800.0, 400.0, 200.0):
        y = _integrate(M, y0, dt, 16000.0)
        errs.append(abs((a + y[2]) * math.cos(y[1]) * y[3] - p0) / abs(p0))
    assert errs[-1] < 1e-9
    for r in _order(errs):
        assert 5.5 < r < 10.5, errs


def test_x_independent_background_keeps_k_exactly():
    grid = synth.fplane_grid(nx=16, ny=16, nz=40)
    x, y, z = synth.node_coords(grid)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    u = 10 + 10 * np.sin(2 * math.pi * Y / (16 * 50e3)) * np.exp(-((Z - 10e3) / 4e3) ** 2)
    bg = (u, np.zeros_like(u), np.full_like(u, 4e-4), np.exp(-Z / 7e3))
    M = model(grid, dict(saturation=0, smoothing=0), bg)
    r = synth.fplane_rays(grid, 64, tag=3)
    M.add_rays(r)
    k0 = dict(zip(M.rays()["id"], M.rays()["k"]))
    for _ in range(10):
        M.step(300.0)
    r1 = M.rays()
    for i, k in zip(r1["id"], r1["k"]):
        assert k == k0[i]


def test_extents_conserved_at_rest():
    """Sec. 3a: in a uniform atmosphere at rest the coordinate extents are exactly conserved."""
    grid = synth.sphere_grid(nx=32, ny=16, nz=20, dz=1000.0, omega=0.0)
    shape = (20, 16, 32)
    bg = (np.zeros(shape), np.zeros(shape), np.full(shape, 4e-4), np.ones(shape))
    M = model(grid, dict(gamma_mode=0, saturation=0, smoothing=0, splitting=0), bg)
    r = synth.sphere_rays(grid, 50, tag=7, z_lo=3e3, z_hi=6e3)
    M.add_rays(r)
    r0 = M.rays()
    for _ in range(5):
        M.step(300.0)
    r1 = M.rays()
    src = {int(i): q for q, i in enumerate(r0["id"])}
    q0 = [src[int(i)] for i in r1["id"]]
    for name in ("ex", "ey", "ez"):
        np.testing.assert_array_equal(r1[name], r0[name][q0])


# ------------------------------------------------------------------ background pieces

def test_gamma_of_isothermal_atmosphere():
    grid = synth.sphere_grid(nx=8, ny=8, nz=30)
    bg = synth.jet_background(grid)
    M = model(grid, None, bg)
    _, H, _ = synth.isothermal(240.0)
    np.testing.assert_allclose(M.gamma2(), 0.25 / H ** 2, rtol=1e-10)
    M0 = model(grid, dict(gamma_mode=0), bg)
    assert np.all(M0.gamma2() == 0.0)


def test_gather_reproduces_linear_fields():
    grid = synth.fplane_grid(nx=32, ny=32, nz=40, dx=50e3, dy=37e3, dz=500.0)
    M = model(grid, bg=linear_background(grid))
    X, Y, Z = 15.37 * 50e3, 16.81 * 37e3, 20.44 * 500.0
    b = M.gather(X, Y, Z)
    assert b[0] == pytest.approx(5.0 + 2e-5 * X - 1e-5 * Y + 1e-3 * Z, rel=1e-13)
    np.testing.assert_allclose(b[4:7], [2e-5, -1e-5, 1e-3], rtol=1e-9)
    np.testing.assert_allclose(b[10:13], [1e-10, -2e-10, 1e-9], rtol=1e-8)


# ------------------------------------------------------------------ sources (Sec. 3c)

def test_source_profile_matches_the_paper():
    rows = np.loadtxt(os.path.join(HERE, "golden", "source_profile.txt"))
    for phi, alpha, fsol in rows:
        assert oracle.alpha_profile(phi) == pytest.approx(alpha, abs=1e-15)
        assert oracle.fam(phi, 0.0, 2.4e-3, 8e-3) == pytest.approx(fsol, abs=1e-15)
        # half a year later the hemispheres swap
        assert oracle.fam(-phi, math.pi, 2.4e-3, 8e-3) == pytest.approx(fsol, abs=1e-15)


def test_launch_counts_and_slab_flux():
    """Sphere workload: all 32 bins launch in the 120 rows with |phi| <= 85 deg, and the
    vertical pseudomomentum flux of one spectral launch integrates to F dz_launch."""
    grid = synth.sphere_grid(nx=16, ny=128, nz=20)
    bg = synth.jet_background(grid)
    M = model(grid, dict(saturation=0, smoothing=0), bg)
    M.launch_background(synth.background_source())
    st = M.stats()
    assert st["n_launched"] == 120 * 16 * 32 and st["n_filtered"] == 0
    # single spectral bins on an f-plane at rest
    gf = synth.fplane_grid(nx=8, ny=8, nz=20, dz=500.0)
    bgf = synth.uniform_background(gf, U=0.0)
    for form in (1, 0):
        Mf = model(gf, dict(flux_form=form, smoothing=0, saturation=0), bgf)
        spec = np.zeros(1, dtype=synth.SPEC_DTYPE)
        spec[0] = (3, 4, 0, 2000.0, 1000.0, 0.7, 20.0, 1e5, 3e-3, 0.1)
        Mf.launch_spectral(spec)
        Mf.diagnose()
        fz_l, fz_p = Mf.field("fz_l"), Mf.field("fz_p")
        r = Mf.rays()
        d = oracle.dispersion(r["k"][0], r["l"][0], r["m"][0], 4e-4, 0.25 / 7000.0 ** 2, 1e-8)
        factor = 1.0 if form == 1 else d[0] ** 2 / (d[0] ** 2 - 1e-8)
        assert fz_l[:, 4, 3].sum() * 500.0 == pytest.approx(3e-3 * math.cos(0.7) * 1000.0 * factor, rel=1e-12)
        assert fz_p[:, 4, 3].sum() * 500.0 == pytest.approx(3e-3 * math.sin(0.7) * 1000.0 * factor, rel=1e-12)


def test_launch_filters_evanescent_bins():
    gf = synth.fplane_grid(nx=8, ny=8, nz=20, dz=500.0)
    M = model(gf, None, synth.uniform_background(gf, U=0.0))
    spec = np.zeros(3, dtype=synth.SPEC_DTYPE)
    spec[0] = (1, 1, 0, 2000.0, 1000.0, 0.0, 400.0, 1e5, 1e-3, 0.1)   # w > N
    spec[1] = (1, 1, 0, 2000.0, 1000.0, 0.0, 0.1, 1e5, 1e-3, 0.1)     # w < f
    spec[2] = (1, 1, 0, 2000.0, 1000.0, 0.0, 20.0, 1e5, 1e-3, 0.1)    # propagating
    M.launch_spectral(spec)
    st = M.stats()
    assert st["n_filtered"] == 2 and st["n_launched"] == 1


# ------------------------------------------------------------------ saturation (Sec. 3c)

def test_monochromatic_saturation_threshold():
    """Eq. instability-threshold reduces to |B|^2 < N^4 / m^2 for one monochromatic wave:
    with E = rho |B|^2 / (2 N^2) and A = E / w, a ray filling its cell exactly at that
    amplitude has P = rho / 2."""
    grid = synth.fplane_grid(nx=8, ny=8, nz=20, dz=500.0, f0=0.0)
    shape = (20, 8, 8)
    N2, rho = 4e-4, 0.9
    bg = (np.zeros(shape), np.zeros(shape), np.full(shape, N2), np.full(shape, rho))
    M = model(grid, dict(gamma_mode=0), bg)
    k, l, m = 2 * math.pi / 2e5, 2 * math.pi / 4e5, -2 * math.pi / 3e3
    w = oracle.dispersion(k, l, m, N2, 0.0, 0.0)[0]
    B2 = N2 ** 2 / m ** 2
    A = rho * B2 / (2 * N2) / w
    dk, dl, dm = 1e-6, 1e-6, 1e-4
    M.add_rays(dict(x=[3.5 * 50e3], y=[2.5 * 50e3], z=[7.5 * 500.0], k=[k], l=[l], m=[m], ex=[50e3],
                    ey=[50e3], ez=[500.0], dk=[dk], dl=[dl], dm=[dm], n=[A / (dk * dl * dm)]))
    P, _ = M.cell_pq()
    assert P[7, 2, 3] == pytest.approx(rho / 2, rel=1e-12)
    assert np.count_nonzero(P) == 1


def test_saturation_brings_cells_exactly_to_threshold():
    grid = synth.fplane_grid(nx=8, ny=8, nz=20, dz=500.0)
    bg = synth.uniform_background(grid, U=0.0)
    M = model(grid, dict(saturation=1, smoothing=0, splitting=0), bg)
    g = np.random.default_rng(31)
    n = 12
    kh = 2 * math.pi / 2e5 * g.uniform(0.9, 1.1, n)
    az = g.uniform(0, 2 * math.pi, n)
    m = -2 * math.pi / 3e3 * g.uniform(0.9, 1.1, n)
    r = dict(x=np.full(n, 3.5 * 50e3), y=np.full(n, 2.5 * 50e3), z=np.full(n, 7.5 * 500.0),
             k=kh * np.cos(az), l=kh * np.sin(az), m=m, ex=np.full(n, 25e3), ey=np.full(n, 25e3),
             ez=np.full(n, 200.0), dk=0.1 * kh, dl=0.1 * kh, dm=0.1 * np.abs(m),
             n=np.full(n, 5e19))
    M.add_rays(r)
    P0, _ = M.cell_pq()
    rho_c = bg[3]
    assert (P0 > 0.5 * rho_c).any()
    w0 = M.stats()["w_total"]
    M.step(60.0)
    P1, _ = M.cell_pq()
    st = M.stats()
    assert st["w_saturated"] > 0
    hit = P1 > 0
    assert np.all(P1[hit] <= 0.5 * rho_c[hit] * (1 + 1e-12))
    sat_cells = np.argwhere(P1 >= 0.5 * rho_c * (1 - 1e-6))
    assert len(sat_cells) >= 1
    for c in sat_cells:
        assert P1[tuple(c)] == pytest.approx(0.5 * rho_c[tuple(c)], rel=1e-12)
    assert st["w_total"] == pytest.approx(w0 - st["w_saturated"] - st["w_exited"], rel=1e-13)


# ------------------------------------------------------------------ projection and tendencies

def _cell_volumes(grid):
    _, y, z = synth.node_coords(grid)
    nx, ny, nz = grid["nx"], grid["ny"], grid["nz"]
    if grid["geometry"] == 1:
        rc = grid["radius"] + z
        vol = (rc ** 2)[:, None] * np.cos(y)[None, :] * (2 * math.pi / nx) * (math.pi / ny) * grid["dz"]
        return np.broadcast_to(vol[:, :, None], (nz, ny, nx))
    return np.full((nz, ny, nx), grid["dx"] * grid["dy"] * grid["dz"])


def test_projected_wave_action_equals_ray_content():
    grid = synth.sphere_grid(nx=32, ny=16, nz=20)
    M = model(grid, dict(smoothing=0, saturation=0), _sphere_bg(grid))
    M.add_rays(synth.sphere_rays(grid, 300, tag=8))
    M.step(180.0)
    wad = M.field("wad")
    total = (wad * _cell_volumes(grid)).sum()
    assert total == pytest.approx(M.stats()["w_total"], rel=1e-12)


def test_single_ray_fluxes_without_rotation():
    """f = 0: the direct fluxes equal the pseudomomentum fluxes, and the vertical flux of a ray
    integrates to k ch_r A w_h dZ over the interfaces."""
    grid = synth.fplane_grid(nx=8, ny=8, nz=30, dz=500.0, f0=0.0)
    bg = synth.uniform_background(grid, U=3.0)
    ray = dict(x=[3.3 * 50e3], y=[5.6 * 50e3], z=[6200.0], k=[3e-5], l=[-2e-5], m=[-2e-3], ex=[30e3], ey=[20e3],
               ez=[1300.0], dk=[3e-6], dl=[2e-6], dm=[2e-4], n=[1e10])
    fields = []
    for form in (0, 1):
        M = model(grid, dict(flux_form=form, smoothing=0, saturation=0, splitting=0), bg)
        M.add_rays(ray)
        M.diagnose()
        fields.append({n: M.field(n) for n in oracle.FIELD_NAMES})
    for n in oracle.FIELD_NAMES:
        np.testing.assert_allclose(fields[0][n], fields[1][n], rtol=1e-13, atol=1e-300)
    d = oracle.dispersion(3e-5, -2e-5, -2e-3, 4e-4, 0.25 / 7000.0 ** 2, 0.0)
    A = 1e10 * 3e-6 * 2e-6 * 2e-4
    wh = 30e3 * 20e3 / (50e3 * 50e3)
    assert fields[0]["fz_l"].sum() * 500.0 == pytest.approx(3e-5 * d[3] * A * wh * 1300.0, rel=1e-12)
    assert fields[0]["fz_p"].sum() * 500.0 == pytest.approx(-2e-5 * d[3] * A * wh * 1300.0, rel=1e-12)
    assert np.all(fields[0]["e_l"] == 0.0)


def _plane_wave_moments(k, m, N2, f, w, u_amp=1.0):
    """Second moments of a plane inertia-gravity wave with wavevector (k, 0, m) from the linear
    Boussinesq equations: v' = -i (f/w) u', w' = -(k/m) u', b' = -i (N^2/w) w'."""
    u = u_amp + 0j
    v = -1j * f / w * u
    ww = -(k / m) * u
    b = -1j * N2 / w * ww
    mom = lambda a, c: 0.5 * (a * np.conj(c)).real
    return dict(uu=mom(u, u), vv=mom(v, v), uv=mom(u, v), wu=mom(ww, u), wv=mom(ww, v),
                ub=mom(u, b), vb=mom(v, b))


def test_fluxes_follow_plane_wave_polarization():
    """Direct fluxes (Eq. fluxes:momentum) and elastic term (Eq. fluxes:buoyancy) of one ray
    against the polarization relations of a plane inertia-gravity wave, for a wave rotated to
    azimuth theta (the fluxes rotate as a tensor, the elastic term as a vector)."""
    f0, N2, rho = 1.2e-4, 4e-4, 1.0
    grid = synth.fplane_grid(nx=8, ny=8, nz=30, dz=500.0, f0=f0)
    shape = (30, 8, 8)
    bg = (np.zeros(shape), np.zeros(shape), np.full(shape, N2), np.full(shape, rho))
    kh, m = 2 * math.pi / 1.5e5, -2 * math.pi / 4e3
    for theta in (0.0, 0.6, 2.2):
        k, l = kh * math.cos(theta), kh * math.sin(theta)
        M = model(grid, dict(gamma_mode=0, smoothing=0, saturation=0, splitting=0), bg)
        M.add_rays(dict(x=[3.5 * 50e3], y=[4.5 * 50e3], z=[7250.0], k=[k], l=[l], m=[m], ex=[50e3], ey=[50e3],
                        ez=[500.0], dk=[1e-6], dl=[1e-6], dm=[1e-4], n=[1e12]))
        M.diagnose()
        c = (14, 4, 3)
        T = np.array([[M.field("f_ll")[c], M.field("f_lp")[c]], [M.field("f_pl")[c], M.field("f_pp")[c]]])
        E = np.array([M.field("e_l")[c], M.field("e_p")[c]])
        w = oracle.dispersion(kh, 0.0, m, N2, 0.0, f0 * f0)[0]
        mo = _plane_wave_moments(kh, m, N2, f0, w)
        R = np.array([[math.cos(theta), -math.sin(theta)], [math.sin(theta), math.cos(theta)]])
        # rho <v'u'> of the wave along x, rotated; first index flux direction, second momentum component
        T0 = np.array([[mo["uu"], mo["uv"]], [mo["uv"], mo["vv"]]])
        Te = R @ T0 @ R.T
        scale = T[0, 0] / Te[0, 0] if abs(Te[0, 0]) > 1e-3 * mo["uu"] else T[1, 1] / Te[1, 1]
        np.testing.assert_allclose(T, scale * Te, rtol=1e-10, atol=1e-12 * abs(scale * mo["uu"]))
        # elastic term (f/g) e_r x <u'b'>, stored as g rho times it
        ub = np.array([mo["ub"], mo["vb"]])
        e0 = f0 * np.array([-ub[1], ub[0]]) * rho
        np.testing.assert_allclose(E, scale * (R @ e0), rtol=1e-10, atol=1e-12 * abs(scale * e0).max())
        # potential-temperature flux (Eq. fluxes:temperature) with theta' = theta-bar b' / g: the
        # projected integrals are g rho <u'theta'> / theta-bar = rho <u'b'>, a vector along e_r x k_h
        Th = np.array([M.field("t_l")[c], M.field("t_p")[c]])
        np.testing.assert_allclose(Th, scale * (R @ (rho * ub)), rtol=1e-10, atol=1e-12 * abs(scale * ub).max())
        # and Eq. fluxes:buoyancy: the elastic term is f e_r x of it
        np.testing.assert_allclose(E, f0 * np.array([-Th[1], Th[0]]), rtol=1e-12)
        # vertical flux of horizontal momentum: rho <w'u'> over the interfaces it covers
        fz = np.array([M.field("fz_l")[:, 4, 3].sum(), M.field("fz_p")[:, 4, 3].sum()])
        wu = R @ np.array([mo["wu"], mo["wv"]])
        np.testing.assert_allclose(fz, scale * wu, rtol=1e-10, atol=1e-12 * abs(scale * mo["wu"]))


def test_divergence_special_cases():
    grid = synth.fplane_grid(nx=16, ny=8, nz=10, dz=500.0)
    bg = synth.uniform_background(grid)
    M = model(grid, None, bg)
    nz, ny, nx = 10, 8, 16
    x, y, z = synth.node_coords(grid)
    Lx = nx * grid["dx"]
    zi = np.arange(nz + 1) * 500.0
    f = {n: np.zeros((nz, ny, nx)) for n in oracle.FIELD_NAMES[2:8]}
    # vertical flux linear in z (zero at the boundaries is not needed for the interior identity)
    f["fz_l"] = np.broadcast_to((0.3 + 2e-4 * zi)[:, None, None], (nz + 1, ny, nx)).copy()
    f["fz_p"] = np.zeros((nz + 1, ny, nx))
    # horizontally uniform horizontal fluxes contribute nothing
    f["f_pl"] = np.full((nz, ny, nx), 7.0)
    f["f_lp"] = np.full((nz, ny, nx), -3.0)
    # a sinusoid in x for F^{xy}: the centred difference has a closed form
    f["f_pp"] = np.zeros((nz, ny, nx))
    f["f_ll"] = np.zeros((nz, ny, nx))
    kx = 2 * math.pi / Lx
    f["f_lp"] = f["f_lp"] + np.sin(kx * x)[None, None, :]
    du, dv = M.divergence(f)
    rho = bg[3]
    np.testing.assert_allclose(du, -2e-4 / rho, rtol=1e-12)
    expect_v = -(np.cos(kx * x) * math.sin(kx * grid["dx"]) / grid["dx"])[None, None, :] / rho
    np.testing.assert_allclose(dv, expect_v, rtol=1e-10, atol=1e-18)


def test_spherical_divergence_is_flux_form():
    """(1/(r cos phi)) d/dphi (cos phi F): a meridional flux F ~ 1/cos(phi) has no divergence in
    the interior rows, a zonally uniform zonal flux none anywhere; the elastic term enters as
    E / (g rho) (Eq. mean-flow-impact)."""
    grid = synth.sphere_grid(nx=16, ny=24, nz=6)
    bg = synth.jet_background(grid)
    M = model(grid, None, bg)
    _, phi, _ = synth.node_coords(grid)
    nz, ny, nx = 6, 24, 16
    f = {n: np.zeros((nz, ny, nx)) for n in oracle.FIELD_NAMES[2:8]}
    f["fz_l"] = np.zeros((nz + 1, ny, nx))
    f["fz_p"] = np.zeros((nz + 1, ny, nx))
    f["f_pl"] = np.broadcast_to((3.0 / np.cos(phi))[None, :, None], (nz, ny, nx)).copy()
    f["f_ll"] = np.full((nz, ny, nx), 5.0)
    f["e_p"] = np.full((nz, ny, nx), 2.0)
    du, dv = M.divergence(f)
    assert np.max(np.abs(du[:, 1:-1, :])) <= 1e-12 * 3.0 / grid["radius"]
    assert np.all(np.abs(du[:, 0, :]) > 0) and np.all(np.abs(du[:, -1, :]) > 0)
    np.testing.assert_allclose(dv, 2.0 / (grid["g"] * bg[3]), rtol=1e-14)


def test_smoothing_preserves_constants_and_means():
    grid = synth.fplane_grid(nx=16, ny=8, nz=4)
    M = model(grid, None, synth.uniform_background(grid))
    c = np.full((4, 8, 16), 2.5)
    np.testing.assert_allclose(M.smooth(c), c, rtol=1e-15)
    g = np.random.default_rng(3).normal(size=(4, 8, 16))
    s = M.smooth(g)
    # doubly periodic: the 1-2-1 x 1-2-1 stencil conserves the plane sums
    np.testing.assert_allclose(s.sum(axis=(1, 2)), g.sum(axis=(1, 2)), rtol=1e-12)


def test_smoothing_response_of_fourier_modes():
    """Reading of App. B.4 on the lat-lon grid (separable 1-2-1 x 1-2-1, periodic in x, the edge row
    reused beyond the pole rows): a shift-invariant 1-2-1 filter multiplies a Fourier mode of angle
    theta per node by (2 + 2 cos theta) / 4 = cos^2(theta / 2); with the edge row reused, the
    half-sample cosines cos(pi q (j + 1/2) / ny) are its eigenvectors up to and including the pole
    rows, with eigenvalue cos^2(pi q / (2 ny)).  Wrong weights, a box or one-axis stencil, or another
    pole rule (mirror about the edge row, zeros beyond it) change these factors."""
    nx, ny = 24, 12
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    for geometry in ("fplane", "sphere"):
        grid = synth.fplane_grid(nx=nx, ny=ny, nz=4) if geometry == "fplane" else synth.sphere_grid(nx=nx, ny=ny, nz=4)
        M = model(grid, None, synth.uniform_background(grid) if geometry == "fplane" else _sphere_bg(grid))
        for p_, q_ in ((1, 1), (3, 2), (5, 5), (11, 3)):
            fx = np.cos(2 * math.pi * p_ * i / nx + 0.3)
            if geometry == "fplane":
                fy = np.cos(2 * math.pi * q_ * j / ny - 0.7)
                lam = math.cos(math.pi * p_ / nx) ** 2 * math.cos(math.pi * q_ / ny) ** 2
            else:
                fy = np.cos(math.pi * q_ * (j + 0.5) / ny)
                lam = math.cos(math.pi * p_ / nx) ** 2 * math.cos(math.pi * q_ / (2 * ny)) ** 2
            F = np.broadcast_to(fx * fy, (4, ny, nx)).copy()
            np.testing.assert_allclose(M.smooth(F), lam * F, rtol=0, atol=1e-14)


def test_node_gradients_exact_for_linear_fields_up_to_the_pole_rows_and_the_top():
    """Reading of App. B.1 at the edges: node gradients are one-sided at the pole rows and at the
    bottom and top levels, and beyond the first/last node every gathered quantity keeps its edge
    value.  For fields linear in latitude and height both differences are exact, so the gathered
    gradient is the field's slope everywhere -- between the pole rows and the poles too -- and the
    value beyond the edge node is the edge node's value."""
    grid = synth.sphere_grid(nx=16, ny=12, nz=10, dz=1000.0)
    x, y, z = synth.node_coords(grid)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    a_u, c_u, a_v, c_v, a_n, c_n = 3.0, 1e-3, -2.0, 5e-4, 1e-5, 2e-9
    bg = (10.0 + a_u * Y + c_u * Z, -1.0 + a_v * Y + c_v * Z, 4e-4 + a_n * Y + c_n * Z, 1.2 * np.exp(-Z / 7000.0))
    M = model(grid, None, bg)
    dphi, dz = math.pi / 12, 1000.0
    lam = 1.234
    phi_n, phi_s = y[-1], y[0]
    cases = [  # (phi, z, phi used by the value, z used by the value)
        (phi_n + 0.4 * dphi, 4300.0, phi_n, 4300.0),    # between the last row centre and the north pole
        (phi_n - 0.3 * dphi, 4300.0, phi_n - 0.3 * dphi, 4300.0),
        (phi_s - 0.45 * dphi, 6100.0, phi_s, 6100.0),   # south of the first row centre
        (0.2, z[-1] + 0.3 * dz, 0.2, z[-1]),            # above the last level centre
        (-0.1, 0.2 * dz, -0.1, z[0]),                   # below the first level centre
    ]
    for phi, zz, pv, zv in cases:
        b = M.gather(lam, phi, zz)
        assert b[0] == pytest.approx(10.0 + a_u * pv + c_u * zv, rel=1e-13)
        assert b[1] == pytest.approx(-1.0 + a_v * pv + c_v * zv, rel=1e-13)
        assert b[2] == pytest.approx(4e-4 + a_n * pv + c_n * zv, rel=1e-12)
        np.testing.assert_allclose(b[4:7], [0.0, a_u, c_u], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(b[7:10], [0.0, a_v, c_v], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(b[10:13], [0.0, a_n, c_n], rtol=1e-9, atol=1e-19)


# ------------------------------------------------------------------ bookkeeping

def test_splitting_halves_and_conserves_action():
    grid = synth.fplane_grid(nx=8, ny=8, nz=30, dz=500.0)
    bg = synth.uniform_background(grid, U=0.0)
    M = model(grid, dict(saturation=0, smoothing=0), bg)
    ray = dict(x=[3.5 * 50e3], y=[2.5 * 50e3], z=[6000.0], k=[3e-5], l=[1e-5], m=[-2e-3], ex=[130e3], ey=[40e3],
               ez=[1300.0], dk=[3e-6], dl=[1e-6], dm=[2e-4], n=[1e10])
    M.add_rays(ray)
    w0 = M.stats()["w_total"]
    s0 = M.rays()
    y = np.array([s0[n][0] for n in oracle.STATE_NAMES])
    adv = M.advance_ray(y, 300.0)
    M.step(300.0)
    r = M.rays()
    st = M.stats()
    assert st["n_split_v"] == 1 and st["n_split_h"] == 2 and st["n_live"] == 4
    assert sorted(r["id"].tolist()) == [0, 1, 2, 3]
    assert st["w_total"] == pytest.approx(w0, rel=1e-15)
    assert np.all(r["ez"] == 0.5 * adv[8]) and np.all(r["ex"] == 0.5 * adv[6]) and np.all(r["ey"] == adv[7])
    np.testing.assert_allclose(sorted(set(np.round(r["z"] - adv[2], 6))), [-0.25 * adv[8], 0.25 * adv[8]])
    np.testing.assert_allclose(r["pz"], 0.5 * adv[11])
    np.testing.assert_allclose(r["px"], 0.5 * adv[9])
    # below the thresholds nothing splits
    M2 = model(grid, dict(saturation=0, smoothing=0), bg)
    ray2 = dict(ray, ex=[120e3], ez=[1200.0])
    M2.add_rays(ray2)
    M2.step(1.0)
    assert M2.stats()["n_live"] == 1


def test_cap_removes_lowest_energy():
    grid = synth.fplane_grid(nx=4, ny=4, nz=30, dz=500.0)
    bg = synth.uniform_background(grid, U=0.0)
    cap = 7
    M = model(grid, dict(saturation=0, smoothing=0, splitting=0, cap_per_column=cap), bg)
    g = np.random.default_rng(41)
    n = 20
    kh = 2 * math.pi / g.uniform(1e5, 5e5, n)
    m = -2 * math.pi / g.uniform(1e3, 5e3, n)
    r = dict(x=np.full(n, 1.5 * 50e3), y=np.full(n, 2.5 * 50e3), z=g.uniform(3e3, 9e3, n), k=kh, l=0 * kh, m=m,
             ex=np.full(n, 1e3), ey=np.full(n, 1e3), ez=np.full(n, 100.0), dk=0.1 * kh, dl=0.1 * kh,
             dm=0.1 * np.abs(m), n=g.uniform(1e10, 1e11, n))
    M.add_rays(r)
    s0 = M.rays()
    E = {}
    for q in range(n):
        y = np.array([s0[nm][q] for nm in oracle.STATE_NAMES])
        E[int(s0["id"][q])] = M.ray_energy(M.advance_ray(y, 100.0))
    M.step(100.0)
    kept = set(M.rays()["id"].tolist())
    st = M.stats()
    assert len(kept) == cap and st["n_capped"] == n - cap
    removed = set(E) - kept
    assert max(E[i] for i in removed) <= min(E[i] for i in kept)


def test_cap_ties_remove_the_larger_ids_first():
    """Reading of App. B.5 (the paper names no tie rule): among ray volumes of equal energy the one
    with the larger id is removed first.  Identical ray volumes have identical energies, so a cap of
    c keeps exactly the c smallest ids; a lower-energy copy goes before any of them."""
    grid = synth.fplane_grid(nx=4, ny=4, nz=30, dz=500.0)
    bg = synth.uniform_background(grid, U=0.0)
    cap, n = 5, 12
    M = model(grid, dict(saturation=0, smoothing=0, splitting=0, cap_per_column=cap), bg)
    kh, m = 2 * math.pi / 2e5, -2 * math.pi / 3e3
    one = dict(x=[1.5 * 50e3], y=[2.5 * 50e3], z=[6e3], k=[kh], l=[0.0], m=[m], ex=[1e3], ey=[1e3], ez=[100.0],
               dk=[0.1 * kh], dl=[0.1 * kh], dm=[0.1 * abs(m)], n=[1e10])
    r = {key: np.array(v * n) for key, v in one.items()}
    r["n"][7] = 0.5e10                     # id 7: the lowest energy, removed first
    M.add_rays(r)
    M.step(100.0)
    kept = sorted(M.rays()["id"].tolist())
    assert kept == [0, 1, 2, 3, 4] and M.stats()["n_capped"] == n - cap


def test_exit_rule_at_the_pole_rows_and_the_top():
    """Reading of the boundaries (the paper gives none for a lat-lon grid): a carrier that ends a
    step poleward of the centre of the last row, or at z >= z_top, leaves; one that ends just inside
    stays.  Each ray volume is placed so that its own RK3 step ends 1e-9 rad (or 1 mm) beyond or
    before the threshold."""
    grid = synth.sphere_grid(nx=16, ny=12, nz=20, dz=1000.0)
    bg = _sphere_bg(grid)
    dt = 600.0
    dphi = math.pi / 12
    phimax = 0.5 * math.pi - 0.5 * dphi
    ztop = 20 * 1000.0
    M = model(grid, dict(saturation=0, smoothing=0, splitting=0, cap_per_column=0), bg)
    kh, m = 2 * math.pi / 1e5, -2 * math.pi / 4e3

    def base(phi, zz, l_sign):
        return np.array([1.0, phi, zz, 0.0, l_sign * kh, m, 0.01, 0.01, 200.0, 1.0, 1.0, 1.0, 1.0])

    def placed(target_phi, target_z, l_sign, which):
        # start so that the advanced carrier lands on the target (the displacement barely depends on
        # the start over such short distances; two fixed-point passes)
        s0 = base(target_phi, target_z, l_sign)
        for _ in range(3):
            adv = M.advance_ray(s0, dt)
            if which == "phi":
                s0[1] += target_phi - adv[1]
            else:
                s0[2] += target_z - adv[2]
        return s0

    starts = [placed(phimax + 1e-9, 10e3, 1.0, "phi"), placed(phimax - 1e-9, 10e3, 1.0, "phi"),
              placed(-phimax - 1e-9, 10e3, -1.0, "phi"), placed(-phimax + 1e-9, 10e3, -1.0, "phi"),
              placed(0.3, ztop + 1e-3, 1.0, "z"), placed(0.3, ztop - 1e-3, 1.0, "z")]
    rays = {nm: np.array([s[q] for s in starts]) for q, nm in enumerate(oracle.STATE_NAMES)}
    rays.update(dk=np.full(6, 0.1 * kh), dl=np.full(6, 0.1 * kh), dm=np.full(6, 0.1 * abs(m)))
    rays = {nm: rays[nm] for nm in ("x", "y", "z", "k", "l", "m", "ex", "ey", "ez", "dk", "dl", "dm", "n")}
    M.add_rays(rays)
    M.step(dt)
    assert sorted(M.rays()["id"].tolist()) == [1, 3, 5] and M.stats()["n_exited"] == 3


def test_exits_at_top_and_budget_closure():
    """Sec. 4 budget: W(t+dt) = W(t) + launched - saturated - exited - capped, to round-off."""
    grid = synth.sphere_grid(nx=32, ny=16, nz=20)
    bg = _sphere_bg(grid)
    M = model(grid, dict(cap_per_column=40), bg)
    M.launch_background(synth.background_source(z_launch=2e3))
    r = synth.sphere_rays(grid, 400, tag=9, z_lo=15e3, z_hi=19.9e3, ext_scale=3.0)
    r["n"] = r["n"] * 30.0
    M.add_rays(r)
    prev = M.stats()
    seen = dict(exit=0, sat=0, cap=0, split=0)
    for step in range(8):
        if step == 4:
            M.launch_background(synth.background_source(z_launch=2e3))
        M.step(300.0)
        st = M.stats()
        lhs = st["w_total"]
        rhs = prev["w_total"] + (st["w_launched"] - prev["w_launched"]) - (st["w_saturated"] - prev["w_saturated"]) \
            - (st["w_exited"] - prev["w_exited"]) - (st["w_capped"] - prev["w_capped"]) \
            - (st["w_invalid"] - prev["w_invalid"])
        assert lhs == pytest.approx(rhs, rel=1e-12)
        seen["exit"] += st["n_exited"] - prev["n_exited"]
        seen["sat"] += st["w_saturated"] > prev["w_saturated"]
        seen["cap"] += st["n_capped"] - prev["n_capped"]
        seen["split"] += st["n_split_v"] + st["n_split_h"] - prev["n_split_v"] - prev["n_split_h"]
        prev = st
    assert all(v > 0 for v in seen.values()), seen
    r = M.rays()
    assert len(np.unique(r["id"])) == len(r["id"])
    # canonical order: ascending (cell, id)
    key = r["cell"].astype(np.int64) * (1 << 40) + r["id"]
    assert np.all(np.diff(key) > 0)


# ------------------------------------------------------------------ columnar mode (MS-GWaM-1D, Sec. 1)

def test_columnar_mode_freezes_horizontal_state_and_follows_vertical_hamiltonian():
    """Single-column approximation: horizontal gradients of the resolved flow neglected and no
    horizontal propagation or advection (Sec. 1).  Then lambda, phi, k, l and the horizontal
    extents stay fixed, while m obeys Hamilton's equation for the vertical coordinate alone,
    dm/dt = -dOmega/dz (no metric terms: the ray does not move over the sphere), and z moves with
    the vertical group velocity -- checked by finite differences of Omega."""
    grid = synth.sphere_grid(nx=64, ny=40, nz=30, dz=1000.0)
    M = model(grid, dict(columnar=1), _sphere_linear_bg(grid))
    g = np.random.default_rng(41)
    dlam, dphi = 2 * math.pi / 64, math.pi / 40
    for _ in range(20):
        lam = (g.integers(2, 60) + g.uniform(0.6, 1.4)) * dlam
        phi = -0.5 * math.pi + (g.integers(6, 32) + g.uniform(0.6, 1.4)) * dphi
        z = (g.integers(3, 25) + g.uniform(0.6, 1.4)) * 1000.0
        k, l = 2 * math.pi / 3e5 * g.normal(size=2)
        m = -2 * math.pi / 4e3
        F = M.rhs([lam, phi, z, k, l, m, 0.0, 0.0, 0.0])
        assert F[0] == 0.0 and F[1] == 0.0 and F[3] == 0.0 and F[4] == 0.0 and F[6] == 0.0 and F[7] == 0.0
        dOdz = fd(lambda t: M.omega(lam, phi, t, k, l, m), z, 0.05)
        dOdm = fd(lambda t: M.omega(lam, phi, z, k, l, t), m, 1e-6 * abs(m))
        assert abs(F[5] + dOdz) <= 1e-5 * abs(dOdz), (F[5], -dOdz)
        assert abs(F[2] - dOdm) <= 1e-5 * abs(dOdm), (F[2], dOdm)
    # a full RK3 step keeps the horizontal components bit for bit
    y0 = [3 * dlam + 0.3 * dlam, 0.2, 12e3, 2e-5, -1e-5, -1.5e-3, 0.05, 0.04, 800.0]
    y1 = M.rk3(y0, 300.0)
    for c in (0, 1, 3, 4, 6, 7):
        assert y1[c] == y0[c]
    assert y1[2] != y0[2] and y1[5] != y0[5]


def test_columnar_mode_equals_3d_in_a_horizontally_uniform_fplane():
    """Where the single-column assumption holds exactly (f-plane, horizontally uniform
    background), the vertical part of the 3-D ray equations (z, m, dZ rates) is the columnar one."""
    w = synth.workload("fplane")
    grid = w["grid"]
    g = np.random.default_rng(43)
    M1 = model(grid, dict(columnar=1), w["background"])
    M3 = model(grid, dict(columnar=0), w["background"])
    for _ in range(20):
        y = [g.uniform(0, 16 * grid["dx"]), g.uniform(0, 16 * grid["dy"]), g.uniform(2e3, 30e3),
             g.normal() * 2e-5, g.normal() * 2e-5, -g.uniform(6e-4, 6e-3), 5e4, 5e4, 500.0]
        F1, F3 = M1.rhs(y), M3.rhs(y)
        for c in (2, 5, 8):
            assert abs(F1[c] - F3[c]) <= 1e-13 * abs(F3[c]) + 1e-300, (c, F1[c], F3[c])


def test_columnar_divergence_keeps_only_the_vertical_flux_and_elastic_terms():
    """Horizontally homogeneous column: the horizontal flux divergence drops out of Eq.
    mean-flow-impact; the vertical flux divergence and the elastic term remain."""
    grid = synth.sphere_grid(nx=16, ny=8, nz=10, dz=1000.0)
    bg = _sphere_bg(grid)
    M = model(grid, dict(columnar=1), bg)
    g = np.random.default_rng(47)
    nz, ny, nx = 10, 8, 16
    f = {n: g.normal(size=(nz, ny, nx)) for n in oracle.FIELD_NAMES[2:8]}
    f["fz_l"] = g.normal(size=(nz + 1, ny, nx))
    f["fz_p"] = g.normal(size=(nz + 1, ny, nx))
    du, dv = M.divergence(f)
    rho = bg[3]
    gr = grid["g"]
    exp_u = -(f["fz_l"][1:] - f["fz_l"][:-1]) / 1000.0 / rho + f["e_l"] / (gr * rho)
    exp_v = -(f["fz_p"][1:] - f["fz_p"][:-1]) / 1000.0 / rho + f["e_p"] / (gr * rho)
    np.testing.assert_allclose(du, exp_u, rtol=1e-12, atol=0)
    np.testing.assert_allclose(dv, exp_v, rtol=1e-12, atol=0)


# ------------------------------------------------------------------ potential temperature (Eq. mean-flow-impact-t)

def test_theta_tendency_closed_forms():
    """d theta/dt = -div <u'theta'> with <u'theta'> = theta-bar/(g rho-bar) T: a sinusoid in x has
    the closed-form centred difference; uniform T contributes nothing; on the sphere T_phi ~ 1/cos
    phi (flux form) gives zero; the columnar mode drops the horizontal divergence."""
    grid = synth.fplane_grid(nx=16, ny=8, nz=10, dz=500.0)
    bg = synth.uniform_background(grid)
    M = model(grid, None, bg)
    rho = bg[3]
    M.set_theta(grid["g"] * rho)               # theta-bar / (g rho-bar) = 1
    x, y, z = synth.node_coords(grid)
    Lx = 16 * grid["dx"]
    kx = 2 * math.pi / Lx
    tl = np.broadcast_to(np.sin(kx * x)[None, None, :], (10, 8, 16)).copy()
    tp = np.full((10, 8, 16), 3.0)
    out = M.theta_divergence(tl, tp)
    expect = -(np.cos(kx * x) * math.sin(kx * grid["dx"]) / grid["dx"])[None, None, :]
    np.testing.assert_allclose(out, np.broadcast_to(expect, out.shape), rtol=1e-10, atol=1e-18)
    Mc = model(grid, dict(columnar=1), bg)
    Mc.set_theta(grid["g"] * rho)
    assert np.all(Mc.theta_divergence(tl, tp) == 0.0)
    sg = synth.sphere_grid(nx=16, ny=10, nz=6, dz=1000.0)
    sbg = _sphere_bg(sg)
    Ms = model(sg, None, sbg)
    Ms.set_theta(sg["g"] * sbg[3])
    _, phi, _ = synth.node_coords(sg)
    tp_s = np.broadcast_to((1.0 / np.cos(phi))[None, :, None], (6, 10, 16)).copy()
    out = Ms.theta_divergence(np.zeros((6, 10, 16)), tp_s)
    np.testing.assert_allclose(out[:, 1:-1, :], 0.0, atol=1e-20)


# ------------------------------------------------------------------ ghost-layer launch (Sec. 3c)

def _spec(i, j, theta, c, flux, z_launch=5e3, dz_launch=1e3, lambda_h=100e3):
    s = np.zeros(1, dtype=synth.SPEC_DTYPE)
    s["i"], s["j"], s["theta"], s["c"], s["flux"] = i, j, theta, c, flux
    s["z_launch"], s["dz_launch"], s["lambda_h"], s["spectral_frac"] = z_launch, dz_launch, lambda_h, 0.1
    return s


def test_ghost_emission_carries_the_source_flux_per_interval():
    """Uniform f-plane: the emitted part of each bin is the slab its wave action crossed the layer top
    in dt, so its action is the pseudomomentum flux times dt times the column area over |k_h|
    (A = F / (|k_h| c_r) and an extent c_r dt), whatever c_r is.  The ghost propagates vertically
    only: position, horizontal wavenumber, extents and N stay those of the launch state, and the
    emitted slab starts at the layer top."""
    grid = synth.fplane_grid(nx=3, ny=2, nz=40, dx=50e3, dy=40e3, dz=500.0, f0=1e-4)
    bg = synth.uniform_background(grid, U=5.0, V=-2.0)
    params = dict(saturation=0, smoothing=0)
    specs = synth.uniform_specs(grid, flux=2e-3)
    kh = 2.0 * math.pi / 100e3
    dt = 60.0
    G = model(grid, params, bg)
    G.launch_ghost_spectral(specs, dt)
    L = model(grid, params, bg)
    L.launch_spectral(specs)
    g, s = G.rays(), L.rays()
    # the bins the wind filters at launch (w_hat <= |f|) are filtered here too; every other bin emits
    assert len(g["id"]) == len(s["id"]) and len(g["id"]) > 0.8 * len(specs)
    W = g["n"] * g["px"] * g["py"] * g["pz"]
    np.testing.assert_allclose(W, 2e-3 / 32 * dt * grid["dx"] * grid["dy"] / kh, rtol=1e-12)
    for n in ("x", "y", "k", "l", "m", "ex", "ey", "px", "py", "n"):
        np.testing.assert_array_equal(g[n], s[n])
    assert np.all(g["ez"] < s["ez"])
    np.testing.assert_allclose(g["z"] - 0.5 * g["ez"], 6e3, rtol=0, atol=1e-9)
    np.testing.assert_allclose(g["pz"] / g["ez"], s["pz"] / s["ez"], rtol=1e-13)   # same dm
    st = G.stats()
    assert st["n_launched"] == len(s["id"]) and st["n_filtered"] == len(specs) - len(s["id"])
    assert st["w_launched"] == pytest.approx(W.sum(), rel=1e-13)


def test_ghost_emission_on_the_sphere_follows_the_source_profile():
    """Background source at rest on the sphere: per row the emitted action is F_am(phi) dt A_c / |k_h|
    (A_c the column area at the launch height, F_am of Sec. 3c) -- the rate the source prescribes."""
    grid = synth.sphere_grid(nx=8, ny=36, nz=30, dz=500.0)
    n2c, H, rho0 = synth.isothermal()
    shape = (30, 36, 8)
    _, phi, z = synth.node_coords(grid)
    bg = (np.zeros(shape), np.zeros(shape), np.full(shape, n2c),
          np.broadcast_to((rho0 * np.exp(-z / H))[:, None, None], shape).copy())
    src = synth.background_source(launch_zero_flux=0)
    kh = 2.0 * math.pi / src["lambda_h"]
    dt = 60.0
    G = model(grid, dict(saturation=0, smoothing=0), bg)
    G.launch_ghost(src, dt)
    r = G.rays()
    W = r["n"] * r["px"] * r["py"] * r["pz"]
    rows = 0
    for j in range(36):
        pdeg = math.degrees(phi[j])
        F = oracle.fam(pdeg, src["tau"], src["f_s"], src["f_w"])
        sel = np.abs(r["y"] - phi[j]) < 1e-12
        if F == 0.0 or abs(pdeg) > src["phi_max_deg"]:
            assert not sel.any()
            continue
        rows += 1
        assert sel.sum() == 8 * src["n_az"] * src["n_c"]
        area = (synth.EARTH_RADIUS + 5.5e3) ** 2 * math.cos(phi[j]) * (2 * math.pi / 8) * (math.pi / 36)
        assert W[sel].sum() == pytest.approx(F * dt * area / kh * 8, rel=1e-12)
    assert rows == 26


def test_ghost_volume_that_left_the_layer_whole_is_emitted_whole():
    """A launch interval longer than the layer's crossing time emits the whole ghost volume: the launch
    state moved up by c_r dt with its action (less than the flux times dt)."""
    grid = synth.fplane_grid(nx=2, ny=2, nz=80, dx=50e3, dy=50e3, dz=500.0, f0=1e-4)
    bg = synth.uniform_background(grid, U=0.0)
    params = dict(saturation=0, smoothing=0)
    sp = _spec(0, 0, 0.0, 50.0, 1e-3)
    kh = 2.0 * math.pi / 100e3
    L = model(grid, params, bg)
    L.launch_spectral(sp)
    s = L.rays()
    c_r = None
    for dt in (60.0, 600.0):
        G = model(grid, params, bg)
        G.launch_ghost_spectral(sp, dt)
        g = G.rays()
        W = g["n"][0] * g["px"][0] * g["py"][0] * g["pz"][0]
        if dt == 60.0:
            c_r = g["ez"][0] / dt                      # the part above the top: c_r dt
            assert W == pytest.approx(1e-3 * dt * 2.5e9 / kh, rel=1e-12)
        else:
            assert c_r * dt > 1e3
            assert g["ez"][0] == pytest.approx(1e3, rel=1e-13)
            assert g["z"][0] == pytest.approx(5.5e3 + c_r * dt, rel=1e-12)
            assert W == pytest.approx(s["n"][0] * s["px"][0] * s["py"][0] * s["pz"][0], rel=1e-13)
            assert W < 1e-3 * dt * 2.5e9 / kh


def test_ghost_reflected_within_the_layer_is_discarded():
    """N^2 falling with height: a bin launched with w_hat just below N at the layer centre meets its
    turning level (N(z) = w_hat) within the layer after |m| / (dm/dt) ~ a second, dm/dt = -d w_hat/dz
    = k_h^2 / (2 w_hat K^2) |dN^2/dz| (Gamma = 0): it turns downward and is discarded.  A slower bin,
    whose turning level is far above, is emitted."""
    grid = synth.fplane_grid(nx=2, ny=2, nz=40, dx=50e3, dy=50e3, dz=500.0, f0=1e-4)
    u, v, n2, rho = synth.uniform_background(grid, U=0.0)
    _, _, z = synth.node_coords(grid)
    N2c, Hn = 4e-4, 4e3
    n2 = np.broadcast_to((N2c * np.exp(-(z - 5.5e3) / Hn))[:, None, None], n2.shape).copy()
    params = dict(saturation=0, smoothing=0, gamma_mode=0)
    kh = 2.0 * math.pi / 100e3
    dt = 60.0
    for frac, reflects in ((0.999, True), (0.99, True), (0.1, False)):
        w = frac * math.sqrt(N2c)
        c = w / kh
        m0 = -kh * math.sqrt((N2c - w * w) / (w * w - 1e-8))
        mdot = kh * kh / (2.0 * w * (kh * kh + m0 * m0)) * N2c / Hn
        assert (abs(m0) / mdot < 0.1 * dt) == reflects
        G = model(grid, params, (u, v, n2, rho))
        G.launch_ghost_spectral(_spec(0, 0, 0.0, c, 1e-3), dt)
        st = G.stats()
        assert (st["n_launched"], st["n_filtered"]) == ((0, 1) if reflects else (1, 0))


def test_ghost_launching_every_interval_gives_the_steady_source_flux():
    """Emitting every interval and stepping, the emitted slabs tile the column above the layer without
    gap or overlap (uniform medium), so the projected vertical pseudomomentum flux (App. A form) at
    every interface inside the filled region is the source flux exactly."""
    grid = synth.fplane_grid(nx=2, ny=2, nz=60, dx=50e3, dy=50e3, dz=500.0, f0=1e-4)
    bg = synth.uniform_background(grid, U=0.0)
    params = dict(saturation=0, smoothing=0, flux_form=1)
    sp = np.concatenate([_spec(i, j, 0.0, 23.2, 1e-3) for j in range(2) for i in range(2)])
    G = model(grid, params, bg)
    dt, n = 120.0, 30
    for _ in range(n):
        G.launch_ghost_spectral(sp, dt)
        G.step(dt, want_tendencies=False)
    r = G.rays()
    delta = r["ez"].max()
    assert np.allclose(r["ez"], delta, rtol=1e-12) and len(r["z"]) == 4 * n
    fz = G.field("fz_l")
    zi = np.arange(grid["nz"] + 1) * grid["dz"]
    inside = (zi - 0.5 * grid["dz"] > 6e3 + delta) & (zi + 0.5 * grid["dz"] < 6e3 + (n + 1) * delta)
    assert inside.sum() >= 8
    np.testing.assert_allclose(fz[inside], 1e-3, rtol=1e-12)
    np.testing.assert_array_equal(G.field("fz_p")[inside], 0.0)


def test_threaded_oracle_is_bit_identical():
    """The optional threads only run independent per-ray and per-level work in parallel; sums,
    bookkeeping and ids stay in array order, so every output is bit-identical to one thread."""
    grid = synth.sphere_grid(nx=32, ny=16, nz=20)
    bg = _sphere_bg(grid)
    outs = []
    for th in (1, 4):
        M = model(grid, dict(cap_per_column=20), bg)
        M.set_threads(th)
        M.launch_background(synth.background_source(z_launch=2e3))
        r = synth.sphere_rays(grid, 300, tag=9, z_lo=15e3, z_hi=19.9e3, ext_scale=3.0)
        r["n"] = r["n"] * 30.0
        M.add_rays(r)
        for _ in range(5):
            du, dv = M.step(300.0)
        outs.append((M.rays(), du, dv, M.stats(), [M.field(n) for n in oracle.ALL_FIELD_NAMES[:8]]))
    a, b = outs
    for key in a[0]:
        np.testing.assert_array_equal(a[0][key], b[0][key])
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[2], b[2])
    assert a[3] == b[3] and a[3]["n_capped"] > 0 and a[3]["w_saturated"] > 0
    for x, y in zip(a[4], b[4]):
        np.testing.assert_array_equal(x, y)
