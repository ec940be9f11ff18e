"""Seeded synthetic inputs for the ray-volume workloads.

This module only generates inputs -- grids, analytic backgrounds, initial ray
populations and launch specifications -- from seeded random streams.  It holds
none of the method's arithmetic (no dispersion relation, no group velocity, no
projection).  Both the CUDA path and the FP64 CPU oracle take their inputs from
here, so the two sides see identical numbers.

Workloads (all synthetic; the paper uses no public dataset for this path):

* ``fplane``  -- doubly periodic f-plane box 16 x 16 columns, dx = 50 km, 64
  levels of 500 m; N = 0.02 1/s, f = 1e-4 1/s, U = 10 m/s, V = 0, isothermal
  density (H = 7 km); 4096 ray volumes with log-uniform horizontal wavelengths
  100-1000 km, uniform azimuth, log-uniform vertical wavelengths 1-10 km (m < 0,
  upward group velocity) and a Gaussian spectrum of wave action.
* ``sphere``  -- global lat-lon 256 x 128 columns x 90 levels of 1 km; two
  60 m/s zonal jets at +-45 deg with a Gaussian vertical profile peaking at
  60 km; N^2 of an isothermal 240 K atmosphere; exponential density; the
  latitude-dependent background source at 5 km (8 azimuths x 4 phase speeds
  5-50 m/s, lambda_h = 100 km) launches ~0.98 M ray volumes.
* ``sphere_fp32`` -- the same at 512 x 256 x 90 (~3.96 M ray volumes).
* ``ensemble`` -- 16 spheres with jet amplitudes U[30, 80] m/s and jet
  latitudes U[30, 60] deg, plus convective spectral launches with
  lognormal(ln 16, 1) rays per column (capped at 512) at 10 km.
"""
from __future__ import annotations

import math

import numpy as np

# planetary constants (ICON-like values; the paper states none)
EARTH_RADIUS = 6.371229e6
EARTH_OMEGA = 7.29212e-5
GRAVITY = 9.80665
R_DRY = 287.04
CP_DRY = 1004.64
P0 = 101325.0

SEED_BASE = 2309_11257

# laid out like the C struct of an explicit spectral launch (aligned: 72 bytes)
SPEC_DTYPE = np.dtype([("i", np.int32), ("j", np.int32), ("member", np.int32), ("z_launch", np.float64),
                       ("dz_launch", np.float64), ("theta", np.float64), ("c", np.float64),
                       ("lambda_h", np.float64), ("flux", np.float64), ("spectral_frac", np.float64)], align=True)

DEFAULT_PARAMS = dict(gamma_mode=1, saturation=1, smoothing=1, flux_form=0, splitting=1,
                      cap_per_column=4800, alpha_s=2.5, min_split_dz=1000.0, columnar=0,
                      theta_flux=0)


def rng(tag: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(tag)))


# ---------------------------------------------------------------- grids

def fplane_grid(nx=16, ny=16, nz=64, dx=50e3, dy=50e3, dz=500.0, f0=1e-4) -> dict:
    return dict(geometry=0, nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz, f0=f0,
                radius=EARTH_RADIUS, omega=0.0, g=GRAVITY)


def sphere_grid(nx=256, ny=128, nz=90, dz=1000.0, omega=EARTH_OMEGA) -> dict:
    return dict(geometry=1, nx=nx, ny=ny, nz=nz, dx=0.0, dy=0.0, dz=dz, f0=0.0,
                radius=EARTH_RADIUS, omega=omega, g=GRAVITY)


def node_coords(grid: dict):
    """Node (cell-centre) coordinates: x or lambda [nx], y or phi [ny], z [nz]."""
    nx, ny, nz, dz = grid["nx"], grid["ny"], grid["nz"], grid["dz"]
    z = (np.arange(nz) + 0.5) * dz
    if grid["geometry"] == 1:
        x = (np.arange(nx) + 0.5) * (2.0 * math.pi / nx)
        y = -0.5 * math.pi + (np.arange(ny) + 0.5) * (math.pi / ny)
    else:
        x = (np.arange(nx) + 0.5) * grid["dx"]
        y = (np.arange(ny) + 0.5) * grid["dy"]
    return x, y, z


# ---------------------------------------------------------------- backgrounds

def uniform_background(grid: dict, U=10.0, V=0.0, N=0.02, rho0=1.2, H=7000.0):
    nx, ny, nz = grid["nx"], grid["ny"], grid["nz"]
    _, _, z = node_coords(grid)
    shape = (nz, ny, nx)
    u = np.full(shape, float(U))
    v = np.full(shape, float(V))
    n2 = np.full(shape, float(N) ** 2)
    rho = np.broadcast_to((rho0 * np.exp(-z / H))[:, None, None], shape).copy()
    return u, v, n2, rho


def isothermal(T=240.0):
    """N^2 = g^2 / (c_p T), H = R T / g, rho_0 = p_0 / (R T) of an isothermal atmosphere."""
    return GRAVITY ** 2 / (CP_DRY * T), R_DRY * T / GRAVITY, P0 / (R_DRY * T)


def jet_background(grid: dict, amp=60.0, lat_deg=45.0, width_deg=10.0, z_peak=60e3, z_width=15e3,
                   T=240.0, amp_s=None, lat_s_deg=None):
    """Two zonal jets U = A exp(-((phi -+ phi_j)/w)^2) exp(-((z - z_j)/h)^2), V = 0, isothermal."""
    nx, ny, nz = grid["nx"], grid["ny"], grid["nz"]
    _, phi, z = node_coords(grid)
    pdeg = np.degrees(phi)
    amp_s = amp if amp_s is None else amp_s
    lat_s = lat_deg if lat_s_deg is None else lat_s_deg
    lat_prof = amp * np.exp(-((pdeg - lat_deg) / width_deg) ** 2) + amp_s * np.exp(-((pdeg + lat_s) / width_deg) ** 2)
    z_prof = np.exp(-((z - z_peak) / z_width) ** 2)
    shape = (nz, ny, nx)
    u = np.broadcast_to(z_prof[:, None, None] * lat_prof[None, :, None], shape).copy()
    v = np.zeros(shape)
    n2c, H, rho0 = isothermal(T)
    n2 = np.full(shape, n2c)
    rho = np.broadcast_to((rho0 * np.exp(-z / H))[:, None, None], shape).copy()
    return u, v, n2, rho


def channel_jet_background(grid: dict, amp=40.0, width=400e3, z_peak=35e3, z_width=12e3, N=0.02,
                           T=240.0):
    """f-plane zonal jet U = A exp(-((y - y_c)/w)^2) exp(-((z - z_j)/h)^2) centred in the box (y_c = L_y/2),
    V = 0, constant N, isothermal density (the jet-refraction run on the f-plane)."""
    nx, ny, nz = grid["nx"], grid["ny"], grid["nz"]
    _, y, z = node_coords(grid)
    yc = 0.5 * ny * grid["dy"]
    shape = (nz, ny, nx)
    prof = amp * np.exp(-((y - yc) / width) ** 2)
    u = np.broadcast_to(np.exp(-((z - z_peak) / z_width) ** 2)[:, None, None] * prof[None, :, None], shape).copy()
    v = np.zeros(shape)
    n2 = np.full(shape, float(N) ** 2)
    _, H, rho0 = isothermal(T)
    rho = np.broadcast_to((rho0 * np.exp(-z / H))[:, None, None], shape).copy()
    return u, v, n2, rho


def perturbed(fields, tag: int, rel=0.05):
    """Background plus a smooth seeded perturbation in all three directions (parity tests)."""
    g = rng(tag)
    u, v, n2, rho = [np.array(f, dtype=np.float64) for f in fields]
    nz, ny, nx = u.shape
    zz = np.linspace(0, 1, nz)[:, None, None]
    yy = np.linspace(0, 1, ny)[None, :, None]
    xx = np.linspace(0, 2 * math.pi, nx, endpoint=False)[None, None, :]
    a = g.uniform(0.5, 1.5, size=6)
    ph = g.uniform(0, 2 * math.pi, size=6)
    u = u + 5.0 * a[0] * np.sin(xx + ph[0]) * np.cos(3 * yy + ph[1]) * np.sin(2 * zz + ph[2])
    v = v + 3.0 * a[1] * np.cos(2 * xx + ph[3]) * np.sin(2 * yy + ph[4]) * np.cos(zz + ph[5])
    n2 = n2 * (1.0 + rel * a[2] * np.sin(xx + ph[1]) * np.cos(yy * 4 + ph[2]) * np.cos(3 * zz + ph[3]))
    rho = rho * (1.0 + rel * a[3] * np.cos(xx + ph[4]) * np.sin(2 * yy + ph[5]) * np.sin(zz + ph[0]))
    return u, v, n2, rho


# ---------------------------------------------------------------- initial ray volumes

def fplane_rays(grid: dict, n: int = 4096, tag: int = 1, z_lo=2e3, z_hi=8e3, ext_z=500.0, frac=0.1,
                action0=1e-3):
    """Initial ray volumes of the f-plane workload (explicit ray list; see module docstring)."""
    g = rng(tag)
    Lx, Ly = grid["nx"] * grid["dx"], grid["ny"] * grid["dy"]
    x = g.uniform(0.0, Lx, n)
    y = g.uniform(0.0, Ly, n)
    z = g.uniform(z_lo, z_hi, n)
    lam_h = np.exp(g.uniform(math.log(100e3), math.log(1000e3), n))
    az = g.uniform(0.0, 2.0 * math.pi, n)
    lam_z = np.exp(g.uniform(math.log(1e3), math.log(10e3), n))
    kh = 2.0 * math.pi / lam_h
    k = kh * np.cos(az)
    l = kh * np.sin(az)
    m = -2.0 * math.pi / lam_z
    spec = np.exp(-0.5 * ((np.log(lam_h / 316e3) / 0.5) ** 2 + (np.log(lam_z / 3.16e3) / 0.5) ** 2))
    A = action0 * spec
    dk = frac * kh
    dl = frac * kh
    dm = frac * np.abs(m)
    return dict(x=x, y=y, z=z, k=k, l=l, m=m,
                ex=np.full(n, grid["dx"]), ey=np.full(n, grid["dy"]), ez=np.full(n, ext_z),
                dk=dk, dl=dl, dm=dm, n=A / (dk * dl * dm))


def sphere_rays(grid: dict, n: int, tag: int = 2, z_lo=3e3, z_hi=20e3, lat_max_deg=70.0, frac=0.1,
                action0=1e-3, ext_scale=1.0):
    """Random explicit ray volumes on the sphere (parity tests): positions, k, extents, N."""
    g = rng(tag)
    nx, ny = grid["nx"], grid["ny"]
    x = g.uniform(0.0, 2.0 * math.pi, n)
    y = np.radians(g.uniform(-lat_max_deg, lat_max_deg, n))
    z = g.uniform(z_lo, z_hi, n)
    lam_h = np.exp(g.uniform(math.log(100e3), math.log(1000e3), n))
    az = g.uniform(0.0, 2.0 * math.pi, n)
    lam_z = np.exp(g.uniform(math.log(1e3), math.log(10e3), n))
    kh = 2.0 * math.pi / lam_h
    k = kh * np.cos(az)
    l = kh * np.sin(az)
    m = -2.0 * math.pi / lam_z
    A = action0 * g.uniform(0.2, 1.0, n)
    dk = frac * kh
    dl = frac * kh
    dm = frac * np.abs(m)
    ex = ext_scale * g.uniform(0.3, 1.0, n) * (2.0 * math.pi / nx)
    ey = ext_scale * g.uniform(0.3, 1.0, n) * (math.pi / ny)
    ez = ext_scale * g.uniform(300.0, 1000.0, n)
    return dict(x=x, y=y, z=z, k=k, l=l, m=m, ex=ex, ey=ey, ez=ez, dk=dk, dl=dl, dm=dm, n=A / (dk * dl * dm))


# ---------------------------------------------------------------- sources

def background_source(tau=0.0, z_launch=5e3, dz_launch=1e3, lambda_h=100e3, c_min=5.0, c_max=50.0,
                      n_az=8, n_c=4, frac=0.1, f_s=2.4e-3, f_w=8e-3, phi_max_deg=85.0, launch_zero_flux=1):
    """Parameters of the latitude-dependent background source (values of Sec. 3c where it gives them)."""
    return dict(f_s=f_s, f_w=f_w, tau=tau, z_launch=z_launch, dz_launch=dz_launch, lambda_h=lambda_h,
                c_min=c_min, c_max=c_max, n_az=n_az, n_c=n_c, spectral_frac=frac,
                phi_max_deg=phi_max_deg, launch_zero_flux=launch_zero_flux)


def convective_specs(grid: dict, tag: int, median=16.0, sigma=1.0, cap=512, z_launch=10e3, dz_launch=1e3,
                     lambda_h=100e3, c_min=5.0, c_max=50.0, frac=0.1, flux_max=5e-3, lat_max_deg=85.0,
                     col_fraction=1.0):
    """Explicit spectral launches standing in for a convective source.

    Per column: count = min(cap, round(lognormal(ln median, sigma))), a column flux
    uniform in [0, flux_max] Pa shared equally by its rays, each ray with a uniform
    azimuth and a log-uniform ground-based phase speed in [c_min, c_max].
    ``col_fraction`` < 1 draws convection in that seeded fraction of columns only.
    """
    g = rng(1000 + tag)
    nx, ny = grid["nx"], grid["ny"]
    _, phi, _ = node_coords(grid)
    ok_rows = np.nonzero(np.abs(np.degrees(phi)) <= lat_max_deg)[0] if grid["geometry"] == 1 else np.arange(ny)
    cols_j = np.repeat(ok_rows, nx)
    cols_i = np.tile(np.arange(nx), len(ok_rows))
    active = g.uniform(size=len(cols_i)) < col_fraction
    counts = np.minimum(cap, np.rint(g.lognormal(math.log(median), sigma, size=len(cols_i)))).astype(np.int64)
    counts[~active] = 0
    colflux = g.uniform(0.0, flux_max, size=len(cols_i))
    total = int(counts.sum())
    out = np.zeros(total, dtype=SPEC_DTYPE)
    out["i"] = np.repeat(cols_i, counts)
    out["j"] = np.repeat(cols_j, counts)
    out["z_launch"] = z_launch
    out["dz_launch"] = dz_launch
    out["theta"] = g.uniform(0.0, 2.0 * math.pi, total)
    out["c"] = np.exp(g.uniform(math.log(c_min), math.log(c_max), total))
    out["lambda_h"] = lambda_h
    per = np.where(counts > 0, colflux / np.maximum(counts, 1), 0.0)
    out["flux"] = np.repeat(per, counts)
    out["spectral_frac"] = frac
    return out


def uniform_specs(grid: dict, n_az=8, c_list=(5.0, 5.0 * 10 ** (1 / 3), 5.0 * 10 ** (2 / 3), 50.0),
                  flux=1e-3, z_launch=5e3, dz_launch=1e3, lambda_h=100e3, frac=0.1, lat_max_deg=85.0,
                  azimuths="half_bin"):
    """Explicit spectral launches, the same in every column: n_az azimuths (even) times the phase
    speeds in c_list, each ray carrying flux / (n_az len(c_list)).

    azimuths="half_bin": +-(a + 1/2) 2 pi / n_az, a = 0 .. n_az/2 - 1: mirror pairs (theta, -theta)
    are exact (l = |k_h| sin(theta) flips sign with no rounding difference), so a background without
    meridional structure sees no net meridional flux; and no azimuth lies on an axis, where a
    wavenumber component would be rounding noise (cos(pi/2) is not 0 in floating point).
    azimuths="axis": a 2 pi / n_az, a = 0 .. n_az - 1, the azimuths of the background source (four of
    them on the axes).
    """
    nx, ny = grid["nx"], grid["ny"]
    _, phi, _ = node_coords(grid)
    rows = np.nonzero(np.abs(np.degrees(phi)) <= lat_max_deg)[0] if grid["geometry"] == 1 else np.arange(ny)
    per = n_az * len(c_list)
    ncol = len(rows) * nx
    if azimuths == "axis":
        theta = np.arange(n_az) * (2.0 * math.pi / n_az)
    else:
        half = (np.arange(n_az // 2) + 0.5) * (2.0 * math.pi / n_az)
        theta = np.concatenate([half, -half])
    out = np.zeros(ncol * per, dtype=SPEC_DTYPE)
    out["j"] = np.repeat(rows, nx * per)
    out["i"] = np.tile(np.repeat(np.arange(nx), per), len(rows))
    out["theta"] = np.tile(np.repeat(theta, len(c_list)), ncol)
    out["c"] = np.tile(np.asarray(c_list, dtype=np.float64), ncol * n_az)
    out["z_launch"] = z_launch
    out["dz_launch"] = dz_launch
    out["lambda_h"] = lambda_h
    out["flux"] = flux / per
    out["spectral_frac"] = frac
    return out


# ---------------------------------------------------------------- named workloads

def workload(name: str) -> dict:
    """Grid, parameters, background and initial-condition recipe of a named workload."""
    if name == "fplane":
        grid = fplane_grid()
        params = dict(DEFAULT_PARAMS, saturation=0, smoothing=0)
        return dict(name=name, grid=grid, params=params, background=uniform_background(grid),
                    rays=fplane_rays(grid, 4096, tag=1), source=None, dt=300.0, steps=100)
    if name == "sphere_ghost":
        # the background source emitted through the ghost layer every 60 s interval (the paper's model
        # step), starting from no rays
        grid = sphere_grid(nx=256, ny=128, nz=90, dz=1000.0)
        return dict(name=name, grid=grid, params=dict(DEFAULT_PARAMS), background=jet_background(grid),
                    rays=None, source=background_source(), dt=60.0, steps=200, ghost=True)
    if name in ("sphere", "sphere_fp32", "sphere_half", "sphere_half_fp32", "sphere_columnar", "sphere_coupled",
                "sphere_theta"):
        nx, ny = {"sphere": (256, 128), "sphere_fp32": (512, 256), "sphere_half": (128, 64),
                  "sphere_half_fp32": (128, 64), "sphere_columnar": (256, 128), "sphere_coupled": (256, 128),
                  "sphere_theta": (256, 128)}[name]
        grid = sphere_grid(nx=nx, ny=ny, nz=90, dz=1000.0)
        # sphere_theta: the potential-temperature flux integrals projected as well (theta_flux)
        params = dict(DEFAULT_PARAMS, columnar=1 if name == "sphere_columnar" else 0,
                      theta_flux=1 if name == "sphere_theta" else 0)
        # sphere_coupled: the background is advanced by the drag after every step (online coupling)
        return dict(name=name, grid=grid, params=params, background=jet_background(grid),
                    rays=None, source=background_source(), dt=180.0, steps=200,
                    coupled=name == "sphere_coupled")
    raise KeyError(name)


def isothermal_theta(grid: dict, T=240.0):
    """Reference potential temperature of the isothermal atmosphere: d ln theta / dz = N^2 / g."""
    n2c, _, _ = isothermal(T)
    _, _, z = node_coords(grid)
    shape = (grid["nz"], grid["ny"], grid["nx"])
    return np.broadcast_to((T * np.exp(n2c * z / GRAVITY))[:, None, None], shape).copy()


def ensemble_members(grid: dict, members: int = 16, tag: int = 4):
    """Backgrounds of the batched ensemble: jet amplitude U[30, 80] m/s, jet latitude U[30, 60] deg."""
    g = rng(tag)
    amps = g.uniform(30.0, 80.0, members)
    lats = g.uniform(30.0, 60.0, members)
    return [jet_background(grid, amp=float(a), lat_deg=float(p)) for a, p in zip(amps, lats)], amps, lats


def ensemble_workload(members: int = 16, nx: int = 256, ny: int = 128, nz: int = 90):
    """Batched ensemble: `members` spheres (jets U[30, 80] m/s at U[30, 60] deg), each with the
    background source at 5 km and convective spectral launches at 10 km: lognormal(ln 16, 1) rays
    per column, capped at 512 (uneven per-column counts)."""
    grid = sphere_grid(nx=nx, ny=ny, nz=nz, dz=1000.0)
    bgs, amps, lats = ensemble_members(grid, members)
    specs = []
    for m in range(members):
        sp = convective_specs(grid, tag=400 + m, median=16.0, sigma=1.0, cap=512, z_launch=10e3)
        sp["member"] = m
        specs.append(sp)
    return dict(name="ensemble", grid=grid, params=dict(DEFAULT_PARAMS), backgrounds=bgs, specs=specs,
                source=background_source(), dt=180.0, members=members, amps=amps, lats=lats)
