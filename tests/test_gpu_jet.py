"""Jet-refraction run with online coupling (Sec. 4, the discussion of horizontally sheared jets).

The paper finds that the 3-D scheme propagates wave action horizontally into a zonal jet, where the
columnar scheme (MS-GWaM-1D) can only produce meridional fluxes from the launch spectrum and vertical
filtering.  Here the mechanism is isolated on an f-plane channel: a zonal jet U(y, z) symmetric about
the channel centre, the same 8-azimuth x 4-phase-speed launch in every column (mirror azimuths
(theta, -theta) in pairs), and the background advanced by the drag after every step (u += dt du/dt,
v += dt dv/dt, then handed back to the tracer).  With a constant f and no metric terms, the only
source of a net meridional wave-action flux is refraction by the jet's shear (the wavenumber equation
of Eq. eikonal: dl/dt = -k dU/dy with V = 0 and uniform N, f):

* columnar mode with the jet, and the 3-D scheme without a jet: the flux of each latitude band
  vanishes to rounding (mirror pairs cancel);
* 3-D scheme with the jet: the flux points into the jet on both flanks (flux convergence at the jet
  core), antisymmetric about the centre.

The meridional wave-action flux of a band is sum_j W_j c_y,j over the ray volumes in it (W the wave
action, c_y the intrinsic meridional group velocity from the oracle's dispersion relation).
A small coupled case is also compared with the oracle coupled to its own tendencies, and the sphere
workload (256 x 128 x 90, ~0.98 M ray volumes) runs coupled to its drag with its budget closing.
"""
import numpy as np
import pytest

import oracle
from paper_2309_11257_gb300 import synth
from parity_util import assert_fields_match, assert_level_errors, assert_rays_match, assert_stats_match

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    from paper_2309_11257_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2309_11257_gb300 import gwam
    return gwam


def _coupled_run(gw, grid, params, bg, launch, steps, dt):
    import torch
    T = gw.Tracer(grid, params, max_rays=int(2.5 * 32 * grid["nx"] * grid["ny"]))
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in bg]
    T.set_background(*dev)
    launch(T)
    du = torch.zeros_like(dev[0])
    dv = torch.zeros_like(dev[0])
    for _ in range(steps):
        T.step(dt, du, dv)
        dev[0].add_(du, alpha=dt)
        dev[1].add_(dv, alpha=dt)
        T.set_background(*dev)
    torch.cuda.synchronize()
    out = (T.rays(), T.stats(), dev[0].cpu().numpy(), dev[1].cpu().numpy(), du.cpu().numpy())
    T.close()
    return out


def _meridional_flux(grid, r, n2, bands, zlo, zhi):
    """Per band (offsets from the channel centre) sum_j W_j c_y,j over zlo < z < zhi, and the scale
    sum_j W_j |c_y,j| over the selection."""
    H = synth.isothermal()[1]
    g2 = 1.0 / (4.0 * H * H)   # Gamma^2 of the isothermal density profile (gamma_mode 1)
    f2 = grid["f0"] ** 2
    cy = np.array([oracle.dispersion(k, l, m, n2, g2, f2)[2] for k, l, m in zip(r["k"], r["l"], r["m"])])
    W = r["n"] * r["px"] * r["py"] * r["pz"]
    sel = (r["z"] > zlo) & (r["z"] < zhi)
    d = r["y"] - 0.5 * grid["ny"] * grid["dy"]
    flux = np.array([np.sum((W * cy)[sel & (d >= b0) & (d < b1)]) for b0, b1 in zip(bands[:-1], bands[1:])])
    scale = np.sum(np.abs(W * cy)[sel & (d >= bands[0]) & (d < bands[-1])])
    return flux, scale


def test_channel_jet_refraction(gw):
    grid = synth.fplane_grid(nx=16, ny=64, nz=60, dx=50e3, dy=50e3, dz=1000.0)
    specs = synth.uniform_specs(grid)
    bands = np.array([-1200, -800, -500, -300, -150, 0, 150, 300, 500, 800, 1200]) * 1e3
    south = slice(0, 5)          # bands with y < y_c
    north = slice(5, 10)
    res = {}
    for tag, columnar, amp in (("3d_jet", 0, 40.0), ("1d_jet", 1, 40.0), ("3d_nojet", 0, 0.0)):
        bg = synth.channel_jet_background(grid, amp=amp)
        params = dict(synth.DEFAULT_PARAMS, columnar=columnar)
        r, st, u, v, du = _coupled_run(gw, grid, params, bg, lambda T: T.launch_spectral(specs), 150, 180.0)
        assert st["n_launched"] == len(specs) and st["n_live"] > 0.5 * len(specs)
        assert np.all(np.isfinite(u)) and np.all(np.isfinite(v))
        if amp > 0:
            assert np.abs(u - bg[0]).max() > 1e-3       # the drag moved the jet
        res[tag] = _meridional_flux(grid, r, 0.02 ** 2, bands, 15e3, 60e3)
    # no jet, or no horizontal propagation: mirror pairs cancel band by band
    for tag in ("1d_jet", "3d_nojet"):
        flux, scale = res[tag]
        assert scale > 0
        assert np.all(np.abs(flux) <= 1e-12 * scale), (tag, flux / scale)
    # 3-D with the jet: wave action flows into the jet from both flanks, symmetric about the centre
    flux, scale = res["3d_jet"]
    assert np.all(flux[south] > 1e-4 * scale), flux / scale
    assert np.all(flux[north] < -1e-4 * scale), flux / scale
    np.testing.assert_allclose(flux[north], -flux[south][::-1], rtol=0, atol=1e-6 * scale)


@pytest.mark.parametrize("azimuths", ["axis", "half_bin"])
def test_coupled_run_parity(gw, azimuths):
    """Both sides coupled to their own tendencies for 9 steps: rays, budget, fields and tendencies
    to the parity bars of the uncoupled cases.  "axis" launches at the background source's azimuths
    (multiples of 45 deg, four on the axes, where one wavenumber component is rounding noise that
    the coupled drag moves differently on each side; the bars measure wavenumbers against |k_h| and
    the fields against orientation-independent scales), "half_bin" at +-(a + 1/2) 45 deg."""
    import torch
    grid = synth.fplane_grid(nx=8, ny=24, nz=30, dx=60e3, dy=60e3, dz=1000.0)
    bg = [np.array(a) for a in synth.channel_jet_background(grid, amp=40.0, width=250e3, z_peak=20e3,
                                                             z_width=8e3)]
    specs = synth.uniform_specs(grid, flux=5e-3, azimuths=azimuths)
    params = dict(synth.DEFAULT_PARAMS)
    T = gw.Tracer(grid, params, max_rays=200000)
    O = oracle.Model(grid, params)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in bg]
    T.set_background(*dev)
    O.set_background(*bg)
    T.launch_spectral(specs)
    O.launch_spectral(specs)
    dt = 300.0
    du = torch.zeros_like(dev[0])
    dv = torch.zeros_like(dev[0])
    for s in range(9):
        T.step(dt, du, dv)
        odu, odv = O.step(dt)
        if s % 4 == 0 or s == 8:
            assert_rays_match(T.rays(), O.rays(), grid)
            assert_stats_match(T.stats(), O.stats())
            su, sv = O.tendency_scale()
            assert_fields_match(du.cpu().numpy(), odu, su, name="dudt")
            assert_fields_match(dv.cpu().numpy(), odv, sv, name="dvdt")
            assert_level_errors(du.cpu().numpy(), odu, su, name="dudt")
            assert_level_errors(dv.cpu().numpy(), odv, sv, name="dvdt")
            for name in oracle.FIELD_NAMES:
                assert_fields_match(T.field(name), O.field(name), O.field_abs(name), name=name)
        dev[0].add_(du, alpha=dt)
        dev[1].add_(dv, alpha=dt)
        T.set_background(*dev)
        bg[0] += dt * odu
        bg[1] += dt * odv
        O.set_background(*bg)
    assert np.abs(bg[0] - synth.channel_jet_background(grid, amp=40.0, width=250e3, z_peak=20e3,
                                                       z_width=8e3)[0]).max() > 1e-6


def test_sphere_coupled_run(gw):
    """The sphere workload (two 60 m/s jets at +-45 deg, background source at 5 km) run for 100 steps
    of 180 s with the background advanced by its own drag: finite throughout, and the wave-action
    budget closes (W = launched - saturated - exited - capped - invalid)."""
    w = synth.workload("sphere")
    r, st, u, v, du = _coupled_run(gw, w["grid"], w["params"], w["background"],
                                   lambda T: T.launch_sources(w["source"]), 100, w["dt"])
    assert st["n_launched"] > 900000 and st["n_invalid"] == 0
    assert np.all(np.isfinite(u)) and np.all(np.isfinite(v)) and np.all(np.isfinite(du))
    assert np.abs(u - w["background"][0]).max() > 1e-2
    rhs = st["w_launched"] - st["w_saturated"] - st["w_exited"] - st["w_capped"] - st["w_invalid"]
    assert st["w_total"] == pytest.approx(rhs, rel=1e-12)
    assert np.all(np.isfinite(r["n"])) and np.all(r["n"] >= 0)
