"""Ghost-layer launch (Sec. 3c) on the GPU against the FP64 oracle.

Each cycle emits, per source bin, the part of a layer-filling ghost ray volume that propagated
(vertically only) out of the launch layer over the interval, then steps every ray volume.  Rays,
budget, fields and tendencies are compared with the oracle running the same cycles, at the parity
bars of the other cases; the reflection discard and the steady source flux of repeated emission
are checked as in the oracle's pins.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2309_11257_gb300 import synth
from parity_util import assert_fields_match, assert_rays_match, assert_stats_match

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    from paper_2309_11257_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2309_11257_gb300 import gwam
    return gwam


def _pair(gw, grid, params, bg, max_rays=400000):
    import torch
    T = gw.Tracer(grid, params, max_rays=max_rays)
    O = oracle.Model(grid, params)
    T.set_background(*[torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in bg])
    O.set_background(*bg)
    return T, O


def _compare(T, O, grid, du, dv, odu, odv):
    assert_rays_match(T.rays(), O.rays(), grid)
    assert_stats_match(T.stats(), O.stats())
    su, sv = O.tendency_scale()
    assert_fields_match(du.cpu().numpy(), odu, su, name="dudt")
    assert_fields_match(dv.cpu().numpy(), odv, sv, name="dvdt")
    for name in oracle.FIELD_NAMES:
        assert_fields_match(T.field(name), O.field(name), O.field_abs(name), name=name)


def _cycles(T, O, grid, launch_t, launch_o, dt, n, check_every=3):
    import torch
    du = torch.zeros((grid["nz"], grid["ny"], grid["nx"]), dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(du)
    for s in range(n):
        launch_t(dt)
        launch_o(dt)
        if s == 0:
            assert_rays_match(T.rays(), O.rays(), grid)
            assert_stats_match(T.stats(), O.stats())
        T.step(dt, du, dv)
        odu, odv = O.step(dt)
        if s % check_every == check_every - 1 or s == n - 1:
            _compare(T, O, grid, du, dv, odu, odv)


def test_ghost_spectral_parity_fplane(gw):
    """Perturbed sheared f-plane, every column emitting 8 azimuths x 4 phase speeds each interval,
    saturation, splitting, smoothing and a per-column cap on; 7 cycles of 240 s."""
    grid = synth.fplane_grid(nx=12, ny=10, nz=40, dx=40e3, dy=30e3, dz=500.0)
    bg = synth.perturbed(synth.uniform_background(grid, U=8.0, V=-3.0), tag=61, rel=0.1)
    params = dict(synth.DEFAULT_PARAMS, cap_per_column=60)
    specs = synth.uniform_specs(grid, flux=4e-3, z_launch=3e3)
    T, O = _pair(gw, grid, params, bg)
    _cycles(T, O, grid, lambda dt: T.launch_ghost_spectral(specs, dt), lambda dt: O.launch_ghost_spectral(specs, dt),
            240.0, 7)
    st = T.stats()
    assert st["n_launched"] > 6 * 0.8 * len(specs) and st["n_capped"] > 0


def test_ghost_source_parity_sphere(gw):
    """Sphere with perturbed jets: the background source of Sec. 3c emitted through the ghost layer
    every interval, 6 cycles of 300 s."""
    grid = synth.sphere_grid(nx=24, ny=16, nz=30, dz=1000.0)
    bg = synth.perturbed(synth.jet_background(grid, z_peak=15e3, z_width=6e3), tag=62)
    params = dict(synth.DEFAULT_PARAMS, cap_per_column=200)
    src = synth.background_source(z_launch=3e3, launch_zero_flux=0)
    T, O = _pair(gw, grid, params, bg)
    _cycles(T, O, grid, lambda dt: T.launch_ghost(src, dt), lambda dt: O.launch_ghost(src, dt), 300.0, 6)
    assert T.stats()["n_launched"] > 0


def test_ghost_reflection_and_steady_flux(gw):
    """As the oracle's pins: a bin reflected within the layer is discarded, a slow one emitted; and
    emitting every interval in a uniform medium gives the source flux at every filled interface."""
    import torch
    grid = synth.fplane_grid(nx=2, ny=2, nz=40, dx=50e3, dy=50e3, dz=500.0, f0=1e-4)
    u, v, n2, rho = synth.uniform_background(grid, U=0.0)
    _, _, z = synth.node_coords(grid)
    n2 = np.broadcast_to((4e-4 * np.exp(-(z - 5.5e3) / 4e3))[:, None, None], n2.shape).copy()
    kh = 2.0 * math.pi / 100e3
    sp = synth.uniform_specs(grid)[:2]
    sp["i"] = sp["j"] = 0
    sp["theta"] = 0.0
    sp["c"] = [0.999 * 0.02 / kh, 0.1 * 0.02 / kh]
    T, O = _pair(gw, grid, dict(synth.DEFAULT_PARAMS, saturation=0, smoothing=0, gamma_mode=0), (u, v, n2, rho))
    T.launch_ghost_spectral(sp, 60.0)
    O.launch_ghost_spectral(sp, 60.0)
    st = T.stats()
    assert (st["n_launched"], st["n_filtered"]) == (1, 1)
    assert_rays_match(T.rays(), O.rays(), grid)

    grid = synth.fplane_grid(nx=2, ny=2, nz=60, dx=50e3, dy=50e3, dz=500.0, f0=1e-4)
    bg = synth.uniform_background(grid, U=0.0)
    sp = synth.uniform_specs(grid, flux=1e-3, c_list=(23.2,), n_az=2)
    sp = sp[sp["theta"] > 0]
    sp["theta"] = 0.0
    sp["flux"] = 1e-3
    T, O = _pair(gw, grid, dict(synth.DEFAULT_PARAMS, saturation=0, smoothing=0, flux_form=1), bg)
    du = torch.zeros((60, 2, 2), dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(du)
    n = 30
    for _ in range(n):
        T.launch_ghost_spectral(sp, 120.0)
        T.step(120.0, du, dv)
    r = T.rays()
    delta = r["ez"].max()
    assert len(r["z"]) == 4 * n
    fz = T.field("fz_l")
    zi = np.arange(61) * 500.0
    inside = (zi - 250.0 > 6e3 + delta) & (zi + 250.0 < 6e3 + (n + 1) * delta)
    assert inside.sum() >= 8
    np.testing.assert_allclose(fz[inside], 1e-3, rtol=1e-12)


def test_ghost_launch_rejects(gw):
    grid = synth.fplane_grid(nx=4, ny=4, nz=20, dx=50e3, dy=50e3, dz=500.0)
    bg = synth.uniform_background(grid)
    specs = synth.uniform_specs(grid)
    T, _ = _pair(gw, grid, dict(synth.DEFAULT_PARAMS), bg)
    for dt in (0.0, -60.0, float("inf"), float("nan")):
        with pytest.raises(gw.GwamError):
            T.launch_ghost_spectral(specs, dt)
    assert T.num_rays() == 0
    bad = specs[:4].copy()
    bad["i"][2] = grid["nx"]
    with pytest.raises(gw.GwamError):
        T.launch_ghost_spectral(bad, 60.0)
    assert T.num_rays() == 0
