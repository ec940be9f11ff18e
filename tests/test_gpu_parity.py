"""CUDA path (libgwam.so through the C ABI) against the FP64 CPU oracle, element by element.

Small cases run both sides over many steps (several tiles and ragged tails: ray counts are not
multiples of the block size, grids not multiples of the divergence tile); the full-size sphere
workload (256 x 128 x 90 columns, 983 040 launched ray volumes, launch configuration of the
benchmark) compares the launch and a complete step in full.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2309_11257_gb300 import synth
from parity_util import (RTOL, assert_fields_match, assert_level_errors, assert_rays_match, assert_stats_match,
                         level_error, odd_field_case, state_errors)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    from paper_2309_11257_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2309_11257_gb300 import gwam
    return gwam


def _pair(gw, grid, params, bg, max_rays):
    import torch
    T = gw.Tracer(grid, params, max_rays=max_rays)
    O = oracle.Model(grid, params)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in bg]
    T.set_background(*dev)
    O.set_background(*bg)
    return T, O


def _step_both(T, O, dt, nz, ny, nx):
    import torch
    du = torch.zeros((nz, ny, nx), dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(du)
    T.step(dt, du, dv)
    odu, odv = O.step(dt)
    return du.cpu().numpy(), dv.cpu().numpy(), odu, odv


def _compare_all(T, O, grid, du=None, dv=None, odu=None, odv=None, fields=True, report=None):
    errs = assert_rays_match(T.rays(), O.rays(), grid)
    assert_stats_match(T.stats(), O.stats())
    if du is not None:
        su, sv = O.tendency_scale()
        eu = assert_fields_match(du, odu, su, name="dudt")
        ev = assert_fields_match(dv, odv, sv, name="dvdt")
        # beside the elementwise bar: the plain per-level relative drag error
        lu = assert_level_errors(du, odu, su, name="dudt")
        lv = assert_level_errors(dv, odv, sv, name="dvdt")
        if report is not None:
            report.append(dict(state=errs, dudt_scaled=eu, dvdt_scaled=ev, dudt_level=lu, dvdt_level=lv))
    if fields:
        for name in oracle.FIELD_NAMES:
            assert_fields_match(T.field(name), O.field(name), O.field_abs(name), name=name)
    return errs


def test_odd_field_lengths_are_cleared_every_step(gw):
    """Fields of odd length: every projected field compared element by element after each of four
    steps (a value left from the previous step would add to this step's sums)."""
    grid, bg, rays, params = odd_field_case()
    T, O = _pair(gw, grid, params, bg, 4096)
    T.add_rays(rays)
    O.add_rays(rays)
    nz, ny, nx = grid["nz"], grid["ny"], grid["nx"]
    for _ in range(4):
        du, dv, odu, odv = _step_both(T, O, 120.0, nz, ny, nx)
        _compare_all(T, O, grid, du, dv, odu, odv)
        assert O.field("wad")[nz - 1, ny - 1, nx - 1] > 0.0      # the odd last element carries action
        assert T.field("wad")[nz - 1, ny - 1, nx - 1] == pytest.approx(O.field("wad")[nz - 1, ny - 1, nx - 1],
                                                                       rel=1e-12)


def test_fplane_workload_parity(gw):
    """f-plane box (16 x 16 x 64), 1000 ray volumes, 20 steps of 300 s."""
    w = synth.workload("fplane")
    grid, params = w["grid"], w["params"]
    rays = synth.fplane_rays(grid, 1000, tag=11)
    # and ray volumes just below the top (32 km), so that some leave the domain (exit path)
    top = synth.fplane_rays(grid, 100, tag=13, z_lo=29.5e3, z_hi=31.5e3)
    T, O = _pair(gw, grid, params, w["background"], 8192)
    for r in (rays, top):
        T.add_rays(r)
        O.add_rays(r)
    _compare_all(T, O, grid, fields=False)
    for s in range(20):
        du, dv, odu, odv = _step_both(T, O, 300.0, grid["nz"], grid["ny"], grid["nx"])
        if s % 5 == 4:
            _compare_all(T, O, grid, du, dv, odu, odv)
    assert O.stats()["n_exited"] > 0


@pytest.mark.parametrize("variant", ["direct", "pseudomomentum_gamma0"])
def test_fplane_inhomogeneous_parity(gw, variant):
    """f-plane with a smoothly perturbed background: refraction, splits, saturation on."""
    grid = synth.fplane_grid(nx=24, ny=20, nz=40, dx=40e3, dy=30e3, dz=500.0)
    bg = synth.perturbed(synth.uniform_background(grid, U=5.0), tag=21, rel=0.1)
    params = dict(synth.DEFAULT_PARAMS, smoothing=1, saturation=1, cap_per_column=12)
    if variant != "direct":
        params.update(flux_form=1, gamma_mode=0)
    rays = synth.fplane_rays(grid, 1500, tag=22, z_lo=3e3, z_hi=15e3, ext_z=1300.0)
    rays["n"] = rays["n"] * 1e8
    T, O = _pair(gw, grid, params, bg, 20000)
    T.add_rays(rays)
    O.add_rays(rays)
    for s in range(12):
        du, dv, odu, odv = _step_both(T, O, 240.0, grid["nz"], grid["ny"], grid["nx"])
        if s % 4 == 3:
            _compare_all(T, O, grid, du, dv, odu, odv)
    st = O.stats()
    assert st["n_split_v"] > 0 and st["w_saturated"] > 0 and st["n_capped"] > 0


def test_sphere_parity_with_launches_caps_and_exits(gw):
    """Sphere 40 x 20 x 24 with jets, two background launches, explicit ray volumes near the top,
    saturation, smoothing, splitting and a per-column cap."""
    grid = synth.sphere_grid(nx=40, ny=20, nz=24, dz=1000.0)
    bg = synth.perturbed(synth.jet_background(grid, z_peak=15e3, z_width=6e3), tag=31)
    params = dict(synth.DEFAULT_PARAMS, cap_per_column=45)
    T, O = _pair(gw, grid, params, bg, 200000)
    src = synth.background_source(z_launch=2e3)
    T.launch_sources(src)
    O.launch_background(src)
    rays = synth.sphere_rays(grid, 777, tag=32, z_lo=14e3, z_hi=23.5e3, ext_scale=3.0)
    rays["n"] = rays["n"] * 30.0
    T.add_rays(rays)
    O.add_rays(rays)
    _compare_all(T, O, grid, fields=False)
    for s in range(10):
        if s == 5:
            T.launch_sources(src)
            O.launch_background(src)
        du, dv, odu, odv = _step_both(T, O, 300.0, grid["nz"], grid["ny"], grid["nx"])
        if s % 3 == 2 or s == 9:
            _compare_all(T, O, grid, du, dv, odu, odv)
    st = O.stats()
    assert st["n_exited"] > 0 and st["n_capped"] > 0 and st["n_split_h"] > 0 and st["w_saturated"] > 0


@pytest.mark.parametrize("geometry", ["sphere", "fplane"])
def test_gamma2_matches_the_oracle(gw, geometry):
    """Gamma^2 = (d ln rho / dz)^2 / 4 (Sec. 2a reading): the device forms the centred differences as
    logarithms of density ratios in double-float; the oracle differences FP64 logarithms.  Same
    nodes, relative 1e-12 (the ratio form is the better conditioned of the two)."""
    if geometry == "sphere":
        grid = synth.sphere_grid(nx=40, ny=20, nz=24, dz=1000.0)
        bg = synth.perturbed(synth.jet_background(grid, z_peak=15e3, z_width=6e3), tag=31)
    else:
        w = synth.workload("fplane")
        grid, bg = w["grid"], synth.perturbed(w["background"], tag=44)
    T, O = _pair(gw, grid, dict(synth.DEFAULT_PARAMS), bg, 1000)
    g, o = T.gamma2(), O.gamma2()
    assert g.shape == o.shape
    np.testing.assert_allclose(g, o, rtol=1e-12, atol=0)


@pytest.mark.parametrize("geometry", ["sphere", "fplane"])
def test_columnar_mode_parity(gw, geometry):
    """Single-column mode (MS-GWaM-1D): the same parity bars as the 3-D model, and the horizontal
    position, wavenumber and extents of every ray volume exactly as launched."""
    if geometry == "sphere":
        grid = synth.sphere_grid(nx=40, ny=20, nz=24, dz=1000.0)
        bg = synth.perturbed(synth.jet_background(grid, z_peak=15e3, z_width=6e3), tag=31)
        rays = synth.sphere_rays(grid, 777, tag=32, z_lo=4e3, z_hi=20e3, ext_scale=1.0)
        dt = 300.0
    else:
        grid = synth.fplane_grid(nx=24, ny=20, nz=40, dx=40e3, dy=30e3, dz=500.0)
        bg = synth.perturbed(synth.uniform_background(grid, U=5.0), tag=21, rel=0.1)
        rays = synth.fplane_rays(grid, 1500, tag=22, z_lo=3e3, z_hi=15e3, ext_z=1300.0)
        dt = 240.0
    rays["n"] = rays["n"] * 30.0
    params = dict(synth.DEFAULT_PARAMS, cap_per_column=45, columnar=1)
    T, O = _pair(gw, grid, params, bg, 200000)
    T.add_rays(rays)
    O.add_rays(rays)
    r0 = T.rays()
    for s in range(8):
        du, dv, odu, odv = _step_both(T, O, dt, grid["nz"], grid["ny"], grid["nx"])
        if s % 3 == 2 or s == 7:
            _compare_all(T, O, grid, du, dv, odu, odv)
    r1 = T.rays()
    assert T.stats()["n_split_h"] == 0
    common, i0, i1 = np.intersect1d(r0["id"], r1["id"], return_indices=True)
    assert len(common) > 0.5 * len(r0["id"])
    for n in ("x", "y", "k", "l", "ex", "ey"):   # vertical splits move z, ez, pz only
        np.testing.assert_array_equal(r1[n][i1], r0[n][i0])


@pytest.mark.parametrize("geometry", ["sphere", "fplane"])
def test_theta_flux_and_tendency_parity(gw, geometry):
    """Potential-temperature flux integrals (Eq. fluxes:temperature) and d theta/dt (Eq.
    mean-flow-impact-t) against the oracle, scaled as the other projected fields; the momentum
    path is unchanged by projecting them."""
    import torch
    if geometry == "sphere":
        grid = synth.sphere_grid(nx=40, ny=20, nz=24, dz=1000.0)
        bg = synth.perturbed(synth.jet_background(grid, z_peak=15e3, z_width=6e3), tag=31)
        rays = synth.sphere_rays(grid, 777, tag=32, z_lo=4e3, z_hi=20e3, ext_scale=3.0)
        dt = 300.0
    else:
        grid = synth.fplane_grid(nx=24, ny=20, nz=40, dx=40e3, dy=30e3, dz=500.0)
        bg = synth.perturbed(synth.uniform_background(grid, U=5.0), tag=21, rel=0.1)
        rays = synth.fplane_rays(grid, 1500, tag=22, z_lo=3e3, z_hi=15e3, ext_z=1300.0)
        dt = 240.0
    rays["n"] = rays["n"] * 30.0
    _, _, z = synth.node_coords(grid)
    theta = 240.0 * np.exp(bg[2] * z[:, None, None] / grid["g"])      # d ln theta/dz = N^2 / g
    params = dict(synth.DEFAULT_PARAMS, cap_per_column=45, theta_flux=1)
    T, O = _pair(gw, grid, params, bg, 200000)
    T0, _ = _pair(gw, grid, dict(params, theta_flux=0), bg, 200000)
    T.set_theta(torch.from_numpy(np.ascontiguousarray(theta)).cuda())
    O.set_theta(theta)
    for X in (T, O, T0):
        X.add_rays(rays)
    for s in range(6):
        du, dv, odu, odv = _step_both(T, O, dt, grid["nz"], grid["ny"], grid["nx"])
        T0.step(dt, *[torch.zeros((grid["nz"], grid["ny"], grid["nx"]), dtype=torch.float64, device="cuda")
                      for _ in range(2)])
        if s % 2 == 1:
            _compare_all(T, O, grid, du, dv, odu, odv)
            for name in oracle.THETA_FIELD_NAMES:
                assert_fields_match(T.field(name), O.field(name), O.field_abs(name), name=name)
            th, sc = O.theta_tendency()
            assert_fields_match(T.theta_tendency(), th, sc, name="dtheta/dt")
            assert np.abs(th).max() > 0.0
    r, r0 = T.rays(), T0.rays()
    for n in oracle.STATE_NAMES:
        np.testing.assert_array_equal(r[n], r0[n])


def test_spectral_launch_parity(gw):
    """Explicit spectral launches (convective-like source) incl. filtered bins."""
    grid = synth.sphere_grid(nx=36, ny=18, nz=30, dz=1000.0)
    bg = synth.jet_background(grid, z_peak=20e3, z_width=8e3)
    specs = synth.convective_specs(grid, tag=41, median=4.0, cap=20, z_launch=8e3)
    specs["c"][::7] = 0.01     # w below |f|: filtered
    T, O = _pair(gw, grid, dict(synth.DEFAULT_PARAMS), bg, 100000)
    T.launch_spectral(specs)
    O.launch_spectral(specs)
    assert T.stats()["n_filtered"] == O.stats()["n_filtered"] > 0
    for _ in range(4):
        du, dv, odu, odv = _step_both(T, O, 300.0, grid["nz"], grid["ny"], grid["nx"])
    _compare_all(T, O, grid, du, dv, odu, odv)


def test_full_size_sphere_launch_and_step(gw):
    """The benchmark configuration: 256 x 128 x 90, background source (983 040 ray volumes),
    one full step of 180 s, compared in full (state, counters, tendencies, fields)."""
    w = synth.workload("sphere")
    grid = w["grid"]
    T, O = _pair(gw, grid, w["params"], w["background"], 2_500_000)
    T.launch_sources(w["source"])
    O.launch_background(w["source"])
    assert T.stats()["n_launched"] == O.stats()["n_launched"] == 120 * 256 * 32
    _compare_all(T, O, grid, fields=False)
    du, dv, odu, odv = _step_both(T, O, w["dt"], grid["nz"], grid["ny"], grid["nx"])
    _compare_all(T, O, grid, du, dv, odu, odv)


def test_sphere_200_steps_compared_every_25(gw):
    """The benchmark's physics over its whole 200-step run (saturation aloft, splits at altitude,
    exits through the top) on a 64 x 32 x 90 sphere: the same jets, background source (61 440 ray
    volumes) and dt of 180 s, compared in full every 25 steps (ids, cells, counters, ray state per
    ray, tendencies elementwise and per level, every projected field)."""
    w = synth.workload("sphere")
    grid = synth.sphere_grid(nx=64, ny=32, nz=90, dz=1000.0)
    T, O = _pair(gw, grid, w["params"], synth.jet_background(grid), 400_000)
    T.launch_sources(w["source"])
    O.launch_background(w["source"])
    report = []
    for s in range(200):
        du, dv, odu, odv = _step_both(T, O, w["dt"], grid["nz"], grid["ny"], grid["nx"])
        if s % 25 == 24:
            _compare_all(T, O, grid, du, dv, odu, odv, report=report)
    for q, r in enumerate(report):
        print("step %d: state %s; dudt %.2e dvdt %.2e of S; per-level %s %s" % (
            25 * (q + 1), {k: "%.1e" % v for k, v in r["state"].items()}, r["dudt_scaled"], r["dvdt_scaled"],
            r["dudt_level"], r["dvdt_level"]))
    st = O.stats()
    assert st["n_exited"] > 0 and st["n_split_v"] + st["n_split_h"] > 0 and st["w_saturated"] > 0


def test_full_size_sampled_rays_over_several_steps(gw):
    """Full-size run for 5 steps on the GPU; sampled ray volumes that neither split nor left are
    advanced one by one from the oracle's own launch state with the oracle's single-ray RK3."""
    w = synth.workload("sphere")
    grid = w["grid"]
    T, O = _pair(gw, grid, dict(w["params"], splitting=0), w["background"], 2_500_000)
    T.launch_sources(w["source"])
    O.launch_background(w["source"])
    r0 = O.rays()
    for _ in range(5):
        T.step(w["dt"])
    g = T.rays()
    pos = {int(i): q for q, i in enumerate(g["id"])}
    rng = np.random.default_rng(5)
    sample = rng.choice(len(r0["id"]), size=600, replace=False)
    checked = 0
    for q in sample:
        s = np.array([r0[n][q] for n in oracle.STATE_NAMES])
        for _ in range(5):
            s = O.advance_ray(s, w["dt"])
        i = int(r0["id"][q])
        if i not in pos:
            continue
        p = pos[i]
        got = np.array([g[n][p] for n in oracle.STATE_NAMES])
        d = got - s
        d[0] = (d[0] + math.pi) % (2 * math.pi) - math.pi
        scale = np.maximum(np.abs(s), 1e-300)
        # per-ray relative error; k, l near zero measured against |k_h|
        kh = math.hypot(s[3], s[4])
        scale[3] = scale[4] = kh
        scale[0] = 2 * math.pi
        assert np.all(np.abs(d) <= 1e-9 * scale), (i, d / scale)
        checked += 1
    assert checked > 500
    # saturation sink and budget closure at full size (W after = W0 + launched - sinks)
    st = T.stats()
    rhs = st["w_launched"] - st["w_saturated"] - st["w_exited"] - st["w_capped"] - st["w_invalid"]
    assert st["w_total"] == pytest.approx(rhs, rel=1e-12)


def test_deterministic_ray_state(gw):
    grid = synth.sphere_grid(nx=40, ny=20, nz=24, dz=1000.0)
    bg = synth.perturbed(synth.jet_background(grid, z_peak=15e3, z_width=6e3), tag=31)
    outs = []
    for _ in range(2):
        T, _ = _pair(gw, grid, dict(synth.DEFAULT_PARAMS), bg, 200000)
        T.launch_sources(synth.background_source(z_launch=2e3))
        for _ in range(6):
            T.step(300.0)
        outs.append((T.rays(), T.stats()))
    for n in ("id", "cell") + tuple(oracle.STATE_NAMES):
        np.testing.assert_array_equal(outs[0][0][n], outs[1][0][n])
    assert outs[0][1] == outs[1][1]


def test_edge_cases(gw):
    import torch
    grid = synth.fplane_grid(nx=8, ny=8, nz=16)
    bg = synth.uniform_background(grid)
    params = dict(synth.DEFAULT_PARAMS, saturation=0, smoothing=0)
    # step before any background
    T = gw.Tracer(grid, params, max_rays=100)
    with pytest.raises(gw.GwamError) as e:
        T.step(10.0)
    assert e.value.code == gw.GWAM_ESTATE
    # empty population: a step is valid and yields zero tendencies
    dev = [torch.from_numpy(a.copy()).cuda() for a in bg]
    T.set_background(*dev)
    du = torch.ones((16, 8, 8), dtype=torch.float64, device="cuda")
    dv = torch.ones_like(du)
    T.step(10.0, du, dv)
    assert float(du.abs().max()) == 0.0 and T.num_rays() == 0
    # invalid dt
    with pytest.raises(gw.GwamError) as e:
        T.step(0.0)
    assert e.value.code == gw.GWAM_EINVAL
    # a ray outside the domain is rejected and nothing is added
    r = synth.fplane_rays(grid, 5, tag=3)
    r["z"][2] = 1e9
    with pytest.raises(gw.GwamError) as e:
        T.add_rays(r)
    assert e.value.code == gw.GWAM_EINVAL and T.num_rays() == 0
    # capacity: more ray volumes than max_rays
    with pytest.raises(gw.GwamError) as e:
        T.add_rays(synth.fplane_rays(grid, 101, tag=4))
    assert e.value.code == gw.GWAM_ECAPACITY
    # a bad background is refused
    bad = [a.copy() for a in bg]
    bad[3][3, 2, 1] = -1.0
    with pytest.raises(gw.GwamError) as e:
        T.set_background(*[torch.from_numpy(a).cuda() for a in bad])
    assert e.value.code == gw.GWAM_ENUMERIC
    bad = [a.copy() for a in bg]
    bad[0][0, 0, 0] = np.nan
    with pytest.raises(gw.GwamError) as e:
        T.set_background(*bad)
    assert e.value.code == gw.GWAM_ENUMERIC
    # capacity reached inside a step (splits) is reported, not written past the buffers
    T2 = gw.Tracer(grid, dict(params, splitting=1), max_rays=12)
    T2.set_background(*dev)
    r = synth.fplane_rays(grid, 10, tag=5, ext_z=2000.0)
    T2.add_rays(r)
    T2.step(10.0)
    with pytest.raises(gw.GwamError) as e:
        T2.stats()
    assert e.value.code == gw.GWAM_ECAPACITY


def test_host_entry_points_match_device_ones(gw):
    """gwam_set_background_host / gwam_step_host give the device-path results, both with pageable
    host buffers (staged copies) and with page-locked ones (read and written by the kernels
    directly); so do the asynchronous entry points (copies on the copy stream, the background set
    before every step so both staging slots are reused)."""
    import torch
    w = synth.workload("fplane")
    grid, params = w["grid"], w["params"]
    rays = synth.fplane_rays(grid, 300, tag=12)
    outs = []
    shape = (grid["nz"], grid["ny"], grid["nx"])
    for mode in ("device", "pageable", "pinned", "async"):
        host = mode != "device"
        T = gw.Tracer(grid, params, max_rays=4096)
        pinned_bg = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in w["background"]]
        if mode == "async":
            T.set_background_async(*pinned_bg)
        elif mode == "pageable":
            T.set_background(*w["background"])
        elif mode == "pinned":
            T.set_background(*[torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in w["background"]])
        else:
            T.set_background(*[torch.from_numpy(a.copy()).cuda() for a in w["background"]])
        T.add_rays(rays)
        if mode == "async":
            du = torch.full(shape, np.nan, dtype=torch.float64).pin_memory().numpy()
            dv = torch.full(shape, np.nan, dtype=torch.float64).pin_memory().numpy()
            for _ in range(3):
                T.set_background_async(*pinned_bg)
                T.step_host_async(300.0, du, dv)
            T.synchronize()
        elif host:
            if mode == "pinned":
                du = torch.full(shape, np.nan, dtype=torch.float64).pin_memory().numpy()
                dv = torch.full(shape, np.nan, dtype=torch.float64).pin_memory().numpy()
            else:
                du, dv = np.zeros(shape), np.zeros(shape)
            for _ in range(3):
                T.step_host(300.0, du, dv)
        else:
            dud = torch.zeros(shape, dtype=torch.float64, device="cuda")
            dvd = torch.zeros_like(dud)
            for _ in range(3):
                T.step(300.0, dud, dvd)
            du, dv = dud.cpu().numpy(), dvd.cpu().numpy()
        outs.append((T.rays(), np.array(du), np.array(dv)))
    for o in outs[1:]:
        for n in oracle.STATE_NAMES:
            np.testing.assert_array_equal(outs[0][0][n], o[0][n])
        assert level_error(o[1], outs[0][1]) <= 1e-12
        assert level_error(o[2], outs[0][2]) <= 1e-12


def test_async_backgrounds_changing_every_step(gw):
    """A background that changes before every step, set asynchronously (double-buffered background
    sets, the set-up of the next overlapping the current step) and synchronously: the same ray state
    bit for bit after every step, and the same tendencies; then a synchronous set-up after the
    asynchronous ones and a checkpoint of the current set."""
    import torch
    w = synth.workload("fplane")
    grid, params = w["grid"], dict(w["params"], saturation=1, smoothing=1)
    rays = synth.fplane_rays(grid, 600, tag=14)
    shape = (grid["nz"], grid["ny"], grid["nx"])
    bgs = []
    for s in range(6):
        u, v, n2, rho = [np.array(a) for a in synth.perturbed(synth.uniform_background(grid, U=10.0), tag=40 + s)]
        bgs.append([torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in (u, v, n2, rho)])
    outs = []
    for mode in ("sync", "async"):
        T = gw.Tracer(grid, params, max_rays=8192)
        T.set_background(*bgs[0])
        T.add_rays(rays)
        du = torch.zeros(shape, dtype=torch.float64).pin_memory().numpy()
        dv = torch.zeros(shape, dtype=torch.float64).pin_memory().numpy()
        states = []
        for s in range(1, 6):
            if mode == "async":
                T.set_background_async(*bgs[s])
                T.step_host_async(300.0, du, dv)
                T.synchronize()
            else:
                T.set_background(*bgs[s])
                T.step_host(300.0, du, dv)
            states.append((T.rays(), du.copy(), dv.copy()))
        T.set_background(*bgs[0])          # synchronous set-up of the current set after async ones
        T.step_host(300.0, du, dv)
        states.append((T.rays(), du.copy(), dv.copy()))
        outs.append(states)
    for a, b in zip(*outs):
        for n in oracle.STATE_NAMES:
            np.testing.assert_array_equal(a[0][n], b[0][n])
        assert level_error(b[1], a[1]) <= 1e-12 and level_error(b[2], a[2]) <= 1e-12


def test_async_host_entry_points_reject_and_report(gw):
    """Pageable buffers are refused (GWAM_EINVAL) by the asynchronous entry points; an invalid
    background (N^2 <= f^2) set asynchronously is reported by the next synchronising call."""
    import torch
    w = synth.workload("fplane")
    grid, params = w["grid"], w["params"]
    shape = (grid["nz"], grid["ny"], grid["nx"])
    T = gw.Tracer(grid, params, max_rays=4096)
    with pytest.raises(gw.GwamError):
        T.set_background_async(*w["background"])
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in w["background"]]
    T.set_background_async(*pinned)
    T.add_rays(synth.fplane_rays(grid, 100, tag=13))
    with pytest.raises(gw.GwamError):
        T.step_host_async(300.0, np.zeros(shape), np.zeros(shape))
    du = torch.zeros(shape, dtype=torch.float64).pin_memory().numpy()
    dv = torch.zeros(shape, dtype=torch.float64).pin_memory().numpy()
    T.step_host_async(300.0, du, dv)
    T.synchronize()
    bad = [a.copy() for a in pinned]
    bad[2][3, 2, 1] = 0.0        # N^2 <= f^2 at one node
    bad = [torch.from_numpy(a).pin_memory().numpy() for a in bad]
    T.set_background_async(*bad)
    T.step_host_async(300.0, du, dv)
    with pytest.raises(gw.GwamError) as e:
        T.synchronize()
    assert e.value.code == -4          # GWAM_ENUMERIC


def test_double_float_near_the_fp32_exponent_limits(gw):
    """The FP64 form computes in double-float pairs of FP32 values, whose exponent range is FP32's.
    Ray volumes at its edges against the oracle, with the parity bars of the other cases: a
    wavenumber component at the rounding level of an axis-aligned launch (cos(pi/2)|k_h| ~ 4e-21 1/m,
    whose square, 1.6e-41, is below FP32's smallest normal), one of 1e-30 (its square flushes to
    zero), and wave-action densities from 1e-2 to 1e25 (actions 1e-17 ... 1e10)."""
    grid = synth.fplane_grid(nx=16, ny=16, nz=32, dz=1000.0)
    bg = synth.perturbed(synth.uniform_background(grid, U=8.0), tag=51, rel=0.05)
    params = dict(synth.DEFAULT_PARAMS, smoothing=1, saturation=1, cap_per_column=0)
    base = synth.fplane_rays(grid, 250, tag=52, z_lo=3e3, z_hi=20e3)
    kh = np.hypot(base["k"], base["l"])
    r = {k: np.array(v, dtype=np.float64) for k, v in base.items()}
    r["k"][:50], r["l"][:50] = np.cos(np.pi / 2) * kh[:50], kh[:50]          # k at the rounding level
    r["k"][50:100], r["l"][50:100] = -kh[50:100], np.sin(np.pi) * kh[50:100]  # l at the rounding level
    r["k"][100:150], r["l"][100:150] = 1e-30, kh[100:150]                  # k^2 flushes to zero in FP32
    r["n"][150:200] = 1e25 * r["n"][150:200] / r["n"][150:200].max()        # very large densities
    r["n"][200:250] = 1e-2                                                 # tiny actions
    assert abs(r["k"][0]) < 1e-19 and abs(r["k"][0]) ** 2 < np.finfo(np.float32).tiny
    T, O = _pair(gw, grid, params, bg, 20000)
    T.add_rays(r)
    O.add_rays(r)
    for s in range(8):
        du, dv, odu, odv = _step_both(T, O, 300.0, grid["nz"], grid["ny"], grid["nx"])
        if s % 4 == 3:
            _compare_all(T, O, grid, du, dv, odu, odv)


@pytest.mark.parametrize("precision", [0, 1])
def test_step_graph_kernel_count(gw, precision):
    """The step graph's kernel nodes, counted by the library from the captured graph, equal the
    eager step's kernels as the benchmark counts them (its gpu_launches)."""
    import sys
    import os
    import torch
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    grid = synth.sphere_grid(nx=40, ny=20, nz=24, dz=1000.0)
    for params in (dict(synth.DEFAULT_PARAMS, smoothing=1, saturation=1, cap_per_column=12),
                   dict(synth.DEFAULT_PARAMS, smoothing=0, saturation=0, cap_per_column=0)):
        params = dict(params, precision=precision)
        T = gw.Tracer(grid, params, max_rays=100000)
        bg = synth.jet_background(grid)
        T.set_background(*[torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in bg])
        T.add_rays(synth.sphere_rays(grid, 500, tag=51))
        assert T.graph_kernel_count() == 0
        du = torch.zeros((grid["nz"], grid["ny"], grid["nx"]), dtype=torch.float64, device="cuda")
        dv = torch.zeros_like(du)
        T.step_graph(300.0, du, dv)
        T.synchronize()
        assert T.graph_kernel_count() == bench.launches_per_step(params, fp32=bool(precision)), params

