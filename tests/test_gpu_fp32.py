"""Precision form (FP32 kinematics, cell index + FP32 offset positions, FP64 accumulation) against
the FP64 CPU oracle.  The errors are stated, not hidden: every output's error is printed, and the
test holds them to the bounds the form is built for:
  * ray state (rays present on both sides): normwise relative error <= 2e-5 per component, and
    per ray against each ray's own scale (as in the FP64 parity tests) <= 1e-4 (measured: at most
    2.7e-5, N after strong saturation on the f-plane, 1.5e-6 otherwise);
  * projected centre fields: |gpu - oracle| <= 1e-4 * S elementwise, S the oracle's sum of
    contribution magnitudes (as in the FP64 parity tests);
  * vertical fluxes and drag: |gpu - oracle| <= 1e-4 * S_col, S_col the largest S of the column.
    A ray's share of a staggered cell is its vertical overlap with it; a position error of d moves
    flux d/dz between neighbouring interfaces of the column, so a ray that just grazes an interface
    (overlap of centimetres out of a kilometre) carries a large relative error there while the
    column's flux is accurate -- the column scale measures that.  The elastic terms E ~ f^2 are
    held the same way: near the equator the relative error of f^2 is the FP32 position resolution
    (about 1e-8 rad) over phi, so a ray within 1e-4 rad of the equator carries a 1e-4 relative
    error in its (vanishing) elastic contribution;
  * integer bookkeeping: counts within 0.5 % (FP32 can move a ray across a threshold);
  * budget terms: relative 1e-5.
"""
import numpy as np
import pytest

import oracle
from paper_2309_11257_gb300 import synth
from parity_util import odd_field_case, scaled_error, state_errors

pytestmark = pytest.mark.gpu

STATE_TOL = 2e-5
STATE_TOL_PER_RAY = 1e-4
FIELD_TOL = 1e-4


@pytest.fixture(scope="module")
def gw():
    from paper_2309_11257_gb300 import build
    build.build()
    from paper_2309_11257_gb300 import gwam
    return gwam


def _run(gw, grid, params, bg, src, rays, steps, dt, specs=None):
    import torch
    T = gw.Tracer(grid, dict(params, precision=1), max_rays=3_000_000)
    T.set_background(*[torch.from_numpy(a.copy()).cuda() for a in bg])
    O = oracle.Model(grid, params)
    O.set_background(*bg)
    if src:
        T.launch_sources(src)
        O.launch_background(src)
    if specs is not None:
        T.launch_spectral(specs)
        O.launch_spectral(specs)
    if rays:
        T.add_rays(rays)
        O.add_rays(rays)
    shape = (grid["nz"], grid["ny"], grid["nx"])
    du = torch.zeros(shape, dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(du)
    for _ in range(steps):
        T.step(dt, du, dv)
        odu, odv = O.step(dt)
    return T, O, du.cpu().numpy(), dv.cpu().numpy(), odu, odv


def _report_and_check(T, O, grid, du, dv, odu, odv, label):
    g, o = T.rays(), O.rays()
    common, ig, io = np.intersect1d(g["id"], o["id"], return_indices=True)
    assert len(common) >= 0.995 * len(o["id"])
    gsel = {n: g[n][ig] for n in oracle.STATE_NAMES}
    osel = {n: o[n][io] for n in oracle.STATE_NAMES + ("n_scale",)}
    errs = state_errors(gsel, osel, grid, mode="normwise")
    errs_ray = state_errors(gsel, osel, grid, mode="per_ray")
    su, sv = O.tendency_scale()
    col = lambda S: np.broadcast_to(S.max(axis=0, keepdims=True), S.shape)
    e_du, e_dv = scaled_error(du, odu, col(su)), scaled_error(dv, odv, col(sv))
    l2 = np.linalg.norm(du - odu) / max(np.linalg.norm(odu), 1e-300)
    field_errs = {}
    for n in oracle.FIELD_NAMES:
        S = O.field_abs(n)
        # vertical fluxes and elastic terms by the column's largest S: a ray grazing an interface
        # carries a large relative error in that interface's share, and E is proportional to f^2,
        # whose relative error near the equator is the FP32 position resolution (1e-8 rad) over phi
        field_errs[n] = scaled_error(T.field(n), O.field(n), col(S) if n.startswith(("fz", "e_")) else S)
    gs, os_ = T.stats(), O.stats()
    print("\n[%s] precision form vs FP64 oracle" % label)
    print("  ray state normwise:", {k: "%.1e" % v for k, v in errs.items()})
    print("  ray state per ray:", {k: "%.1e" % v for k, v in errs_ray.items()})
    print("  du/dt column-scaled %.2e (rel L2 %.2e), dv/dt column-scaled %.2e" % (e_du, l2, e_dv))
    print("  fields scaled:", {k: "%.1e" % v for k, v in field_errs.items()})
    print("  counts gpu/oracle:", {k: (gs[k], os_[k]) for k in ("n_live", "n_split_v", "n_split_h", "n_exited",
                                                                "n_capped")})
    assert max(errs.values()) <= STATE_TOL, errs
    assert max(errs_ray.values()) <= STATE_TOL_PER_RAY, errs_ray
    assert e_du <= FIELD_TOL and e_dv <= FIELD_TOL
    assert max(field_errs.values()) <= FIELD_TOL, field_errs
    for k in ("n_live", "n_launched", "n_filtered", "n_split_v", "n_split_h", "n_exited", "n_capped"):
        assert abs(gs[k] - os_[k]) <= 0.005 * max(os_[k], 200), (k, gs[k], os_[k])
    for k in ("w_total", "w_launched"):
        assert abs(gs[k] - os_[k]) <= 1e-5 * abs(os_[k]), k


def test_precision_form_small_sphere(gw):
    grid = synth.sphere_grid(nx=40, ny=20, nz=24, dz=1000.0)
    bg = synth.perturbed(synth.jet_background(grid, z_peak=15e3, z_width=6e3), tag=31)
    rays = synth.sphere_rays(grid, 500, tag=71, z_lo=4e3, z_hi=20e3, ext_scale=2.5)
    rays["n"] = rays["n"] * 30.0
    out = _run(gw, grid, dict(synth.DEFAULT_PARAMS, cap_per_column=45), bg, synth.background_source(z_launch=2e3),
               rays, 10, 300.0)
    _report_and_check(*out[:2], grid, *out[2:], "sphere 40x20x24, 10 steps")


def test_precision_form_fplane(gw):
    grid = synth.fplane_grid(nx=24, ny=20, nz=40, dx=40e3, dy=30e3, dz=500.0)
    bg = synth.perturbed(synth.uniform_background(grid, U=5.0), tag=21, rel=0.1)
    rays = synth.fplane_rays(grid, 1500, tag=22, z_lo=3e3, z_hi=15e3, ext_z=1300.0)
    rays["n"] = rays["n"] * 1e8
    out = _run(gw, grid, dict(synth.DEFAULT_PARAMS, cap_per_column=12), bg, None, rays, 12, 240.0)
    _report_and_check(*out[:2], grid, *out[2:], "f-plane 24x20x40, 12 steps")


def test_precision_form_columnar_sphere(gw):
    """The columnar (single-column) mode in the precision form: same bars as the 3-D form."""
    grid = synth.sphere_grid(nx=40, ny=20, nz=24, dz=1000.0)
    bg = synth.perturbed(synth.jet_background(grid, z_peak=15e3, z_width=6e3), tag=31)
    rays = synth.sphere_rays(grid, 500, tag=71, z_lo=4e3, z_hi=20e3, ext_scale=2.5)
    rays["n"] = rays["n"] * 30.0
    out = _run(gw, grid, dict(synth.DEFAULT_PARAMS, cap_per_column=45, columnar=1), bg,
               synth.background_source(z_launch=2e3), rays, 10, 300.0)
    _report_and_check(*out[:2], grid, *out[2:], "columnar sphere 40x20x24, 10 steps")


def test_precision_form_ghost_layer_launch(gw):
    """Ghost-layer emission every interval in the precision form (the ghost integrated in double-float
    on nodes the context allocates at its first ghost launch): sheared f-plane, 8 cycles, then the
    bars above against the FP64 oracle running the same cycles."""
    import torch
    grid = synth.fplane_grid(nx=12, ny=10, nz=40, dx=40e3, dy=30e3, dz=500.0)
    bg = synth.perturbed(synth.uniform_background(grid, U=8.0, V=-3.0), tag=61, rel=0.1)
    params = dict(synth.DEFAULT_PARAMS, cap_per_column=60)
    specs = synth.uniform_specs(grid, flux=4e-3, z_launch=3e3)
    T = gw.Tracer(grid, dict(params, precision=1), max_rays=400000)
    T.set_background(*[torch.from_numpy(a.copy()).cuda() for a in bg])
    O = oracle.Model(grid, params)
    O.set_background(*bg)
    shape = (grid["nz"], grid["ny"], grid["nx"])
    du = torch.zeros(shape, dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(du)
    for _ in range(8):
        T.launch_ghost_spectral(specs, 240.0)
        O.launch_ghost_spectral(specs, 240.0)
        T.step(240.0, du, dv)
        odu, odv = O.step(240.0)
    assert T.stats()["n_launched"] > 7 * 0.8 * len(specs)
    _report_and_check(T, O, grid, du.cpu().numpy(), dv.cpu().numpy(), odu, odv, "ghost f-plane 12x10x40, 8 cycles")


@pytest.mark.parametrize("geometry", ["sphere", "fplane"])
def test_precision_form_theta_flux(gw, geometry):
    """Potential-temperature flux integrals (Eq. fluxes:temperature) and d theta/dt (Eq.
    mean-flow-impact-t) in the precision form: the field bar above, by the column's largest
    contribution sum like the elastic terms (f^2 and f share the FP32 latitude resolution), and
    the tendency by the same column scale of its error scale."""
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
    T = gw.Tracer(grid, dict(params, precision=1), max_rays=200000)
    T.set_background(*[torch.from_numpy(a.copy()).cuda() for a in bg])
    T.set_theta(torch.from_numpy(np.ascontiguousarray(theta)).cuda())
    O = oracle.Model(grid, params)
    O.set_background(*bg)
    O.set_theta(theta)
    T.add_rays(rays)
    O.add_rays(rays)
    shape = (grid["nz"], grid["ny"], grid["nx"])
    du = torch.zeros(shape, dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(du)
    for _ in range(6):
        T.step(dt, du, dv)
        odu, odv = O.step(dt)
    _report_and_check(T, O, grid, du.cpu().numpy(), dv.cpu().numpy(), odu, odv, "theta " + geometry)
    col = lambda S: np.broadcast_to(S.max(axis=0, keepdims=True), S.shape)
    errs = {n: scaled_error(T.field(n), O.field(n), col(O.field_abs(n))) for n in oracle.THETA_FIELD_NAMES}
    th, sc = O.theta_tendency()
    errs["dtheta/dt"] = scaled_error(T.theta_tendency(), th, col(sc))
    print("  theta fields and tendency:", {k: "%.1e" % v for k, v in errs.items()})
    assert np.abs(th).max() > 0.0
    assert max(errs.values()) <= FIELD_TOL, errs


def test_precision_form_full_size_sphere(gw):
    """The precision-form benchmark physics at the FP64 workload's size: launch and 2 steps."""
    w = synth.workload("sphere")
    out = _run(gw, w["grid"], w["params"], w["background"], w["source"], None, 2, w["dt"])
    _report_and_check(*out[:2], w["grid"], *out[2:], "sphere 256x128x90, 2 steps")


def test_precision_form_ensemble_and_graph(gw):
    """Two members in the precision form: graph replay is bit-identical to eager steps, the budget
    closes, the members stay independent."""
    import torch
    grid = synth.sphere_grid(nx=32, ny=16, nz=20, dz=1000.0)
    outs = []
    for graph in (False, True):
        T = gw.Tracer(grid, dict(synth.DEFAULT_PARAMS, precision=1), max_rays=400000, members=2)
        for m in range(2):
            bg = synth.perturbed(synth.jet_background(grid, amp=30 + 30 * m, z_peak=12e3, z_width=5e3), tag=80 + m)
            T.set_member_background(m, *[torch.from_numpy(a.copy()).cuda() for a in bg])
        T.launch_sources(synth.background_source(z_launch=2e3))
        du = torch.zeros((2, 20, 16, 32), dtype=torch.float64, device="cuda")
        dv = torch.zeros_like(du)
        for _ in range(6):
            (T.step_graph if graph else T.step)(300.0, du, dv)
        st = T.stats()
        rhs = st["w_launched"] - st["w_saturated"] - st["w_exited"] - st["w_capped"] - st["w_invalid"]
        assert abs(st["w_total"] - rhs) <= 1e-12 * st["w_total"]
        r = T.rays()
        assert set(np.unique(r["member"]).tolist()) == {0, 1}
        assert np.isfinite(du.cpu().numpy()).all()
        outs.append(r)
    for n in ("id", "member", "cell") + tuple(oracle.STATE_NAMES):
        np.testing.assert_array_equal(outs[0][n], outs[1][n])


def test_odd_field_lengths_are_cleared_every_step(gw):
    """Fields of odd length (3 x 5 columns of 21 levels): the bulk copies clear the fields' 16-byte
    part and thread 0 the last element, the top cell of the last column, where ray volumes are
    placed; the fields are compared after each of four steps."""
    import torch
    grid, bg, rays, params = odd_field_case()
    T = gw.Tracer(grid, dict(params, precision=1), max_rays=4096)
    T.set_background(*[torch.from_numpy(a.copy()).cuda() for a in bg])
    O = oracle.Model(grid, params)
    O.set_background(*bg)
    T.add_rays(rays)
    O.add_rays(rays)
    nz, ny, nx = grid["nz"], grid["ny"], grid["nx"]
    du = torch.zeros((nz, ny, nx), dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(du)
    for _ in range(4):
        T.step(120.0, du, dv)
        odu, odv = O.step(120.0)
        _report_and_check(T, O, grid, du.cpu().numpy(), dv.cpu().numpy(), odu, odv, "odd field lengths")
        o_last = O.field("wad")[nz - 1, ny - 1, nx - 1]
        assert o_last > 0.0
        assert T.field("wad")[nz - 1, ny - 1, nx - 1] == pytest.approx(o_last, rel=FIELD_TOL)
