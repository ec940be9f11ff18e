"""Comparison helpers for CUDA-path vs oracle parity (used by the gpu tests and the smoke check).

Tolerances (FP64 path):
  * integer bookkeeping -- ids, cells, canonical order, counters -- bit-exact;
  * ray state, per ray volume: |gpu - oracle| <= 1e-9 * s with s the ray's own scale of that
    component -- its value for the positive components (z, extents, P_x, P_y, P_z), its
    wave-action density before the step's saturation for N (the damping factor 1 - 2 kappa K^2 dt
    is formed with a rounding error relative to 1), |k_h| for k and l and |k| for m (a wave vector
    along one axis has a rounding-level component along the other); only the horizontal position,
    which crosses zero and is periodic, is compared normwise (max |gpu - oracle| over rays
    <= 1e-9 max |oracle|, modulo the period);
  * du/dt, dv/dt and the grid fields, which are sums over ray volumes: elementwise
    |gpu - oracle| <= 1e-9 * S, with S the oracle's sum of the magnitudes of the contributions
    (pushed through the divergence for the tendencies), each taken with the ray volume's wave
    action before this step's saturation: the damping factor 1 - 2 kappa K^2 dt is a difference
    of terms of size 1, so a nearly fully damped ray volume carries an error of the unit roundoff
    times its undamped contribution.  Sums whose contributions cancel (opposite
    azimuths) carry only rounding noise relative to their own size, so a plain relative error of
    the result would measure summation order, not parity;
  * budget terms: relative 1e-9.
"""
import numpy as np

STATE_NAMES = ("x", "y", "z", "k", "l", "m", "ex", "ey", "ez", "px", "py", "pz", "n")
RTOL = 1e-9
# Tendency errors measured against the oracle stay below ERR_PER_S of their rounding scale S (at most
# 1.6e-10 over the 200-step sphere run), so a level's plain relative error is gated where its largest
# tendency is at least SIGNIFICANT of S.
ERR_PER_S = 2e-10
SIGNIFICANT = ERR_PER_S / RTOL
INT_STATS = ("n_live", "n_launched", "n_filtered", "n_split_v", "n_split_h", "n_exited", "n_capped", "n_merged",
             "n_invalid", "n_steps")
W_STATS = ("w_total", "w_launched", "w_saturated", "w_exited", "w_capped", "w_invalid")


def periods(grid):
    if grid["geometry"] == 1:
        return {"x": 2 * np.pi}
    return {"x": grid["nx"] * grid["dx"], "y": grid["ny"] * grid["dy"]}


def _component_scale(name, o):
    """Per-ray error scale of one state component (see the module docstring), or None for the
    normwise components."""
    if name in ("x", "y"):
        return None
    if name == "z":
        return np.maximum(np.abs(o["z"]), np.abs(o["ez"]))
    if name in ("k", "l"):
        return np.hypot(o["k"], o["l"])
    if name == "m":
        return np.sqrt(o["k"] ** 2 + o["l"] ** 2 + o["m"] ** 2)
    if name == "n" and "n_scale" in o:
        return np.maximum(np.asarray(o["n_scale"]), np.abs(o["n"]))
    return np.abs(o[name])


def state_errors(g, o, grid, mode="per_ray"):
    """Relative error per state component (rays in the same canonical order): per ray against the
    ray's own scale (mode "per_ray"), or normwise against max |oracle| over the rays ("normwise")."""
    per = periods(grid)
    out = {}
    for name in STATE_NAMES:
        a, b = g[name], o[name]
        d = a - b
        if name in per:
            L = per[name]
            d = (d + 0.5 * L) % L - 0.5 * L
        d = np.abs(d)
        if not len(b):
            out[name] = 0.0
            continue
        sc = _component_scale(name, o) if mode == "per_ray" else None
        if sc is None:
            scale = np.abs(b).max()
            out[name] = float(d.max() / scale) if scale > 0 else float(d.max())
        else:
            if np.any((sc == 0) & (d != 0)):
                out[name] = float("inf")
                continue
            out[name] = float(np.where(sc > 0, d / np.where(sc > 0, sc, 1.0), 0.0).max())
    return out


def assert_rays_match(g, o, grid, rtol=RTOL):
    assert len(g["id"]) == len(o["id"]), (len(g["id"]), len(o["id"]))
    np.testing.assert_array_equal(g["id"], o["id"])          # canonical order, bit-exact
    np.testing.assert_array_equal(g["cell"], o["cell"])
    errs = state_errors(g, o, grid)
    bad = {k: v for k, v in errs.items() if not v <= rtol}
    assert not bad, bad
    return errs


def level_errors(a, b):
    """Per level: max|a - b| / max|b| on that level (inf where b == 0 and a != b; 0 where both 0)."""
    out = np.zeros(a.shape[0])
    for lev in range(a.shape[0]):
        s = np.abs(b[lev]).max()
        d = np.abs(a[lev] - b[lev]).max()
        out[lev] = (d / s) if s > 0 else (0.0 if d == 0 else np.inf)
    return out


def assert_level_errors(a, b, scale, rtol=RTOL, significant=SIGNIFICANT, name=""):
    """The plain per-level relative error of a tendency, max|gpu - oracle| / max|oracle| per level,
    bounded by rtol on every level whose largest value is at least `significant` times the level's
    largest rounding scale S (sum of |contribution| pushed through the divergence).  The elementwise
    bar holds the error below about ERR_PER_S * S (measured), so a level whose net tendency is at
    least `significant` of its S meets rtol when ERR_PER_S / significant <= rtol; below that the
    level's net tendency is mostly cancellation (opposite azimuths) and only the elementwise bar
    applies.  Returns (worst gated level error, number of gated levels, levels, worst ungated)."""
    errs = level_errors(a, b)
    gated, other = [], []
    for lev in range(a.shape[0]):
        big = np.abs(b[lev]).max()
        sc = np.abs(scale[lev]).max()
        (gated if sc > 0 and big >= significant * sc else other).append(errs[lev])
    worst = max(gated) if gated else 0.0
    assert worst <= rtol, (name, "per-level relative error", worst)
    return worst, len(gated), a.shape[0], (max(other) if other else 0.0)


def level_error(a, b):
    """max over levels of max|a-b| / max|b| on that level (levels with b == 0 need a == 0)."""
    worst = 0.0
    for lev in range(a.shape[0]):
        s = np.abs(b[lev]).max()
        d = np.abs(a[lev] - b[lev]).max()
        if s == 0.0:
            if d != 0.0:
                return float("inf")
            continue
        worst = max(worst, d / s)
    return worst


def scaled_error(a, b, scale):
    """max |a - b| / scale elementwise (scale 0 requires equality)."""
    d = np.abs(a - b)
    if np.any((scale == 0) & (d != 0)):
        return float("inf")
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(scale > 0, d / np.where(scale > 0, scale, 1.0), 0.0)
    return float(r.max()) if r.size else 0.0


def assert_fields_match(gf, of, scale, rtol=RTOL, name=""):
    e = scaled_error(gf, of, scale)
    assert e <= rtol, (name, e)
    return e


def assert_stats_match(gs, os_, rtol=RTOL):
    for k in INT_STATS:
        assert gs[k] == os_[k], (k, gs[k], os_[k])
    for k in W_STATS:
        a, b = gs[k], os_[k]
        assert abs(a - b) <= rtol * max(abs(b), 1e-300), (k, a, b)


def odd_field_case():
    """3 x 5 columns of 21 levels: the centre fields hold 315 values, an odd count, whose last
    element (the top cell of the last column) the ray-step kernels clear apart from their 16-byte
    stores; ray volumes are placed in that cell, propagating downward so that they stay."""
    from paper_2309_11257_gb300 import synth
    grid = synth.fplane_grid(nx=3, ny=5, nz=21, dx=50e3, dy=50e3, dz=500.0)
    bg = synth.perturbed(synth.uniform_background(grid, U=5.0), tag=41, rel=0.1)
    rays = synth.fplane_rays(grid, 300, tag=42, z_lo=1e3, z_hi=9e3)
    top = synth.fplane_rays(grid, 40, tag=43, z_lo=10.1e3, z_hi=10.4e3, ext_z=100.0)
    g = synth.rng(44)
    top["x"] = g.uniform(2.05, 2.95, 40) * grid["dx"]
    top["y"] = g.uniform(4.05, 4.95, 40) * grid["dy"]
    top["m"] = -top["m"]
    rays = {k: np.concatenate([rays[k], top[k]]) for k in rays}
    params = dict(synth.DEFAULT_PARAMS, smoothing=0, saturation=1)
    return grid, bg, rays, params
