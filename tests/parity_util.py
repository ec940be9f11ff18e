"""Comparison helpers for CUDA-path vs oracle parity (used by the gpu tests and the smoke check).

Tolerances (FP64 path):
  * integer bookkeeping -- ids, cells, canonical order, counters -- bit-exact;
  * ray state: per component max |gpu - oracle| <= 1e-9 * max |oracle| over the rays
    (normwise, since positions and wavenumbers cross zero), periodic coordinates compared
    modulo their period;
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
INT_STATS = ("n_live", "n_launched", "n_filtered", "n_split_v", "n_split_h", "n_exited", "n_capped", "n_merged",
             "n_invalid", "n_steps")
W_STATS = ("w_total", "w_launched", "w_saturated", "w_exited", "w_capped", "w_invalid")


def periods(grid):
    if grid["geometry"] == 1:
        return {"x": 2 * np.pi}
    return {"x": grid["nx"] * grid["dx"], "y": grid["ny"] * grid["dy"]}


def state_errors(g, o, grid):
    """Normwise relative error per state component (rays in the same canonical order)."""
    per = periods(grid)
    out = {}
    for name in STATE_NAMES:
        a, b = g[name], o[name]
        d = a - b
        if name in per:
            L = per[name]
            d = (d + 0.5 * L) % L - 0.5 * L
        scale = np.abs(b).max() if len(b) else 1.0
        out[name] = float(np.abs(d).max() / scale) if len(b) and scale > 0 else float(np.abs(d).max() if len(d) else 0)
    return out


def assert_rays_match(g, o, grid, rtol=RTOL):
    assert len(g["id"]) == len(o["id"]), (len(g["id"]), len(o["id"]))
    np.testing.assert_array_equal(g["id"], o["id"])          # canonical order, bit-exact
    np.testing.assert_array_equal(g["cell"], o["cell"])
    errs = state_errors(g, o, grid)
    bad = {k: v for k, v in errs.items() if not v <= rtol}
    assert not bad, bad
    return errs


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
