"""Checkpoint and resume (gwam_save / gwam_load): a context restored from a checkpoint steps on
exactly as the saved one does -- ray state, ids, cells and counters bit for bit; budget terms and
tendencies equal up to the order of FP64 atomic additions (which two uninterrupted runs share
too)."""
import numpy as np
import pytest

import oracle
from paper_2309_11257_gb300 import synth
from parity_util import level_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    from paper_2309_11257_gb300 import build
    build.build()
    from paper_2309_11257_gb300 import gwam
    return gwam


def _setup(gw, precision):
    import torch
    grid = synth.sphere_grid(nx=40, ny=20, nz=24, dz=1000.0)
    bg = synth.perturbed(synth.jet_background(grid, z_peak=15e3, z_width=6e3), tag=31)
    params = dict(synth.DEFAULT_PARAMS, cap_per_column=45, precision=precision)
    T = gw.Tracer(grid, params, max_rays=200000)
    T.set_background(*[torch.from_numpy(a.copy()).cuda() for a in bg])
    return grid, params, T


def _steps(T, grid, k):
    import torch
    shape = (grid["nz"], grid["ny"], grid["nx"])
    du = torch.zeros(shape, dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(du)
    for _ in range(k):
        T.step(300.0, du, dv)
    return du.cpu().numpy(), dv.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1])
def test_resume_from_checkpoint_matches_uninterrupted_run(gw, tmp_path, precision):
    grid, params, T = _setup(gw, precision)
    src = synth.background_source(z_launch=2e3)
    T.launch_sources(src)
    rays = synth.sphere_rays(grid, 777, tag=32, z_lo=14e3, z_hi=23.5e3, ext_scale=3.0)
    rays["n"] = rays["n"] * 30.0
    T.add_rays(rays)
    _steps(T, grid, 3)
    path = str(tmp_path / "state.gwam")
    T.save(path)
    T.launch_sources(src)
    du0, dv0 = _steps(T, grid, 3)
    r0, s0 = T.rays(), T.stats()

    T2 = gw.Tracer(grid, params, max_rays=200000)
    T2.load(path)
    T2.launch_sources(src)
    du1, dv1 = _steps(T2, grid, 3)
    r1, s1 = T2.rays(), T2.stats()
    np.testing.assert_array_equal(r0["id"], r1["id"])
    np.testing.assert_array_equal(r0["cell"], r1["cell"])
    for n in oracle.STATE_NAMES:
        np.testing.assert_array_equal(r0[n], r1[n])
    for k, v in s0.items():
        if isinstance(v, float):
            # per-block partial sums over the over-full columns follow the (atomic) order in which
            # the columns were listed: equal up to rounding
            assert abs(v - s1[k]) <= 1e-12 * max(abs(v), 1e-300), (k, v, s1[k])
        else:
            assert v == s1[k], (k, v, s1[k])
    assert level_error(du1, du0) <= 1e-12 and level_error(dv1, dv0) <= 1e-12
    assert s1["n_split_h"] > 0 and s1["n_capped"] > 0


def test_load_rejects_other_configurations_and_bad_files(gw, tmp_path):
    grid, params, T = _setup(gw, 0)
    T.launch_sources(synth.background_source(z_launch=2e3))
    path = str(tmp_path / "state.gwam")
    T.save(path)
    other = gw.Tracer(synth.sphere_grid(nx=40, ny=20, nz=20, dz=1000.0), params, max_rays=200000)
    with pytest.raises(gw.GwamError):
        other.load(path)
    f32 = gw.Tracer(grid, dict(params, precision=1), max_rays=200000)
    with pytest.raises(gw.GwamError):
        f32.load(path)
    small = gw.Tracer(grid, params, max_rays=1000)
    with pytest.raises(gw.GwamError):
        small.load(path)
    data = open(path, "rb").read()
    cut = str(tmp_path / "cut.gwam")
    open(cut, "wb").write(data[: len(data) // 2])
    T3 = gw.Tracer(grid, params, max_rays=200000)
    with pytest.raises(gw.GwamError):
        T3.load(cut)
    with pytest.raises(gw.GwamError):
        T3.load(str(tmp_path / "missing.gwam"))
    # the failed loads left the context usable: a good checkpoint still loads
    T3.load(path)
    assert T3.num_rays() == T.num_rays()
