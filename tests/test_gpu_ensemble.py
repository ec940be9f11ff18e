"""Batched ensemble form: several members (own background, own ray population) advanced together
in one set of launches; each member against its own FP64 oracle instance.  Also CUDA-graph replay
against eager steps, and the autotuner."""
import numpy as np
import pytest

import oracle
from paper_2309_11257_gb300 import synth
from parity_util import RTOL, assert_fields_match, scaled_error, state_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    from paper_2309_11257_gb300 import build
    build.build()
    from paper_2309_11257_gb300 import gwam
    return gwam


GRID = synth.sphere_grid(nx=32, ny=16, nz=20, dz=1000.0)
PARAMS = dict(synth.DEFAULT_PARAMS, cap_per_column=34)


def _members(M):
    return [synth.perturbed(synth.jet_background(GRID, amp=30.0 + 20 * m, lat_deg=35.0 + 8 * m, z_peak=12e3,
                                                 z_width=5e3), tag=50 + m) for m in range(M)]


def _specs(M):
    out = []
    for m in range(M):
        sp = synth.convective_specs(GRID, tag=60 + m, median=3.0, cap=12, z_launch=4e3)
        sp["member"] = m
        out.append(sp)
    return out


def _setup(gw, M, bgs, specs):
    import torch
    T = gw.Tracer(GRID, PARAMS, max_rays=400000, members=M)
    for m in range(M):
        T.set_member_background(m, *[torch.from_numpy(a.copy()).cuda() for a in bgs[m]])
    src = synth.background_source(z_launch=2e3)
    T.launch_sources(src)
    T.launch_spectral(np.concatenate(specs))
    Os = []
    for m in range(M):
        O = oracle.Model(GRID, PARAMS)
        O.set_background(*bgs[m])
        O.launch_background(src)
        O.launch_spectral(specs[m])
        Os.append(O)
    return T, Os


def _compare_members(T, Os, du=None, dv=None, oout=None):
    g = T.rays()
    M = len(Os)
    for m in range(M):
        sel = g["member"] == m
        o = Os[m].rays()
        assert sel.sum() == len(o["id"]), (m, sel.sum(), len(o["id"]))
        gid = g["id"][sel]
        # ids are issued per event in the same order on both sides: map by rank
        rank_g = {int(i): r for r, i in enumerate(np.sort(gid))}
        rank_o = {int(i): r for r, i in enumerate(np.sort(o["id"]))}
        np.testing.assert_array_equal([rank_g[int(i)] for i in gid], [rank_o[int(i)] for i in o["id"]])
        np.testing.assert_array_equal(g["cell"][sel], o["cell"])
        gm = {n: g[n][sel] for n in oracle.STATE_NAMES}
        errs = state_errors(gm, o, GRID)
        assert max(errs.values()) <= RTOL, (m, errs)
        if du is not None:
            su, sv = Os[m].tendency_scale()
            assert_fields_match(du[m], oout[m][0], su, name="dudt[%d]" % m)
            assert_fields_match(dv[m], oout[m][1], sv, name="dvdt[%d]" % m)
    st = T.stats()
    for key in ("n_launched", "n_filtered", "n_split_v", "n_split_h", "n_exited", "n_capped", "n_invalid"):
        assert st[key] == sum(O.stats()[key] for O in Os), key
    for key in ("w_total", "w_launched", "w_saturated", "w_exited", "w_capped"):
        ref = sum(O.stats()[key] for O in Os)
        assert abs(st[key] - ref) <= RTOL * max(abs(ref), 1e-300), key


def test_ensemble_members_match_separate_oracles(gw):
    import torch
    M = 3
    T, Os = _setup(gw, M, _members(M), _specs(M))
    _compare_members(T, Os)
    shape = (M, GRID["nz"], GRID["ny"], GRID["nx"])
    du = torch.zeros(shape, dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(du)
    for _ in range(6):
        T.step(300.0, du, dv)
        oout = [O.step(300.0) for O in Os]
    _compare_members(T, Os, du.cpu().numpy(), dv.cpu().numpy(), oout)
    st = T.stats()
    assert st["n_capped"] > 0 and st["n_split_h"] > 0 and st["w_saturated"] > 0


def test_graph_replay_matches_eager_steps(gw):
    import torch
    M = 2
    bgs, specs = _members(M), _specs(M)
    shape = (M, GRID["nz"], GRID["ny"], GRID["nx"])
    outs = []
    for use_graph in (False, True):
        T, _ = _setup(gw, M, bgs, specs)
        du = torch.zeros(shape, dtype=torch.float64, device="cuda")
        dv = torch.zeros_like(du)
        for s in range(7):
            if s == 3:      # a launch between replays: the graph reads counts from device memory
                T.launch_sources(synth.background_source(z_launch=3e3))
            (T.step_graph if use_graph else T.step)(300.0, du, dv)
        if use_graph:
            # the graphs' phase events: the five phase times of the last replays, all positive
            phases, n = T.graph_profile_read()
            assert n == 2 and all(v > 0.0 for v in phases.values()), phases
        outs.append((T.rays(), du.cpu().numpy(), T.stats()))
    for n in ("id", "member", "cell") + tuple(oracle.STATE_NAMES):
        np.testing.assert_array_equal(outs[0][0][n], outs[1][0][n])
    scale = np.abs(outs[0][1]).max()
    assert np.abs(outs[0][1] - outs[1][1]).max() <= 1e-12 * scale
    assert outs[0][2]["n_steps"] == outs[1][2]["n_steps"] == 7


def test_autotune_keeps_parity(gw):
    import torch
    M = 2
    T, Os = _setup(gw, M, _members(M), _specs(M))
    cfg = T.autotune(300.0, steps_per_candidate=1)
    for name, (threads, blocks) in cfg.items():
        assert threads in (64, 128, 256) and blocks >= 1
    for _ in range(7):           # the autotuner advanced 7 candidate steps
        for O in Os:
            O.step(300.0)
    shape = (M, GRID["nz"], GRID["ny"], GRID["nx"])
    du = torch.zeros(shape, dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(du)
    T.step_graph(300.0, du, dv)
    oout = [O.step(300.0) for O in Os]
    _compare_members(T, Os, du.cpu().numpy(), dv.cpu().numpy(), oout)


def test_precision_form_members_track_their_oracles(gw):
    """The precision form with members: each member's drag against its own FP64 oracle within the
    precision form's bars (column-scaled 1e-4), its live count within 0.5 %, the summed wave action
    within 1e-5 (member-major arrays, the fields of all members cleared by the ray-step kernel)."""
    import torch
    M = 2
    bgs, specs = _members(M), _specs(M)
    p32 = dict(PARAMS, precision=1)
    T = gw.Tracer(GRID, p32, max_rays=400000, members=M)
    for m in range(M):
        T.set_member_background(m, *[torch.from_numpy(a.copy()).cuda() for a in bgs[m]])
    src = synth.background_source(z_launch=2e3)
    T.launch_sources(src)
    T.launch_spectral(np.concatenate(specs))
    Os = []
    for m in range(M):
        O = oracle.Model(GRID, PARAMS)
        O.set_background(*bgs[m])
        O.launch_background(src)
        O.launch_spectral(specs[m])
        Os.append(O)
    shape = (M, GRID["nz"], GRID["ny"], GRID["nx"])
    du = torch.zeros(shape, dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(du)
    for _ in range(5):
        T.step_graph(300.0, du, dv)
        oout = [O.step(300.0) for O in Os]
    g = T.rays()
    col = lambda S: np.broadcast_to(S.max(axis=0, keepdims=True), S.shape)
    for m in range(M):
        n_g = int((g["member"] == m).sum())
        n_o = len(Os[m].rays()["id"])
        assert abs(n_g - n_o) <= 0.005 * max(n_o, 200), (m, n_g, n_o)
        su, sv = Os[m].tendency_scale()
        e_u = scaled_error(du[m].cpu().numpy(), oout[m][0], col(su))
        e_v = scaled_error(dv[m].cpu().numpy(), oout[m][1], col(sv))
        assert e_u <= 1e-4 and e_v <= 1e-4, (m, e_u, e_v)
        assert np.abs(oout[m][0]).max() > 0.0
    w = sum(O.stats()["w_total"] for O in Os)
    assert abs(T.stats()["w_total"] - w) <= 1e-5 * abs(w)

