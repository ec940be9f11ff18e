"""Latitude-band domain decomposition (App. B.2: ray volumes stored per parent column and handed to
the neighbouring domain after each step) over a world of `gloo` ranks on the CPU, against the
single-domain oracle.

Each rank runs the oracle's step phases on its own band through
`paper_2309_11257_gb300.domain.BandDecomposition`: provisional ids made global by an exclusive scan,
migration of the ray volumes that left the band (variable all-to-all), a halo of two rows of the
projected fields, and the band's rows of du/dt, dv/dt.  Joined over the ranks, the ray volumes (ids,
cells, every state component), the tendencies and the integer counters equal the single domain's
bit for bit; the wave-action terms, summed over the ranks in another order, agree to 1e-12.
No GPU is involved (unmeasured on hardware: every run of this build has one GPU).
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STEPS = 8
DT = 300.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _setup():
    sys.path.insert(0, ROOT)
    from paper_2309_11257_gb300 import synth
    grid = synth.sphere_grid(nx=32, ny=16, nz=30, dz=1000.0)
    bg = synth.perturbed(synth.jet_background(grid, z_peak=15e3, z_width=6e3), tag=31)
    params = dict(synth.DEFAULT_PARAMS, cap_per_column=40)
    src = synth.background_source(z_launch=2e3)
    rays = synth.sphere_rays(grid, 600, tag=32, z_lo=4e3, z_hi=25e3, lat_max_deg=80.0, ext_scale=3.0)
    rays["n"] = rays["n"] * 1e6          # strong enough to saturate
    # explicit rays in row order: the order in which one domain and the bands in rank order issue ids
    dphi = np.pi / grid["ny"]
    rows = np.floor((rays["y"] + 0.5 * np.pi) / dphi).astype(int)
    order = np.argsort(rows, kind="stable")
    rays = {k: np.asarray(v)[order] for k, v in rays.items()}
    rows = rows[order]
    return grid, bg, params, src, rays, rows


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2309_11257_gb300 import domain
        grid, bg, params, src, rays, rows = _setup()
        M = oracle.Model(grid, params)
        M.set_background(*bg)
        D = domain.BandDecomposition(M, grid["ny"])
        D.launch(lambda e: e.launch_background(src))
        mine = (rows >= D.j0) & (rows < D.j1)
        D.launch(lambda e: e.add_rays({k: v[mine] for k, v in rays.items()}))
        res = []
        sent = 0
        for _ in range(STEPS):
            du, dv = D.step(DT)
            sent += D.last_migrated
            st = D.stats()
            r = M.rays()
            res.append(dict(rays={k: r[k] for k in ("id", "cell") + oracle.STATE_NAMES}, du=du, dv=dv, stats=st))
        left = D.migrate()   # nothing may be left outside after a step's own migration
        out.put((rank, D.j0, D.j1, res, left, sent))
    finally:
        dist.destroy_process_group()


def _single_domain():
    sys.path.insert(0, ROOT)
    import oracle
    grid, bg, params, src, rays, rows = _setup()
    M = oracle.Model(grid, params)
    M.set_background(*bg)
    M.launch_background(src)
    M.add_rays(rays)
    out = []
    for _ in range(STEPS):
        du, dv = M.step(DT)
        out.append(dict(rays=M.rays(), du=du, dv=dv, stats=M.stats()))
    return out


@pytest.mark.parametrize("world", [2, 3])
def test_band_decomposition_matches_one_domain(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = _single_domain()
    import oracle
    for s in range(STEPS):
        one = ref[s]
        joined = {k: np.concatenate([p[3][s]["rays"][k] for p in parts]) for k in ("id", "cell") + oracle.STATE_NAMES}
        order = np.lexsort((joined["id"], joined["cell"]))
        for k in joined:
            np.testing.assert_array_equal(joined[k][order], one["rays"][k], err_msg="step %d %s" % (s, k))
        du = np.concatenate([p[3][s]["du"] for p in parts], axis=1)
        dv = np.concatenate([p[3][s]["dv"] for p in parts], axis=1)
        np.testing.assert_array_equal(du, one["du"])
        np.testing.assert_array_equal(dv, one["dv"])
        st = parts[0][3][s]["stats"]
        for k in ("n_live", "n_launched", "n_filtered", "n_split_v", "n_split_h", "n_exited", "n_capped", "n_invalid"):
            assert st[k] == one["stats"][k], (s, k, st[k], one["stats"][k])
        for k in ("w_total", "w_launched", "w_saturated", "w_exited", "w_capped"):
            assert st[k] == pytest.approx(one["stats"][k], rel=1e-12, abs=1e-300), (s, k)
    for p in parts:
        assert p[4] == 0
    # the case exercises what it claims: volumes crossing band edges, splits, saturation, cap, exits
    final = ref[-1]["stats"]
    assert final["n_split_v"] + final["n_split_h"] > 0 and final["w_saturated"] > 0 and final["n_capped"] > 0
    assert final["n_exited"] > 0
    assert all(p[5] > 0 for p in parts)       # every band handed ray volumes to a neighbour


def test_band_bounds_and_owners():
    sys.path.insert(0, ROOT)
    from paper_2309_11257_gb300 import domain
    b = domain.band_bounds(128, 3)
    assert b == [(0, 43), (43, 86), (86, 128)]
    np.testing.assert_array_equal(domain.owner_of_rows(np.array([0, 42, 43, 85, 86, 127]), b), [0, 0, 1, 1, 2, 2])
    with pytest.raises(ValueError):
        domain.band_bounds(5, 3)
