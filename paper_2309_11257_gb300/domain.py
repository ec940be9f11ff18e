"""Latitude-band domain decomposition of the ray-volume step across ranks (App. B.2).

The paper parallelises the scheme over the dynamical core's domains: ray volumes are stored with
their parent column, and after each propagation step the volumes that left a domain are handed to
the neighbouring one.  Here each rank owns a contiguous band of latitude rows [j0, j1) of the
lat-lon grid and the ray volumes whose carrier column lies in it.  One step, given a per-rank
engine that runs the step in three phases:

1. ``engine.step_advance(dt)`` -- RK3, exits and splits of the band's ray volumes, in array order.
   New ids are issued in array order from a provisional base and then made global.  A band's array
   is its part of the single domain's array: the canonical (row-major cell) order left by the last
   step -- the bands in rank order -- followed by the ray volumes of each launch since then, again
   the bands in rank order.  So the ids issued within each such segment are offset by an exclusive
   scan over (segment, rank), and the global ids are exactly those one domain would issue.
2. Migration -- the volumes whose carrier row left the band go to the owning band (a
   variable-size all-to-all; only neighbours exchange anything, since a step moves a carrier far
   less than a band).
3. ``engine.step_local(dt)`` -- canonical order, per-column cap, saturation and projection: all
   local to a carrier cell or column.
4. Halo exchange -- ``HALO`` = 2 rows of the raw projected fields from each neighbour: one for the
   3 x 3 smoothing and one for the centred meridional difference of the divergence.
5. ``engine.step_grid()`` -- smoothing and divergence; the band's rows of du/dt, dv/dt are those of
   a single domain bit for bit.
6. Budget -- counters and wave-action terms summed over the ranks.

The engine is duck-typed (methods ``set_owned_rows``, ``step_advance``, ``step_local``,
``step_grid``, ``take_rays_outside``, ``put_rays``, ``remap_ids``, ``issued_before``, ``next_id``,
``field``, ``set_field``, ``stats``, ``n_rays``).  All exchanges go through ``torch.distributed``
(``all_gather`` and ``all_to_all_single``), so the same code runs over ``gloo`` on the CPU and over
NCCL.
"""
from __future__ import annotations

import numpy as np

HALO = 2
NSTATE = 13
# provisional ids issued during a phase, before the global offsets are known
PROVISIONAL = 1 << 62
# fields smoothed and differenced by the grid phase (vertical fluxes, the six horizontal centre
# fields incl. the elastic terms, the wave-action diagnostic)
HALO_FIELDS = ("fz_l", "fz_p", "f_ll", "f_lp", "f_pl", "f_pp", "e_l", "e_p", "wad")
INT_STATS = ("n_launched", "n_filtered", "n_split_v", "n_split_h", "n_exited", "n_capped", "n_merged",
             "n_invalid")
W_STATS = ("w_total", "w_launched", "w_saturated", "w_exited", "w_capped", "w_invalid")


def band_bounds(ny: int, world: int):
    """Contiguous bands of rows, sizes differing by at most one; each band holds at least HALO rows
    (so that its halo comes from its immediate neighbours)."""
    if ny < HALO * world:
        raise ValueError("%d rows cannot give %d bands of at least %d rows" % (ny, world, HALO))
    base, extra = divmod(ny, world)
    out, j = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((j, j + n))
        j += n
    return out


def owner_of_rows(rows: np.ndarray, bounds) -> np.ndarray:
    """Rank owning each row."""
    starts = np.array([b[0] for b in bounds])
    return np.searchsorted(starts, np.asarray(rows), side="right") - 1


def _dist():
    import torch.distributed as dist
    return dist


def gather_counts(counts, group=None) -> np.ndarray:
    """Every rank's vector of counts (the same length on every rank): array [world, len]."""
    import torch
    dist = _dist()
    world = dist.get_world_size(group)
    t = torch.tensor([int(c) for c in counts], dtype=torch.int64)
    parts = [torch.zeros(len(counts), dtype=torch.int64) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    return np.stack([p.numpy() for p in parts]) if len(counts) else np.zeros((world, 0), dtype=np.int64)


def segment_offsets(counts: np.ndarray, rank: int):
    """Offsets of this rank's part of each segment in the order (segment, rank): counts[r, s] items
    of segment s on rank r; returns (offset of each of this rank's segments, total)."""
    flat = counts.T.reshape(-1)                       # segment-major, ranks in order
    starts = np.concatenate([[0], np.cumsum(flat)[:-1]]).reshape(counts.shape[1], counts.shape[0])
    return starts[:, rank], int(flat.sum())


def alltoallv(chunks, dtype, width: int, group=None):
    """Variable-size all-to-all: chunks[r] (rows of `width` values) goes to rank r; returns the list
    of the chunks received from each rank."""
    import torch
    dist = _dist()
    world = dist.get_world_size(group)
    counts = torch.tensor([len(c) for c in chunks], dtype=torch.int64)
    recv_counts = torch.empty(world, dtype=torch.int64)
    dist.all_to_all_single(recv_counts, counts, group=group)
    rc = [int(x) for x in recv_counts.tolist()]
    send = np.concatenate([np.asarray(c, dtype=dtype).reshape(-1, width) for c in chunks], axis=0) \
        if any(len(c) for c in chunks) else np.zeros((0, width), dtype=dtype)
    send_t = torch.from_numpy(np.ascontiguousarray(send).reshape(-1))
    recv_t = torch.empty(sum(rc) * width, dtype=send_t.dtype)
    dist.all_to_all_single(recv_t, send_t, output_split_sizes=[c * width for c in rc],
                           input_split_sizes=[len(c) * width for c in chunks], group=group)
    recv = recv_t.numpy().reshape(-1, width)
    out, o = [], 0
    for c in rc:
        out.append(recv[o:o + c])
        o += c
    return out


class BandDecomposition:
    """One rank's part of a domain-decomposed run (see the module docstring)."""

    def __init__(self, engine, ny: int, group=None, next_id: int = 0):
        dist = _dist()
        self.engine = engine
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.ny = ny
        self.bounds = band_bounds(ny, self.world)
        self.j0, self.j1 = self.bounds[self.rank]
        engine.set_owned_rows(self.j0, self.j1)
        self.next_id = int(next_id)
        engine.next_id = self.next_id
        # the band's array as segments: the canonical part left by the last step, then one per launch
        self.segments = [engine.n_rays]
        self.last_migrated = 0

    # -- ids
    def _remap(self, issued_per_segment):
        """Provisional ids issued segment by segment (in array order) -> the single domain's ids."""
        counts = gather_counts(issued_per_segment, self.group)
        offs, total = segment_offsets(counts, self.rank)
        lo = PROVISIONAL
        for s, c in enumerate(issued_per_segment):
            if c:
                self.engine.remap_ids(lo, lo + c, self.next_id + int(offs[s]))
            lo += c
        self.next_id += total
        self.engine.next_id = self.next_id

    def launch(self, launch_fn):
        """A launch into the band's own columns (launch_fn(engine) calls the engine's launch, the
        same launch on every rank); ids as one domain issues them (rows ascending)."""
        n0 = self.engine.n_rays
        self.engine.next_id = PROVISIONAL
        launch_fn(self.engine)
        self._remap([self.engine.next_id - PROVISIONAL])
        self.segments.append(self.engine.n_rays - n0)

    def advance(self, dt: float):
        """RK3, exits and splits of the band's ray volumes, ids made global."""
        self.engine.next_id = PROVISIONAL
        self.engine.step_advance(dt)
        ends = np.cumsum(self.segments)
        starts = np.concatenate([[0], ends[:-1]])
        self._remap([self.engine.issued_before(int(b)) - self.engine.issued_before(int(a))
                     for a, b in zip(starts, ends)])

    # -- migration
    def migrate(self):
        """Hand the ray volumes whose carrier row left the band to the owning ranks; returns the
        number sent."""
        st, ids, rows = self.engine.take_rays_outside()
        dest = owner_of_rows(rows, self.bounds) if len(ids) else np.zeros(0, dtype=np.int64)
        if np.any(dest == self.rank):
            raise RuntimeError("a ray volume inside the band was handed out")
        st_chunks = [st[dest == r] for r in range(self.world)]
        id_chunks = [ids[dest == r].reshape(-1, 1) for r in range(self.world)]
        got_st = alltoallv(st_chunks, np.float64, NSTATE, self.group)
        got_id = alltoallv(id_chunks, np.int64, 1, self.group)
        states = np.concatenate(got_st, axis=0) if got_st else np.zeros((0, NSTATE))
        rids = np.concatenate(got_id, axis=0).reshape(-1) if got_id else np.zeros(0, dtype=np.int64)
        if len(rids):
            self.engine.put_rays(states, rids)
        return len(ids)

    # -- halo
    def _neighbour_rows(self):
        """(rank, rows it needs from this band) for the bands whose halo reaches into this one."""
        out = []
        for r, (a, b) in enumerate(self.bounds):
            if r == self.rank:
                continue
            need = [j for j in list(range(a - HALO, a)) + list(range(b, b + HALO)) if self.j0 <= j < self.j1]
            out.append((r, need))
        return out

    def exchange_halo(self, names=HALO_FIELDS):
        """Copy HALO rows of every named field from the neighbouring bands into this band's arrays."""
        fields = {n: self.engine.field(n) for n in names}
        width = sum(f.shape[0] * f.shape[2] for f in fields.values())
        want = dict(self._neighbour_rows())
        chunks, rows_sent = [], []
        for r in range(self.world):
            rows = want.get(r, [])
            rows_sent.append(rows)
            chunks.append(np.stack([np.concatenate([fields[n][:, j, :].reshape(-1) for n in names]) for j in rows])
                          if rows else np.zeros((0, width)))
        got = alltoallv(chunks, np.float64, width, self.group)
        for r in range(self.world):
            if r == self.rank or not len(got[r]):
                continue
            a, b = self.bounds[r]
            rows = [j for j in list(range(self.j0 - HALO, self.j0)) + list(range(self.j1, self.j1 + HALO))
                    if a <= j < b]
            assert len(rows) == len(got[r])
            for j, vec in zip(rows, got[r]):
                o = 0
                for n in names:
                    f = fields[n]
                    size = f.shape[0] * f.shape[2]
                    f[:, j, :] = vec[o:o + size].reshape(f.shape[0], f.shape[2])
                    o += size
        for n in names:
            self.engine.set_field(n, fields[n])

    # -- the step
    def step(self, dt: float):
        """One step of the band; returns du/dt, dv/dt on the band's rows [nz][j1 - j0][nx]."""
        self.advance(dt)
        self.last_migrated = self.migrate()
        self.engine.step_local(dt)
        self.segments = [self.engine.n_rays]
        self.exchange_halo()
        du, dv = self.engine.step_grid()
        return du[:, self.j0:self.j1, :], dv[:, self.j0:self.j1, :]

    def stats(self) -> dict:
        """Counters and wave-action terms summed over the ranks (the live count too)."""
        import torch
        dist = _dist()
        s = self.engine.stats()
        ints = torch.tensor([s[k] for k in INT_STATS] + [self.engine.n_rays], dtype=torch.int64)
        ws = torch.tensor([s[k] for k in W_STATS], dtype=torch.float64)
        dist.all_reduce(ints, group=self.group)
        dist.all_reduce(ws, group=self.group)
        out = {k: int(v) for k, v in zip(INT_STATS, ints.tolist()[:-1])}
        out["n_live"] = int(ints[-1])
        out.update({k: float(v) for k, v in zip(W_STATS, ws.tolist())})
        return out
