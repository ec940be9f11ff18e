"""FP64 CPU oracle of the MS-GWaM-3D ray-volume step (arXiv:2309.11257).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this package.  The
library under ``paper_2309_11257_gb300`` never imports it, and this package
imports nothing from the library: the two share no code.

The arithmetic lives in ``gwam_oracle.c`` (plain C, FP64, no FMA contraction,
single threaded unless set_threads asks for more: the per-ray loops then run
under OpenMP with bit-identical results); this module compiles it with gcc on
first use and wraps it with ctypes.  Grid fields are numpy arrays in C order ``[nz][ny][nx]``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gwam_oracle.c")
_HDR = os.path.join(_HERE, "gwam_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NSTATE = 13
STATE_NAMES = ("x", "y", "z", "k", "l", "m", "ex", "ey", "ez", "px", "py", "pz", "n")


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, no FP contraction; OpenMP for the optional
    threaded per-ray loops, left out if the compiler lacks it)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + ".tmp%d" % os.getpid()
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
        r = subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], capture_output=True, text=True)
        if r.returncode != 0:
            subprocess.run(base + ["-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Grid(C.Structure):
    _fields_ = [("geometry", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("f0", C.c_double),
                ("radius", C.c_double), ("omega", C.c_double), ("g", C.c_double)]


class Params(C.Structure):
    _fields_ = [("gamma_mode", C.c_int), ("saturation", C.c_int), ("smoothing", C.c_int),
                ("flux_form", C.c_int), ("splitting", C.c_int), ("cap_per_column", C.c_int),
                ("alpha_s", C.c_double), ("min_split_dz", C.c_double), ("columnar", C.c_int)]


class Stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("n_live", "n_launched", "n_filtered", "n_split_v", "n_split_h",
                                         "n_exited", "n_capped", "n_merged", "n_invalid", "n_steps")] + \
               [(n, C.c_double) for n in ("w_total", "w_launched", "w_saturated", "w_exited", "w_capped",
                                          "w_invalid")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class BgSource(C.Structure):
    _fields_ = [("f_s", C.c_double), ("f_w", C.c_double), ("tau", C.c_double), ("z_launch", C.c_double),
                ("dz_launch", C.c_double), ("lambda_h", C.c_double), ("c_min", C.c_double),
                ("c_max", C.c_double), ("n_az", C.c_int), ("n_c", C.c_int), ("spectral_frac", C.c_double),
                ("phi_max_deg", C.c_double), ("launch_zero_flux", C.c_int)]


class Spec(C.Structure):
    _fields_ = [("i", C.c_int), ("j", C.c_int), ("pad_", C.c_int), ("z_launch", C.c_double),
                ("dz_launch", C.c_double), ("theta", C.c_double), ("c", C.c_double),
                ("lambda_h", C.c_double), ("flux", C.c_double), ("spectral_frac", C.c_double)]


_P = C.POINTER
_D = _P(C.c_double)


def _declare(lib):
    lib.orc_create.restype = C.c_void_p
    lib.orc_create.argtypes = [_P(Grid), _P(Params)]
    lib.orc_destroy.argtypes = [C.c_void_p]
    lib.orc_set_background.argtypes = [C.c_void_p, _D, _D, _D, _D]
    lib.orc_add_rays.argtypes = [C.c_void_p, C.c_int64] + [_D] * 13
    lib.orc_launch_background.argtypes = [C.c_void_p, _P(BgSource)]
    lib.orc_launch_spectral.argtypes = [C.c_void_p, C.c_int64, _P(Spec)]
    lib.orc_launch_ghost.argtypes = [C.c_void_p, _P(BgSource), C.c_double]
    lib.orc_launch_ghost_spectral.argtypes = [C.c_void_p, C.c_int64, _P(Spec), C.c_double]
    lib.orc_step.argtypes = [C.c_void_p, C.c_double, _D, _D]
    lib.orc_diagnose.argtypes = [C.c_void_p, _D, _D]
    lib.orc_num_rays.restype = C.c_int64
    lib.orc_num_rays.argtypes = [C.c_void_p]
    lib.orc_get_rays.argtypes = [C.c_void_p, _D, _P(C.c_int64), _P(C.c_int32)]
    lib.orc_get_stats.argtypes = [C.c_void_p, _P(Stats)]
    lib.orc_get_action_scale.argtypes = [C.c_void_p, _D]
    lib.orc_set_threads.restype = C.c_int
    lib.orc_set_threads.argtypes = [C.c_void_p, C.c_int]
    lib.orc_step_advance.argtypes = [C.c_void_p, C.c_double]
    lib.orc_step_local.argtypes = [C.c_void_p, C.c_double]
    lib.orc_step_grid.argtypes = [C.c_void_p, _D, _D]
    lib.orc_set_owned_rows.argtypes = [C.c_void_p, C.c_long, C.c_long]
    lib.orc_get_next_id.restype = C.c_int64
    lib.orc_get_next_id.argtypes = [C.c_void_p]
    lib.orc_set_next_id.argtypes = [C.c_void_p, C.c_int64]
    lib.orc_remap_ids.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int64]
    lib.orc_issued_before.restype = C.c_int64
    lib.orc_issued_before.argtypes = [C.c_void_p, C.c_int64]
    lib.orc_count_rays_outside.restype = C.c_int64
    lib.orc_count_rays_outside.argtypes = [C.c_void_p]
    lib.orc_take_rays_outside.restype = C.c_int64
    lib.orc_take_rays_outside.argtypes = [C.c_void_p, _D, _P(C.c_int64), _P(C.c_int32), C.c_int64]
    lib.orc_put_rays.argtypes = [C.c_void_p, C.c_int64, _D, _P(C.c_int64)]
    lib.orc_set_field.argtypes = [C.c_void_p, C.c_int, _D]
    lib.orc_get_field.argtypes = [C.c_void_p, C.c_int, _D]
    lib.orc_get_gamma2.argtypes = [C.c_void_p, _D]
    lib.orc_get_field_abs.argtypes = [C.c_void_p, C.c_int, _D]
    lib.orc_tendency_scale.argtypes = [C.c_void_p, _D, _D]
    lib.orc_set_theta.argtypes = [C.c_void_p, _D]
    lib.orc_theta_tendency.argtypes = [C.c_void_p, _D, _D]
    lib.orc_theta_divergence.argtypes = [C.c_void_p, _D, _D, _D]
    lib.orc_gather.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, _D]
    lib.orc_dispersion.argtypes = [C.c_double] * 6 + [_D]
    lib.orc_rhs.argtypes = [C.c_void_p, _D, _D]
    lib.orc_omega.restype = C.c_double
    lib.orc_omega.argtypes = [C.c_void_p] + [C.c_double] * 6
    lib.orc_rk3.argtypes = [C.c_void_p, _D, C.c_double]
    lib.orc_advance_ray.argtypes = [C.c_void_p, _D, C.c_double]
    lib.orc_cell_pq.argtypes = [C.c_void_p, _D, _D]
    lib.orc_alpha_profile.restype = C.c_double
    lib.orc_alpha_profile.argtypes = [C.c_double]
    lib.orc_fam.restype = C.c_double
    lib.orc_fam.argtypes = [C.c_double] * 4
    lib.orc_divergence.argtypes = [C.c_void_p] + [_D] * 10
    lib.orc_smooth.argtypes = [C.c_void_p, _D, C.c_int]
    lib.orc_ray_energy.restype = C.c_double
    lib.orc_ray_energy.argtypes = [C.c_void_p, _D]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            h = C.CDLL(path)
            _declare(h)
            _lib = h
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


FIELD_NAMES = ("fz_l", "fz_p", "f_ll", "f_lp", "f_pl", "f_pp", "e_l", "e_p", "wad")
THETA_FIELD_NAMES = ("t_l", "t_p")          # potential-temperature flux integrals (Eq. fluxes:temperature)
ALL_FIELD_NAMES = FIELD_NAMES + THETA_FIELD_NAMES


def _struct(cls, d: dict):
    s = cls()
    for name, _ in cls._fields_:
        if name in d:
            setattr(s, name, d[name])
    return s


def alpha_profile(phi_deg: float) -> float:
    return lib().orc_alpha_profile(float(phi_deg))


def fam(phi_deg: float, tau: float, f_s: float, f_w: float) -> float:
    return lib().orc_fam(float(phi_deg), float(tau), float(f_s), float(f_w))


def dispersion(k, l, m, n2, g2, f2):
    """(w_hat, ch_x, ch_y, ch_r, K2) of the positive intrinsic branch."""
    out = np.zeros(5)
    lib().orc_dispersion(float(k), float(l), float(m), float(n2), float(g2), float(f2), _dp(out))
    return out


class Model:
    """One oracle instance: grid, parameters, background, ray volumes."""

    def __init__(self, grid: dict, params: dict):
        self._lib = lib()
        self.grid = dict(grid)
        self.params = dict(params)
        self._g = _struct(Grid, grid)
        self._p = _struct(Params, params)
        self._h = self._lib.orc_create(C.byref(self._g), C.byref(self._p))
        if not self._h:
            raise ValueError("oracle rejected the grid/params")
        self.nx, self.ny, self.nz = grid["nx"], grid["ny"], grid["nz"]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    # -- inputs
    def set_threads(self, n: int) -> int:
        """Threads for the independent per-ray loops (results identical for any count); returns
        the count in effect."""
        return int(self._lib.orc_set_threads(self._h, int(n)))

    # -- the phases of a step and the latitude-band hooks of a domain-decomposed run (App. B.2)
    def step_advance(self, dt: float):
        if self._lib.orc_step_advance(self._h, float(dt)) != 0:
            raise ValueError("step failed")

    def step_local(self, dt: float):
        self._lib.orc_step_local(self._h, float(dt))

    def step_grid(self):
        shape = (self.nz, self.ny, self.nx)
        du, dv = np.zeros(shape), np.zeros(shape)
        self._lib.orc_step_grid(self._h, _dp(du), _dp(dv))
        return du, dv

    def set_owned_rows(self, j0: int, j1: int):
        if self._lib.orc_set_owned_rows(self._h, int(j0), int(j1)) != 0:
            raise ValueError("bad band")

    @property
    def next_id(self) -> int:
        return int(self._lib.orc_get_next_id(self._h))

    @next_id.setter
    def next_id(self, v: int):
        self._lib.orc_set_next_id(self._h, int(v))

    def remap_ids(self, lo: int, hi: int, to: int):
        """ids in [lo, hi) become id - lo + to"""
        self._lib.orc_remap_ids(self._h, int(lo), int(hi), int(to))

    def issued_before(self, q: int) -> int:
        """new ids issued by the rays before array position q in the last advance"""
        return int(self._lib.orc_issued_before(self._h, int(q)))

    def take_rays_outside(self):
        """Ray volumes whose carrier row left the owned band, removed: (states [n, 13], ids [n],
        carrier rows [n])."""
        n = int(self._lib.orc_count_rays_outside(self._h))
        st = np.zeros((n, NSTATE))
        ids = np.zeros(n, dtype=np.int64)
        rows = np.zeros(n, dtype=np.int32)
        if n:
            got = self._lib.orc_take_rays_outside(self._h, _dp(st), ids.ctypes.data_as(_P(C.c_int64)),
                                                  rows.ctypes.data_as(_P(C.c_int32)), n)
            assert got == n
        return st, ids, rows

    def put_rays(self, states, ids):
        st = np.ascontiguousarray(states, dtype=np.float64).reshape(-1, NSTATE)
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        if len(ids):
            self._lib.orc_put_rays(self._h, len(ids), _dp(st), ids.ctypes.data_as(_P(C.c_int64)))

    def set_field(self, name: str, values):
        which = ALL_FIELD_NAMES.index(name)
        a = _f64(values)
        if self._lib.orc_set_field(self._h, which, _dp(a)) != 0:
            raise ValueError(name)

    def set_background(self, u, v, n2, rho):
        arrs = [_f64(a).reshape(self.nz, self.ny, self.nx) for a in (u, v, n2, rho)]
        rc = self._lib.orc_set_background(self._h, *[_dp(a) for a in arrs])
        if rc != 0:
            raise ValueError("oracle rejected the background (%d)" % rc)

    def add_rays(self, r: dict):
        """r: dict of arrays x y z k l m ex ey ez dk dl dm n."""
        names = ("x", "y", "z", "k", "l", "m", "ex", "ey", "ez", "dk", "dl", "dm", "n")
        arrs = [_f64(r[n]) for n in names]
        rc = self._lib.orc_add_rays(self._h, len(arrs[0]), *[_dp(a) for a in arrs])
        if rc != 0:
            raise ValueError("oracle rejected a ray")

    def launch_background(self, src: dict):
        s = _struct(BgSource, src)
        if self._lib.orc_launch_background(self._h, C.byref(s)) != 0:
            raise ValueError("launch rejected")

    @staticmethod
    def _specs(specs: np.ndarray):
        n = len(specs)
        arr = (Spec * max(n, 1))()
        for q in range(n):
            for name, _ in Spec._fields_:
                if name in specs.dtype.names:
                    setattr(arr[q], name, specs[name][q].item())
        return n, arr

    def launch_spectral(self, specs: np.ndarray):
        """specs: structured array with fields of Spec (see synth.SPEC_DTYPE)."""
        n, arr = self._specs(specs)
        if self._lib.orc_launch_spectral(self._h, n, arr) != 0:
            raise ValueError("spectral launch rejected")

    def launch_ghost(self, src: dict, dt: float):
        """Ghost-layer emission of the background source over one launch interval dt."""
        s = _struct(BgSource, src)
        if self._lib.orc_launch_ghost(self._h, C.byref(s), float(dt)) != 0:
            raise ValueError("ghost launch rejected")

    def launch_ghost_spectral(self, specs: np.ndarray, dt: float):
        n, arr = self._specs(specs)
        if self._lib.orc_launch_ghost_spectral(self._h, n, arr, float(dt)) != 0:
            raise ValueError("ghost spectral launch rejected")

    # -- step
    def step(self, dt: float, want_tendencies: bool = True):
        shape = (self.nz, self.ny, self.nx)
        du = np.zeros(shape)
        dv = np.zeros(shape)
        rc = self._lib.orc_step(self._h, float(dt), _dp(du), _dp(dv))
        if rc != 0:
            raise ValueError("oracle step failed (%d)" % rc)
        return du, dv

    def diagnose(self):
        """Project the current ray volumes (no advance); returns du/dt, dv/dt."""
        shape = (self.nz, self.ny, self.nx)
        du = np.zeros(shape)
        dv = np.zeros(shape)
        if self._lib.orc_diagnose(self._h, _dp(du), _dp(dv)) != 0:
            raise ValueError("diagnose failed")
        return du, dv

    # -- outputs
    @property
    def n_rays(self) -> int:
        return int(self._lib.orc_num_rays(self._h))

    def rays(self) -> dict:
        """Ray state in array order: dict of the 13 state arrays plus id and cell."""
        n = self.n_rays
        st = np.zeros((NSTATE, n))
        ids = np.zeros(n, dtype=np.int64)
        cells = np.zeros(n, dtype=np.int32)
        if n:
            self._lib.orc_get_rays(self._h, _dp(st), ids.ctypes.data_as(_P(C.c_int64)),
                                   cells.ctypes.data_as(_P(C.c_int32)))
        out = {name: st[q].copy() for q, name in enumerate(STATE_NAMES)}
        out["id"] = ids
        out["cell"] = cells
        # scale of the rounding error of N: its value before the last step's saturation
        out["n_scale"] = np.zeros(n)
        if n:
            self._lib.orc_get_action_scale(self._h, _dp(out["n_scale"]))
        return out

    def stats(self) -> dict:
        s = Stats()
        self._lib.orc_get_stats(self._h, C.byref(s))
        return s.as_dict()

    def field(self, name: str) -> np.ndarray:
        which = ALL_FIELD_NAMES.index(name)
        nl = self.nz + 1 if which < 2 else self.nz
        out = np.zeros((nl, self.ny, self.nx))
        self._lib.orc_get_field(self._h, which, _dp(out))
        return out

    def field_abs(self, name: str) -> np.ndarray:
        """Sum of |contribution| of a projected field (the scale of its rounding error), each
        contribution taken with the ray volume's wave action before the step's saturation and with
        the wavenumber and group-velocity components replaced by the magnitudes of their vectors."""
        which = ALL_FIELD_NAMES.index(name)
        nl = self.nz + 1 if which < 2 else self.nz
        out = np.zeros((nl, self.ny, self.nx))
        self._lib.orc_get_field_abs(self._h, which, _dp(out))
        return out

    def set_theta(self, theta):
        """Reference potential temperature [nz][ny][nx] (positive)."""
        t = _f64(theta)
        if self._lib.orc_set_theta(self._h, _dp(t)) != 0:
            raise ValueError("oracle rejected theta")

    def theta_divergence(self, tl, tp):
        """d theta/dt of given integrals T_l, T_p [nz][ny][nx]."""
        out = np.zeros((self.nz, self.ny, self.nx))
        if self._lib.orc_theta_divergence(self._h, _dp(_f64(tl)), _dp(_f64(tp)), _dp(out)) != 0:
            raise ValueError("no theta set")
        return out

    def theta_tendency(self):
        """(d theta/dt of the last step, its error scale), [nz][ny][nx] each."""
        shape = (self.nz, self.ny, self.nx)
        out = np.zeros(shape)
        sc = np.zeros(shape)
        if self._lib.orc_theta_tendency(self._h, _dp(out), _dp(sc)) != 0:
            raise ValueError("no theta set")
        return out, sc

    def tendency_scale(self):
        """Error scales of du/dt and dv/dt of the last step (magnitudes through the divergence)."""
        shape = (self.nz, self.ny, self.nx)
        du = np.zeros(shape)
        dv = np.zeros(shape)
        self._lib.orc_tendency_scale(self._h, _dp(du), _dp(dv))
        return du, dv

    def gamma2(self) -> np.ndarray:
        out = np.zeros((self.nz, self.ny, self.nx))
        self._lib.orc_get_gamma2(self._h, _dp(out))
        return out

    # -- single-ray pieces
    def gather(self, X, Y, Z) -> np.ndarray:
        out = np.zeros(16)
        self._lib.orc_gather(self._h, float(X), float(Y), float(Z), _dp(out))
        return out

    def rhs(self, y9) -> np.ndarray:
        y = _f64(y9).copy()
        f = np.zeros(9)
        self._lib.orc_rhs(self._h, _dp(y), _dp(f))
        return f

    def omega(self, X, Y, Z, k, l, m) -> float:
        return self._lib.orc_omega(self._h, float(X), float(Y), float(Z), float(k), float(l), float(m))

    def rk3(self, y9, dt) -> np.ndarray:
        y = _f64(y9).copy()
        self._lib.orc_rk3(self._h, _dp(y), float(dt))
        return y

    def advance_ray(self, state13, dt) -> np.ndarray:
        s = _f64(state13).copy()
        self._lib.orc_advance_ray(self._h, _dp(s), float(dt))
        return s

    def cell_pq(self):
        shape = (self.nz, self.ny, self.nx)
        p = np.zeros(shape)
        q = np.zeros(shape)
        self._lib.orc_cell_pq(self._h, _dp(p), _dp(q))
        return p, q

    def divergence(self, fields: dict):
        shape = (self.nz, self.ny, self.nx)
        du = np.zeros(shape)
        dv = np.zeros(shape)
        arrs = [_f64(fields[n]) for n in FIELD_NAMES[:8]]
        self._lib.orc_divergence(self._h, *[_dp(a) for a in arrs], _dp(du), _dp(dv))
        return du, dv

    def smooth(self, field: np.ndarray) -> np.ndarray:
        f = _f64(field).copy()
        self._lib.orc_smooth(self._h, _dp(f), f.shape[0])
        return f

    def ray_energy(self, state13) -> float:
        s = _f64(state13).copy()
        return self._lib.orc_ray_energy(self._h, _dp(s))
