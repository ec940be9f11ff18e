"""ctypes binding of libgwam.so (include/gwam.h).

Argument marshalling only: every step of the ray-volume path runs in the library's CUDA
kernels.  Device buffers are torch CUDA tensors (float64, contiguous); the context's stream
is the torch stream current at construction.  Importing this module loads libgwam.so and
raises if it is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgwam.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libgwam.so is not built (run __graft_entry__.build() or paper_2309_11257_gb300/build.py); "
                      "the ray-volume path has no CPU fallback")

_lib = C.CDLL(LIB_PATH)

GWAM_OK, GWAM_EINVAL, GWAM_ENOMEM, GWAM_ECAPACITY, GWAM_ENUMERIC, GWAM_ECUDA, GWAM_ETIMEOUT, GWAM_ESTATE = \
    0, -1, -2, -3, -4, -5, -6, -7
STATUS_NAMES = {0: "GWAM_OK", -1: "GWAM_EINVAL", -2: "GWAM_ENOMEM", -3: "GWAM_ECAPACITY", -4: "GWAM_ENUMERIC",
                -5: "GWAM_ECUDA", -6: "GWAM_ETIMEOUT", -7: "GWAM_ESTATE"}
STATE_NAMES = ("x", "y", "z", "k", "l", "m", "ex", "ey", "ez", "px", "py", "pz", "n")
MEMBER_SHIFT = 56     # ray ids carry the ensemble member in their top 8 bits
FIELD_NAMES = ("fz_l", "fz_p", "f_ll", "f_lp", "f_pl", "f_pp", "e_l", "e_p", "wad", "t_l", "t_p")


class GwamError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, code), msg))
        self.code = code


class Grid(C.Structure):
    _fields_ = [("geometry", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("f0", C.c_double),
                ("radius", C.c_double), ("omega", C.c_double), ("g", C.c_double)]


class Params(C.Structure):
    _fields_ = [("precision", C.c_int), ("gamma_mode", C.c_int), ("saturation", C.c_int), ("smoothing", C.c_int),
                ("flux_form", C.c_int), ("splitting", C.c_int), ("cap_per_column", C.c_int),
                ("alpha_s", C.c_double), ("min_split_dz", C.c_double), ("max_rays", C.c_int64),
                ("members", C.c_int), ("columnar", C.c_int), ("theta_flux", C.c_int)]


class BgSource(C.Structure):
    _fields_ = [("f_s", C.c_double), ("f_w", C.c_double), ("tau", C.c_double), ("z_launch", C.c_double),
                ("dz_launch", C.c_double), ("lambda_h", C.c_double), ("c_min", C.c_double),
                ("c_max", C.c_double), ("n_az", C.c_int), ("n_c", C.c_int), ("spectral_frac", C.c_double),
                ("phi_max_deg", C.c_double), ("launch_zero_flux", C.c_int)]


class Spec(C.Structure):
    _fields_ = [("i", C.c_int), ("j", C.c_int), ("member", C.c_int), ("z_launch", C.c_double),
                ("dz_launch", C.c_double), ("theta", C.c_double), ("c", C.c_double),
                ("lambda_h", C.c_double), ("flux", C.c_double), ("spectral_frac", C.c_double)]


class RayInput(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("x", "y", "z", "k", "l", "m", "ex", "ey", "ez", "dk", "dl", "dm", "n")]


class Stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("n_live", "n_launched", "n_filtered", "n_split_v", "n_split_h",
                                         "n_exited", "n_capped", "n_merged", "n_invalid", "n_steps",
                                         "ray_steps")] + \
               [(n, C.c_double) for n in ("w_total", "w_launched", "w_saturated", "w_exited", "w_capped",
                                          "w_invalid")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class MlpConfig(C.Structure):
    _fields_ = [("n_in", C.c_int), ("n_hidden", C.c_int), ("n_layers", C.c_int), ("n_out", C.c_int),
                ("nlev", C.c_int), ("max_batch", C.c_int), ("seed", C.c_uint64), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float)]


_vp = C.c_void_p
_P = C.POINTER
# name -> (restype, argtypes); every entry point declared in include/gwam.h
SIGNATURES = {
    "gwam_init": (C.c_int, [_P(_vp), _P(Grid), _P(Params), _vp]),
    "gwam_destroy": (None, [_vp]),
    "gwam_set_background": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "gwam_set_background_host": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "gwam_set_member_background": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp]),
    "gwam_set_member_background_host": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp]),
    "gwam_add_rays": (C.c_int, [_vp, _P(RayInput), C.c_int64]),
    "gwam_add_rays_host": (C.c_int, [_vp, _P(RayInput), C.c_int64]),
    "gwam_launch_sources": (C.c_int, [_vp, _P(BgSource)]),
    "gwam_launch_spectral": (C.c_int, [_vp, _vp, C.c_int64]),
    "gwam_launch_spectral_host": (C.c_int, [_vp, _vp, C.c_int64]),
    "gwam_launch_ghost": (C.c_int, [_vp, _P(BgSource), C.c_double]),
    "gwam_launch_ghost_spectral": (C.c_int, [_vp, _vp, C.c_int64, C.c_double]),
    "gwam_launch_ghost_spectral_host": (C.c_int, [_vp, _vp, C.c_int64, C.c_double]),
    "gwam_step": (C.c_int, [_vp, C.c_double, _vp, _vp]),
    "gwam_step_host": (C.c_int, [_vp, C.c_double, _vp, _vp]),
    "gwam_step_graph": (C.c_int, [_vp, C.c_double, _vp, _vp]),
    "gwam_set_background_host_async": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "gwam_step_host_async": (C.c_int, [_vp, C.c_double, _vp, _vp]),
    "gwam_set_launch_config": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int]),
    "gwam_get_launch_config": (C.c_int, [_vp, C.c_int, _P(C.c_int), _P(C.c_int)]),
    "gwam_autotune": (C.c_int, [_vp, C.c_double, C.c_int, _vp, _vp]),
    "gwam_num_rays": (C.c_int, [_vp, _P(C.c_int64)]),
    "gwam_get_rays_host": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int64]),
    "gwam_get_stats": (C.c_int, [_vp, _P(Stats)]),
    "gwam_get_field_host": (C.c_int, [_vp, C.c_int, _vp]),
    "gwam_get_gamma2_host": (C.c_int, [_vp, _vp]),
    "gwam_synchronize": (C.c_int, [_vp]),
    "gwam_cell_offsets": (C.c_int, [_vp, C.c_int64, C.c_int32, _vp, _vp]),
    "gwam_cell_offsets_noalloc": (C.c_int, [_vp, C.c_int64, C.c_int32, _vp, _vp]),
    "gwam_selftest_math": (C.c_int, [_vp, C.c_int64, _vp, _vp, _vp]),
    "gwam_selftest_widen": (C.c_int, [_vp, C.c_int64, _vp, _vp, _vp]),
    "gwam_selftest_narrow": (C.c_int, [_vp, C.c_int64, _vp, _vp]),
    "gwam_selftest_split": (C.c_int, [_vp, C.c_int64, _vp, _vp, _vp]),
    "gwam_selftest_logratio": (C.c_int, [_vp, _vp, C.c_int64, _vp, _vp]),
    "gwam_save": (C.c_int, [_vp, C.c_char_p]),
    "gwam_set_theta": (C.c_int, [_vp, _vp]),
    "gwam_get_theta_tendency_host": (C.c_int, [_vp, _vp]),
    "gwam_load": (C.c_int, [_vp, C.c_char_p]),
    "gwam_gemm_bf16": (C.c_int, [_vp, _vp, C.c_int, C.c_int, C.c_int, _vp, C.c_int, C.c_int, C.c_int, _vp, _vp]),
    "gwam_selftest_gemm_timeout": (C.c_int, [_vp, _vp, C.c_int, C.c_int, C.c_int, C.c_int, _vp, C.c_uint, _vp]),
    "gwam_mlp_create": (C.c_int, [_P(_vp), _P(MlpConfig), _vp]),
    "gwam_mlp_destroy": (None, [_vp]),
    "gwam_mlp_last_error": (C.c_char_p, [_vp]),
    "gwam_mlp_set_normalization_host": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "gwam_mlp_fit_normalization": (C.c_int, [_vp, _vp, _vp, C.c_int64, C.c_float, _vp]),
    "gwam_mlp_set_params_host": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "gwam_mlp_get_params_host": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp]),
    "gwam_mlp_train_step": (C.c_int, [_vp, _vp, _vp, C.c_int64, _vp, C.c_int, C.c_uint64, C.c_float]),
    "gwam_mlp_last_loss_host": (C.c_int, [_vp, _P(C.c_double)]),
    "gwam_mlp_output_host": (C.c_int, [_vp, _vp, C.c_int]),
    "gwam_mlp_infer": (C.c_int, [_vp, _vp, C.c_int64, _vp, _vp, _vp, _vp]),
    "gwam_mlp_status": (C.c_int, [_vp]),
    "gwam_mlp_profile_enable": (C.c_int, [_vp, C.c_int]),
    "gwam_mlp_profile_read": (C.c_int, [_vp, _vp, _P(C.c_int64)]),
    "gwam_mlp_merge_fallback": (C.c_int, [_vp, C.c_int64, C.c_int, _vp, _vp, _vp, _vp, _vp]),
    "gwam_column_features": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int, C.c_int64, _vp, C.c_int, C.c_int, _vp, _vp]),
    "gwam_column_targets": (C.c_int, [_vp, _vp, C.c_int, C.c_int64, C.c_double, _vp, _vp]),
    "gwam_profile_enable": (C.c_int, [_vp, C.c_int]),
    "gwam_profile_read": (C.c_int, [_vp, _vp, _P(C.c_int64)]),
    "gwam_graph_profile_read": (C.c_int, [_vp, _vp, _P(C.c_int)]),
    "gwam_graph_kernel_count": (C.c_int, [_vp, _P(C.c_int)]),
    "gwam_selftest_scan": (C.c_int, [_vp, _vp, _vp, C.c_int64, _vp, _vp, C.c_int64]),
    "gwam_last_error": (C.c_char_p, [_vp]),
    "gwam_version": (C.c_char_p, []),
}
for _name, (_res, _args) in SIGNATURES.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def lib():
    return _lib


def version() -> str:
    return _lib.gwam_version().decode()


def _struct(cls, d: dict):
    s = cls()
    for name, _ in cls._fields_:
        if name in d:
            setattr(s, name, d[name])
    return s


def _ptr(t):
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return C.c_void_p(t.data_ptr())


def cell_offsets(cells, ncell: int, offsets=None, stream=None):
    """Per-cell segment offsets (ncell + 1 int32) of a cell-ordered int32 CUDA tensor of cells."""
    import torch
    if offsets is None:
        offsets = torch.empty(ncell + 1, dtype=torch.int32, device=cells.device)
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = _lib.gwam_cell_offsets(_ptr(cells) if cells.numel() else None, cells.numel(), int(ncell), _ptr(offsets),
                                C.c_void_p(s.cuda_stream))
    if rc != 0:
        raise GwamError(rc, "gwam_cell_offsets")
    return offsets


class Tracer:
    """One ray-volume context on the current CUDA device."""

    def __init__(self, grid: dict, params: dict, max_rays: int, stream=None, members: int = 1):
        import torch
        self.grid = dict(grid)
        self.params = dict(params, members=members)
        self.members = members
        self.nx, self.ny, self.nz = grid["nx"], grid["ny"], grid["nz"]
        self.max_rays = int(max_rays)
        p = dict(params, max_rays=self.max_rays, members=members)
        p.setdefault("precision", 0)
        self._g = _struct(Grid, grid)
        self._p = _struct(Params, p)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        h = C.c_void_p()
        rc = _lib.gwam_init(C.byref(h), C.byref(self._g), C.byref(self._p), C.c_void_p(s.cuda_stream))
        if rc != 0:
            raise GwamError(rc, "gwam_init")
        self._h = h

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.gwam_destroy(h)
            self._h = None

    def __del__(self):
        self.close()

    def _check(self, rc, what):
        if rc != 0:
            raise GwamError(rc, "%s: %s" % (what, _lib.gwam_last_error(self._h).decode()))

    # -------------------------------------------------------------- inputs
    def set_background(self, u, v, n2, rho):
        """Device tensors (float64, [nz][ny][nx]) or numpy arrays (host path)."""
        if isinstance(u, np.ndarray):
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (u, v, n2, rho)]
            self._check(_lib.gwam_set_background_host(self._h, *[a.ctypes.data_as(_vp) for a in arrs]),
                        "set_background_host")
        else:
            self._check(_lib.gwam_set_background(self._h, *[_ptr(a) for a in (u, v, n2, rho)]), "set_background")

    def set_member_background(self, member: int, u, v, n2, rho):
        if isinstance(u, np.ndarray):
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (u, v, n2, rho)]
            self._check(_lib.gwam_set_member_background_host(self._h, member, *[a.ctypes.data_as(_vp) for a in arrs]),
                        "set_member_background_host")
        else:
            self._check(_lib.gwam_set_member_background(self._h, member, *[_ptr(a) for a in (u, v, n2, rho)]),
                        "set_member_background")

    def add_rays(self, r: dict):
        names = ("x", "y", "z", "k", "l", "m", "ex", "ey", "ez", "dk", "dl", "dm", "n")
        arrs = [np.ascontiguousarray(r[n], dtype=np.float64) for n in names]
        ri = RayInput(*[a.ctypes.data_as(_vp) for a in arrs])
        self._check(_lib.gwam_add_rays_host(self._h, C.byref(ri), len(arrs[0])), "add_rays_host")

    def launch_sources(self, src: dict):
        s = _struct(BgSource, src)
        self._check(_lib.gwam_launch_sources(self._h, C.byref(s)), "launch_sources")

    @staticmethod
    def _specs(specs: np.ndarray) -> np.ndarray:
        specs = np.ascontiguousarray(specs)
        assert specs.dtype.itemsize == C.sizeof(Spec) and all(
            specs.dtype.fields[n][1] == getattr(Spec, n).offset for n, _ in Spec._fields_), "spec layout"
        return specs

    def launch_spectral(self, specs: np.ndarray):
        """specs: numpy structured array laid out like gwam_spec (synth.SPEC_DTYPE, host memory)."""
        specs = self._specs(specs)
        self._check(_lib.gwam_launch_spectral_host(self._h, specs.ctypes.data_as(_vp), len(specs)),
                    "launch_spectral_host")

    def launch_ghost(self, src: dict, dt: float):
        """Ghost-layer emission of the background source over one launch interval dt (FP64 form)."""
        s = _struct(BgSource, src)
        self._check(_lib.gwam_launch_ghost(self._h, C.byref(s), float(dt)), "launch_ghost")

    def launch_ghost_spectral(self, specs: np.ndarray, dt: float):
        specs = self._specs(specs)
        self._check(_lib.gwam_launch_ghost_spectral_host(self._h, specs.ctypes.data_as(_vp), len(specs),
                                                          float(dt)), "launch_ghost_spectral_host")

    # -------------------------------------------------------------- step
    def step(self, dt: float, dudt=None, dvdt=None):
        """Stream-ordered step; dudt/dvdt: device tensors [nz][ny][nx] float64 or None."""
        self._check(_lib.gwam_step(self._h, float(dt), _ptr(dudt) if dudt is not None else None,
                                   _ptr(dvdt) if dvdt is not None else None), "step")

    def step_graph(self, dt: float, dudt=None, dvdt=None):
        """Step replayed from a captured CUDA graph (captured on first use for these buffers)."""
        self._check(_lib.gwam_step_graph(self._h, float(dt), _ptr(dudt) if dudt is not None else None,
                                         _ptr(dvdt) if dvdt is not None else None), "step_graph")

    KERNELS = ("advance", "materialize", "project")

    def launch_config(self) -> dict:
        out = {}
        for k, name in enumerate(self.KERNELS):
            t, b = C.c_int(), C.c_int()
            self._check(_lib.gwam_get_launch_config(self._h, k, C.byref(t), C.byref(b)), "get_launch_config")
            out[name] = (t.value, b.value)
        return out

    def set_launch_config(self, cfg: dict):
        for k, name in enumerate(self.KERNELS):
            if name in cfg:
                t, b = cfg[name]
                self._check(_lib.gwam_set_launch_config(self._h, k, int(t), int(b)), "set_launch_config")

    def autotune(self, dt: float, steps_per_candidate: int = 2, dudt=None, dvdt=None) -> dict:
        """Advance the simulation while timing candidate launch shapes; keep the fastest per kernel."""
        self._check(_lib.gwam_autotune(self._h, float(dt), int(steps_per_candidate),
                                       _ptr(dudt) if dudt is not None else None,
                                       _ptr(dvdt) if dvdt is not None else None), "autotune")
        return self.launch_config()

    def step_host(self, dt: float, dudt: np.ndarray, dvdt: np.ndarray):
        """Step with host (numpy, ideally pinned) output buffers; synchronising."""
        self._check(_lib.gwam_step_host(self._h, float(dt), dudt.ctypes.data_as(_vp), dvdt.ctypes.data_as(_vp)),
                    "step_host")

    # -------------------------------------------------------------- potential temperature
    def set_background_async(self, u, v, n2, rho):
        """Page-locked numpy arrays [nz][ny][nx]: copied on the context's upload stream, set up without
        waiting (keep them unchanged until the next synchronising call)."""
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (u, v, n2, rho)]
        self._check(_lib.gwam_set_background_host_async(self._h, *[a.ctypes.data_as(_vp) for a in arrs]),
                    "set_background_host_async")

    def step_host_async(self, dt: float, dudt: np.ndarray, dvdt: np.ndarray):
        """Page-locked numpy outputs, valid after the next synchronising call."""
        self._check(_lib.gwam_step_host_async(self._h, float(dt), dudt.ctypes.data_as(_vp),
                                              dvdt.ctypes.data_as(_vp)), "step_host_async")

    def set_theta(self, theta):
        """Reference potential temperature: a float64 CUDA tensor [members][nz][ny][nx] (or [nz][ny][nx])."""
        self._check(_lib.gwam_set_theta(self._h, _ptr(theta)), "set_theta")

    def theta_tendency(self) -> np.ndarray:
        """d theta/dt of the last step (needs theta_flux = 1 and set_theta)."""
        out = np.zeros((self.members, self.nz, self.ny, self.nx))
        self._check(_lib.gwam_get_theta_tendency_host(self._h, out.ctypes.data_as(_vp)), "get_theta_tendency_host")
        return out[0] if self.members == 1 else out

    # -------------------------------------------------------------- checkpoints
    def save(self, path: str):
        """Write the complete step state (rays, ids, counters, budget, background) to `path`."""
        self._check(_lib.gwam_save(self._h, os.fsencode(path)), "save")

    def load(self, path: str):
        """Read a checkpoint written by a tracer of the same grid, parameters and precision."""
        self._check(_lib.gwam_load(self._h, os.fsencode(path)), "load")

    # -------------------------------------------------------------- outputs
    def num_rays(self) -> int:
        n = C.c_int64()
        self._check(_lib.gwam_num_rays(self._h, C.byref(n)), "num_rays")
        return n.value

    def rays(self) -> dict:
        n = self.num_rays()
        cap = max(n, 1)
        st = np.zeros((13, cap))
        ids = np.zeros(cap, dtype=np.int64)
        cells = np.zeros(cap, dtype=np.int32)
        self._check(_lib.gwam_get_rays_host(self._h, st.ctypes.data_as(_vp), ids.ctypes.data_as(_vp),
                                            cells.ctypes.data_as(_vp), cap), "get_rays_host")
        out = {name: st[q, :n].copy() for q, name in enumerate(STATE_NAMES)}
        out["id"] = ids[:n] & ((1 << MEMBER_SHIFT) - 1)
        out["member"] = (ids[:n] >> MEMBER_SHIFT).astype(np.int32)
        ncell = self.nx * self.ny * self.nz
        out["cell"] = cells[:n] - out["member"] * ncell
        return out

    def stats(self) -> dict:
        s = Stats()
        self._check(_lib.gwam_get_stats(self._h, C.byref(s)), "get_stats")
        return s.as_dict()

    def field(self, name: str) -> np.ndarray:
        which = FIELD_NAMES.index(name)
        nl = self.nz + 1 if which < 2 else self.nz
        out = np.zeros((self.members, nl, self.ny, self.nx))
        self._check(_lib.gwam_get_field_host(self._h, which, out.ctypes.data_as(_vp)), "get_field_host")
        return out[0] if self.members == 1 else out

    def gamma2(self) -> np.ndarray:
        out = np.zeros((self.members, self.nz, self.ny, self.nx))
        self._check(_lib.gwam_get_gamma2_host(self._h, out.ctypes.data_as(_vp)), "get_gamma2_host")
        return out[0] if self.members == 1 else out

    PHASES = ("advance", "rebin", "saturation", "projection", "grid")

    def profile(self, enable: bool = True):
        self._check(_lib.gwam_profile_enable(self._h, 1 if enable else 0), "profile_enable")

    def profile_read(self):
        ms = np.zeros(5)
        n = C.c_int64()
        self._check(_lib.gwam_profile_read(self._h, ms.ctypes.data_as(_vp), C.byref(n)), "profile_read")
        return dict(zip(self.PHASES, ms.tolist())), n.value

    def graph_profile_read(self):
        """Phase times (ms) of the last replay of each step graph, averaged; and how many graphs."""
        ms = np.zeros(5)
        n = C.c_int()
        self._check(_lib.gwam_graph_profile_read(self._h, ms.ctypes.data_as(_vp), C.byref(n)), "graph_profile_read")
        return dict(zip(self.PHASES, ms.tolist())), n.value

    def selftest_scan(self, in0, out0, n0, in1=None, out1=None, n1=0):
        """Exclusive scans of device int32 arrays by the step's scan kernels (pointers as ints)."""
        self._check(_lib.gwam_selftest_scan(self._h, _vp(in0), _vp(out0), int(n0), _vp(in1) if in1 else None,
                                            _vp(out1) if out1 else None, int(n1)), "selftest_scan")

    def graph_kernel_count(self):
        """Kernel launches per step-graph replay, counted from the captured graph."""
        n = C.c_int()
        self._check(_lib.gwam_graph_kernel_count(self._h, C.byref(n)), "graph_kernel_count")
        return n.value

    def synchronize(self):
        self._check(_lib.gwam_synchronize(self._h), "synchronize")


# ------------------------------------------------------------------ drag surrogate
def _stream_ptr():
    import torch
    return _vp(torch.cuda.current_stream().cuda_stream)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


class Surrogate:
    """The column drag surrogate (gwam_mlp_* in include/gwam.h).  Data sets and outputs are torch
    CUDA tensors; the stream is torch's current stream at construction."""

    def __init__(self, n_in=368, n_out=180, n_hidden=512, n_layers=4, nlev=90, max_batch=32768, seed=1,
                 beta1=0.9, beta2=0.999, eps=1e-8):
        self._h = _vp()
        cfg = MlpConfig(n_in=n_in, n_hidden=n_hidden, n_layers=n_layers, n_out=n_out, nlev=nlev,
                        max_batch=max_batch, seed=seed, beta1=beta1, beta2=beta2, eps=eps)
        self._stream = _stream_ptr()
        rc = _lib.gwam_mlp_create(C.byref(self._h), C.byref(cfg), self._stream)
        if rc != GWAM_OK:
            raise GwamError(rc, "gwam_mlp_create")
        self.n_in, self.n_out, self.n_hidden, self.n_layers, self.nlev = n_in, n_out, n_hidden, n_layers, nlev
        self.max_batch = max_batch
        self.dims = (n_in,) + (n_hidden,) * n_layers + (n_out,)

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.gwam_mlp_destroy(self._h)
            self._h = _vp()

    def _check(self, rc, what):
        if rc != GWAM_OK:
            raise GwamError(rc, "%s: %s" % (what, _lib.gwam_mlp_last_error(self._h).decode()))

    def set_normalization(self, x_mu, x_sigma, y_mu, y_sigma, lo, hi):
        arrs = [_f32(a) for a in (x_mu, x_sigma, y_mu, y_sigma, lo, hi)]
        self._check(_lib.gwam_mlp_set_normalization_host(self._h, *[a.ctypes.data_as(_vp) for a in arrs]),
                    "set_normalization")

    def fit_normalization(self, X, Y, margin=0.05):
        st = np.zeros(4 * self.n_in + 2 * self.n_out, dtype=np.float32)
        self._check(_lib.gwam_mlp_fit_normalization(self._h, _ptr(X), _ptr(Y), X.shape[0], float(margin),
                                                    st.ctypes.data_as(_vp)), "fit_normalization")
        ni, no = self.n_in, self.n_out
        return {"x_mu": st[:ni], "x_sigma": st[ni:2 * ni], "lo": st[2 * ni:3 * ni], "hi": st[3 * ni:4 * ni],
                "y_mu": st[4 * ni:4 * ni + no], "y_sigma": st[4 * ni + no:]}

    def set_params(self, params):
        for l, (W, b) in enumerate(params, start=1):
            W, b = _f32(W), _f32(b)
            self._check(_lib.gwam_mlp_set_params_host(self._h, l, W.ctypes.data_as(_vp), b.ctypes.data_as(_vp)),
                        "set_params")

    def _get(self, which):
        out = []
        for l in range(1, len(self.dims)):
            W = np.zeros((self.dims[l], self.dims[l - 1]), dtype=np.float32)
            b = np.zeros(self.dims[l], dtype=np.float32)
            self._check(_lib.gwam_mlp_get_params_host(self._h, l, which, W.ctypes.data_as(_vp),
                                                      b.ctypes.data_as(_vp)), "get_params")
            out.append((W, b))
        return out

    def params(self):
        return self._get(0)

    def grads(self):
        return self._get(1)

    def train_step(self, X, Y, batch, seed=0, lr=1e-3, rows=None):
        self._check(_lib.gwam_mlp_train_step(self._h, _ptr(X), _ptr(Y), X.shape[0],
                                             _ptr(rows) if rows is not None else None, int(batch), int(seed),
                                             float(lr)), "train_step")

    def loss(self) -> float:
        v = C.c_double()
        self._check(_lib.gwam_mlp_last_loss_host(self._h, C.byref(v)), "last_loss")
        return v.value

    def output(self, rows):
        out = np.zeros((rows, self.n_out), dtype=np.float32)
        self._check(_lib.gwam_mlp_output_host(self._h, out.ctypes.data_as(_vp), int(rows)), "output")
        return out

    def infer(self, X, dudt, dvdt, mask, n_fallback):
        """Drag of the in-envelope columns into dudt/dvdt ([nlev][ncol] float64 tensors); mask and
        n_fallback (int32 tensors) receive the fallback flags and their count.  Asynchronous."""
        self._check(_lib.gwam_mlp_infer(self._h, _ptr(X), X.shape[0], _ptr(dudt), _ptr(dvdt), _ptr(mask),
                                        _ptr(n_fallback)), "infer")

    def status(self):
        self._check(_lib.gwam_mlp_status(self._h), "status")

    def profile(self, enable=True):
        self._check(_lib.gwam_mlp_profile_enable(self._h, 1 if enable else 0), "profile_enable")

    def profile_read(self):
        ms = np.zeros(2)
        n = C.c_int64()
        self._check(_lib.gwam_mlp_profile_read(self._h, ms.ctypes.data_as(_vp), C.byref(n)), "profile_read")
        return {"pack_ms": ms[0], "gemm_ms": ms[1]}, n.value


def merge_fallback(mask, du_tracer, dv_tracer, dudt, dvdt):
    ncol = mask.shape[0]
    nlev = dudt.numel() // ncol
    rc = _lib.gwam_mlp_merge_fallback(_ptr(mask), ncol, nlev, _ptr(du_tracer), _ptr(dv_tracer), _ptr(dudt),
                                      _ptr(dvdt), _stream_ptr())
    if rc != GWAM_OK:
        raise GwamError(rc, "merge_fallback")


def column_features(u, v, n2, rho, src, out):
    """Features [ncol][4 nz + n_src] of [nz][ny][nx] float64 tensors; src: float32 tensor [n_src]
    (shared) or [ncol][n_src]."""
    nz = u.shape[0]
    ncol = u.numel() // nz
    n_src = src.shape[-1]
    stride = 0 if src.dim() == 1 else n_src
    rc = _lib.gwam_column_features(_ptr(u), _ptr(v), _ptr(n2), _ptr(rho), nz, ncol, _ptr(src), n_src, stride,
                                   _ptr(out), _stream_ptr())
    if rc != GWAM_OK:
        raise GwamError(rc, "column_features")


def column_targets(du_sum, dv_sum, scale, out):
    nz = du_sum.shape[0]
    ncol = du_sum.numel() // nz
    rc = _lib.gwam_column_targets(_ptr(du_sum), _ptr(dv_sum), nz, ncol, float(scale), _ptr(out), _stream_ptr())
    if rc != GWAM_OK:
        raise GwamError(rc, "column_targets")
