"""The C-ABI library builds, loads without a GPU and exports every symbol include/gwam.h declares.
Argument checks that return before any CUDA call are exercised here too."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(gwam_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def gw():
    from paper_2309_11257_gb300 import build
    build.build()
    from paper_2309_11257_gb300 import gwam
    return gwam


def test_every_declared_symbol_is_exported(gw):
    declared = _declared()
    assert len(declared) >= 19
    lib = gw.lib()
    for name in sorted(declared):
        assert hasattr(lib, name), name
    # the binding wraps exactly the declared set
    assert set(gw.SIGNATURES) == declared


def test_version_string(gw):
    assert "sm_103a" in gw.version()


def test_init_rejects_bad_arguments_before_touching_the_device(gw):
    lib = gw.lib()
    h = C.c_void_p()
    grid = gw.Grid(geometry=1, nx=1, ny=8, nz=8, dz=1000.0, radius=6.4e6, g=9.8)
    params = gw.Params(precision=0, gamma_mode=1, alpha_s=2.5, min_split_dz=1000.0, max_rays=1000)
    assert lib.gwam_init(C.byref(h), C.byref(grid), C.byref(params), None) == gw.GWAM_EINVAL
    grid.nx = 8
    params.max_rays = 0
    assert lib.gwam_init(C.byref(h), C.byref(grid), C.byref(params), None) == gw.GWAM_EINVAL
    params.max_rays = 100
    params.flux_form = 3
    assert lib.gwam_init(C.byref(h), C.byref(grid), C.byref(params), None) == gw.GWAM_EINVAL
    assert lib.gwam_init(None, C.byref(grid), C.byref(params), None) == gw.GWAM_EINVAL
    assert not h.value
    # null context everywhere
    assert lib.gwam_step(None, 1.0, None, None) == gw.GWAM_EINVAL
    assert lib.gwam_synchronize(None) == gw.GWAM_EINVAL
    assert lib.gwam_last_error(None) == b"null context"


def test_struct_layouts_match_the_header(gw, tmp_path):
    """sizeof/offsetof of every POD struct as gcc lays out include/gwam.h, against the binding."""
    structs = {"gwam_grid": gw.Grid, "gwam_params": gw.Params, "gwam_bg_source": gw.BgSource,
               "gwam_spec": gw.Spec, "gwam_stats": gw.Stats, "gwam_ray_input": gw.RayInput,
               "gwam_mlp_config": gw.MlpConfig}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gwam.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(out[cname]) == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(out["%s.%s" % (cname, fname)]) == getattr(py, fname).offset, (cname, fname)


def test_surrogate_rejects_bad_configs_before_touching_the_device(gw):
    lib = gw.lib()
    h = C.c_void_p()
    good = dict(n_in=368, n_hidden=512, n_layers=4, n_out=180, nlev=90, max_batch=1024, seed=1, beta1=0.9,
                beta2=0.999, eps=1e-8)
    for bad in (dict(n_hidden=500), dict(max_batch=1000), dict(n_layers=0), dict(nlev=91), dict(beta1=1.0),
                dict(eps=0.0), dict(n_in=0)):
        cfg = gw.MlpConfig(**dict(good, **bad))
        assert lib.gwam_mlp_create(C.byref(h), C.byref(cfg), None) == gw.GWAM_EINVAL, bad
        assert not h.value
    assert lib.gwam_mlp_create(None, None, None) == gw.GWAM_EINVAL
    assert lib.gwam_mlp_train_step(None, None, None, 0, None, 64, 0, 0.0) == gw.GWAM_EINVAL
    assert lib.gwam_mlp_infer(None, None, 0, None, None, None, None) == gw.GWAM_EINVAL
    assert lib.gwam_mlp_merge_fallback(None, 0, 0, None, None, None, None, None) == gw.GWAM_EINVAL
    assert lib.gwam_gemm_bf16(None, None, 128, 64, 64, None, 0, 0, 0, None, None) == gw.GWAM_EINVAL
