"""gwam_cell_offsets_noalloc: the allocation-free entry point for callers that cannot allocate.

Host models that give all device memory to their own pool at start-up (or run under a fixed memory
budget) cannot let a library call cudaMalloc.  This checks, through the C ABI, that the
allocation-free entry point returns exactly what gwam_cell_offsets returns (integer results: bit
for bit), on two calls in a row with different inputs -- the second call must not see the first
call's scratch -- and that sizes beyond its fixed maximum are refused.  The file is named so that
pytest collects it last; it must pass alone in a fresh process and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw():
    from paper_2309_11257_gb300 import build
    build.build()
    from paper_2309_11257_gb300 import gwam
    return gwam


def _call(gw, name, cells, ncell, offsets, stream):
    fn = getattr(gw.lib(), name)
    return fn(C.c_void_p(cells.data_ptr()) if cells.numel() else None, cells.numel(), ncell,
              C.c_void_p(offsets.data_ptr()), C.c_void_p(stream.cuda_stream))


def test_noalloc_matches_allocating_entry_point_twice(gw):
    import torch
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(7)
    cases = [(np.sort(rng.integers(0, 2_949_120, 1_000_000)).astype(np.int32), 2_949_120),
             (np.sort(rng.integers(0, 4099, 12345)).astype(np.int32), 4099)]
    for cells_np, ncell in cases:       # two calls in a row, different sizes and contents
        cells = torch.from_numpy(cells_np).cuda()
        ref = torch.full((ncell + 1,), -7, dtype=torch.int32, device="cuda")
        got = torch.full((ncell + 1,), -7, dtype=torch.int32, device="cuda")
        assert _call(gw, "gwam_cell_offsets", cells, ncell, ref, stream) == gw.GWAM_OK
        assert _call(gw, "gwam_cell_offsets_noalloc", cells, ncell, got, stream) == gw.GWAM_OK
        torch.testing.assert_close(got, ref, rtol=0, atol=0)
        assert int(got[-1]) == len(cells_np)


def test_noalloc_reports_bad_cells_then_recovers(gw):
    import torch
    stream = torch.cuda.current_stream()
    bad = torch.tensor([0, 3, 99], dtype=torch.int32, device="cuda")
    out = torch.empty(11, dtype=torch.int32, device="cuda")
    assert _call(gw, "gwam_cell_offsets_noalloc", bad, 10, out, stream) == gw.GWAM_EINVAL
    good = torch.tensor([0, 3, 3, 9], dtype=torch.int32, device="cuda")
    assert _call(gw, "gwam_cell_offsets_noalloc", good, 10, out, stream) == gw.GWAM_OK   # flag cleared
    np.testing.assert_array_equal(out.cpu().numpy(), [0, 1, 1, 1, 3, 3, 3, 3, 3, 3, 4])


def test_noalloc_refuses_sizes_beyond_its_maximum(gw):
    import torch
    stream = torch.cuda.current_stream()
    cells = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    too_many = 16775168 + 1
    assert _call(gw, "gwam_cell_offsets_noalloc", cells, too_many, out, stream) == gw.GWAM_ECAPACITY
