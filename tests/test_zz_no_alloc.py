"""gwam_cell_offsets_noalloc: the allocation-free entry point for callers that cannot allocate.

Host models that give all device memory to their own pool at start-up (or run under a fixed memory
budget) cannot let a library call cudaMalloc.  This checks, through the C ABI, that the
allocation-free entry point returns exactly what gwam_cell_offsets returns (integer results: bit
for bit), on two calls in a row with different inputs -- the second call must not see the first
call's scratch -- and that sizes beyond its fixed maximum are refused.  The file is named so that
pytest collects it last; it must pass alone in a fresh process and after the other tests.
"""
import ctypes as C
import ctypes.util
import glob
import os

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


def test_noalloc_works_at_its_maximum_size(gw):
    # at GWAM_NOALLOC_MAX_CELLS the scan's block sums fill the fixed array right up to the error flag:
    # an off-by-one in that arithmetic would overwrite the flag (a spurious GWAM_EINVAL) or the array
    import torch
    stream = torch.cuda.current_stream()
    ncell = 16775168
    rng = np.random.default_rng(11)
    cells_np = np.sort(np.concatenate([rng.integers(0, ncell, 5000), [0, ncell - 1, ncell - 1]])).astype(np.int32)
    cells = torch.from_numpy(cells_np).cuda()
    ref = torch.full((ncell + 1,), -7, dtype=torch.int32, device="cuda")
    got = torch.full((ncell + 1,), -7, dtype=torch.int32, device="cuda")
    assert _call(gw, "gwam_cell_offsets", cells, ncell, ref, stream) == gw.GWAM_OK
    assert _call(gw, "gwam_cell_offsets_noalloc", cells, ncell, got, stream) == gw.GWAM_OK
    torch.testing.assert_close(got, ref, rtol=0, atol=0)
    assert int(got[-1]) == len(cells_np) and int(got[ncell - 1]) == len(cells_np) - 2


def _cudart():
    """The CUDA runtime, to read the device's free memory and its default pool's counters."""
    cands = [ctypes.util.find_library("cudart")]
    cands += sorted(glob.glob("/usr/local/cuda/lib64/libcudart.so*"))
    try:
        import torch
        base = os.path.dirname(os.path.dirname(torch.__file__))
        cands += sorted(glob.glob(os.path.join(base, "nvidia", "cu*", "lib", "libcudart.so*")))
        cands += sorted(glob.glob(os.path.join(base, "nvidia", "cuda_runtime", "lib", "libcudart.so*")))
    except Exception:
        pass
    for c in cands:
        if not c:
            continue
        try:
            return C.CDLL(c)
        except OSError:
            continue
    pytest.skip("libcudart not found")


_USED_HIGH, _RESERVED_HIGH, _USED_CUR, _RESERVED_CUR = 8, 6, 7, 5   # cudaMemPoolAttr values


class _MemProbe:
    """Free device memory (cudaMemGetInfo) and the high-water marks of the device's default
    stream-ordered pool, which any cudaMallocAsync inside a call would raise."""

    def __init__(self, dev):
        self.rt = _cudart()
        self.pool = C.c_void_p()
        assert self.rt.cudaDeviceGetDefaultMemPool(C.byref(self.pool), C.c_int(dev)) == 0

    def _attr(self, a):
        v = C.c_uint64()
        assert self.rt.cudaMemPoolGetAttribute(self.pool, C.c_int(a), C.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = C.c_uint64(0)
        for a in (_USED_HIGH, _RESERVED_HIGH):   # setting 0 resets a high-water mark to the current value
            assert self.rt.cudaMemPoolSetAttribute(self.pool, C.c_int(a), C.byref(zero)) == 0

    def free(self):
        f, t = C.c_size_t(), C.c_size_t()
        assert self.rt.cudaMemGetInfo(C.byref(f), C.byref(t)) == 0
        return f.value

    def snapshot(self):
        return dict(free=self.free(), used=self._attr(_USED_CUR), reserved=self._attr(_RESERVED_CUR),
                    used_high=self._attr(_USED_HIGH), reserved_high=self._attr(_RESERVED_HIGH))


def test_noalloc_allocates_nothing(gw):
    # the promise the entry point exists for: several calls of different sizes leave the device's free
    # memory and the default pool's used/reserved high-water marks where they were
    import torch
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(5)
    cases = []
    for ncell, n in ((2_949_120, 300_000), (777, 5000), (16775168, 1000), (1, 0)):
        cells = torch.from_numpy(np.sort(rng.integers(0, ncell, n)).astype(np.int32)).cuda()
        cases.append((cells, ncell, torch.empty(ncell + 1, dtype=torch.int32, device="cuda")))
    for cells, ncell, out in cases:             # warm-up: modules loaded, scratch address looked up
        assert _call(gw, "gwam_cell_offsets_noalloc", cells, ncell, out, stream) == gw.GWAM_OK
    torch.cuda.synchronize()
    probe = _MemProbe(torch.cuda.current_device())
    probe.reset_high()
    before = probe.snapshot()
    for _ in range(2):
        for cells, ncell, out in cases:
            assert _call(gw, "gwam_cell_offsets_noalloc", cells, ncell, out, stream) == gw.GWAM_OK
    torch.cuda.synchronize()
    after = probe.snapshot()
    assert after["free"] == before["free"], (before, after)
    assert after["used_high"] <= before["used"] and after["reserved_high"] <= before["reserved"], (before, after)
    # the probe sees a stream-ordered allocation: the allocating entry point raises the used mark
    probe.reset_high()
    base = probe.snapshot()
    cells, ncell, out = cases[0]
    assert _call(gw, "gwam_cell_offsets", cells, ncell, out, stream) == gw.GWAM_OK
    torch.cuda.synchronize()
    assert probe.snapshot()["used_high"] > base["used"]
