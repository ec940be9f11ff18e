"""The step's exclusive scans (re-binning offsets, App. B.2 parent-cell storage) against numpy:
exclusive prefix sums with the total at out[n], for sizes across the part and tile boundaries
(empty, one item, ragged tails), 16-byte-aligned and unaligned arrays (the vector and the scalar
path), in place and out of place, one scan or two independent scans in the same launches, in a
context with few parts (small grid) and one with two parts per SM."""
import numpy as np
import pytest

from paper_2309_11257_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [0, 1, 3, 31, 1023, 1024, 1025, 4101, 65537, 1_000_003]


@pytest.fixture(scope="module")
def gw():
    from paper_2309_11257_gb300 import build
    build.build()
    from paper_2309_11257_gb300 import gwam
    return gwam


def _context(gw, kind):
    if kind == "small":
        grid = synth.fplane_grid(nx=4, ny=4, nz=8)
        return gw.Tracer(grid, dict(synth.DEFAULT_PARAMS), max_rays=512)
    grid = synth.sphere_grid(nx=64, ny=32, nz=90)
    return gw.Tracer(grid, dict(synth.DEFAULT_PARAMS), max_rays=200_000)


def _buffers(torch, vals, off, in_place):
    n = len(vals)
    src = torch.zeros(n + 2 + off, dtype=torch.int32, device="cuda")
    src[off:off + n] = torch.from_numpy(vals)
    if in_place:
        return src[off:], src[off:]
    dst = torch.full((n + 2 + off,), -7, dtype=torch.int32, device="cuda")
    return src[off:], dst[off:]


def _expect(vals):
    return np.concatenate([[0], np.cumsum(vals.astype(np.int64))])


@pytest.mark.parametrize("kind", ["small", "sphere"])
def test_single_scans_match_numpy(gw, kind):
    import torch
    T = _context(gw, kind)
    g = synth.rng(61)
    for n in SIZES:
        for off in (0, 1):
            for in_place in (False, True):
                vals = g.integers(0, 6, n).astype(np.int32)
                src, dst = _buffers(torch, vals, off, in_place)
                T.selftest_scan(src.data_ptr(), dst.data_ptr(), n)
                got = dst[:n + 1].cpu().numpy().astype(np.int64)
                np.testing.assert_array_equal(got, _expect(vals), err_msg="n=%d off=%d in_place=%s" % (n, off, in_place))
    T.close()


@pytest.mark.parametrize("kind", ["small", "sphere"])
def test_paired_scans_match_numpy(gw, kind):
    import torch
    T = _context(gw, kind)
    g = synth.rng(62)
    pairs = [(0, 5), (1, 1), (1025, 3), (65537, 1_000_003), (1_000_003, 4101)]
    for n0, n1 in pairs:
        for off in (0, 1):
            v0 = g.integers(0, 4, n0).astype(np.int32)
            v1 = g.integers(0, 9, n1).astype(np.int32)
            s0, d0 = _buffers(torch, v0, off, True)       # the step scans its first array in place
            s1, d1 = _buffers(torch, v1, 0, False)
            T.selftest_scan(s0.data_ptr(), d0.data_ptr(), n0, s1.data_ptr(), d1.data_ptr(), n1)
            np.testing.assert_array_equal(d0[:n0 + 1].cpu().numpy().astype(np.int64), _expect(v0))
            np.testing.assert_array_equal(d1[:n1 + 1].cpu().numpy().astype(np.int64), _expect(v1))
            # the second array's input is untouched when scanned out of place
            np.testing.assert_array_equal(s1[:n1].cpu().numpy(), v1)
    T.close()


def test_scan_arguments_are_checked(gw):
    import torch
    T = _context(gw, "small")
    buf = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(RuntimeError):
        T.selftest_scan(buf.data_ptr(), buf.data_ptr(), -1)
    with pytest.raises(RuntimeError):
        T.selftest_scan(buf.data_ptr(), 0, 4)
    T.close()
