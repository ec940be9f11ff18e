"""The Newton-Raphson reciprocal and reciprocal square root used in place of FP64 division and
square root, against the GPU's IEEE results: within 2 ulp over the operand range of the path."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_rcp_and_rsqrt_within_two_ulp():
    import torch
    from paper_2309_11257_gb300 import build
    build.build()
    from paper_2309_11257_gb300 import gwam
    rng = np.random.default_rng(1)
    x = np.concatenate([10.0 ** rng.uniform(-30, 30, 200_000), rng.uniform(0.5, 2.0, 50_000),
                        [1.0, 2.0, 0.5, 3.0, 1e-300, 1e300]])
    xd = torch.from_numpy(x).cuda()
    r = torch.empty_like(xd)
    q = torch.empty_like(xd)
    s = torch.cuda.current_stream()
    rc = gwam.lib().gwam_selftest_math(C.c_void_p(xd.data_ptr()), len(x), C.c_void_p(r.data_ptr()),
                                       C.c_void_p(q.data_ptr()), C.c_void_p(s.cuda_stream))
    assert rc == 0
    ref_r = (1.0 / xd).cpu().numpy()
    ref_q = (1.0 / torch.sqrt(xd)).cpu().numpy()
    for got, ref in ((r.cpu().numpy(), ref_r), (q.cpu().numpy(), ref_q)):
        ulp = np.abs(got - ref) / np.spacing(np.abs(ref))
        assert np.all(np.isfinite(got))
        assert ulp.max() <= 2.0, ulp.max()


def test_integer_widening_and_double_float_action():
    """float -> double by integer re-biasing equals the hardware conversion bit for bit; the
    double-float product of four floats is within 2^-46 of the exact (FP64-evaluated) product."""
    import torch
    from paper_2309_11257_gb300 import build
    build.build()
    from paper_2309_11257_gb300 import gwam
    rng = np.random.default_rng(2)
    special = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45, 1.17549435e-38,
                        1.1754942e-38, 3.4028235e38, -3.4028235e38, 5.877472e-39, 2.0 ** -149, 2.0 ** -126],
                       dtype=np.float32)
    bits = rng.integers(0, 2 ** 32, size=200_000, dtype=np.uint64).astype(np.uint32).view(np.float32)
    mags = (10.0 ** rng.uniform(-30, 30, 100_000) * rng.choice([-1, 1], 100_000)).astype(np.float32)
    x = np.concatenate([special, bits, mags])
    xd = torch.from_numpy(x).cuda()
    w = torch.empty(len(x), dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    assert gwam.lib().gwam_selftest_widen(C.c_void_p(xd.data_ptr()), len(x), C.c_void_p(w.data_ptr()), None,
                                          C.c_void_p(s.cuda_stream)) == 0
    ref = xd.double().cpu().numpy().view(np.uint64)
    got = w.cpu().numpy().view(np.uint64)
    nan = np.isnan(x)
    np.testing.assert_array_equal(got[~nan], ref[~nan])
    assert np.isnan(w.cpu().numpy()[nan]).all()
    # double-float action on positive, moderate values (the ray-volume range)
    y = (10.0 ** rng.uniform(-7, 7, 50_000)).astype(np.float32)   # products stay normal in FP32
    yd = torch.from_numpy(y).cuda()
    w2 = torch.empty(len(y), dtype=torch.float64, device="cuda")
    a = torch.empty_like(w2)
    assert gwam.lib().gwam_selftest_widen(C.c_void_p(yd.data_ptr()), len(y), C.c_void_p(w2.data_ptr()),
                                          C.c_void_p(a.data_ptr()), C.c_void_p(s.cuda_stream)) == 0
    yy = y.astype(np.float64)
    n = len(y)
    idx = np.arange(n)
    exact = yy * yy[(idx + 1) % n] * yy[(idx + 2) % n] * yy[(idx + 3) % n]
    rel = np.abs(a.cpu().numpy() - exact) / exact
    assert rel.max() <= 2.0 ** -46, rel.max()


def test_integer_narrowing_matches_the_hardware_conversion():
    """double -> float by integer rounding (nearest even) equals the hardware conversion bit for
    bit: random bit patterns, the float range edges, subnormal results, ties, overflow."""
    import torch
    from paper_2309_11257_gb300 import build
    build.build()
    from paper_2309_11257_gb300 import gwam
    rng = np.random.default_rng(3)
    bits = rng.integers(0, 2 ** 63, size=300_000, dtype=np.uint64) | \
        (rng.integers(0, 2, size=300_000, dtype=np.uint64) << np.uint64(63))
    x = bits.view(np.float64)
    mags = 10.0 ** rng.uniform(-50, 45, 200_000) * rng.choice([-1, 1], 200_000)
    f32 = np.finfo(np.float32)
    special = np.array([0.0, -0.0, 1.0, np.inf, -np.inf, np.nan, float(f32.max), float(f32.max) * (1 + 2 ** -25),
                        float(f32.max) * (1 + 2 ** -23), float(f32.tiny), float(f32.tiny) / 3, 2.0 ** -149,
                        2.0 ** -150, 2.0 ** -150 * 1.0000001, 3 * 2.0 ** -151, 1.0 + 2 ** -24, 1.0 + 3 * 2 ** -24,
                        5e-324, -5e-324, 1e-320])
    # exact ties at every float exponent: 1 + 2^-24 scaled
    ties = (1.0 + 2.0 ** -24) * 2.0 ** rng.integers(-149, 127, 20_000).astype(np.float64)
    allx = np.concatenate([special, x, mags, ties])
    xd = torch.from_numpy(allx).cuda()
    out = torch.empty(len(allx), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream()
    assert gwam.lib().gwam_selftest_narrow(C.c_void_p(xd.data_ptr()), len(allx), C.c_void_p(out.data_ptr()),
                                           C.c_void_p(s.cuda_stream)) == 0
    ref = xd.float().cpu().numpy()
    got = out.cpu().numpy()
    nan = np.isnan(allx)
    np.testing.assert_array_equal(got[~nan].view(np.uint32), ref[~nan].view(np.uint32))
    assert np.isnan(got[nan]).all()


def test_double_float_split_is_exact():
    """The split x = hi + lo of the FP64 form: hi = RN32(x), lo = RN32(x - hi) bit for bit, over 100
    decades, at rounding ties (x = float + half an ulp, both ways of even), at the ends of the
    integer-only range (2^-74, 2^127) and outside it (tiny, subnormal, huge, zero, infinities)."""
    import torch
    from paper_2309_11257_gb300 import build
    build.build()
    from paper_2309_11257_gb300 import gwam
    rng = np.random.default_rng(12)
    h = rng.uniform(1.0, 2.0, 20_000).astype(np.float32).astype(np.float64)
    half_ulp = np.spacing(h.astype(np.float32)).astype(np.float64) / 2
    x = np.concatenate([rng.normal(size=200_000) * 10.0 ** rng.uniform(-50, 50, 200_000),
                        h + half_ulp, -(h + half_ulp), h - half_ulp / 2,
                        2.0 ** -74 * rng.uniform(1, 2, 1000), 2.0 ** 126 * rng.uniform(1, 1.9999, 1000),
                        2.0 ** rng.integers(-140, 140, 1000).astype(float),
                        np.array([0.0, -0.0, 5e-324, 1e-310, 1e300, -1e300, np.inf, -np.inf])])
    xd = torch.from_numpy(x).cuda()
    hi = torch.empty(len(x), dtype=torch.float32, device="cuda")
    lo = torch.empty_like(hi)
    s = torch.cuda.current_stream()
    assert gwam.lib().gwam_selftest_split(C.c_void_p(xd.data_ptr()), len(x), C.c_void_p(hi.data_ptr()),
                                          C.c_void_p(lo.data_ptr()), C.c_void_p(s.cuda_stream)) == 0
    with np.errstate(over="ignore", invalid="ignore"):
        rhi = x.astype(np.float32)
        rlo = (x - rhi.astype(np.float64)).astype(np.float32)
    ghi, glo = hi.cpu().numpy(), lo.cpu().numpy()
    fin = np.isfinite(rhi)
    np.testing.assert_array_equal(ghi.view(np.uint32), rhi.view(np.uint32))
    np.testing.assert_array_equal(glo[fin].view(np.uint32), rlo[fin].view(np.uint32))


def test_double_float_log_ratio():
    """ln(a/b) in double-float (atanh series after range reduction, as used for the Gamma^2
    differences) against numpy's FP64 logarithms: ratios across 70 decades, near 1, exactly 1 and
    at powers of two; relative error within 2^-44 (exactly 0 for a == b)."""
    import torch
    from paper_2309_11257_gb300 import build
    build.build()
    from paper_2309_11257_gb300 import gwam
    rng = np.random.default_rng(8)
    b = 10.0 ** rng.uniform(-30, 30, 200_000)
    r = np.concatenate([10.0 ** rng.uniform(-35, 35, 100_000), np.exp(rng.uniform(-0.5, 0.5, 80_000)),
                        1.0 + rng.uniform(-1e-9, 1e-9, 10_000), 2.0 ** rng.integers(-100, 100, 9_998).astype(float),
                        np.array([1.0, np.sqrt(2.0)])])
    a = b * r
    ad, bd = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    out = torch.empty(len(a), dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    assert gwam.lib().gwam_selftest_logratio(C.c_void_p(ad.data_ptr()), C.c_void_p(bd.data_ptr()), len(a),
                                             C.c_void_p(out.data_ptr()), C.c_void_p(s.cuda_stream)) == 0
    # FP64 reference: log1p of the exact difference over b near 1 (Sterbenz), log of the quotient
    # elsewhere; both within a few 2^-53 of |ln(a/b)|
    near = np.abs(a / b - 1.0) < 0.5
    with np.errstate(divide="ignore", invalid="ignore"):
        ref = np.where(near, np.log1p((a - b) / b), np.log(a / np.where(near, 1.0, b)))
    got = out.cpu().numpy()
    tol = 2.0 ** -44 * np.abs(ref)
    err = np.abs(got - ref)
    assert np.all(err <= tol), (err / tol).max()
