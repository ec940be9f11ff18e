"""The surrogate's tcgen05/TMA BF16 GEMM against FP64 products of the same BF16 values.

Products of BF16 numbers are exact in FP32; only the FP32 sums round, so every element must lie
within 2e-5 * S of the FP64 result, S = sum_k |a_ik b_jk| (K <= 512: the worst case K 2^-24 is
3e-5, the typical sqrt(K) 2^-24 is 1.3e-6).  A layout or descriptor mistake gives O(S) errors."""
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


def _gelu(z):
    from scipy.special import erf
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


CASES = [
    (128, 64, 64, 64, False, False),
    (300, 180, 384, 0, True, True),
    (256, 512, 512, 0, True, False),
    (1000, 256, 128, 256, True, True),
    (129, 40, 192, 64, False, True),
    (513, 192, 512, 192, True, False),
    (2048, 512, 512, 128, False, False),
]


@pytest.mark.parametrize("M,N,K,bn,bias,gelu", CASES)
def test_gemm_matches_fp64(gw, M, N, K, bn, bias, gelu):
    import torch
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = (torch.randn(N, K, generator=g) / 8).to(torch.bfloat16)
    b = torch.randn(N, generator=g).float() if bias else None
    Ad, Bd = A.cuda(), B.cuda()
    bd = b.cuda() if bias else None
    Cd = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream()
    rc = gw.lib().gwam_gemm_bf16(C.c_void_p(Ad.data_ptr()), C.c_void_p(Bd.data_ptr()), M, N, K,
                                 C.c_void_p(bd.data_ptr() if bias else 0), int(gelu), bn, 0,
                                 C.c_void_p(Cd.data_ptr()), C.c_void_p(s.cuda_stream))
    assert rc == 0
    a, bb = A.double().numpy(), B.double().numpy()
    z = a @ bb.T + (b.double().numpy() if bias else 0.0)
    S = np.abs(a) @ np.abs(bb).T
    ref = _gelu(z) if gelu else z
    got = Cd.cpu().double().numpy()
    err = np.abs(got - ref)
    assert np.isfinite(got).all()
    assert (err <= 2e-5 * S + 1e-6 * np.abs(ref)).all(), (err / (S + 1e-30)).max()


@pytest.mark.parametrize("M,N,K,bn,bias,gelu", CASES)
def test_gemm_bf16_output_through_tma_store(gw, M, N, K, bn, bias, gelu):
    """BF16 output (TMA stores from swizzled shared memory when N % 8 == 0): the FP32 result of the
    same kernel rounded to BF16, bit for bit."""
    import torch
    g = torch.Generator().manual_seed(M * 5 + N + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = (torch.randn(N, K, generator=g) / 8).to(torch.bfloat16).cuda()
    b = torch.randn(N, generator=g).float().cuda() if bias else None
    Cf = torch.empty((M, N), dtype=torch.float32, device="cuda")
    Cb = torch.full((M, N), float("nan"), dtype=torch.bfloat16, device="cuda")
    s = torch.cuda.current_stream()
    lib = gw.lib()
    args = (C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()), M, N, K, C.c_void_p(b.data_ptr() if bias else 0),
            int(gelu), bn)
    assert lib.gwam_gemm_bf16(*args, 0, C.c_void_p(Cf.data_ptr()), C.c_void_p(s.cuda_stream)) == 0
    assert lib.gwam_gemm_bf16(*args, 1, C.c_void_p(Cb.data_ptr()), C.c_void_p(s.cuda_stream)) == 0
    ref = Cf.to(torch.bfloat16)
    assert torch.equal(Cb.view(torch.int16), ref.view(torch.int16))


def test_gemm_rejects_bad_shapes(gw):
    import torch
    A = torch.zeros(128, 64, dtype=torch.bfloat16, device="cuda")
    Cd = torch.zeros(128, 64, device="cuda")
    lib = gw.lib()
    p = C.c_void_p(A.data_ptr())
    assert lib.gwam_gemm_bf16(p, p, 128, 64, 60, None, 0, 0, 0, C.c_void_p(Cd.data_ptr()), None) == -1
    assert lib.gwam_gemm_bf16(p, p, 128, 64, 64, None, 0, 96, 0, C.c_void_p(Cd.data_ptr()), None) == -1
    assert lib.gwam_gemm_bf16(p, p, 0, 64, 64, None, 0, 0, 0, C.c_void_p(Cd.data_ptr()), None) == -1


@pytest.mark.parametrize("bn", [64, 128, 192, 256])
def test_bounded_waits_give_up_and_the_context_stays_usable(gw, bn):
    """Failure detection of the library's spin-waits without a GPU fault: the GEMM's producer is
    told to issue no copies and every mbarrier wait is limited to 2 ms, so its MMA and epilogue warps
    wait on stages that never fill.  They give up, release their tensor memory and report: the call
    returns GWAM_ETIMEOUT within a fraction of a second.  The next GEMM of the same tile width (whose
    CTAs allocate the same tensor memory) and of another width then run to the correct result."""
    import time
    import torch
    M, N, K = 512, bn, 256
    g = torch.Generator().manual_seed(bn)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = (torch.randn(N, K, generator=g) / 8).to(torch.bfloat16)
    Ad, Bd = A.cuda(), B.cuda()
    Cd = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream()
    lib = gw.lib()
    t0 = time.perf_counter()
    rc = lib.gwam_selftest_gemm_timeout(C.c_void_p(Ad.data_ptr()), C.c_void_p(Bd.data_ptr()), M, N, K, bn,
                                        C.c_void_p(Cd.data_ptr()), 2000, C.c_void_p(s.cuda_stream))
    elapsed = time.perf_counter() - t0
    assert rc == gw.GWAM_ETIMEOUT
    assert elapsed < 1.0
    assert lib.gwam_selftest_gemm_timeout(None, None, M, N, K, bn, None, 2000, None) == gw.GWAM_EINVAL
    assert lib.gwam_selftest_gemm_timeout(C.c_void_p(Ad.data_ptr()), C.c_void_p(Bd.data_ptr()), M, N, K, bn,
                                          C.c_void_p(Cd.data_ptr()), 0, C.c_void_p(s.cuda_stream)) == gw.GWAM_EINVAL
    ref = A.double().numpy() @ B.double().numpy().T
    S = np.abs(A.double().numpy()) @ np.abs(B.double().numpy()).T
    for width in (bn, 64 if bn != 64 else 128):
        Cd.fill_(float("nan"))
        rc = lib.gwam_gemm_bf16(C.c_void_p(Ad.data_ptr()), C.c_void_p(Bd.data_ptr()), M, N, K, C.c_void_p(0), 0,
                                width, 0, C.c_void_p(Cd.data_ptr()), C.c_void_p(s.cuda_stream))
        assert rc == 0
        got = Cd.cpu().double().numpy()
        assert (np.abs(got - ref) <= 2e-5 * S + 1e-6 * np.abs(ref)).all()
    torch.cuda.synchronize()
    assert float(torch.ones(4, device="cuda").sum()) == 4.0     # the context answers
