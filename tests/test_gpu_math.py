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
