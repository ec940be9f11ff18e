"""The surrogate trained on the ray tracer's drag at full size: 1 048 576 columns generated by the
FP64 tracer on 256 x 128 x 90 spheres (the sphere workload's jets and the batched ensemble's jet
distribution, background and convective sources), training with early stopping on validation
members, and an honest evaluation on held-out members (unseen jets, perturbations and sources):
the drag relative L2 against the stated bound, the envelope fallback, and the gain -- skill over
the training-mean baseline, and columns per second over the tracer's."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NLEV = 90
# stated bound on the held-out drag relative L2 (measured 0.66-0.68 on the held-out members; the
# training-mean baseline is 0.94): the convective spectra are drawn at random per column and are not
# among the features, so part of every column's drag cannot be predicted from them
DRAG_REL_L2_BOUND = 0.72


@pytest.fixture(scope="module")
def gw():
    from paper_2309_11257_gb300 import build
    build.build()
    from paper_2309_11257_gb300 import gwam
    return gwam


def test_surrogate_on_one_million_tracer_columns(gw):
    import torch
    from paper_2309_11257_gb300 import surrogate
    X, Y, infos = surrogate.generate_1m()
    assert X.shape == (1_048_576, 368) and Y.shape == (1_048_576, 180)
    assert torch.isfinite(X).all() and torch.isfinite(Y).all()
    assert float(Y.abs().max()) > 0.0
    ncol = infos[0]["ncol"]
    tr, va, te = surrogate.member_split(4, 8, ncol)
    Xtr, Ytr = X[tr].contiguous(), Y[tr].contiguous()
    Xva, Yva = X[va].contiguous(), Y[va].contiguous()
    Xte, Yte = X[te].contiguous(), Y[te].contiguous()
    assert Xtr.shape[0] == 26 * ncol and Xte.shape[0] == 4 * ncol
    S = gw.Surrogate(max_batch=32768, seed=1)
    S.fit_normalization(Xtr, Ytr, margin=0.05)
    best, step, hist = surrogate.train_early_stopping(S, Xtr, Ytr, Xva, Yva, NLEV, **surrogate.TRAIN_1M)
    te_err = surrogate.drag_error(S, Xte, Yte, NLEV)
    # baseline: the training-mean drag of every output, on the same in-envelope held-out columns
    mean = Ytr.double().mean(dim=0)
    mk = torch.zeros(Xte.shape[0], dtype=torch.int32, device="cuda")
    d0 = torch.zeros((NLEV, Xte.shape[0]), dtype=torch.float64, device="cuda")
    S.infer(Xte, d0, torch.zeros_like(d0), mk, torch.zeros(1, dtype=torch.int32, device="cuda"))
    ref = Yte.double()[mk == 0]
    base = float(torch.linalg.norm(ref - mean) / torch.linalg.norm(ref))
    # speed: surrogate inference over 32 768-column batches vs the tracer's step over its columns
    B = 32768
    Xb = Xte[:B].contiguous()
    du = torch.zeros((NLEV, B), dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(du)
    mask = torch.zeros(B, dtype=torch.int32, device="cuda")
    nfb = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(3):
        S.infer(Xb, du, dv, mask, nfb)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        S.infer(Xb, du, dv, mask, nfb)
    e1.record()
    e1.synchronize()
    sur_cps = B * 10 / (e0.elapsed_time(e1) * 1e-3)
    tr_cps = 8 * ncol / (infos[0]["tracer_ms_per_step"] * 1e-3)
    print("\n[surrogate] validation history %s" % [(a, round(b, 3), round(c, 3)) for a, b, c in hist])
    print("  kept weights of step %d (validation rel L2 %.3f); held-out rel L2 %.3f (baseline %.3f), "
          "fallback %d of %d held-out columns" % (step, best, te_err["rel_l2"], base, te_err["n_fallback"],
                                                   Xte.shape[0]))
    print("  columns/s: surrogate %.3e, tracer %.3e (x%.0f)" % (sur_cps, tr_cps, sur_cps / tr_cps))
    assert te_err["n_fallback"] <= 0.01 * Xte.shape[0]
    assert te_err["rel_l2"] <= DRAG_REL_L2_BOUND
    assert te_err["rel_l2"] < base - 0.2          # skill over the climatological baseline on unseen members
    assert sur_cps > 30 * tr_cps                   # far cheaper than the tracer per column
