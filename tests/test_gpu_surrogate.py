"""The surrogate trained on the ray tracer's drag: data generation, training, honest evaluation on
held-out ensemble members (unseen jets and perturbations), the envelope fallback, and the gain --
skill over the training-mean baseline, and columns per second over the tracer's."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NLEV = 90


@pytest.fixture(scope="module")
def gw():
    from paper_2309_11257_gb300 import build
    build.build()
    from paper_2309_11257_gb300 import gwam
    return gwam


def test_surrogate_gain_over_baseline_and_tracer(gw):
    import torch
    from paper_2309_11257_gb300 import surrogate
    X, Y, info = surrogate.generate(members=16, nx=64, ny=32, nz=NLEV, steps=120, avg=40, launch_every=5, tag=1)
    assert X.shape == (16 * 2048, 368) and Y.shape == (16 * 2048, 180)
    assert torch.isfinite(X).all() and torch.isfinite(Y).all()
    assert float(Y.abs().max()) > 0.0
    ncol = info["ncol"]
    ntr = 12 * ncol
    Xtr, Ytr, Xte, Yte = X[:ntr], Y[:ntr], X[ntr:], Y[ntr:]
    S = gw.Surrogate(max_batch=4096, seed=1)
    S.fit_normalization(Xtr, Ytr, margin=0.05)
    hist = surrogate.train(S, Xtr, Ytr, steps=800, batch=2048, lr=1e-3, log_every=200)
    tr = surrogate.drag_error(S, Xtr, Ytr, NLEV)
    te = surrogate.drag_error(S, Xte, Yte, NLEV)
    # baseline: the training-mean drag of every output, on the same in-envelope held-out columns
    mean = Ytr.double().mean(dim=0)
    mk = torch.zeros(Xte.shape[0], dtype=torch.int32, device="cuda")
    d0 = torch.zeros((NLEV, Xte.shape[0]), dtype=torch.float64, device="cuda")
    S.infer(Xte, d0, torch.zeros_like(d0), mk, torch.zeros(1, dtype=torch.int32, device="cuda"))
    ref = Yte.double()[mk == 0]
    base = float(torch.linalg.norm(ref - mean) / torch.linalg.norm(ref))
    # speed: surrogate inference over all columns vs the tracer's step over the same columns
    du = torch.zeros((NLEV, X.shape[0]), dtype=torch.float64, device="cuda")
    dv = torch.zeros_like(du)
    mask = torch.zeros(X.shape[0], dtype=torch.int32, device="cuda")
    nfb = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(3):
        S.infer(X, du, dv, mask, nfb)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        S.infer(X, du, dv, mask, nfb)
    e1.record()
    e1.synchronize()
    sur_cps = X.shape[0] * 10 / (e0.elapsed_time(e1) * 1e-3)
    tr_cps = X.shape[0] / (info["tracer_ms_per_step"] * 1e-3)
    print("\n[surrogate] loss history %s" % hist)
    print("  train rel L2 %.3f, held-out rel L2 %.3f (baseline %.3f), fallback %d of %d held-out columns"
          % (tr["rel_l2"], te["rel_l2"], base, te["n_fallback"], Xte.shape[0]))
    print("  columns/s: surrogate %.3e, tracer %.3e (x%.1f); rays %d" % (sur_cps, tr_cps, sur_cps / tr_cps,
                                                                       info["rays"]))
    assert te["n_inside"] > 0.5 * Xte.shape[0]
    assert te["rel_l2"] < base          # skill over the climatological baseline on unseen members
    assert tr["rel_l2"] < te["rel_l2"] + 0.5
    assert sur_cps > tr_cps             # cheaper than the tracer per column
