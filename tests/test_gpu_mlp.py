"""The surrogate's training and inference kernels against the FP64 reference (oracle/mlp.py).

Both sides start from the same BF16-rounded weights and the same BF16-rounded normalised inputs
(the kernel's FP32 normalisation (x - mu) * (1/sigma) is reproduced in FP32 here), so the
remaining differences are the kernels' BF16 rounding of the hidden activations and of the
back-propagated gradients (unit roundoff 2^-9 ~ 2e-3 each, 4 activation and 5 gradient roundings)
and FP32 accumulation.  Derived bars (normwise relative): outputs 1e-2, gradients 3e-2 per
layer; the integer envelope decisions are bit-exact (same FP32 arithmetic on both sides); the
Adam update, given the same gradient, agrees to FP32 rounding."""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu

N_IN, N_OUT, NLEV = 368, 180, 90


@pytest.fixture(scope="module")
def gw():
    from paper_2309_11257_gb300 import build
    build.build()
    from paper_2309_11257_gb300 import gwam
    return gwam


def _bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).double().numpy()


def _data(n, seed):
    r = np.random.default_rng(seed)
    scales = np.concatenate([np.full(90, 20.0), np.full(90, 5.0), np.full(90, 1e-4), np.full(90, 2.0),
                             np.array([1e-3, 5e3, 1e5, 5.0, 50.0, 1e-3, 3.0, 1e-4])])
    offs = np.concatenate([np.zeros(90), np.zeros(90), np.full(90, 4e-4), -np.linspace(0, 12, 90),
                           np.array([8e-3, 5e3, 1e5, 5.0, 50.0, 2e-3, 2.0, 0.0])])
    X = (r.standard_normal((n, N_IN)) * scales + offs).astype(np.float32)
    Y = (r.standard_normal((n, N_OUT)) * 1e-4 + 2e-5).astype(np.float32)
    return X, Y


def _norm(X, Y):
    mu = X.mean(axis=0).astype(np.float32)
    sd = X.std(axis=0).astype(np.float32)
    ymu = Y.mean(axis=0).astype(np.float32)
    ysd = Y.std(axis=0).astype(np.float32)
    return mu, sd, ymu, ysd


def _xhat32(X, mu, sd):
    """The kernel's FP32 normalisation: (x - mu) * (1 / sigma), each operation rounded to FP32."""
    isd = (np.float32(1.0) / sd).astype(np.float32)
    return ((X - mu).astype(np.float32) * isd).astype(np.float32)


def _relnorm(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def setup(gw):
    import torch
    X, Y = _data(1000, 3)
    mu, sd, ymu, ysd = _norm(X, Y)
    lo, hi = np.full(N_IN, -50.0, np.float32), np.full(N_IN, 50.0, np.float32)
    S = gw.Surrogate(max_batch=256, seed=7)
    S.set_normalization(mu, sd, ymu, ysd, lo, hi)
    params = mlp.init_params(mlp.DIMS, seed=5)
    params = [(W.astype(np.float32), (0.05 * np.random.default_rng(l).standard_normal(len(b))).astype(np.float32))
              for l, (W, b) in enumerate(params)]
    S.set_params(params)
    rows = np.random.default_rng(9).choice(len(X), 256, replace=False).astype(np.int32)
    return dict(S=S, X=X, Y=Y, Xd=torch.from_numpy(X).cuda(), Yd=torch.from_numpy(Y).cuda(), mu=mu, sd=sd,
                ymu=ymu, ysd=ysd, lo=lo, hi=hi, params=params, rows=rows, rows_d=torch.from_numpy(rows).cuda())


def _reference(st):
    p64 = [(_bf16(W), b.astype(np.float64)) for W, b in st["params"]]
    Xn = _bf16(_xhat32(st["X"][st["rows"]], st["mu"], st["sd"]))
    Tn = _xhat32(st["Y"][st["rows"]], st["ymu"], st["ysd"]).astype(np.float64)
    Yo, cache = mlp.forward(p64, Xn)
    grads = mlp.backward(p64, cache, mlp.loss_grad(Yo, Tn))
    return Yo, mlp.loss(Yo, Tn), grads


def test_forward_loss_and_gradients(gw, setup):
    st = setup
    S = st["S"]
    S.train_step(st["Xd"], st["Yd"], 256, rows=st["rows_d"], lr=0.0)
    loss = S.loss()
    Yg = S.output(256).astype(np.float64)
    gr = S.grads()
    Yo, lo_, go = _reference(st)
    e_out, e_loss = _relnorm(Yg, Yo), abs(loss - lo_) / lo_
    e_w = [_relnorm(gr[l][0].astype(np.float64), go[l][0]) for l in range(5)]
    e_b = [_relnorm(gr[l][1].astype(np.float64), go[l][1]) for l in range(5)]
    print("\n[surrogate vs FP64] output %.2e loss %.2e dW %s db %s" % (
        e_out, e_loss, ["%.1e" % e for e in e_w], ["%.1e" % e for e in e_b]))
    assert e_out <= 1e-2 and e_loss <= 1e-2
    assert max(e_w) <= 3e-2 and max(e_b) <= 3e-2


def test_gradients_are_deterministic(gw, setup):
    st = setup
    S = st["S"]
    S.train_step(st["Xd"], st["Yd"], 256, rows=st["rows_d"], lr=0.0)
    g1 = S.grads()
    S.train_step(st["Xd"], st["Yd"], 256, rows=st["rows_d"], lr=0.0)
    g2 = S.grads()
    for a, b in zip(g1, g2):
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])


def test_adam_step_matches_reference_update(gw, setup):
    st = setup
    S = st["S"]
    S.set_params(st["params"])
    S.train_step(st["Xd"], st["Yd"], 256, rows=st["rows_d"], lr=0.0)
    g = S.grads()
    p0 = S.params()
    lr = 1e-3
    S.train_step(st["Xd"], st["Yd"], 256, rows=st["rows_d"], lr=lr)
    p1 = S.params()
    ref, _ = mlp.adam_step([(W.astype(np.float64), b.astype(np.float64)) for W, b in p0],
                           [(W.astype(np.float64), b.astype(np.float64)) for W, b in g],
                           mlp.adam_init(p0), 1, lr)
    for l in range(5):
        for q in (0, 1):
            d_gpu = p1[l][q].astype(np.float64) - p0[l][q]
            d_ref = ref[l][q] - p0[l][q]
            tol = 2e-6 * lr + 1e-7 * np.abs(p0[l][q])
            assert np.all(np.abs(d_gpu - d_ref) <= tol), (l, q, np.abs(d_gpu - d_ref).max())
    S.set_params(st["params"])


def test_training_reduces_loss(gw):
    """A learnable target (a fixed smooth function of the inputs): 300 Adam steps cut the loss."""
    import torch
    r = np.random.default_rng(4)
    n = 8192
    X = r.standard_normal((n, N_IN)).astype(np.float32)
    A = r.standard_normal((N_IN, N_OUT)) / np.sqrt(N_IN)
    Y = (np.tanh(X @ A) + 0.3 * (X[:, :N_OUT] ** 2)).astype(np.float32)
    S = gw.Surrogate(max_batch=1024, seed=3)
    mu, sd, ymu, ysd = _norm(X, Y)
    S.set_normalization(mu, sd, ymu, ysd, np.full(N_IN, -1e3, np.float32), np.full(N_IN, 1e3, np.float32))
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    S.train_step(Xd, Yd, 1024, seed=0, lr=0.0)
    l0 = S.loss()
    for it in range(300):
        S.train_step(Xd, Yd, 1024, seed=it + 1, lr=1e-3)
    l1 = S.loss()
    print("\n[training] loss %.4f -> %.4f" % (l0, l1))
    assert l1 < 0.3 * l0


def test_inference_envelope_and_fallback_routing(gw, setup):
    import torch
    st = setup
    S = st["S"]
    S.set_params(st["params"])
    ncol = 1000                      # not a multiple of the 128-row tile
    X = st["X"][:ncol].copy()
    r = np.random.default_rng(12)
    out_cols = r.choice(ncol, 37, replace=False)
    feats = r.integers(0, N_IN, size=37)
    lo = np.full(N_IN, -3.0, np.float32)
    hi = np.full(N_IN, 3.0, np.float32)
    for c, f in zip(out_cols, feats):   # push one feature of each chosen column outside the box
        X[c, f] = st["mu"][f] + (4.0 + r.uniform()) * st["sd"][f] * (1 if r.uniform() < 0.5 else -1)
    X[out_cols[0], 5] = np.nan
    S.set_normalization(st["mu"], st["sd"], st["ymu"], st["ysd"], lo, hi)
    Xd = torch.from_numpy(X).cuda()
    du = torch.full((NLEV, ncol), 7.5, dtype=torch.float64, device="cuda")
    dv = torch.full((NLEV, ncol), -7.5, dtype=torch.float64, device="cuda")
    mask = torch.full((ncol,), -1, dtype=torch.int32, device="cuda")
    nfb = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.infer(Xd, du, dv, mask, nfb)
    S.status()
    xh = _xhat32(X, st["mu"], st["sd"])
    ref_mask = mlp.envelope_mask(xh, lo, hi)
    m = mask.cpu().numpy()
    np.testing.assert_array_equal(m, ref_mask)
    assert int(nfb.item()) == int(ref_mask.sum()) >= 37
    p64 = [(_bf16(W), b.astype(np.float64)) for W, b in st["params"]]
    Yo, _ = mlp.forward(p64, _bf16(np.where(np.isfinite(xh), xh, 0)))
    drag = Yo * st["ysd"].astype(np.float64) + st["ymu"].astype(np.float64)
    dug, dvg = du.cpu().numpy(), dv.cpu().numpy()
    inside = m == 0
    e_u = _relnorm(dug[:, inside].T, drag[inside, :NLEV])
    e_v = _relnorm(dvg[:, inside].T, drag[inside, NLEV:])
    print("\n[inference vs FP64] du %.2e dv %.2e, fallback %d of %d" % (e_u, e_v, m.sum(), ncol))
    assert e_u <= 1e-2 and e_v <= 1e-2
    assert np.all(dug[:, ~inside] == 7.5) and np.all(dvg[:, ~inside] == -7.5)
    # routing: fallback columns take the ray tracer's values, the rest keep the surrogate's
    tu = torch.full_like(du, 1.25)
    tv = torch.full_like(dv, -1.25)
    gw.merge_fallback(mask, tu, tv, du, dv)
    dug2, dvg2 = du.cpu().numpy(), dv.cpu().numpy()
    assert np.all(dug2[:, ~inside] == 1.25) and np.all(dvg2[:, ~inside] == -1.25)
    np.testing.assert_array_equal(dug2[:, inside], dug[:, inside])
    S.set_normalization(st["mu"], st["sd"], st["ymu"], st["ysd"], st["lo"], st["hi"])


def test_bad_arguments(gw, setup):
    import torch
    st = setup
    S = st["S"]
    with pytest.raises(gw.GwamError):
        S.train_step(st["Xd"], st["Yd"], 100, lr=0.0)          # not a multiple of 64
    with pytest.raises(gw.GwamError):
        S.train_step(st["Xd"], st["Yd"], 512, lr=0.0)          # above max_batch
    bad = torch.full((256,), 5000, dtype=torch.int32, device="cuda")
    S.train_step(st["Xd"], st["Yd"], 256, rows=bad, lr=0.0)  # row outside the data set: device error
    with pytest.raises(gw.GwamError):
        S.loss()
