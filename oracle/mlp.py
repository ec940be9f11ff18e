"""FP64 CPU reference of the column drag surrogate -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline/reference leg may import this
module; the product path never does.

The surrogate is not part of the paper: it is a multilayer perceptron that maps the features of
one model column (u, v, N^2, ln rho on the column's levels plus the source parameters) to the
column's wave drag (du/dt, dv/dt on the levels), trained on drag computed by the ray tracer.  What
it computes is fixed by textbook definitions, written out here one operation at a time in FP64:
  * dense layers z = W a + b, W of shape [n_out, n_in] (row i holds the weights of output i);
  * GELU(z) = z * Phi(z), Phi the standard normal CDF (Hendrycks & Gimpel 2016), on every hidden
    layer, none on the output layer;
  * loss L = mean over batch rows and the n_out true outputs of (y - t)^2 (t the normalised target);
  * backpropagation of L by the chain rule;
  * Adam (Kingma & Ba 2015, Algorithm 1): m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
    w <- w - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps);
  * feature normalisation x_hat = (x - mu) / sigma and the envelope test lo <= x_hat <= hi on every
    feature (a column outside it goes to the ray tracer).
"""
import math

import numpy as np
from scipy.special import erf

DIMS = (368, 512, 512, 512, 512, 180)
SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def gelu(z):
    """GELU(z) = z Phi(z) with Phi(z) = (1 + erf(z / sqrt 2)) / 2."""
    return 0.5 * z * (1.0 + erf(z / SQRT2))


def gelu_grad(z):
    """d GELU / dz = Phi(z) + z phi(z), phi the standard normal density."""
    return 0.5 * (1.0 + erf(z / SQRT2)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


def init_params(dims, seed):
    """Seeded initial weights: W ~ N(0, 1/n_in), b = 0 (FP64 lists of (W, b))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for n_in, n_out in zip(dims[:-1], dims[1:]):
        out.append((rng.standard_normal((n_out, n_in)) / math.sqrt(n_in), np.zeros(n_out)))
    return out


def forward(params, X):
    """Y = W_L a_{L-1} + b_L with a_l = GELU(W_l a_{l-1} + b_l), a_0 = X (rows are columns).
    Returns Y and the cache (inputs of every layer, pre-activations of the hidden layers)."""
    a = np.asarray(X, dtype=np.float64)
    acts, zs = [a], []
    for li, (W, b) in enumerate(params):
        z = a @ W.T + b
        if li < len(params) - 1:
            zs.append(z)
            a = gelu(z)
            acts.append(a)
        else:
            return z, (acts, zs)


def loss(Y, T):
    """Mean squared error over all rows and outputs."""
    d = Y - T
    return float(np.mean(d * d))


def loss_grad(Y, T):
    """dL/dY of the mean squared error."""
    return 2.0 * (Y - T) / Y.size


def backward(params, cache, dY):
    """Gradients (dW, db) of every layer given dL/dY, by the chain rule from the output back."""
    acts, zs = cache
    grads = [None] * len(params)
    d = dY
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        grads[li] = (d.T @ acts[li], d.sum(axis=0))
        if li > 0:
            d = (d @ W) * gelu_grad(zs[li - 1])
    return grads


def adam_init(params):
    return [(np.zeros_like(W), np.zeros_like(W), np.zeros_like(b), np.zeros_like(b)) for W, b in params]


def adam_step(params, grads, state, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns new params and state."""
    new_p, new_s = [], []
    c1, c2 = 1.0 - b1 ** t, 1.0 - b2 ** t
    for (W, b), (gW, gb), (mW, vW, mb, vb) in zip(params, grads, state):
        out = []
        for w, g, m, v in ((W, gW, mW, vW), (b, gb, mb, vb)):
            m = b1 * m + (1.0 - b1) * g
            v = b2 * v + (1.0 - b2) * g * g
            w = w - lr * (m / c1) / (np.sqrt(v / c2) + eps)
            out.append((w, m, v))
        (W2, mW2, vW2), (b2_, mb2, vb2) = out
        new_p.append((W2, b2_))
        new_s.append((mW2, vW2, mb2, vb2))
    return new_p, new_s


def normalize(X, mu, sigma):
    return (np.asarray(X, dtype=np.float64) - mu) / sigma


def column_stats(X):
    """Per-feature mean and standard deviation (population); a constant feature gets sigma = 1."""
    X = np.asarray(X, dtype=np.float64)
    mu = X.mean(axis=0)
    sd = X.std(axis=0)
    return mu, np.where(sd > 0, sd, 1.0)


def envelope_mask(Xn, lo, hi):
    """1 for rows with some feature outside the closed box [lo, hi] or not finite (fallback to the
    ray tracer), else 0."""
    Xn = np.asarray(Xn, dtype=np.float64)
    return np.any(~((Xn >= lo) & (Xn <= hi)), axis=1).astype(np.int32)
