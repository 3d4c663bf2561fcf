"""Plain FP64 reference of the learned pre-screen: an MLP surrogate of one
benchmark function, its training step and the top-k screen.

TEST INFRASTRUCTURE ONLY: like the rest of ``oracle/`` this module is what the
GPU library is checked against; only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code
with the CUDA library.

The paper has no learned part; the model below is this project's definition of
it, and each function states the published method it follows.

Model.  u = x / 128 (exact in every binary format); then
    a1 = W1 u + b1,  h1 = gelu(a1)          W1: 256 x 100
    a2 = W2 h1 + b2, h2 = gelu(a2)          W2: 256 x 256
    y  = w3 . h2 + b3                       w3: 256
with gelu(a) = a Phi(a), Phi the standard normal CDF (Hendrycks and Gimpel,
"Gaussian Error Linear Units", 2016, the exact form, not its tanh fit).  y predicts the
standardised target (t - mu) / sd with t = log(f - f_opt + 1), mu and sd the
mean and standard deviation of t over the training set.  Loss: mean squared
error over the batch.  Optimiser: AdamW (Loshchilov and Hutter, "Decoupled
Weight Decay Regularization", 2019), decay applied as w <- w (1 - lr wd)
before the Adam step, bias-corrected moments, eps added to sqrt(v_hat).

BF16 storage.  The GPU contracts BF16 operands with FP32 accumulation: the
weights W1, W2, w3 are BF16 copies of FP32 masters; u and h1 are BF16 where
they enter a contraction, and so are the back-propagated delta2 and delta1
where they enter one.  With ``bf16_points=True`` the functions here round at
those points (to nearest, ties to even) and do everything else in FP64;
biases and the bias gradients stay unrounded.

Pins (tests/test_oracle_surrogate.py): forward and gradients equal PyTorch's
float64 modules and autograd (bf16=False), gradients equal central finite
differences, AdamW equals torch.optim.AdamW over several steps, the BF16
rounding equals PyTorch's float32 -> bfloat16 conversion, the selection equals
a full sort, Spearman's rho equals scipy.stats.spearmanr.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

D_IN = 100
H = 256
U_SCALE = 1.0 / 128.0


# --------------------------------------------------------------------- BF16
def bf16(a):
    """Round to the nearest BF16 value (8 significant bits), ties to even.
    Inputs are FP64 arrays; the result is FP64 holding BF16 values."""
    a = np.asarray(a, dtype=np.float64)
    m, e = np.frexp(a)                       # a = m 2^e, 0.5 <= |m| < 1
    r = np.round(m * 256.0) / 256.0          # np.round: half to even
    return np.ldexp(r, e)


# --------------------------------------------------------------------- GELU
def Phi(a):
    """Standard normal CDF, erfc(-a / sqrt 2) / 2 (no cancellation for a < 0)."""
    return 0.5 * erfc(-np.asarray(a, dtype=np.float64) / math.sqrt(2.0))


def gelu(a):
    """a Phi(a)."""
    return a * Phi(a)


def gelu_grad(a):
    """d/da [a Phi(a)] = Phi(a) + a phi(a), phi the standard normal density."""
    return Phi(a) + a * np.exp(-0.5 * a * a) / math.sqrt(2.0 * math.pi)


# ------------------------------------------------------------------- target
def target(f, f_opt=100.0):
    """t = log(f - f_opt + 1); f >= f_opt for every benchmark function, and a
    value a rounding below f_opt is taken as f_opt."""
    return np.log1p(np.maximum(np.asarray(f, dtype=np.float64) - f_opt, 0.0))


def standardise(t):
    """mean and (population) standard deviation of the training targets."""
    t = np.asarray(t, dtype=np.float64)
    mu = t.mean()
    sd = math.sqrt(((t - mu) ** 2).mean())
    return mu, sd


# ------------------------------------------------------------------ network
def _weights(p, bf):
    r = bf16 if bf else (lambda v: np.asarray(v, dtype=np.float64))
    return r(p["W1"]), r(p["W2"]), r(p["w3"])


def forward(p, x, bf16_points=False):
    """Forward pass on candidates x (n x 100); returns the intermediates."""
    W1, W2, w3 = _weights(p, bf16_points)
    u = np.asarray(x, dtype=np.float64) * U_SCALE
    if bf16_points:
        u = bf16(u)
    a1 = u @ W1.T + p["b1"]
    h1 = gelu(a1)
    h1c = bf16(h1) if bf16_points else h1          # operand of the second layer
    a2 = h1c @ W2.T + p["b2"]
    h2 = gelu(a2)
    y = h2 @ w3 + float(p["b3"])
    return {"u": u, "a1": a1, "h1": h1c, "a2": a2, "h2": h2, "y": y}


def loss_and_grads(p, x, ts, bf16_points=False):
    """Mean squared error against standardised targets ts and its gradient
    with respect to every parameter (back-propagation written out)."""
    W1, W2, w3 = _weights(p, bf16_points)
    fw = forward(p, x, bf16_points)
    n = len(ts)
    r = fw["y"] - np.asarray(ts, dtype=np.float64)
    loss = float((r * r).mean())
    d3 = 2.0 * r / n                                    # dL/dy
    d2 = d3[:, None] * w3[None, :] * gelu_grad(fw["a2"])  # dL/da2
    d2c = bf16(d2) if bf16_points else d2
    d1 = (d2c @ W2) * gelu_grad(fw["a1"])              # dL/da1
    d1c = bf16(d1) if bf16_points else d1
    g = {
        "W1": d1c.T @ fw["u"],
        "b1": d1.sum(axis=0),
        "W2": d2c.T @ fw["h1"],
        "b2": d2.sum(axis=0),
        "w3": fw["h2"].T @ d3,
        "b3": float(d3.sum()),
    }
    return loss, g


def init_state():
    return {"t": 0, "m": {}, "v": {}}


def adamw_step(p, g, state, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=1e-4):
    """One AdamW step on every parameter, in place on copies; returns the new
    parameters.  Decoupled decay first, then the bias-corrected Adam step."""
    state["t"] += 1
    t = state["t"]
    out = {}
    for k, w in p.items():
        w = np.asarray(w, dtype=np.float64)
        gk = np.asarray(g[k], dtype=np.float64)
        m = state["m"].get(k, np.zeros_like(w))
        v = state["v"].get(k, np.zeros_like(w))
        m = beta1 * m + (1.0 - beta1) * gk
        v = beta2 * v + (1.0 - beta2) * gk * gk
        state["m"][k], state["v"][k] = m, v
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        w = w * (1.0 - lr * wd)
        out[k] = w - lr * mhat / (np.sqrt(vhat) + eps)
    return out


# ------------------------------------------------------------------- screen
def select_smallest(v, k):
    """Indices of the k smallest values of v, equal values taken in index
    order; returned in ascending index order."""
    v = np.asarray(v)
    order = np.lexsort((np.arange(len(v)), v))
    return np.sort(order[:k])


def ranks(a):
    """1-based ranks, tied values sharing the mean of their ranks."""
    a = np.asarray(a, dtype=np.float64)
    n = len(a)
    order = np.argsort(a, kind="stable")
    sa = a[order]
    starts = np.r_[0, np.flatnonzero(sa[1:] != sa[:-1]) + 1]
    ends = np.r_[starts[1:], n] - 1
    mean_rank = 0.5 * (starts + ends) + 1.0
    r = np.empty(n)
    r[order] = np.repeat(mean_rank, ends - starts + 1)
    return r


def spearman(a, b):
    """Spearman's rank correlation: Pearson's correlation of the ranks."""
    ra, rb = ranks(a), ranks(b)
    ra -= ra.mean()
    rb -= rb.mean()
    return float((ra @ rb) / math.sqrt((ra @ ra) * (rb @ rb)))


def regret(f_selected, f_pool):
    """Best exact value among the screened candidates minus the best in the
    whole pool (0 when the screen keeps the pool's best)."""
    return float(np.min(f_selected) - np.min(f_pool))
