"""Pins for the oracle of the learned pre-screen (oracle/surrogate.py).

The forward pass, the back-propagated gradients and the AdamW step are checked
against PyTorch's float64 modules, autograd and torch.optim.AdamW (library
routines that implement the same published definitions), and the gradients
also against central finite differences; the BF16 rounding against PyTorch's
bfloat16 conversion; the selection against a full sort; Spearman's rho
against scipy.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import surrogate as S  # noqa: E402


def params(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.normal(0, scale / math.sqrt(100), (256, 100)),
        "b1": rng.normal(0, 0.1, 256),
        "W2": rng.normal(0, scale / math.sqrt(256), (256, 256)),
        "b2": rng.normal(0, 0.1, 256),
        "w3": rng.normal(0, 1 / math.sqrt(256), 256),
        "b3": 0.3,
    }


def torch_model(p):
    import torch.nn as nn
    net = nn.Sequential(nn.Linear(100, 256), nn.GELU(), nn.Linear(256, 256), nn.GELU(),
                        nn.Linear(256, 1)).double()
    with torch.no_grad():
        net[0].weight.copy_(torch.from_numpy(p["W1"]))
        net[0].bias.copy_(torch.from_numpy(p["b1"]))
        net[2].weight.copy_(torch.from_numpy(p["W2"]))
        net[2].bias.copy_(torch.from_numpy(p["b2"]))
        net[4].weight.copy_(torch.from_numpy(p["w3"][None, :]))
        net[4].bias.fill_(p["b3"])
    return net


def batch(n=64, seed=1):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-100, 100, (n, 100))
    ts = rng.normal(0, 1, n)
    return x, ts


def test_gelu_matches_normal_cdf_and_its_derivative():
    from scipy.stats import norm
    a = np.linspace(-8, 8, 801)
    assert np.allclose(S.gelu(a), a * norm.cdf(a), rtol=1e-13, atol=1e-300)
    h = 1e-6
    fd = (S.gelu(a + h) - S.gelu(a - h)) / (2 * h)
    assert np.max(np.abs(fd - S.gelu_grad(a))) < 1e-8
    assert S.gelu(0.0) == 0.0 and abs(S.gelu_grad(0.0) - 0.5) < 1e-16


def test_forward_equals_torch():
    p = params()
    x, _ = batch()
    y = S.forward(p, x)["y"]
    ref = torch_model(p)(torch.from_numpy(x / 128.0)).detach().numpy()[:, 0]
    assert np.allclose(y, ref, rtol=1e-12, atol=1e-12)


def test_gradients_equal_autograd():
    p = params()
    x, ts = batch()
    loss, g = S.loss_and_grads(p, x, ts)
    net = torch_model(p)
    out = net(torch.from_numpy(x / 128.0))[:, 0]
    lt = ((out - torch.from_numpy(ts)) ** 2).mean()
    lt.backward()
    assert abs(loss - lt.item()) < 1e-12 * max(1, abs(loss))
    ref = {"W1": net[0].weight.grad, "b1": net[0].bias.grad, "W2": net[2].weight.grad,
           "b2": net[2].bias.grad, "w3": net[4].weight.grad[0], "b3": net[4].bias.grad[0]}
    for k, t in ref.items():
        assert np.allclose(g[k], t.numpy(), rtol=1e-10, atol=1e-14), k


@pytest.mark.parametrize("key,idx", [("W1", (3, 7)), ("W1", (200, 99)), ("b1", (11,)),
                                     ("W2", (0, 255)), ("W2", (128, 5)), ("b2", (77,)),
                                     ("w3", (9,)), ("b3", None)])
def test_gradients_equal_finite_differences(key, idx):
    p = params(scale=2.0)
    x, ts = batch(32, 5)
    _, g = S.loss_and_grads(p, x, ts)
    h = 1e-6
    q = {k: (np.array(v, copy=True) if k != "b3" else v) for k, v in p.items()}

    def L(delta):
        r = {k: (np.array(v, copy=True) if k != "b3" else v) for k, v in q.items()}
        if key == "b3":
            r["b3"] = q["b3"] + delta
        else:
            r[key][idx] += delta
        return S.loss_and_grads(r, x, ts)[0]

    fd = (L(h) - L(-h)) / (2 * h)
    an = g[key] if key == "b3" else g[key][idx]
    assert abs(fd - an) <= 1e-6 * max(1e-3, abs(an)), (fd, an)


def test_adamw_equals_torch_over_steps():
    p = params()
    x, ts = batch()
    tp = {k: torch.tensor(np.array(v, dtype=np.float64), requires_grad=True) for k, v in p.items()}
    opt = torch.optim.AdamW(list(tp.values()), lr=3e-3, betas=(0.9, 0.999), eps=1e-8,
                            weight_decay=1e-2)
    st = S.init_state()
    cur = {k: np.array(v, dtype=np.float64) for k, v in p.items()}
    rng = np.random.default_rng(3)
    for step in range(4):
        g = {k: rng.normal(0, 10 ** rng.uniform(-6, 0), np.shape(v)) for k, v in cur.items()}
        for k, t in tp.items():
            t.grad = torch.from_numpy(np.array(g[k], dtype=np.float64))
        opt.step()
        cur = S.adamw_step(cur, g, st, lr=3e-3, wd=1e-2)
        for k, t in tp.items():
            assert np.allclose(cur[k], t.detach().numpy(), rtol=1e-13, atol=1e-16), (step, k)


def test_bf16_rounding_equals_torch():
    rng = np.random.default_rng(4)
    v = np.concatenate([rng.normal(0, 1, 4000) * 10.0 ** rng.integers(-8, 8, 4000),
                        [0.0, 1.0, -1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -9,
                         -(1 + 2.0 ** -8), 255.5, 256.5]]).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    got = S.bf16(v.astype(np.float64))
    assert np.array_equal(got, ref)
    # ties to even: 1 + 2^-8 sits half-way between 1 and 1 + 2^-7
    assert S.bf16(1 + 2.0 ** -8) == 1.0 and S.bf16(1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6


def test_bf16_points_change_little_and_only_where_stated():
    p = params()
    x, ts = batch()
    exact = S.forward(p, x)
    q = S.forward(p, x, bf16_points=True)
    assert np.max(np.abs(exact["y"] - q["y"])) < 0.05
    assert np.array_equal(q["u"], S.bf16(x / 128.0))
    assert np.array_equal(q["h1"], S.bf16(q["h1"]))


def test_selection_equals_sort_with_ties():
    rng = np.random.default_rng(6)
    v = rng.integers(0, 50, 10_000).astype(np.float32)   # many ties
    for k in (0, 1, 137, 5000, 10_000):
        got = S.select_smallest(v, k)
        order = sorted(range(len(v)), key=lambda i: (v[i], i))[:k]
        assert np.array_equal(got, np.sort(np.array(order, dtype=np.int64)))


def test_spearman_equals_scipy():
    from scipy.stats import spearmanr
    rng = np.random.default_rng(7)
    a = rng.normal(size=5000)
    b = a + rng.normal(size=5000)
    b[::10] = b[5]  # ties
    assert abs(S.spearman(a, b) - spearmanr(a, b).statistic) < 1e-12
    assert S.spearman(a, 3 * a + 1) == pytest.approx(1.0, abs=1e-14)
    assert S.spearman(a, -a) == pytest.approx(-1.0, abs=1e-14)


def test_target_and_regret():
    assert S.target(100.0) == 0.0
    assert S.target(100.0 - 1e-9) == 0.0
    assert S.target(100.0 + math.e - 1) == pytest.approx(1.0, abs=1e-14)
    mu, sd = S.standardise([1.0, 3.0])
    assert (mu, sd) == (2.0, 1.0)
    assert S.regret([5.0, 7.0], [7.0, 5.0, 9.0]) == 0.0
    assert S.regret([6.0], [7.0, 5.0]) == 1.0
