"""Pins of the FP64 gate network in the oracle (oracle/mlp.py).

The network is an addition to the paper's scheme (a troubled-cell gate for
the WENO reconstruction of Sec. 3.4); these tests check its reference
implementation against independent routines: central finite differences of
the loss, PyTorch's float64 layers and logistic loss, PyTorch's bfloat16
conversion, and the closed form of Adam's first step.
"""
import numpy as np
import pytest

from oracle import mlp
from paper_2306_04467_gb300 import inputs

torch = pytest.importorskip("torch")


def params(seed=7):
    P = inputs.gate_init(seed).astype(np.float64)
    # nonzero biases and normalisation so every term of the formula matters
    rng = np.random.default_rng(seed)
    P[mlp.B1:mlp.W2] = 0.1 * rng.standard_normal(32)
    P[mlp.B2:mlp.W3] = 0.1 * rng.standard_normal(32)
    P[mlp.B3] = -0.3
    P[mlp.MEAN:mlp.ISTD] = 0.05 * rng.standard_normal(24)
    P[mlp.ISTD:] = 1.0 + 0.2 * rng.random(24)
    return P


def test_layout_sizes():
    assert mlp.NPARAM == inputs.GATE_NPARAM == 1937
    assert mlp.NTRAIN == 1889


def test_forward_matches_torch_layers():
    P = params()
    X, _ = inputs.gate_samples(300, seed=11)
    p = mlp.unpack(P)
    net = torch.nn.Sequential(torch.nn.Linear(24, 32), torch.nn.ReLU(), torch.nn.Linear(32, 32), torch.nn.ReLU(),
                              torch.nn.Linear(32, 1)).double()
    with torch.no_grad():
        net[0].weight.copy_(torch.from_numpy(p["W1"]))
        net[0].bias.copy_(torch.from_numpy(p["b1"]))
        net[2].weight.copy_(torch.from_numpy(p["W2"]))
        net[2].bias.copy_(torch.from_numpy(p["b2"]))
        net[4].weight.copy_(torch.from_numpy(p["w3"][None, :]))
        net[4].bias.fill_(float(p["b3"]))
        xn = (torch.from_numpy(X.astype(np.float64)) - torch.from_numpy(p["mean"])) * torch.from_numpy(p["istd"])
        ref = net(xn)[:, 0].numpy()
    s = mlp.forward(P, X)
    assert np.abs(s - ref).max() <= 1e-13 * (1 + np.abs(ref).max())


def test_loss_matches_torch_weighted_logistic_loss():
    P = params()
    X, y = inputs.gate_samples(257, seed=12)
    s = mlp.forward(P, X)
    for pos_w in (1.0, 3.5):
        ref = torch.nn.functional.binary_cross_entropy_with_logits(
            torch.from_numpy(s), torch.from_numpy(y.astype(np.float64)), pos_weight=torch.tensor(pos_w, dtype=torch.float64),
            reduction="sum").item()
        assert abs(mlp.loss(P, X, y, pos_w) - ref) <= 1e-12 * abs(ref)


def test_gradient_matches_central_differences():
    P = params()
    X, y = inputs.gate_samples(40, seed=13)
    pos_w = 2.5
    _, g = mlp.loss_grad(P, X, y, pos_w)
    h = 1e-6
    fd = np.zeros(mlp.NTRAIN)
    for k in range(mlp.NTRAIN):
        Pp, Pm = P.copy(), P.copy()
        Pp[k] += h
        Pm[k] -= h
        fd[k] = (mlp.loss(Pp, X, y, pos_w) - mlp.loss(Pm, X, y, pos_w)) / (2 * h)
    # ReLU kinks within h of a sample would break the check: none here
    assert np.abs(g - fd).max() <= 1e-6 * (1 + np.abs(fd).max()), np.abs(g - fd).max()


def test_gradient_matches_torch_autograd():
    P = params(9)
    X, y = inputs.gate_samples(500, seed=14)
    p = mlp.unpack(P)
    t = {k: torch.tensor(np.asarray(v, np.float64), requires_grad=True) for k, v in p.items()
         if k not in ("mean", "istd")}
    x = (torch.from_numpy(X.astype(np.float64)) - torch.from_numpy(p["mean"])) * torch.from_numpy(p["istd"])
    h1 = torch.relu(x @ t["W1"].T + t["b1"])
    h2 = torch.relu(h1 @ t["W2"].T + t["b2"])
    s = h2 @ t["w3"] + t["b3"]
    L = torch.nn.functional.binary_cross_entropy_with_logits(s, torch.from_numpy(y.astype(np.float64)),
                                                             pos_weight=torch.tensor(1.7, dtype=torch.float64), reduction="sum")
    L.backward()
    ref = np.concatenate([t["W1"].grad.numpy().ravel(), t["b1"].grad.numpy(), t["W2"].grad.numpy().ravel(),
                          t["b2"].grad.numpy(), t["w3"].grad.numpy(), [t["b3"].grad.item()]])
    _, g = mlp.loss_grad(P, X, y, 1.7)
    assert np.abs(g - ref).max() <= 1e-12 * (1 + np.abs(ref).max())


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-6, 6, 10000),
                        # exact ties between two bfloat16 values, both parities
                        (np.arange(1, 2000, dtype=np.float64) * 2.0 + 1.0) * 2.0 ** -8,
                        [0.0, -0.0, 1.0, -3.0, 65504.0]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), ref)


def test_bf16_model_is_close_to_exact():
    P = params()
    X, y = inputs.gate_samples(400, seed=15)
    s = mlp.forward(P, X)
    sb = mlp.forward(P, X, use_bf16=True)
    assert np.abs(s - sb).max() <= 0.05 * (1 + np.abs(s).max())
    # the training convention's forward, too
    st = mlp._forward(P, X, True)[0]
    assert np.abs(st - s).max() <= 0.05 * (1 + np.abs(s).max())
    _, g = mlp.loss_grad(P, X, y, 2.0)
    _, gb = mlp.loss_grad(P, X, y, 2.0, use_bf16=True)
    cos = g @ gb / np.linalg.norm(g) / np.linalg.norm(gb)
    assert cos >= 0.999


def test_adam_first_step_closed_form():
    # after one step from zero moments the bias-corrected update is lr * g / (|g| + eps)
    P = params()
    G = np.linspace(-2.0, 3.0, mlp.NTRAIN)
    m = np.zeros(mlp.NTRAIN)
    v = np.zeros(mlp.NTRAIN)
    P1 = P.copy()
    mlp.adam(P1, G, m, v, 1, 1e-2, 0.5)
    gs = 0.5 * G
    assert np.allclose(P1[:mlp.NTRAIN], P[:mlp.NTRAIN] - 1e-2 * gs / (np.abs(gs) + 1e-8), rtol=0, atol=1e-15)
    assert np.array_equal(P1[mlp.NTRAIN:], P[mlp.NTRAIN:])
