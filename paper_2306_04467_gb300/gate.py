"""Learned troubled-cell gate: training data from the solver's own runs and
training on the GPU with the library's BF16 tensor-core kernels.

The gate is not part of the paper. The compact reconstruction (Sec. 3.4)
blends a P3 least-squares polynomial with three P1 candidates through WENO-Z
weights; where the data are smooth those weights stay at the linear ones and
the result is the P3 polynomial. The gate, a 24 -> 32 -> 32 -> 1 MLP, predicts
that from the cell's and its face neighbours' averages and gradients. It runs
as its own kernel on a second stream beside a stage's interface and edge
kernels and decides for the next stage: cells it calls smooth skip the
smoothness indicators and weights there, and a tile of 32 such cells skips
loading their operators. Labels are the method's own: a cell is troubled when
any of its WENO weights departs from the linear one by more than `tol`
(relative).

Everything numeric here runs in the library (gks2l_harvest, gks2l_mlp_grad,
gks2l_mlp_adam, gks2l_mlp_forward); PyTorch holds device memory.
"""
from __future__ import annotations

import math

import numpy as np

from . import gks2l as g
from . import inputs

N_IN = 24
# A cell is smooth when the predicted probability of trouble is below this.
# With the interlayer source taken from each cell's own reconstruction, a
# troubled cell called smooth costs more accuracy; 0.15 keeps the smooth
# periodic case's L1 against the FP64 oracle at 5.6e-6 (0.3: 1.4e-5) while
# the large configuration still takes 99% of its cells smooth.
THRESHOLD = 0.15
MEAN = g.GKS2L_MLP_NTRAIN
ISTD = MEAN + N_IN


def collect(problems, precision=g.GKS2L_FP32, snapshots=8, stride=20, tol=3e-3):
    """Harvest (features, labels) from runs of each problem: every cell every
    `stride` stages. The reconstruction decides with the gate its previous
    stage computed, so a cell's label marks it troubled at this stage or the
    next. Returns device tensors [n, 24], [n]."""
    import torch
    Xs, ys = [], []
    for prob in problems:
        s = g.problem_solver(prob, precision=precision)
        for k in range(snapshots):
            X, y, _ = s.harvest(tol)
            s.advance(1)
            _, y1, _ = s.harvest(tol)
            Xs.append(X)
            ys.append(torch.maximum(y, y1))
            if k + 1 < snapshots:
                s.advance(stride - 1)
        s.close()
    return torch.cat(Xs), torch.cat(ys)


def training_problems(scale=1):
    """The seeded runs the default gate learns from (meshes and seeds of their
    own): an interface dam break, the smooth periodic case and the periodic
    translation at coarse to moderate resolutions, an internal wave over a
    ridge and an ensemble member with Fourier bathymetry."""
    probs = [inputs.interface_dambreak(96 * scale, seed=7101),
             inputs.internal_wave_ridge(160 * scale, 20 * scale, seed=7103),
             inputs.ensemble_member(48 * scale, seed=7104)]
    probs += [inputs.smooth_periodic(n * scale, seed=7110 + n) for n in (12, 16, 24, 32, 48)]
    probs += [inputs.translation(n * scale, seed=7130 + n) for n in (12, 24)]
    return probs


def train(X, y, steps=1500, batch=8192, lr=3e-3, pos_weight=None, seed=2312, log_every=0):
    """Adam on the weighted logistic loss over shuffled minibatches of (X, y)
    (device tensors). Returns the float32 parameter vector (host) and the
    loss history (mean loss per sample, every `log_every` steps)."""
    import torch
    dev = X.device
    n = int(y.numel())
    if n < 16:
        raise ValueError("too few samples")
    P0 = inputs.gate_init(seed)
    Xh = X.double().cpu().numpy()
    mean = Xh.mean(0)
    std = Xh.std(0)
    P0[MEAN:ISTD] = mean
    P0[ISTD:] = 1.0 / np.maximum(std, 1e-3)
    npos = float(y.sum().item())
    if pos_weight is None:
        pos_weight = min(50.0, max(1.0, 2.0 * (n - npos) / max(npos, 1.0)))
    P = torch.from_numpy(P0).to(dev)
    G = torch.zeros(g.GKS2L_MLP_NTRAIN, dtype=torch.float32, device=dev)
    m = torch.zeros_like(G)
    v = torch.zeros_like(G)
    L = torch.zeros(1, dtype=torch.float32, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    perm = torch.randperm(n, generator=gen, device=dev)
    Xs = X[perm].contiguous()
    ys = y[perm].contiguous()
    batch = min(batch, n)
    hist = []
    off = 0
    for step in range(1, steps + 1):
        if off + batch > n:
            off = 0
        g.mlp_grad(Xs[off:off + batch], ys[off:off + batch], P, pos_weight, G, L)
        g.mlp_adam(P, G, m, v, step, lr * (0.5 * (1 + math.cos(math.pi * step / steps)) * 0.9 + 0.1), 1.0 / batch)
        off += batch
        if log_every and step % log_every == 0:
            hist.append(L.item() / batch)
    torch.cuda.synchronize(dev)
    return P.cpu().numpy().astype(np.float32), hist


def evaluate(X, y, P, threshold=THRESHOLD):
    """Gate quality on (X, y): the fraction it calls smooth, the fraction of
    troubled cells it calls smooth (misses) and of smooth cells it flags."""
    import torch
    Pd = torch.from_numpy(np.ascontiguousarray(P, np.float32)).to(X.device)
    s = torch.empty(y.numel(), dtype=torch.float32, device=X.device)
    g.mlp_forward(X, Pd, s)
    smooth = s < math.log(threshold / (1 - threshold))
    pos = y > 0.5
    npos = max(int(pos.sum().item()), 1)
    nneg = max(int((~pos).sum().item()), 1)
    return dict(smooth_fraction=float(smooth.float().mean().item()),
                missed=float((smooth & pos).sum().item()) / npos,
                flagged=float((~smooth & ~pos).sum().item()) / nneg,
                label_fraction=float(pos.float().mean().item()))


def default_gate(precision=g.GKS2L_FP32, tol=3e-3, steps=1500, seed=2312, scale=1):
    """Harvest from `training_problems(scale)` and train: the gate the
    benchmark and tests use. Returns (params, quality on the training set)."""
    X, y = collect(training_problems(scale), precision=precision, tol=tol)
    P, _ = train(X, y, steps=steps, seed=seed)
    return P, evaluate(X, y, P)
