"""Learned troubled-cell gate on the GPU, through the C ABI, against the oracle.

The gate (not part of the paper) lets cells whose WENO weights (Sec. 3.4)
would stay at the linear ones take the P3 polynomial directly. Checked here:
the BF16 tensor-core forward, loss gradient and Adam step against the FP64
network of the oracle (with the same BF16 operand rounding, and without it),
the harvested features and labels against the oracle's, the fused gate in
the reconstruction against the oracle's linear mask, and what a network
trained on the method's own runs gains over the method without it.
"""
import math

import numpy as np
import pytest

from oracle import mlp
from oracle.oracle import Oracle
from paper_2306_04467_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2306_04467_gb300 import gks2l as g  # noqa: E402
from paper_2306_04467_gb300 import gate  # noqa: E402

from test_gpu_parity import max_rel, areas  # noqa: E402

DEV = torch.device("cuda", 0)


def params(seed=7):
    P = inputs.gate_init(seed).astype(np.float64)
    rng = np.random.default_rng(seed)
    P[mlp.B1:mlp.W2] = 0.1 * rng.standard_normal(32)
    P[mlp.B2:mlp.W3] = 0.1 * rng.standard_normal(32)
    P[mlp.B3] = -0.3
    P[mlp.MEAN:mlp.ISTD] = 0.05 * rng.standard_normal(24)
    P[mlp.ISTD:] = 1.0 + 0.2 * rng.random(24)
    return P.astype(np.float32)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(DEV)


def constant_gate(logit):
    P = np.zeros(mlp.NPARAM, np.float32)
    P[mlp.B3] = logit
    P[mlp.ISTD:] = 1.0
    return P


@pytest.mark.parametrize("n", [1, 31, 5000])
def test_forward_matches_oracle(n):
    P = params()
    X, _ = inputs.gate_samples(n, seed=21)
    s = torch.empty(n, dtype=torch.float32, device=DEV)
    g.mlp_forward(dev(X), dev(P), s)
    s = s.cpu().numpy().astype(np.float64)
    ref = mlp.forward(P, X, use_bf16=True)
    err = np.abs(s - ref) / (1 + np.abs(ref))
    # identical BF16 operands, FP32 sums: rare one-ulp flips of a rounded
    # hidden activation are the only larger differences
    assert np.quantile(err, 0.99) <= 1e-5 and err.max() <= 1e-2, (np.quantile(err, 0.99), err.max())
    exact = mlp.forward(P, X)
    assert np.abs(s - exact).max() <= 0.05 * (1 + np.abs(exact).max())


@pytest.mark.parametrize("n", [16, 3001])
def test_gradient_matches_oracle(n):
    P = params(8)
    X, y = inputs.gate_samples(n, seed=22)
    G = torch.empty(mlp.NTRAIN, dtype=torch.float32, device=DEV)
    L = torch.empty(1, dtype=torch.float32, device=DEV)
    g.mlp_grad(dev(X), dev(y), dev(P), 2.5, G, L)
    G = G.cpu().numpy().astype(np.float64)
    Lr, Gr = mlp.loss_grad(P, X, y, 2.5, use_bf16=True)
    assert abs(L.item() - Lr) <= 1e-4 * abs(Lr)
    scale = np.abs(Gr).max()
    assert np.abs(G - Gr).max() <= 2e-3 * scale, np.abs(G - Gr).max() / scale
    assert np.linalg.norm(G - Gr) <= 1e-3 * np.linalg.norm(Gr)
    _, Ge = mlp.loss_grad(P, X, y, 2.5)
    assert G @ Ge / np.linalg.norm(G) / np.linalg.norm(Ge) >= 0.999


def test_gradient_is_reproducible():
    P = params(8)
    X, y = inputs.gate_samples(20000, seed=23)
    out = []
    for _ in range(2):
        G = torch.empty(mlp.NTRAIN, dtype=torch.float32, device=DEV)
        L = torch.empty(1, dtype=torch.float32, device=DEV)
        g.mlp_grad(dev(X), dev(y), dev(P), 1.5, G, L)
        out.append((G.cpu().numpy(), L.item()))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]


def test_adam_matches_oracle():
    P = params(9)
    rng = np.random.default_rng(4)
    Pd = dev(P)
    m = torch.zeros(mlp.NTRAIN, dtype=torch.float32, device=DEV)
    v = torch.zeros_like(m)
    Pr = P.astype(np.float64)
    mr = np.zeros(mlp.NTRAIN)
    vr = np.zeros(mlp.NTRAIN)
    for step in (1, 2, 3):
        G = rng.standard_normal(mlp.NTRAIN).astype(np.float32)
        g.mlp_adam(Pd, dev(G), m, v, step, 1e-2, 0.25)
        mlp.adam(Pr, G.astype(np.float64), mr, vr, step, 1e-2, 0.25)
    out = Pd.cpu().numpy().astype(np.float64)
    assert np.abs(out - Pr).max() <= 1e-6
    assert np.array_equal(out[mlp.NTRAIN:], P[mlp.NTRAIN:].astype(np.float64))


@pytest.mark.parametrize("precision", [g.GKS2L_FP64, g.GKS2L_FP32])
def test_harvest_matches_oracle(precision):
    prob = inputs.interface_dambreak(24)
    s = g.problem_solver(prob, precision=precision)
    s.advance(10)
    X, y, _ = s.harvest(1e-2)
    o = Oracle.from_problem(prob)
    o.advance(10)
    Xr = o.gate_features()
    o.reconstruct()
    d = o.weight_departure().max(1)
    X = X.cpu().numpy().astype(np.float64)
    y = y.cpu().numpy()
    ftol = 1e-6 if precision == g.GKS2L_FP64 else 1e-4
    assert np.abs(X - Xr).max() <= ftol, np.abs(X - Xr).max()
    margin = 1e-6 if precision == g.GKS2L_FP64 else 1e-3
    sure = np.abs(d - 1e-2) > margin
    assert sure.mean() > 0.95
    assert np.array_equal(y[sure], (d[sure] > 1e-2).astype(np.float32))
    assert 0.02 < y.mean() < 0.9
    # harvesting leaves the state alone
    a0, g0 = s.get_state()
    s2 = g.problem_solver(prob, precision=precision)
    s2.advance(10)
    a1, g1 = s2.get_state()
    assert np.array_equal(a0, a1) and np.array_equal(g0, g1)


# mma.sync warp tiles, tcgen05 CTA tiles, the same with two and four times the blocks
GATE_KERNELS = list(range(g.GKS2L_GATE_KERNELS))
# each kernel beside the edge kernels, then beside the reconstruction; both
# with the fused edge pass, then with the plain edge kernels
GATE_VARIANTS = list(range(g.GKS2L_GATE_VARIANTS))


@pytest.mark.parametrize("variant", GATE_KERNELS)
@pytest.mark.parametrize("case", ["ensemble", "dambreak"])
def test_fused_gate_logits_match_oracle(case, variant):
    """Logits of the gate kernel (either variant) vs the oracle network on
    the oracle's features of the same seeded state (392 and 800 cells: the
    tensor-memory variant's last 128-cell tile is ragged)."""
    prob = inputs.ensemble_member(14, seed=31) if case == "ensemble" else inputs.interface_dambreak(20)
    P = params(10)
    s = g.problem_solver(prob, precision=g.GKS2L_FP64, indicator=g.GKS2L_INDICATOR_MLP)
    s.set_launch_shapes([1, 1, 1, variant])
    s.set_mlp(P)
    logits = torch.empty(prob.mesh.n_tri, dtype=torch.float32, device=DEV)
    s.harvest(1e-2, logits=logits)
    o = Oracle.from_problem(prob)
    ref = mlp.forward(P, o.gate_features(), use_bf16=True)
    got = logits.cpu().numpy().astype(np.float64)
    err = np.abs(got - ref) / (1 + np.abs(ref))
    assert np.quantile(err, 0.99) <= 1e-4 and err.max() <= 2e-2, (np.quantile(err, 0.99), err.max())


def test_gate_kernels_agree():
    """The two gate kernels on the same state and network: logits equal up to
    the FP32 accumulation order inside the MMAs, and so the same decisions
    away from the threshold (5,408 cells with features everywhere, ragged
    last tile)."""
    prob = inputs.ensemble_member(52, seed=33)
    P = params(11)
    out = []
    for variant in GATE_KERNELS:
        s = g.problem_solver(prob, precision=g.GKS2L_FP32, indicator=g.GKS2L_INDICATOR_MLP)
        s.set_launch_shapes([1, 1, 1, variant])
        s.set_mlp(P)
        logits = torch.empty(prob.mesh.n_tri, dtype=torch.float32, device=DEV)
        s.harvest(1e-2, logits=logits)
        out.append(logits.cpu().numpy().astype(np.float64))
    for k in range(1, len(out)):
        err = np.abs(out[k] - out[0]) / (1 + np.abs(out[0]))
        assert err.max() <= 1e-3 and np.quantile(err, 0.99) <= 1e-5, (k, err.max(), np.quantile(err, 0.99))


@pytest.mark.parametrize("variant", GATE_VARIANTS)
@pytest.mark.parametrize("case", ["smooth", "dambreak"])
def test_all_smooth_gate_matches_oracle_linear_mask(case, variant):
    """A gate that calls every cell smooth: the first stage (no decisions yet)
    is the plain method, every later one the P3 polynomial."""
    prob, n = (inputs.smooth_periodic(16), 100) if case == "smooth" else (inputs.interface_dambreak(16), 40)
    s = g.problem_solver(prob, precision=g.GKS2L_FP64, indicator=g.GKS2L_INDICATOR_MLP)
    s.set_launch_shapes([1, 1, 1, variant])
    s.set_mlp(constant_gate(-30.0))
    s.advance(n)
    a, gr = s.get_state()
    st = s.stats()
    assert st["status"] == 0 and abs(st["smooth_fraction"] - (n - 1) / n) < 1e-12
    o = Oracle.from_problem(prob)
    o.advance(1)
    o.set_linear_mask(np.ones(prob.mesh.n_tri, np.uint8))
    o.advance(n - 1)
    ao, go = o.get_state()
    ra, rg = max_rel(prob, a, gr, ao, go)
    assert ra <= 1e-11 and rg <= 1e-11, (ra, rg)


def test_set_state_runs_the_gate_for_the_first_stage():
    """A state set while the gate is on gets the gate's decisions on that
    state for its first stage: with a gate that calls every cell smooth,
    every stage (the first included) is the P3 polynomial."""
    prob, n = inputs.smooth_periodic(16), 10
    s = g.problem_solver(prob, precision=g.GKS2L_FP64, indicator=g.GKS2L_INDICATOR_MLP)
    s.set_mlp(constant_gate(-30.0))
    s.set_state(prob.avg, prob.grad)
    s.advance(n)
    a, gr = s.get_state()
    st = s.stats()
    assert st["status"] == 0 and st["smooth_fraction"] == 1.0
    o = Oracle.from_problem(prob)
    o.set_linear_mask(np.ones(prob.mesh.n_tri, np.uint8))
    o.advance(n)
    ao, go = o.get_state()
    ra, rg = max_rel(prob, a, gr, ao, go)
    assert ra <= 1e-11 and rg <= 1e-11, (ra, rg)


@pytest.mark.parametrize("variant", GATE_VARIANTS)
def test_no_smooth_gate_is_the_plain_method(variant):
    prob = inputs.interface_dambreak(16)
    s = g.problem_solver(prob, precision=g.GKS2L_FP32, indicator=g.GKS2L_INDICATOR_MLP)
    s.set_launch_shapes([1, 1, 1, variant])
    s.set_mlp(constant_gate(30.0))
    s.advance(20)
    a, gr = s.get_state()
    assert s.stats()["smooth_fraction"] == 0.0
    s2 = g.problem_solver(prob, precision=g.GKS2L_FP32)
    s2.advance(20)
    b, h = s2.get_state()
    assert np.array_equal(a, b) and np.array_equal(gr, h)


@pytest.mark.parametrize("kernel", GATE_KERNELS)
def test_gate_placement_changes_no_result(kernel):
    """A network that calls some cells smooth and some not (its output bias
    puts the oracle's median logit of the initial state at the threshold 1/2),
    run beside the edge kernels and beside the reconstruction, each with the
    fused edge pass and with the plain edge kernels: the same decisions reach
    the same reconstructions and edges, so 20 stages agree bit for bit."""
    prob = inputs.ensemble_member(16, seed=33)
    P = params(10)
    ref = mlp.forward(P, Oracle.from_problem(prob).gate_features(), use_bf16=True)
    P[mlp.B3] -= np.float32(np.median(ref))
    out = []
    K = g.GKS2L_GATE_KERNELS
    for variant in (kernel, kernel + K, kernel + 2 * K, kernel + 3 * K):
        s = g.problem_solver(prob, precision=g.GKS2L_FP32, indicator=g.GKS2L_INDICATOR_MLP,
                             indicator_threshold=0.5)
        s.set_launch_shapes([1, 1, 1, variant])
        s.set_mlp(P)
        s.advance(20)
        a, gr = s.get_state()
        st = s.stats()
        assert st["status"] == 0
        out.append((a, gr, st["smooth_fraction"]))
    assert 0.0 < out[0][2] < 1.0, out[0][2]
    for o in out[1:]:
        assert o[2] == out[0][2]
        assert np.array_equal(o[0], out[0][0]) and np.array_equal(o[1], out[0][1])


def test_set_mlp_rejects_bad_input():
    prob = inputs.smooth_periodic(4)
    s = g.problem_solver(prob, precision=g.GKS2L_FP32, indicator=g.GKS2L_INDICATOR_MLP)
    with pytest.raises(g.GKSError):
        s.set_mlp(np.zeros(10, np.float32))
    bad = constant_gate(0.0)
    bad[3] = np.nan
    with pytest.raises(g.GKSError):
        s.set_mlp(bad)


@pytest.fixture(scope="module")
def trained():
    P, quality = gate.default_gate()
    return P, quality


def gated_solver(prob, P, precision=g.GKS2L_FP32):
    s = g.problem_solver(prob, precision=precision, indicator=g.GKS2L_INDICATOR_MLP,
                         indicator_threshold=gate.THRESHOLD)
    s.set_mlp(P)
    return s


def test_training_learns_the_labels(trained):
    P, q = trained
    # few troubled cells are called smooth; most smooth ones are
    print(q)
    assert q["missed"] <= 0.03, q
    assert q["smooth_fraction"] >= 0.5 * (1 - q["label_fraction"]), q


def test_trained_gate_keeps_smooth_cases_within_l1_of_oracle(trained):
    P, _ = trained
    for prob in (inputs.smooth_periodic(16), inputs.translation(16)):
        s = gated_solver(prob, P)
        s.advance(100)
        a, _ = s.get_state()
        assert s.stats()["smooth_fraction"] > 0.3
        o = Oracle.from_problem(prob)
        o.advance(100)
        ao, _ = o.get_state()
        area = areas(prob.mesh)
        for v in (0, 3):
            l1 = np.sum(area * np.abs(a[v] - ao[v])) / np.sum(area * np.abs(ao[v]))
            assert l1 <= 1e-5, (prob.name, v, l1)


def test_trained_gate_gain_on_dambreak(trained):
    """What the gate gains on an unseen interface dam break (another seed and
    size than the training runs): the share of cells it lets skip the WENO
    weights, the reconstruction time saved, and the L1 change of the result
    against the plain nonlinear reconstruction, against which its error is measured."""
    P, _ = trained
    prob = inputs.interface_dambreak(256, seed=99)
    plain = g.problem_solver(prob, precision=g.GKS2L_FP32)
    gated = gated_solver(prob, P)
    plain.advance(200)
    gated.advance(200)
    a, _ = plain.get_state()
    b, _ = gated.get_state()
    frac = gated.stats()["smooth_fraction"]
    area = areas(prob.mesh)
    l1 = max(np.sum(area * np.abs(a[v] - b[v])) / np.sum(area * np.abs(a[v])) for v in (0, 3))
    ms_plain = plain.profile_kernels(20)
    ms_gated = gated.profile_kernels(20)
    print("smooth fraction %.3f, L1 change %.2e, recon ms plain %.4f gated %.4f"
          % (frac, l1, ms_plain["recon"], ms_gated["recon"]))
    assert frac >= 0.9
    assert l1 <= 2e-4
    assert ms_gated["recon"] < ms_plain["recon"]


def test_full_size_dambreak_with_gate(trained):
    """The learned-indicator configuration at full size: interface dam break
    on a 1,602,050-triangle mesh of [-1, 1]^2, FP32 with the gate. After 200
    stages both layers keep their mass, the gate calls most cells smooth, and
    the result stays within a stated L1 distance of the plain method's."""
    P, _ = trained
    prob = inputs.interface_dambreak(895)
    assert prob.mesh.n_tri == 1602050
    plain = g.problem_solver(prob, precision=g.GKS2L_FP32)
    plain.advance(200)
    a, _ = plain.get_state()
    del plain
    gated = gated_solver(prob, P)
    gated.advance(200)
    b, _ = gated.get_state()
    st = gated.stats()
    assert st["status"] == 0 and st["smooth_fraction"] >= 0.9
    area = areas(prob.mesh)
    for v in (0, 3):
        m0, m1 = area @ prob.avg[v], area @ b[v]
        assert abs(m1 - m0) <= 1e-12 * m0
    l1 = max(np.sum(area * np.abs(a[v] - b[v])) / np.sum(area * np.abs(a[v])) for v in (0, 3))
    print("full-size dam break: smooth fraction %.3f, L1 change %.2e" % (st["smooth_fraction"], l1))
    assert l1 <= 1e-4


def test_large_internal_wave(trained):
    """The large configuration: internal wave over a ridge on 7,997,584
    triangles, FP32 + learned gate + FP64 balance terms, all 2000 stages at
    the paper's CFL 0.5. Both layers keep their mass to rounding, the depths
    stay positive and the discharges stay at the internal wave's scale: the
    linear wave of an interface depression a = 0.1 carries a layer discharge
    of about c_i a h2 / (h1 + h2) = 0.0074 (c_i = sqrt((1 - chi) G h1 h2 /
    (h1 + h2)) = 0.25), so |hu| <= 0.02 leaves room for the ridge's
    amplification, and the flow across the channel, which only the mesh's
    irregularity drives, stays below 0.01."""
    P, _ = trained
    prob = inputs.internal_wave_ridge()
    assert prob.mesh.n_tri == 7997584
    s = gated_solver(prob, P)
    s.advance(2000)
    a, _ = s.get_state()
    st = s.stats()
    assert st["status"] == 0 and np.isfinite(a).all() and a[0].min() > 0 and a[3].min() > 0
    area = areas(prob.mesh)
    for v in (0, 3):
        m0, m1 = area @ prob.avg[v], area @ a[v]
        assert abs(m1 - m0) <= 1e-12 * m0
    hu, hv = np.abs(a[[1, 4]]).max(), np.abs(a[[2, 5]]).max()
    print("large internal wave: t %.4f after 2000 stages, smooth fraction %.3f, max |hu| %.3g, max |hv| %.3g"
          % (st["t"], st["smooth_fraction"], hu, hv))
    assert hu <= 0.02 and hv <= 0.01, (hu, hv)
