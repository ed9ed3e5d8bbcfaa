"""BF16 tensor-core MLP kernels of the LES closure against the FP64 oracle
fed the same BF16-rounded operands: forward values, loss, every parameter
gradient, and the Adam update."""

import numpy as np
import pytest

from oracle import les

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


@pytest.fixture(scope="module")
def ps():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_01309_gb300 import ps as _ps
    return _ps


def pack(p):
    return np.concatenate([p[k].reshape(-1) for k in ORDER]).astype(np.float32)


def unpack(v):
    out, o = {}, 0
    for k, shape in (("W1", (5, 64)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64, 6)), ("b3", (6,))):
        n = int(np.prod(shape))
        out[k] = v[o:o + n].reshape(shape).astype(np.float64)
        o += n
    return out


def _case(seed, B):
    rng = np.random.default_rng(seed)
    p = les.init_params(seed=seed)
    for k in p:
        p[k] = p[k] + 0.2 * rng.standard_normal(p[k].shape)
    X = rng.standard_normal((B, 5)).astype(np.float32)
    T = rng.standard_normal((B, 6)).astype(np.float32)
    # the kernel sees FP32 parameters: give the oracle the same values
    p = unpack(pack(p))
    return p, X, T


def relerr(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("B", [16, 1000, 70001])
def test_forward_matches_oracle(ps, B):
    p, X, _ = _case(1, B)
    dev = "cuda"
    Y = torch.empty((B, 6), device=dev, dtype=torch.float32)
    ps.ps_mlp_forward(torch.from_numpy(pack(p)).to(dev), torch.from_numpy(X).to(dev), Y, B)
    y_ref, _ = les.mlp_forward(p, X.astype(np.float64), rnd=les.bf16_round)
    got = Y.cpu().numpy()
    assert relerr(got, y_ref) < 2e-3
    # the unrounded FP64 network differs only by the BF16 operand rounding
    y64, _ = les.mlp_forward(p, X.astype(np.float64))
    assert relerr(got, y64) < 3e-2


@pytest.mark.parametrize("B", [100, 4096, 50000])
def test_gradients_match_oracle(ps, B):
    p, X, T = _case(2, B)
    dev = "cuda"
    grad = torch.empty(ps.MLP_NPARAM, device=dev, dtype=torch.float32)
    loss = torch.empty(1, device=dev, dtype=torch.float64)
    ps.ps_mlp_grad(torch.from_numpy(pack(p)).to(dev), torch.from_numpy(X).to(dev), torch.from_numpy(T).to(dev),
                   B, grad, loss)
    L_ref, g_ref = les.mse_and_grads(p, X.astype(np.float64), T.astype(np.float64), rnd=les.bf16_round)
    assert abs(float(loss.item()) - L_ref) < 1e-4 * L_ref
    g = unpack(grad.cpu().numpy())
    for k in ORDER:
        assert relerr(g[k], g_ref[k]) < 2e-2, k


def test_adam_update_closed_form(ps):
    rng = np.random.default_rng(5)
    n = ps.MLP_NPARAM
    p0 = rng.standard_normal(n).astype(np.float32)
    dev = "cuda"
    P = torch.from_numpy(p0.copy()).to(dev)
    M = torch.zeros(n, device=dev)
    V = torch.zeros(n, device=dev)
    ref_p, ref_m, ref_v = p0.astype(np.float64), np.zeros(n), np.zeros(n)
    for step in range(1, 4):
        g = rng.standard_normal(n).astype(np.float32)
        ps.ps_mlp_adam(P, torch.from_numpy(g).to(dev), M, V, step, 1e-2)
        ref_m = 0.9 * ref_m + 0.1 * g
        ref_v = 0.999 * ref_v + 0.001 * g.astype(np.float64) ** 2
        ref_p = ref_p - 1e-2 * (ref_m / (1 - 0.9 ** step)) / (np.sqrt(ref_v / (1 - 0.999 ** step)) + 1e-8)
    assert np.max(np.abs(P.cpu().numpy() - ref_p)) < 1e-5


def test_training_reduces_the_loss(ps):
    """Fit a smooth synthetic map with the GPU kernels only."""
    rng = np.random.default_rng(7)
    B = 8192
    X = rng.standard_normal((B, 5)).astype(np.float32)
    Wt = rng.standard_normal((5, 6)) * 0.5
    T = np.tanh(X @ Wt).astype(np.float32)
    dev = "cuda"
    P = torch.from_numpy(pack(les.init_params(seed=3))).to(dev)
    M = torch.zeros_like(P)
    V = torch.zeros_like(P)
    G = torch.empty_like(P)
    L = torch.empty(1, device=dev, dtype=torch.float64)
    Xd, Td = torch.from_numpy(X).to(dev), torch.from_numpy(T).to(dev)
    losses = []
    for step in range(1, 301):
        ps.ps_mlp_grad(P, Xd, Td, B, G, L)
        ps.ps_mlp_adam(P, G, M, V, step, 3e-3)
        if step in (1, 300):
            losses.append(float(L.item()))
    assert losses[1] < 0.1 * losses[0]


@pytest.mark.parametrize("B", [100, 40000])
def test_tensor_basis_gradients_match_oracle(ps, B):
    p, X, _ = _case(4, B)
    rng = np.random.default_rng(9)
    A = rng.standard_normal((B, 9)).astype(np.float32)
    T = rng.standard_normal((B, 6)).astype(np.float32)
    s_A, s_tau = 1.7, 0.3
    dev = "cuda"
    grad = torch.empty(ps.MLP_NPARAM, device=dev, dtype=torch.float32)
    loss = torch.empty(1, device=dev, dtype=torch.float64)
    ps.ps_mlp_grad_tb(torch.from_numpy(pack(p)).to(dev), torch.from_numpy(X).to(dev), torch.from_numpy(A).to(dev),
                      torch.from_numpy(T).to(dev), B, s_A, s_tau, grad, loss)
    Bas = les.tensor_basis(A.astype(np.float64).T.reshape(3, 3, B), s_A).transpose(2, 1, 0)
    L_ref, g_ref = les.mse_and_grads_tb(p, X.astype(np.float64), Bas, T.astype(np.float64) / s_tau,
                                        rnd=les.bf16_round)
    assert abs(float(loss.item()) - L_ref) < 1e-4 * L_ref
    g = unpack(grad.cpu().numpy())
    for k in ORDER:
        assert relerr(g[k], g_ref[k]) < 2e-2, k
