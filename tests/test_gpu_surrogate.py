"""GPU tests of the neural-operator surrogate kernels and model: the BF16
tensor-core GEMM against float64 products of the same BF16 values; the whole
network's forward output and every parameter gradient against a float64
CPU reference (plain torch ops with autograd, same weights, same DFT
matrices) on a tiny grid; a short training run lowers the loss; the gate
falls back to the exact path bit for bit."""
import math

import numpy as np
import pytest
import torch
import torch.nn.functional as F

from paper_2506_10812_gb300 import _native as N
from paper_2506_10812_gb300 import build as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built(cuda_device):
    B.build()
    N.load()


def bf(t):
    return t.to(torch.bfloat16)


GEMM_CASES = [
    (1, 64, 64, 32, False, 1.0, 0.0, False), (3, 100, 70, 45, False, 0.5, 1.0, True),
    (2, 33, 130, 200, True, 1.0, 0.0, False), (5, 7, 2, 4096, True, 1.0, 0.5, True),
    (1, 1000, 32, 7, False, 1.0, 0.0, True),
    # 16-byte load paths (leading dimensions multiples of 8) with ragged tiles
    (2, 72, 40, 96, True, 1.0, 0.0, True), (1, 130, 24, 40, False, 2.0, 0.0, False),
    (4, 64, 64, 64, False, 1.0, 1.0, True),
    # several 128-row and 128-column tiles, ragged in M, N and K; K = 16 (one
    # product of a 64-deep step); the surrogate's azimuthal-DFT shape
    (2, 300, 300, 136, False, 1.0, 0.0, True), (1, 257, 520, 72, True, 1.0, 1.0, False),
    (3, 1024, 32, 16, False, 1.0, 0.0, False), (8, 32, 32, 1024, False, 1.0, 0.0, False)]


@pytest.fixture(params=["tcgen05", "mma_sync"])
def gemm_engine(request):
    lib = N.load()
    eng = {"tcgen05": N.SG_NN_GEMM_TCGEN05, "mma_sync": N.SG_NN_GEMM_MMA_SYNC}[request.param]
    assert lib.sg_nn_set_gemm_engine(eng) == N.SG_OK
    yield request.param
    assert lib.sg_nn_set_gemm_engine(N.SG_NN_GEMM_TCGEN05) == N.SG_OK


@pytest.mark.parametrize("batch,M,Nn,K,trans_a,alpha,beta,bias", GEMM_CASES)
def test_gemm(gemm_engine, batch, M, Nn, K, trans_a, alpha, beta, bias):
    """Both engines against float64 products of the same BF16 values; the
    tcgen05 engine's device waits all completed (sg_nn_check)."""
    dev = torch.device("cuda:0")
    g = torch.Generator().manual_seed(M * 7 + K)
    A = torch.randn(batch, K, M, generator=g) if trans_a else torch.randn(batch, M, K, generator=g)
    Bm = torch.randn(batch, K, Nn, generator=g)
    C0 = torch.randn(batch, M, Nn, generator=g)
    bv = torch.randn(Nn, generator=g)
    Ad, Bd = bf(A).to(dev), bf(Bm).to(dev)
    Cd = C0.to(dev).contiguous()
    Cb = torch.empty(batch, M, Nn, dtype=torch.bfloat16, device=dev)
    lib = N.load()
    vp = lambda t: t.data_ptr() if t is not None else None
    st = lib.sg_nn_gemm(batch, M, Nn, K, alpha, vp(Ad), M if trans_a else K, Ad[0].numel(), int(trans_a), vp(Bd),
                        Nn, Bd[0].numel(), beta, vp(Cd), Nn, M * Nn, vp(Cb),
                        vp(bv.to(dev)) if bias else None, None)
    assert st == 0
    torch.cuda.synchronize()
    Af = bf(A).double()
    opA = Af.transpose(1, 2) if trans_a else Af
    ref = alpha * opA @ bf(Bm).double() + beta * C0.double() + (bv.double() if bias else 0.0)
    got = Cd.double().cpu()
    assert (got - ref).abs().max() <= 1e-5 * ref.abs().max() * math.sqrt(K) + 1e-6
    assert torch.allclose(Cb.double().cpu(), got, rtol=1e-2, atol=1e-2 * ref.abs().max())
    assert lib.sg_nn_check(None) == N.SG_OK


@pytest.mark.parametrize("batch,M,Nn,K,beta", [(7, 32, 32, 1024, 0.0), (5, 48, 24, 200, 1.0),
                                                (3, 130, 64, 72, 0.5), (6, 20, 40, 96, 0.0), (1, 64, 32, 256, 0.0)])
def test_gemm_shared_a(gemm_engine, batch, M, Nn, K, beta):
    """One A for the whole batch (stride 0) with K > 64: the tcgen05 engine
    folds several batch entries into one 128-column tile (ragged last group,
    N = 24 and 40 leaving tile columns unused)."""
    dev = torch.device("cuda:0")
    g = torch.Generator().manual_seed(batch * 1000 + K)
    A = torch.randn(M, K, generator=g)
    Bm = torch.randn(batch, K, Nn, generator=g)
    C0 = torch.randn(batch, M, Nn, generator=g)
    Ad, Bd = bf(A).to(dev), bf(Bm).to(dev)
    Cd = C0.to(dev).contiguous()
    Cb = torch.empty(batch, M, Nn, dtype=torch.bfloat16, device=dev)
    lib = N.load()
    vp = lambda t: t.data_ptr()
    st = lib.sg_nn_gemm(batch, M, Nn, K, 1.0, vp(Ad), K, 0, 0, vp(Bd), Nn, K * Nn, beta, vp(Cd), Nn, M * Nn,
                        vp(Cb), None, None)
    assert st == 0
    torch.cuda.synchronize()
    ref = bf(A).double() @ bf(Bm).double() + beta * C0.double()
    got = Cd.double().cpu()
    assert (got - ref).abs().max() <= 1e-5 * ref.abs().max() * math.sqrt(K) + 1e-6
    assert torch.allclose(Cb.double().cpu(), got, rtol=1e-2, atol=1e-2 * ref.abs().max())
    assert lib.sg_nn_check(None) == N.SG_OK


def test_gemm_random_shapes(gemm_engine):
    """40 seeded random shapes (M, N, K up to 700, batch up to 6, transposed
    or not, shared or per-entry A, odd leading dimensions that force the
    element-wise load paths) against float64 products of the same BF16
    values."""
    dev = torch.device("cuda:0")
    lib = N.load()
    rng = np.random.default_rng(2506)
    vp = lambda t: t.data_ptr() if t is not None else None
    for case in range(40):
        batch = int(rng.integers(1, 7))
        M, Nn, K = (int(x) for x in rng.integers(1, 700, 3))
        if case % 4 == 0:
            K = int(rng.integers(65, 700))            # several 64-deep steps
        trans_a = bool(rng.integers(0, 2))
        shared_a = bool(rng.integers(0, 2)) and not trans_a
        if case % 5 == 0:
            Nn = 8 * int(rng.integers(1, 9))         # batch folding candidates
        pad = int(rng.integers(0, 3))                 # leading dimensions beyond the matrix
        lda = (M if trans_a else K) + pad
        ldb, ldc = Nn + pad, Nn + pad
        g = torch.Generator().manual_seed(case)
        rows_a = K if trans_a else M
        A = torch.randn(1 if shared_a else batch, rows_a, lda, generator=g)
        Bm = torch.randn(batch, K, ldb, generator=g)
        C0 = torch.randn(batch, M, ldc, generator=g)
        beta = float(rng.choice([0.0, 1.0, 0.5]))
        bias = torch.randn(Nn, generator=g) if rng.integers(0, 2) else None
        Ad, Bd = bf(A).to(dev), bf(Bm).to(dev)
        Cd = C0.to(dev).contiguous()
        st = lib.sg_nn_gemm(batch, M, Nn, K, 1.0, vp(Ad), lda, 0 if shared_a else rows_a * lda, int(trans_a),
                            vp(Bd), ldb, K * ldb, beta, vp(Cd), ldc, M * ldc, None,
                            vp(bias.to(dev)) if bias is not None else None, None)
        assert st == 0, case
        torch.cuda.synchronize()
        Af = bf(A).double()[..., :M] if trans_a else bf(A).double()[..., :K]
        opA = Af.transpose(1, 2) if trans_a else Af
        if shared_a:
            opA = opA.expand(batch, -1, -1)
        ref = opA @ bf(Bm).double()[..., :Nn] + beta * C0.double()[..., :Nn]
        if bias is not None:
            ref = ref + bias.double()
        got = Cd.double().cpu()
        assert (got[..., :Nn] - ref).abs().max() <= 1e-5 * ref.abs().max() * math.sqrt(K) + 1e-6, case
        # columns beyond N (the leading-dimension padding) are untouched
        assert torch.equal(got[..., Nn:], C0.double()[..., Nn:]), case
    assert lib.sg_nn_check(None) == N.SG_OK


def test_gemm_engine_argument_checks():
    lib = N.load()
    assert lib.sg_nn_set_gemm_engine(2) == N.SG_ERR_ARG
    assert lib.sg_nn_set_gemm_engine(-1) == N.SG_ERR_ARG
    assert lib.sg_nn_set_gemm_engine(N.SG_NN_GEMM_TCGEN05) == N.SG_OK


# ---------------------------------------------------------------- network
def reference_loss(S):
    """The surrogate's forward pass and loss in float64 on the CPU (torch
    ops, autograd), from the model's own weights and DFT matrices."""
    Bn, R, P, C, M1, K1 = S.B, S.nr, S.nphi, 32, S.M1, S.K1
    n = Bn * R * P
    d = lambda t: t.detach().double().cpu()
    leaf = {}

    def w(name, use_bf16):
        src = S.P[name]["b"] if use_bf16 else S.P[name]["w"]
        t = d(src).clone().requires_grad_(True)
        leaf[name] = t
        return t

    x = d(S.x)
    tgt = d(S.tgt)
    Fphi, Gr, Hr, Hre, Him = d(S.Fphi), d(S.Gr), d(S.Hr), d(S.Hre), d(S.Him)
    v = x @ w("Pw", True) + w("Pb", False)
    for l in range(4):
        vi = v.reshape(Bn, R, P, C)
        V1 = torch.einsum("jp,brpc->brjc", Fphi, vi)
        T = torch.einsum("kr,brjc->bkjc", Gr, V1)
        Tc, Ts = T[:, :K1], T[:, K1:]
        V2r = Tc[:, :, 0::2] - Ts[:, :, 1::2]
        V2i = Tc[:, :, 1::2] + Ts[:, :, 0::2]
        Sw = w(f"S{l}", False)
        Wr, Wi = Sw[..., 0], Sw[..., 1]
        Or = torch.einsum("bkmi,kmio->bkmo", V2r, Wr) - torch.einsum("bkmi,kmio->bkmo", V2i, Wi)
        Oi = torch.einsum("bkmi,kmio->bkmo", V2r, Wi) + torch.einsum("bkmi,kmio->bkmo", V2i, Wr)
        U1 = torch.einsum("rk,bkmc->brmc", Hr, torch.cat([Or, Oi], dim=1))
        u = torch.einsum("pm,brmc->brpc", Hre, U1[:, :R]) + torch.einsum("pm,brmc->brpc", Him, U1[:, R:])
        pre = u.reshape(n, C) + v @ w(f"W{l}", True) + w(f"b{l}", False)
        v = F.gelu(pre) if l < 3 else pre
    q = F.gelu(v @ w("Q1", True) + w("q1", False))
    out = q @ w("Q2", True) + w("q2", False)
    o, t = out.reshape(Bn, -1, 2), tgt.reshape(Bn, -1, 2)
    loss = (((o - t) ** 2).sum(1) / (t ** 2).sum(1)).mean()
    loss.backward()
    return out.detach(), loss.detach(), {k: v.grad for k, v in leaf.items()}


def rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


@pytest.mark.parametrize("modes_phi,modes_r", [(16, 32), (16, 16)])
def test_forward_and_gradients_match_reference(modes_phi, modes_r):
    """Both retained-mode sizes (16 azimuthal x 32 radial, and 16 x 16), with
    every GEMM on the tcgen05 engine."""
    from paper_2506_10812_gb300.surrogate import Surrogate
    S = Surrogate(nr=32, nphi=64, batch=2, seed=3, modes_phi=modes_phi, modes_r=modes_r)
    S.load([11, 12])
    S.forward()
    L, _ = S.loss(grad=True)
    S.backward()
    torch.cuda.synchronize()
    out, Lref, grads = reference_loss(S)
    assert rel(S.out.double().cpu(), out) < 3e-2
    assert abs(L - float(Lref)) < 3e-2 * float(Lref)
    for name, g in grads.items():
        got = S.P[name]["g"].double().cpu().reshape(g.shape)
        assert rel(got, g) < 1e-1, (name, rel(got, g))
    assert N.load().sg_nn_check(None) == N.SG_OK


def test_training_lowers_the_loss_and_gate():
    from paper_2506_10812_gb300 import Plan
    from paper_2506_10812_gb300.surrogate import GATE, Surrogate
    S = Surrogate(nr=32, nphi=64, batch=2, seed=5)
    hist = S.train(60, lr=3e-3, seed0=100)
    assert np.mean(hist[-10:]) < 0.5 * np.mean(hist[:5])
    rel_val = S.validate([900, 901, 902, 903])
    assert S.val_error == pytest.approx(float(np.max(rel_val)))
    # above the gate: the exact path, bit for bit
    S.val_error = 10 * GATE
    S.load([77, 78])
    h_g, St = 0.05, 0.1
    gr, gphi, used = S.solve(S.sg[0].clone(), S.sd[0].clone(), h_g, St)
    assert not used
    p = S._plan(h_g, St)
    ref = p.solve(S.sg[0].clone(), S.sd[0].clone(), outputs=("gr", "gphi"))
    assert torch.equal(gr, ref["gr_g"]) and torch.equal(gphi, ref["gphi_g"])
    # within the gate: the network's fields
    S.val_error = 0.0
    gr2, gphi2, used2 = S.solve(S.sg[0].clone(), S.sd[0].clone(), h_g, St)
    assert used2 and torch.isfinite(gr2).all() and not torch.equal(gr2, gr)
