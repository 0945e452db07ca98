"""Spectral neural-operator surrogate of the field solve, trained on fields the
exact FFT path labels and gated against it.

The network maps (Sigma_g, Sigma_d, h_g, h_d) on the log-polar grid to the
gas accelerations (g_r, g_phi):

    lifting   v0 = x P + p                      (7 input channels -> C = 32)
    4 layers  v_{l+1} = act(S_l(v_l) + v_l W_l + b_l)   (act = GELU, none last)
    output    y = GELU(v4 Q1 + q1) Q2 + q2       (C -> 64 -> 2)

where S_l is a spectral convolution that keeps M1 azimuthal modes m and K1
radial modes k (K1 / 2 non-negative, K1 / 2 negative; defaults 16 and 32,
and 16 x 16 as the other studied size): a truncated DFT along phi and r, a
complex C x C channel mix per kept mode, and the inverse truncated DFT.  With truncated modes every transform is a product with a fixed DFT
matrix, so the forward and backward passes are batched BF16 tensor-core
GEMMs (sg_nn_gemm, FP32 accumulation) plus the mode-mixing, activation and
loss kernels of sg_nn.cu; weights are FP32 masters with BF16 copies and
Adam.  This module only sequences library calls (argument marshalling).

`Surrogate.solve` returns the network's fields when its validation error
(relative L2 against the exact path, worst channel) is at or below the gate
(1e-3), and otherwise the exact path's fields.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _native as N
from .plan import Plan

C = 32            # width
M1 = 16           # azimuthal modes kept (default)
K1 = 32           # radial modes kept (default; half non-negative, half negative)
CIN = 7
QH = 64           # projection hidden width
NF = 32           # random Fourier features of the training fields
NPAR = 8 + 4 * NF + 12 + 12
GATE = 1e-3
ALPHA_DUST = 1e-3


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class _Lib:
    def __init__(self, device):
        self.lib = N.load()
        self.device = device
        self.count = None      # when a dict: launches, GEMM flops and operand bytes are tallied into it

    def _s(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def call(self, name, *args):
        st = getattr(self.lib, name)(*args, self._s())
        N.check(st, None, name)
        if self.count is not None:
            self.count["launches"] = self.count.get("launches", 0) + 1

    def gemm(self, batch, M, Nn, K, A, lda, sa, B, ldb, sb, C=None, ldc=0, sc=0, Cb=None, alpha=1.0, beta=0.0,
             bias=None, trans_a=False, a_off=0):
        Ap = ctypes.c_void_p(A.data_ptr() + a_off * A.element_size())
        self.call("sg_nn_gemm", batch, M, Nn, K, alpha, Ap, lda, sa, 1 if trans_a else 0, _p(B), ldb, sb, beta,
                  _p(C), ldc, sc, _p(Cb), _p(bias))
        if self.count is not None:
            c = self.count
            c["gemm_flops"] = c.get("gemm_flops", 0) + 2 * batch * M * Nn * K
            # each operand once: broadcast (stride 0) operands count once for the batch
            nb = (batch if sa else 1) * M * K * 2 + (batch if sb else 1) * K * Nn * 2
            nb += batch * M * Nn * ((4 if C is not None else 0) + (4 if beta != 0 else 0) +
                                    (2 if Cb is not None else 0))
            c["gemm_bytes"] = c.get("gemm_bytes", 0) + nb
            c["gemms"] = c.get("gemms", 0) + 1


def field_params(seed, nr, nphi, r_in, r_out):
    """Per-sample parameters of one C5 training field (seeded numpy)."""
    rng = np.random.default_rng(seed)
    du = math.log(r_out / r_in) / nr
    q = np.zeros(NPAR, dtype=np.float32)
    q[0], q[1], q[2] = math.log(r_in), du, 2 * math.pi / nphi
    q[3] = rng.uniform(0.2, 0.4)                      # log-normal width
    q[4] = rng.uniform(0.005, 0.02)                   # dust-to-gas ratio
    q[5] = np.array([rng.integers(1, 2**31)], dtype=np.uint32).view(np.float32)[0]
    q[6] = 1.0 / math.tan(math.radians(rng.uniform(10.0, 25.0)))
    f = q[8:8 + 4 * NF].reshape(NF, 4)
    f[:, 0] = rng.normal(0.0, 2 * math.pi / (12 * du), NF)        # radial wavenumber (~12-cell correlation)
    f[:, 1] = np.round(rng.normal(0.0, 8.0, NF))                  # integer azimuthal wavenumber
    f[:, 2] = math.sqrt(2.0 / NF)
    f[:, 3] = rng.uniform(0, 2 * math.pi, NF)
    sp = q[8 + 4 * NF:8 + 4 * NF + 12].reshape(6, 2)
    sp[:, 0] = rng.uniform(0.0, 0.08, 6)
    sp[:, 1] = rng.uniform(0, 2 * math.pi, 6)
    cl = q[8 + 4 * NF + 12:].reshape(3, 4)
    rc, pc = rng.uniform(0.5, 3.0, 3), rng.uniform(0, 2 * math.pi, 3)
    cl[:, 0], cl[:, 1] = rc * np.cos(pc), rc * np.sin(pc)
    cl[:, 2] = rng.uniform(0.0, 5.0, 3)
    cl[:, 3] = rng.uniform(0.05, 0.25, 3)
    h_g = float(rng.choice([0.03, 0.05, 0.07, 0.1]))
    St = float(rng.choice([0.01, 0.1, 1.0]))
    return q, h_g, St


class Surrogate:
    """Spectral neural operator on an nr x nphi grid (C5: 512 x 1024)."""

    def __init__(self, nr=512, nphi=1024, r_in=0.1, r_out=5.0, G=1.0, batch=2, seed=0, device=None,
                 modes_phi=M1, modes_r=K1):
        if modes_r % 2 or not (2 <= modes_r <= nr) or not (1 <= modes_phi <= nphi // 2):
            raise ValueError("modes_r must be even and <= nr, modes_phi <= nphi / 2")
        self.M1, self.K1 = int(modes_phi), int(modes_r)
        self.dev = torch.device("cuda") if device is None else torch.device(device)
        if self.dev.index is None:
            self.dev = torch.device("cuda", torch.cuda.current_device())
        self.nr, self.nphi, self.r_in, self.r_out, self.G, self.B = nr, nphi, r_in, r_out, G, batch
        self.npix = nr * nphi
        self.k = _Lib(self.dev)
        self.plans = {}
        self.val_error = math.inf
        self.step_count = 0
        rng = np.random.default_rng(seed)
        f32 = dict(dtype=torch.float32, device=self.dev)
        bf = dict(dtype=torch.bfloat16, device=self.dev)

        def param(shape, scale):
            w = torch.tensor(rng.normal(0.0, scale, shape).astype(np.float32), **f32)
            return {"w": w, "m": torch.zeros_like(w), "v": torch.zeros_like(w), "g": torch.zeros_like(w),
                    "b": torch.empty(shape, **bf) if len(shape) == 2 else None}

        self.P = {"Pw": param((CIN, C), 1 / math.sqrt(CIN)), "Pb": param((C,), 0.0),
                  "Q1": param((C, QH), 1 / math.sqrt(C)), "q1": param((QH,), 0.0),
                  "Q2": param((QH, 2), 0.1 / math.sqrt(QH)), "q2": param((2,), 0.0)}
        for l in range(4):
            self.P[f"W{l}"] = param((C, C), 1 / math.sqrt(C))
            self.P[f"b{l}"] = param((C,), 0.0)
            sw = param((self.K1, self.M1, C, C, 2), 0.5 / C)
            self.P[f"S{l}"] = sw
        for v in self.P.values():
            if v["b"] is not None:
                self.k.call("sg_nn_cast", v["w"].numel(), _p(v["w"]), _p(v["b"]))
        self._build_dft()
        self._alloc()

    # ------------------------------------------------------------ constants
    def _bf(self, a):
        t = torch.tensor(np.ascontiguousarray(a, dtype=np.float32), dtype=torch.float32, device=self.dev)
        out = torch.empty(t.shape, dtype=torch.bfloat16, device=self.dev)
        self.k.call("sg_nn_cast", t.numel(), _p(t), _p(out))
        return out

    def _build_dft(self):
        M1, K1 = self.M1, self.K1
        R, Pn = self.nr, self.nphi
        p = np.arange(Pn)
        m = np.arange(M1)
        ang = 2 * np.pi * np.outer(m, p) / Pn                        # [M1][P]
        Fphi = np.empty((2 * M1, Pn))
        Fphi[0::2], Fphi[1::2] = np.cos(ang) / Pn, -np.sin(ang) / Pn  # rows 2m (re), 2m+1 (im)
        h = K1 // 2
        kv = np.concatenate([np.arange(h), np.arange(R - h, R)])     # kept radial frequencies
        r = np.arange(R)
        angr = 2 * np.pi * np.outer(kv, r) / R                       # [K1][R]
        Gr = np.concatenate([np.cos(angr), -np.sin(angr)]) / R       # [2 K1][R]
        Hr = np.block([[np.cos(angr).T, -np.sin(angr).T], [np.sin(angr).T, np.cos(angr).T]])   # [2R][2 K1]
        w = np.where(m == 0, 1.0, 2.0)
        Hre = np.cos(ang).T * w                                      # [P][M1]
        Him = -np.sin(ang).T * w
        self.Fphi, self.FphiT = self._bf(Fphi), self._bf(Fphi.T)
        self.Gr, self.GrT = self._bf(Gr), self._bf(Gr.T)
        self.Hr, self.HrT = self._bf(Hr), self._bf(Hr.T)
        self.Hre, self.Him = self._bf(Hre), self._bf(Him)
        self.HreT, self.HimT = self._bf(Hre.T), self._bf(Him.T)

    def _alloc(self):
        M1, K1 = self.M1, self.K1
        B, R, Pn, n = self.B, self.nr, self.nphi, self.B * self.npix
        f32 = dict(dtype=torch.float32, device=self.dev)
        bf = dict(dtype=torch.bfloat16, device=self.dev)
        self.x = torch.empty((n, CIN), **bf)
        self.v = [torch.empty((n, C), **bf) for _ in range(5)]
        self.pre = [torch.empty((n, C), **f32) for _ in range(5)]      # pre[4]: lifting output
        self.V1 = torch.empty((B * R, 2 * M1, C), **bf)
        self.T = torch.empty((B, 2 * K1, 2 * M1 * C), **f32)
        self.V2 = [torch.empty((B, K1, M1, C, 2), **f32) for _ in range(4)]
        self.O = torch.empty((B, 2, K1, M1, C), **bf)
        self.U1 = torch.empty((2, B * R, M1, C), **bf)
        self.qpre = torch.empty((n, QH), **f32)
        self.q = torch.empty((n, QH), **bf)
        self.out = torch.empty((n, 2), **f32)
        self.tgt = torch.empty((n, 2), **f32)
        self.stats = torch.empty((B * 2 * 2,), **f32)
        # backward
        self.dout = torch.empty((n, 2), **f32)
        self.dout_b = torch.empty((n, 2), **bf)
        self.dq = torch.empty((n, QH), **f32)
        self.dq_b = torch.empty((n, QH), **bf)
        self.dv = torch.empty((n, C), **f32)
        self.dv2 = torch.empty((n, C), **f32)
        self.dpre_b = torch.empty((n, C), **bf)
        self.dU1 = torch.empty((2, B * R, M1, C), **bf)
        self.dO = torch.empty((B, 2, K1, M1, C), **f32)
        self.dV2 = torch.empty((B, K1, M1, C, 2), **f32)
        self.dT = torch.empty((B, 2 * K1, 2 * M1 * C), **bf)
        self.dV1 = torch.empty((B * R, 2 * M1, C), **bf)
        self.nsplit = 512
        self.part = torch.empty((self.nsplit, QH * C), **f32)
        self.WT = torch.empty((QH * C,), **bf)
        self.sg = torch.empty((B, R, Pn), **f32)
        self.sd = torch.empty((B, R, Pn), **f32)
        self.gr = torch.empty((B, R, Pn), **f32)
        self.gphi = torch.empty((B, R, Pn), **f32)
        self.per = torch.empty((B, 4), **f32)
        self.scale = torch.empty((B,), **f32)
        self.sums = torch.empty((1,), **f32)

    # ------------------------------------------------------------ forward
    def _spectral(self, l, v, pre):
        M1, K1 = self.M1, self.K1
        k, B, R, Pn = self.k, self.B, self.nr, self.nphi
        k.gemm(B * R, 2 * M1, C, Pn, self.Fphi, Pn, 0, v, C, Pn * C, Cb=self.V1, ldc=C, sc=2 * M1 * C)
        k.gemm(B, 2 * K1, 2 * M1 * C, R, self.Gr, R, 0, self.V1, 2 * M1 * C, R * 2 * M1 * C, C=self.T,
               ldc=2 * M1 * C, sc=2 * K1 * 2 * M1 * C)
        k.call("sg_nn_spec_combine", B, K1, M1, C, _p(self.T), _p(self.V2[l]))
        k.call("sg_nn_modemix", B, K1, M1, C, _p(self.V2[l]), _p(self.P[f"S{l}"]["w"]), _p(self.O))
        for ri in range(2):   # U1[ri] = Hr[ri R : (ri + 1) R] O[b]
            k.gemm(B, R, M1 * C, 2 * K1, self.Hr, 2 * K1, 0, self.O, M1 * C, 2 * K1 * M1 * C,
                   Cb=self.U1[ri], ldc=M1 * C, sc=R * M1 * C, a_off=ri * R * 2 * K1)
        k.gemm(B * R, Pn, C, M1, self.Hre, M1, 0, self.U1[0], C, M1 * C, C=pre, ldc=C, sc=Pn * C)
        k.gemm(B * R, Pn, C, M1, self.Him, M1, 0, self.U1[1], C, M1 * C, C=pre, ldc=C, sc=Pn * C, beta=1.0)

    def forward(self):
        """x -> out (FP32 [B npix][2]); keeps the activations for backward."""
        k, n = self.k, self.B * self.npix
        k.gemm(1, n, C, CIN, self.x, CIN, 0, self.P["Pw"]["b"], C, 0, C=self.pre[4], ldc=C,
               bias=self.P["Pb"]["w"])
        k.call("sg_nn_act", n * C, _p(self.pre[4]), _p(self.v[0]), 0)
        for l in range(4):
            self._spectral(l, self.v[l], self.pre[l])
            k.gemm(1, n, C, C, self.v[l], C, 0, self.P[f"W{l}"]["b"], C, 0, C=self.pre[l], ldc=C, beta=1.0,
                   bias=self.P[f"b{l}"]["w"])
            k.call("sg_nn_act", n * C, _p(self.pre[l]), _p(self.v[l + 1]), 1 if l < 3 else 0)
        k.gemm(1, n, QH, C, self.v[4], C, 0, self.P["Q1"]["b"], QH, 0, C=self.qpre, ldc=QH, bias=self.P["q1"]["w"])
        k.call("sg_nn_act", n * QH, _p(self.qpre), _p(self.q), 1)
        k.gemm(1, n, 2, QH, self.q, QH, 0, self.P["Q2"]["b"], 2, 0, C=self.out, ldc=2, bias=self.P["q2"]["w"])

    # ------------------------------------------------------------ backward
    def _wgrad(self, A, Mm, Bm, Nn, name):
        """dW = A^T B over all rows, split along K in nsplit chunks."""
        k, n = self.k, self.B * self.npix
        kc = n // self.nsplit
        k.gemm(self.nsplit, Mm, Nn, kc, A, Mm, kc * Mm, Bm, Nn, kc * Nn, C=self.part, ldc=Nn, sc=Mm * Nn,
               trans_a=True)
        k.call("sg_nn_colsum", self.nsplit, Mm * Nn, _p(self.part), _p(self.P[name]["g"]), 0)

    def _transpose(self, name, rows, cols):
        self.k.call("sg_nn_transpose", rows, cols, _p(self.P[name]["w"]), _p(self.WT))
        return self.WT

    def backward(self):
        M1, K1 = self.M1, self.K1
        k, B, R, Pn, n = self.k, self.B, self.nr, self.nphi, self.B * self.npix
        k.call("sg_nn_cast", n * 2, _p(self.dout), _p(self.dout_b))
        self._wgrad(self.q, QH, self.dout_b, 2, "Q2")
        k.call("sg_nn_colsum", n, 2, _p(self.dout), _p(self.P["q2"]["g"]), 0)
        k.gemm(1, n, QH, 2, self.dout_b, 2, 0, self._transpose("Q2", QH, 2), QH, 0, C=self.dq, ldc=QH)
        k.call("sg_nn_act_bwd", n * QH, _p(self.qpre), _p(self.dq), _p(self.dq), _p(self.dq_b), 1)
        self._wgrad(self.v[4], C, self.dq_b, QH, "Q1")
        k.call("sg_nn_colsum", n, QH, _p(self.dq), _p(self.P["q1"]["g"]), 0)
        k.gemm(1, n, C, QH, self.dq_b, QH, 0, self._transpose("Q1", C, QH), C, 0, C=self.dv, ldc=C)
        for l in (3, 2, 1, 0):
            # d pre_l (FP32 in dv, in place) and its BF16 copy
            k.call("sg_nn_act_bwd", n * C, _p(self.pre[l]), _p(self.dv), _p(self.dv), _p(self.dpre_b),
                   1 if l < 3 else 0)
            self._wgrad(self.v[l], C, self.dpre_b, C, f"W{l}")
            k.call("sg_nn_colsum", n, C, _p(self.dv), _p(self.P[f"b{l}"]["g"]), 0)
            k.gemm(1, n, C, C, self.dpre_b, C, 0, self._transpose(f"W{l}", C, C), C, 0, C=self.dv2, ldc=C)
            # spectral path
            k.gemm(B * R, M1, C, Pn, self.HreT, Pn, 0, self.dpre_b, C, Pn * C, Cb=self.dU1[0], ldc=C, sc=M1 * C)
            k.gemm(B * R, M1, C, Pn, self.HimT, Pn, 0, self.dpre_b, C, Pn * C, Cb=self.dU1[1], ldc=C, sc=M1 * C)
            for ri in range(2):   # dO[b] += HrT[:, ri R : (ri + 1) R] dU1[ri][b]
                k.gemm(B, 2 * K1, M1 * C, R, self.HrT, 2 * R, 0, self.dU1[ri], M1 * C, R * M1 * C, C=self.dO,
                       ldc=M1 * C, sc=2 * K1 * M1 * C, beta=float(ri), a_off=ri * R)
            k.call("sg_nn_modemix_bwd", B, K1, M1, C, _p(self.V2[l]), _p(self.P[f"S{l}"]["w"]), _p(self.dO),
                   _p(self.dV2), _p(self.P[f"S{l}"]["g"]))
            k.call("sg_nn_spec_combine_bwd", B, K1, M1, C, _p(self.dV2), _p(self.dT))
            k.gemm(B, R, 2 * M1 * C, 2 * K1, self.GrT, 2 * K1, 0, self.dT, 2 * M1 * C, 2 * K1 * 2 * M1 * C,
                   Cb=self.dV1, ldc=2 * M1 * C, sc=R * 2 * M1 * C)
            k.gemm(B * R, Pn, C, 2 * M1, self.FphiT, 2 * M1, 0, self.dV1, C, 2 * M1 * C, C=self.dv2, ldc=C,
                   sc=Pn * C, beta=1.0)
            self.dv, self.dv2 = self.dv2, self.dv
        # lifting (no activation): dv is d pre[4]
        k.call("sg_nn_cast", n * C, _p(self.dv), _p(self.dpre_b))
        self._wgrad(self.x, CIN, self.dpre_b, C, "Pw")
        k.call("sg_nn_colsum", n, C, _p(self.dv), _p(self.P["Pb"]["g"]), 0)

    def adam(self, lr):
        self.step_count += 1
        for v in self.P.values():
            self.k.call("sg_nn_adam", v["w"].numel(), _p(v["w"]), _p(v["g"]), _p(v["m"]), _p(v["v"]), lr, 0.9,
                        0.999, 1e-8, self.step_count, _p(v["b"]))

    # ------------------------------------------------------------ data
    def _plan(self, h_g, St):
        key = (h_g, St)
        if key not in self.plans:
            self.plans[key] = Plan(self.nr, self.nphi, self.r_in, self.r_out, h_g,
                                   h_g * math.sqrt(ALPHA_DUST / (ALPHA_DUST + St)), G=self.G, device=self.dev)
        return self.plans[key]

    def _sum(self, t):
        self.k.call("sg_nn_colsum", t.numel(), 1, _p(t), _p(self.sums), 0)
        return float(self.sums.item())

    def load(self, seeds):
        """Generate the fields of `seeds` (len B), label them with the exact
        path, and pack network inputs and targets."""
        B = self.B
        params, hs = [], []
        for s in seeds:
            q, h_g, St = field_params(int(s), self.nr, self.nphi, self.r_in, self.r_out)
            params.append(q)
            hs.append((h_g, St))
        pt = torch.tensor(np.stack(params), dtype=torch.float32, device=self.dev)
        self.k.call("sg_nn_fields", B, self.nr, self.nphi, _p(pt), _p(self.sg), _p(self.sd))
        per, scale = np.zeros((B, 4), np.float32), np.zeros(B, np.float32)
        for b, (h_g, St) in enumerate(hs):
            plan = self._plan(h_g, St)
            plan.solve(self.sg[b], self.sd[b], out={"gr_g": self.gr[b], "gphi_g": self.gphi[b]})
            mg = self._sum(self.sg[b]) / self.npix
            per[b] = (1.0 / mg, 50.0 / mg, h_g / 0.05, plan.h_d / 0.05)
            scale[b] = 1.0 / (self.G * mg)
        self.per.copy_(torch.from_numpy(per))
        self.scale.copy_(torch.from_numpy(scale))
        self.k.call("sg_nn_pack_inputs", B, self.nr, self.nphi, _p(self.sg), _p(self.sd), _p(self.per), _p(self.x))
        self.k.call("sg_nn_pack_targets", B, self.npix, _p(self.gr), _p(self.gphi), _p(self.scale), _p(self.tgt), 0)
        return hs

    def loss(self, grad=True):
        """Mean over samples and channels of |pred - target|^2 / |target|^2;
        with grad also d loss / d out into self.dout.  Returns (loss, per
        (sample, channel) relative L2)."""
        self.k.call("sg_nn_rel_l2", self.B, self.npix, 2, _p(self.out), _p(self.tgt), _p(self.stats),
                    _p(self.dout) if grad else None)
        st = self.stats.view(self.B, 2, 2).cpu().numpy()
        rel = np.sqrt(st[..., 0] / st[..., 1])
        return float(np.mean(st[..., 0] / st[..., 1])), rel

    def train(self, steps, lr=1e-3, seed0=1000, log=None):
        """`steps` Adam steps on fresh seeded fields (B per step; seeds
        seed0 + B step + b), cosine-decayed learning rate."""
        hist = []
        for s in range(steps):
            self.load([seed0 + self.B * s + b for b in range(self.B)])
            self.forward()
            L, rel = self.loss(grad=True)
            self.backward()
            self.adam(lr * 0.5 * (1 + math.cos(math.pi * s / max(steps, 1))))
            hist.append(L)
            if log and (s % log == 0 or s == steps - 1):
                print(f"step {s:5d} loss {L:.4e} rel-L2 {rel.mean(axis=0)}", flush=True)
        return hist

    def validate(self, seeds):
        """Relative L2 against the exact path on held-out seeds, per channel
        (g_r, g_phi); sets val_error = the worse channel's mean."""
        rels = []
        for i in range(0, len(seeds), self.B):
            self.load(seeds[i:i + self.B])
            self.forward()
            rels.append(self.loss(grad=False)[1])
        rel = np.concatenate(rels).mean(axis=0)
        self.val_error = float(rel.max())
        return rel

    def solve(self, sigma_g, sigma_d, h_g, St):
        """(g_r, g_phi) of the gas for one disc: the network's fields if the
        validated error is within the gate, else the exact FFT path's.
        Returns (g_r, g_phi, used_surrogate)."""
        plan = self._plan(h_g, St)
        if not self.val_error <= GATE:
            out = plan.solve(sigma_g, sigma_d, outputs=("gr", "gphi"))
            return out["gr_g"], out["gphi_g"], False
        self.sg[0].copy_(sigma_g)
        self.sd[0].copy_(sigma_d)
        mg = self._sum(self.sg[0]) / self.npix
        per = np.zeros((self.B, 4), np.float32)
        per[:] = (1.0 / mg, 50.0 / mg, h_g / 0.05, plan.h_d / 0.05)
        self.per.copy_(torch.from_numpy(per))
        self.scale.copy_(torch.full((self.B,), 1.0 / (self.G * mg), dtype=torch.float32))
        self.k.call("sg_nn_pack_inputs", self.B, self.nr, self.nphi, _p(self.sg), _p(self.sd), _p(self.per),
                    _p(self.x))
        self.forward()
        self.k.call("sg_nn_pack_targets", self.B, self.npix, _p(self.gr), _p(self.gphi), _p(self.scale),
                    _p(self.out), 1)
        return self.gr[0].clone(), self.gphi[0].clone(), True
