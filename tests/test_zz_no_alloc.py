"""sg_direct_noalloc: the direct pair sum for callers that cannot let a
library allocate device memory (device memory owned by the host code's own
allocator or pool, or loops that must not enter the CUDA allocator).  It
keeps its scratch in a fixed array inside the library instead of a plan.

Checked through the C ABI against the plan-based entry point (sg_solve of a
DIRECT plan) on two calls in a row, with the tolerances of the other parity
tests, and checked to leave the device's free memory unchanged.  This file
is collected last so that a stop-at-first-failure run has already run every
other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2506_10812_gb300 import _native as N
from paper_2506_10812_gb300 import build as B
from paper_2506_10812_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {torch.float64: (1e-11, 1e-11), torch.float32: (1e-5, 1e-4)}
KEYS = ("phi_g", "gr_g", "gphi_g", "phi_d", "gr_d", "gphi_d")


def params_of(d, dtype):
    p = N.SgParams()
    p.nr, p.nphi, p.r_in, p.r_out = d.nr, d.nphi, d.r_in, d.r_out
    p.h_g, p.h_d = d.h_g, (d.h_d or 0.0)
    p.G = d.G
    p.dtype = N.SG_F64 if dtype == torch.float64 else N.SG_F32
    p.method = N.SG_METHOD_DIRECT
    return p


def rel(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return np.linalg.norm(a - b) / np.linalg.norm(b), np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_direct_matches_plan_two_calls(cuda_device, dtype):
    B.build()
    lib = N.load()
    from paper_2506_10812_gb300 import Plan
    discs = [inputs.ragged_noise(24, 48, bifluid=True), inputs.small_gas(nr=16, nphi=32)]
    dev = cuda_device
    ref, tens, outs = [], [], []
    for d in discs:
        sg = torch.tensor(d.sigma_g, dtype=dtype, device=dev)
        sd = None if d.sigma_d is None else torch.tensor(d.sigma_d, dtype=dtype, device=dev)
        with Plan(d.nr, d.nphi, d.r_in, d.r_out, d.h_g, d.h_d, G=d.G, dtype=dtype, method="direct",
                  device=dev) as plan:
            ref.append(plan.solve(sg, sd))
        tens.append((sg, sd))
        outs.append({k: torch.full((d.nr, d.nphi), float("nan"), dtype=dtype, device=dev) for k in ref[-1]})
    torch.cuda.synchronize()
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)

    def call(i):
        d, (sg, sd), out = discs[i], tens[i], outs[i]
        ptr = [ctypes.c_void_p(out[k].data_ptr()) if k in out else None for k in KEYS]
        p = params_of(d, dtype)
        st = lib.sg_direct_noalloc(ctypes.byref(p), ctypes.c_void_p(sg.data_ptr()),
                                   None if sd is None else ctypes.c_void_p(sd.data_ptr()), *ptr, stream)
        assert st == N.SG_OK

    call(1)                                   # first call on this device: address lookup, kernel load
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    call(0)                                   # two calls in a row, different grids and fluids
    call(1)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0
    for r, o in zip(ref, outs):
        for k, v in r.items():
            e2, em = rel(o[k], v)
            assert e2 <= TOL[dtype][0] and em <= TOL[dtype][1], (k, e2, em)


def test_noalloc_rejects_oversize_grid(cuda_device):
    lib = N.load()
    d = inputs.small_gas()
    p = params_of(d, torch.float32)
    p.nr, p.nphi = 2048, 64
    x = torch.ones((8, 8), device=cuda_device)
    assert lib.sg_direct_noalloc(ctypes.byref(p), ctypes.c_void_p(x.data_ptr()), None,
                                 ctypes.c_void_p(x.data_ptr()), None, None, None, None, None, None) \
        == N.SG_ERR_UNSUPPORTED
    p.nr, p.nphi, p.method = 16, 32, N.SG_METHOD_FFT
    assert lib.sg_direct_noalloc(ctypes.byref(p), ctypes.c_void_p(x.data_ptr()), None,
                                 ctypes.c_void_p(x.data_ptr()), None, None, None, None, None, None) == N.SG_ERR_ARG
