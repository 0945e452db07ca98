"""GPU tests of the tensor-core column engines (split-precision DFT-as-GEMM
stages, the precision study of the FFT path): error against the FP64 oracle
on the precision-study discs, agreement with the FP32 FFT engine, the
single-term modes' larger error, and the engine's argument checks."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_10812_gb300 import _native as N
from paper_2506_10812_gb300 import build as B
from paper_2506_10812_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL32 = (1e-5, 1e-4)


@pytest.fixture(scope="module", autouse=True)
def built(cuda_device):
    B.build()
    N.load()
    oracle.build()


def rounded(d):
    import copy
    e = copy.copy(d)
    e.sigma_g = d.sigma_g.astype(np.float32).astype(np.float64)
    return e


def solve(d, engine):
    from paper_2506_10812_gb300 import Plan
    dev = torch.device("cuda:0")
    with Plan(d.nr, d.nphi, d.r_in, d.r_out, d.h_g, None, G=d.G, device=dev) as plan:
        plan.set_column_engine(engine)
        assert plan.launches_per_solve() == (3 if engine == "fft32" else 4)
        sg = torch.tensor(d.sigma_g, dtype=torch.float32, device=dev)
        out = plan.solve(sg)
        plan.sync()
        return {k: v.double().cpu().numpy() for k, v in out.items()}


def errors(out, ref):
    return {k: (oracle.rel_l2(v, ref[k]), oracle.rel_max(v, ref[k])) for k, v in out.items()}


@pytest.fixture(scope="module")
def disc_1024():
    d = rounded(inputs.lognormal_gas(1024, 2048))
    ref = oracle.fft64(oracle.Grid(d.nr, d.nphi, d.r_in, d.r_out), d.sigma_g, h_g=d.h_g, G=d.G)
    return d, ref


def test_fp16x3_meets_fp32_tolerance(disc_1024):
    """FP16 hi + lo operands, three products, FP32 accumulation: the FP32
    tolerance against the FP64 oracle (Phi, g_r, g_phi)."""
    d, ref = disc_1024
    err = errors(solve(d, "dft_fp16x3"), ref)
    for k, (e2, em) in err.items():
        assert e2 <= TOL32[0] and em <= TOL32[1], (k, e2, em)


def test_engines_against_fft32_and_oracle(disc_1024):
    """Every engine against the FP32 FFT engine and the oracle: the split
    modes stay within 10x the FP32 tolerance of the oracle; a single FP16 or
    BF16 product is orders of magnitude worse (what the split recovers)."""
    d, ref = disc_1024
    base = errors(solve(d, "fft32"), ref)
    for k, (e2, em) in base.items():
        assert e2 <= TOL32[0] and em <= TOL32[1], ("fft32", k, e2, em)
    split = {e: errors(solve(d, e), ref) for e in ("dft_fp16x3", "dft_bf16x3")}
    single = {e: errors(solve(d, e), ref) for e in ("dft_fp16", "dft_bf16")}
    for e, err in split.items():
        for k, (e2, em) in err.items():
            assert e2 <= 10 * TOL32[0] and em <= 10 * TOL32[1], (e, k, e2, em)
    for e, err in single.items():
        worst = max(e2 for e2, _ in err.values())
        assert worst > 10 * max(max(e2 for e2, _ in s.values()) for s in split.values()), (e, err)


def test_fp16x3_full_size():
    """2048 x 4096 (column length 4096: three radix-16 stages)."""
    d = rounded(inputs.lognormal_gas(2048, 4096))
    ref = oracle.fft64(oracle.Grid(d.nr, d.nphi, d.r_in, d.r_out), d.sigma_g, h_g=d.h_g, G=d.G)
    err = errors(solve(d, "dft_fp16x3"), ref)
    for k, (e2, em) in err.items():
        assert e2 <= TOL32[0] and em <= TOL32[1], (k, e2, em)


@pytest.mark.parametrize("engine", ["tc_bf16x3", "tc_tf32x3", "tc_fp16x3"])
def test_tcgen05_split_engines_meet_fp32_tolerance(disc_1024, engine):
    """tcgen05 engines (each radix-16 DFT one tensor-core product per
    128-butterfly tile: operands in tensor and shared memory, FP32
    accumulators in tensor memory; BF16, TF32 or FP16 (per-tile power-of-two
    scaling) hi + lo operands, three products): the FP32 tolerance against
    the FP64 oracle at 1024 x 2048 (column length 2048: two radix-16 stages
    on the tensor cores)."""
    d, ref = disc_1024
    err = errors(solve(d, engine), ref)
    for k, (e2, em) in err.items():
        assert e2 <= TOL32[0] and em <= TOL32[1], (engine, k, e2, em)


def test_tcgen05_single_product_is_worse(disc_1024):
    """One BF16 product on the tcgen05 path is orders of magnitude less
    accurate than the split engines: what the hi + lo split recovers."""
    d, ref = disc_1024
    split = max(e2 for e2, _ in errors(solve(d, "tc_bf16x3"), ref).values())
    single = max(e2 for e2, _ in errors(solve(d, "tc_bf16"), ref).values())
    assert single > 10 * split, (single, split)


@pytest.mark.parametrize("engine", ["tc_bf16x3", "tc_tf32x3", "tc_fp16x3"])
def test_tcgen05_full_size(engine):
    """2048 x 4096 (column length 4096: all three radix-16 stages on the
    tensor cores, two 128-butterfly tiles per product)."""
    d = rounded(inputs.lognormal_gas(2048, 4096))
    ref = oracle.fft64(oracle.Grid(d.nr, d.nphi, d.r_in, d.r_out), d.sigma_g, h_g=d.h_g, G=d.G)
    err = errors(solve(d, engine), ref)
    for k, (e2, em) in err.items():
        assert e2 <= TOL32[0] and em <= TOL32[1], (engine, k, e2, em)


def test_engine_argument_checks():
    from paper_2506_10812_gb300 import Plan
    dev = torch.device("cuda:0")
    d = inputs.ragged_noise(512, 64)
    with Plan(d.nr, d.nphi, d.r_in, d.r_out, d.h_g, None, device=dev) as plan:
        for engine in ("dft_fp16x3", "tc_bf16x3"):
            with pytest.raises(N.SgError) as ei:
                plan.set_column_engine(engine)               # nr = 512
            assert ei.value.status == N.SG_ERR_UNSUPPORTED
        assert plan._lib.sg_set_column_engine(plan._h, 9) == N.SG_ERR_ARG
    with Plan(1024, 64, 0.1, 5.0, 0.05, 0.01, device=dev) as plan:  # gas + dust
        with pytest.raises(N.SgError) as ei:
            plan.set_column_engine("dft_bf16x3")
        assert ei.value.status == N.SG_ERR_UNSUPPORTED
    with Plan(1024, 64, 0.1, 5.0, 0.05, dtype=torch.float64, device=dev) as plan:
        with pytest.raises(N.SgError) as ei:
            plan.set_column_engine("dft_fp16")
        assert ei.value.status == N.SG_ERR_UNSUPPORTED


@pytest.mark.parametrize("engine,tol", [("tc_bf16x3", 5e-5), ("tc_tf32x3", 5e-6), ("tc_fp16x3", 5e-6),
                                        ("tc_bf16", None)])
@pytest.mark.parametrize("inverse", [False, True])
def test_tcgen05_single_stage_against_fp64_dft(engine, tol, inverse):
    """One radix-16 stage of each tcgen05 engine alone (sg_tc_dft16): 4096
    seeded 16-point DFTs against float64 DFTs.  Each 128-DFT tile (one
    tensor-core product) has its own magnitude, the 32 tiles spanning six
    decades, which exercises the FP16 engine's per-tile scaling; the error
    of each output sequence is measured against its own largest value.  The
    single BF16 product is orders of magnitude worse than the split
    engines."""
    import ctypes
    lib = N.load()
    rng = np.random.default_rng(1606)
    count = 4096
    mag = np.repeat(10.0 ** rng.uniform(-3, 3, (count // 128, 1)), 128, axis=0)
    x = (rng.standard_normal((count, 16)) + 1j * rng.standard_normal((count, 16))) * mag
    xin = torch.tensor(np.stack([x.real, x.imag], -1).astype(np.float32), device="cuda:0").contiguous()
    out = torch.empty_like(xin)
    st = lib.sg_tc_dft16(N.ENGINES[engine], count, ctypes.c_void_p(xin.data_ptr()),
                         ctypes.c_void_p(out.data_ptr()), int(inverse), None)
    assert st == N.SG_OK
    torch.cuda.synchronize()
    xr = xin.double().cpu().numpy()
    z = xr[..., 0] + 1j * xr[..., 1]
    ref = np.fft.ifft(z, axis=1) * 16 if inverse else np.fft.fft(z, axis=1)
    o = out.double().cpu().numpy()
    got = o[..., 0] + 1j * o[..., 1]
    err = float(np.max(np.abs(got - ref).max(axis=1) / np.abs(ref).max(axis=1)))
    if tol is None:
        assert err > 1e-3, err
    else:
        assert err <= tol, (engine, err)


def test_tcgen05_single_stage_argument_checks():
    import ctypes
    lib = N.load()
    buf = torch.empty(256 * 16 * 2, device="cuda:0")
    p = ctypes.c_void_p(buf.data_ptr())
    assert lib.sg_tc_dft16(N.ENGINES["fft32"], 256, p, p, 0, None) == N.SG_ERR_ARG
    assert lib.sg_tc_dft16(N.ENGINES["dft_fp16x3"], 256, p, p, 0, None) == N.SG_ERR_ARG
    assert lib.sg_tc_dft16(N.ENGINES["tc_bf16x3"], 100, p, p, 0, None) == N.SG_ERR_ARG
    assert lib.sg_tc_dft16(N.ENGINES["tc_bf16x3"], 0, p, p, 0, None) == N.SG_ERR_ARG
    assert lib.sg_tc_dft16(N.ENGINES["tc_bf16x3"], 256, None, p, 0, None) == N.SG_ERR_ARG
    # misaligned or overlapping device buffers are refused, not launched
    out = torch.empty(256 * 16 * 2, device="cuda:0")
    q = ctypes.c_void_p(out.data_ptr())
    assert lib.sg_tc_dft16(N.ENGINES["tc_bf16x3"], 256, p, p, 0, None) == N.SG_ERR_ARG
    assert lib.sg_tc_dft16(N.ENGINES["tc_bf16x3"], 256, ctypes.c_void_p(buf.data_ptr() + 4), q, 0,
                           None) == N.SG_ERR_ARG
    src = torch.randn(256 * 16 * 2, device="cuda:0")
    assert lib.sg_tc_dft16(N.ENGINES["tc_bf16x3"], 256, ctypes.c_void_p(src.data_ptr()), q, 0, None) == N.SG_OK
    torch.cuda.synchronize()
