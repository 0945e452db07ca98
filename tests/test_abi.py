"""The C ABI library builds, loads and exports every function include/sg.h
declares; host-side argument checks reject bad plans before any CUDA call.
(No compute call here: this file runs without a GPU.)"""
import ctypes
import os
import re

import pytest

from paper_2506_10812_gb300 import _native as N
from paper_2506_10812_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return N.load()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "sg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sg_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_five_paper_entry_points():
    names = declared_functions()
    for f in ("sg_plan_create", "sg_kernel_table", "sg_potential", "sg_accel", "sg_destroy"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert set(names) == set(N.EXPORTS)
    for f in names:
        assert hasattr(lib, f), f


def test_library_is_built_for_sm103a():
    # the build passes exactly one -gencode, for sm_103a
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(B.LIB_PATH)


def _params(**kw):
    p = N.SgParams()
    p.nr, p.nphi, p.r_in, p.r_out, p.h_g, p.h_d, p.G = 64, 128, 0.2, 2.5, 0.05, 0.0, 1.0
    p.dtype, p.method = N.SG_F32, N.SG_METHOD_FFT
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("kw,status", [
    (dict(r_in=2.0, r_out=1.0), N.SG_ERR_ARG),
    (dict(r_in=0.0), N.SG_ERR_ARG),
    (dict(nr=0), N.SG_ERR_ARG),
    (dict(h_g=0.0), N.SG_ERR_ARG),
    (dict(h_g=float("nan")), N.SG_ERR_ARG),
    (dict(G=float("inf")), N.SG_ERR_ARG),
    (dict(dtype=7), N.SG_ERR_ARG),
    (dict(method=5), N.SG_ERR_ARG),
    (dict(nr=48), N.SG_ERR_UNSUPPORTED),
    (dict(nphi=16), N.SG_ERR_UNSUPPORTED),
    (dict(nr=8192), N.SG_ERR_UNSUPPORTED),
    (dict(H_g_field=1234), N.SG_ERR_NOT_FFT_COMPATIBLE),
])
def test_plan_argument_checks(lib, kw, status):
    h = ctypes.c_void_p(99)
    p = _params(**kw)
    st = lib.sg_plan_create(ctypes.byref(h), ctypes.byref(p), None)
    assert st == status
    assert not h.value


def test_null_arguments(lib):
    assert lib.sg_plan_create(None, None, None) == N.SG_ERR_ARG
    h = ctypes.c_void_p()
    assert lib.sg_plan_create(ctypes.byref(h), None, None) == N.SG_ERR_ARG
    assert lib.sg_solve(None, *([None] * 9)) == N.SG_ERR_ARG
    assert lib.sg_potential(None, None, None, None, None, None) == N.SG_ERR_ARG
    assert lib.sg_accel(None, *([None] * 7)) == N.SG_ERR_ARG
    assert lib.sg_kernel_table(None, 0, 0, None, None) == N.SG_ERR_ARG
    assert lib.sg_launches_per_solve(None, 7) == 0
    lib.sg_destroy(None)
    assert lib.sg_last_error(None) == b""
    # batch entry points reject NULL / empty batches before any CUDA call
    assert lib.sg_batch_create(None, None, 0, None, None, None, None, None) == N.SG_ERR_ARG
    assert lib.sg_batch_create(ctypes.byref(h), None, 1, None, None, None, None, None) == N.SG_ERR_ARG
    assert h.value is None
    plans = (ctypes.c_void_p * 1)(None)
    assert lib.sg_batch_create(ctypes.byref(h), plans, 0, plans, plans, plans, None, None) == N.SG_ERR_ARG
    for fn in (lib.sg_batch_solve, lib.sg_batch_solve_loop, lib.sg_batch_sync):
        assert fn(None, None) == N.SG_ERR_ARG
    assert lib.sg_batch_release(None) == N.SG_ERR_ARG
    assert lib.sg_batch_config(None, None, None, None, None) == N.SG_ERR_ARG
    assert lib.sg_batch_tune_results(None, 0, None, None) == -1
    lib.sg_batch_destroy(None)
    assert lib.sg_batch_last_error(None) == b""


def test_tc_dft16_argument_checks(lib):
    """The single-stage tensor-core entry point rejects a non-tcgen05 engine,
    a count that is not a positive multiple of 256, NULL, misaligned and
    overlapping buffers before any CUDA call (the pointers are never
    dereferenced)."""
    tc = N.ENGINES["tc_bf16x3"]
    a, b = ctypes.c_void_p(0x10000000), ctypes.c_void_p(0x20000000)
    span = 256 * 16 * 8
    assert lib.sg_tc_dft16(N.ENGINES["fft32"], 256, a, b, 0, None) == N.SG_ERR_ARG
    assert lib.sg_tc_dft16(tc, 255, a, b, 0, None) == N.SG_ERR_ARG
    assert lib.sg_tc_dft16(tc, -256, a, b, 0, None) == N.SG_ERR_ARG
    assert lib.sg_tc_dft16(tc, 256, None, b, 0, None) == N.SG_ERR_ARG
    assert lib.sg_tc_dft16(tc, 256, ctypes.c_void_p(0x10000004), b, 0, None) == N.SG_ERR_ARG
    assert lib.sg_tc_dft16(tc, 256, a, ctypes.c_void_p(0x20000004), 0, None) == N.SG_ERR_ARG
    assert lib.sg_tc_dft16(tc, 256, a, a, 0, None) == N.SG_ERR_ARG
    assert lib.sg_tc_dft16(tc, 256, a, ctypes.c_void_p(0x10000000 + span - 8), 0, None) == N.SG_ERR_ARG
    assert lib.sg_tc_dft16(tc, 256, ctypes.c_void_p(0x10000000 + span - 8), a, 0, None) == N.SG_ERR_ARG


def test_nn_gemm_argument_checks(lib):
    """sg_nn_gemm refuses short leading dimensions, negative strides and
    pointers not aligned to their element before any CUDA call."""
    a, b, c = ctypes.c_void_p(0x10000000), ctypes.c_void_p(0x20000000), ctypes.c_void_p(0x30000000)
    M, Nn, K = 64, 32, 48

    def call(A=a, lda=K, sa=0, ta=0, B=b, ldb=Nn, sb=0, beta=0.0, C=c, ldc=Nn, sc=0, Cb=None, bias=None):
        return lib.sg_nn_gemm(2, M, Nn, K, 1.0, A, lda, sa, ta, B, ldb, sb, beta, C, ldc, sc, Cb, bias, None)

    assert call(lda=K - 1) == N.SG_ERR_ARG
    assert call(ta=1, lda=M - 1) == N.SG_ERR_ARG
    assert call(ldb=Nn - 1) == N.SG_ERR_ARG
    assert call(ldc=Nn - 1) == N.SG_ERR_ARG
    assert call(sa=-1) == N.SG_ERR_ARG
    assert call(sb=-1) == N.SG_ERR_ARG
    assert call(sc=-1) == N.SG_ERR_ARG
    assert call(A=ctypes.c_void_p(0x10000001)) == N.SG_ERR_ARG
    assert call(B=ctypes.c_void_p(0x20000001)) == N.SG_ERR_ARG
    assert call(C=ctypes.c_void_p(0x30000002)) == N.SG_ERR_ARG
    assert call(C=None, Cb=ctypes.c_void_p(0x30000001)) == N.SG_ERR_ARG
    assert call(bias=ctypes.c_void_p(0x40000002)) == N.SG_ERR_ARG
    assert call(C=None, beta=1.0, Cb=c) == N.SG_ERR_ARG


def test_nn_pieces_refuse_misaligned_pointers(lib):
    """The surrogate's elementwise and spectral entry points refuse pointers
    not aligned to their element and int-overflowing counts before any CUDA
    call."""
    f4, odd = ctypes.c_void_p(0x10000000), ctypes.c_void_p(0x10000002)
    c8 = ctypes.c_void_p(0x20000000)
    assert lib.sg_nn_spec_combine(2, 4, 4, 8, f4, odd, None) == N.SG_ERR_ARG
    assert lib.sg_nn_spec_combine(2, 4, 4, 8, odd, c8, None) == N.SG_ERR_ARG
    assert lib.sg_nn_spec_combine(65536, 1024, 64, 64, f4, c8, None) == N.SG_ERR_ARG
    assert lib.sg_nn_spec_combine_bwd(2, 4, 4, 8, ctypes.c_void_p(0x20000004), f4, None) == N.SG_ERR_ARG
    assert lib.sg_nn_modemix(2, 4, 4, 8, c8, ctypes.c_void_p(0x20000004), f4, None) == N.SG_ERR_ARG
    assert lib.sg_nn_modemix_bwd(2, 4, 4, 8, c8, c8, odd, c8, None, None) == N.SG_ERR_ARG
    assert lib.sg_nn_act(16, odd, f4, 1, None) == N.SG_ERR_ARG
    assert lib.sg_nn_act(16, f4, ctypes.c_void_p(0x10000001), 1, None) == N.SG_ERR_ARG
    assert lib.sg_nn_cast(16, odd, f4, None) == N.SG_ERR_ARG
    assert lib.sg_nn_colsum(4, 4, f4, odd, 0, None) == N.SG_ERR_ARG
    assert lib.sg_nn_transpose(65536, 65536, f4, f4, None) == N.SG_ERR_ARG
    assert lib.sg_nn_pack_targets(1, 16, f4, f4, f4, odd, 0, None) == N.SG_ERR_ARG


def test_status_strings(lib):
    for s in range(8):
        assert lib.sg_status_string(s)
    assert lib.sg_status_string(N.SG_OK) == b"ok"
