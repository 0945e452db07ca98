"""ctypes declarations of the C ABI in ``include/sg.h`` (``libsg.so``).

Loading fails loudly when the library has not been built: there is no CPU
fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsg.so")

SG_OK, SG_ERR_ARG, SG_ERR_UNSUPPORTED, SG_ERR_NOT_FFT_COMPATIBLE, SG_ERR_CUDA, SG_ERR_OOM, \
    SG_ERR_NONFINITE, SG_ERR_TIMEOUT = range(8)
SG_F32, SG_F64 = 0, 1
SG_METHOD_FFT, SG_METHOD_DIRECT, SG_METHOD_SEMISPECTRAL = 0, 1, 2
SG_PAIR_GG, SG_PAIR_GD, SG_PAIR_DG, SG_PAIR_DD = 0, 1, 2, 3
SG_COMP_PHI, SG_COMP_R, SG_COMP_AZ = 0, 1, 2
SG_CHECK_FINITE = 2
SG_BATCH_HOST_GATE = 4
SG_BATCH_ORDER_PIPELINED, SG_BATCH_ORDER_STAGED = 0, 1
SG_NN_GEMM_TCGEN05, SG_NN_GEMM_MMA_SYNC = 0, 1
SG_COLS_STAGE_ALL, SG_COLS_STAGE_STEP = 0, 1
SG_ENGINE_FFT32, SG_ENGINE_DFT_FP16X3, SG_ENGINE_DFT_BF16X3, SG_ENGINE_DFT_FP16, SG_ENGINE_DFT_BF16, \
    SG_ENGINE_TC_BF16X3, SG_ENGINE_TC_TF32X3, SG_ENGINE_TC_BF16 = range(8)
ENGINES = {"fft32": 0, "dft_fp16x3": 1, "dft_bf16x3": 2, "dft_fp16": 3, "dft_bf16": 4,
           "tc_bf16x3": 5, "tc_tf32x3": 6, "tc_bf16": 7, "tc_fp16x3": 8}

# Every symbol include/sg.h declares (checked by the ABI test).
EXPORTS = ("sg_plan_create", "sg_kernel_table", "sg_potential", "sg_accel", "sg_solve",
           "sg_solve_host", "sg_indirect", "sg_sync", "sg_set_stage_events", "sg_stage_times", "sg_launches_per_solve", "sg_direct_noalloc", "sg_set_column_engine", "sg_tc_dft16", "sg_get_tiles", "sg_set_tiles", "sg_batch_create", "sg_batch_solve",
           "sg_batch_solve_loop", "sg_batch_release", "sg_batch_sync", "sg_batch_config", "sg_batch_tune_results", "sg_batch_tile_trials", "sg_batch_destroy",
           "sg_batch_last_error", "sg_nn_set_gemm_engine", "sg_nn_check", "sg_nn_gemm", "sg_nn_spec_combine", "sg_nn_spec_combine_bwd", "sg_nn_modemix",
           "sg_nn_modemix_bwd", "sg_nn_act", "sg_nn_act_bwd", "sg_nn_colsum", "sg_nn_rel_l2", "sg_nn_adam", "sg_nn_cast",
           "sg_nn_transpose", "sg_nn_fields", "sg_nn_pack_inputs", "sg_nn_pack_targets", "sg_destroy", "sg_status_string", "sg_last_error")


class SgParams(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int32), ("nphi", ctypes.c_int32),
                ("r_in", ctypes.c_double), ("r_out", ctypes.c_double),
                ("h_g", ctypes.c_double), ("h_d", ctypes.c_double),
                ("H_g_field", ctypes.c_void_p), ("H_d_field", ctypes.c_void_p),
                ("G", ctypes.c_double), ("dtype", ctypes.c_int32), ("method", ctypes.c_int32),
                ("flags", ctypes.c_uint32)]


class SgBatchOpts(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("order", ctypes.c_int32),
                ("specialize", ctypes.c_int32), ("autotune", ctypes.c_int32), ("flags", ctypes.c_uint32), ("timeout_ms", ctypes.c_double),
                ("streams", ctypes.c_int32)]


class SgTiles(ctypes.Structure):
    _fields_ = [("rows_fwd", ctypes.c_int32), ("rows_inv", ctypes.c_int32), ("cols_staging", ctypes.c_int32)]


class SgTileTrial(ctypes.Structure):
    _fields_ = [("disc", ctypes.c_int32), ("nr", ctypes.c_int32), ("nphi", ctypes.c_int32),
                ("nsrc", ctypes.c_int32), ("tiles", SgTiles), ("ms", ctypes.c_float), ("chosen", ctypes.c_int32)]


COLS_STAGING = {"all": 0, "step": 1}


class SgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None


def load() -> ctypes.CDLL:
    """Load ``libsg.so`` (built in-tree by ``paper_2506_10812_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                           "(python -m paper_2506_10812_gb300.build)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32
    st = ctypes.c_int
    lib.sg_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(SgParams), vp]
    lib.sg_plan_create.restype = st
    lib.sg_kernel_table.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp]
    lib.sg_kernel_table.restype = st
    lib.sg_potential.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.sg_potential.restype = st
    lib.sg_accel.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.sg_accel.restype = st
    lib.sg_solve.argtypes = [vp] * 10
    lib.sg_solve.restype = st
    lib.sg_solve_host.argtypes = [vp] * 10
    lib.sg_solve_host.restype = st
    lib.sg_indirect.argtypes = [vp, vp, vp, vp, vp]
    lib.sg_indirect.restype = st
    lib.sg_sync.argtypes = [vp, vp]
    lib.sg_sync.restype = st
    lib.sg_set_stage_events.argtypes = [vp, ctypes.POINTER(vp)]
    lib.sg_set_stage_events.restype = st
    lib.sg_stage_times.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_float)]
    lib.sg_stage_times.restype = st
    lib.sg_direct_noalloc.argtypes = [ctypes.POINTER(SgParams)] + [vp] * 9
    lib.sg_direct_noalloc.restype = st
    lib.sg_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), i32, ctypes.POINTER(vp),
                                    ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(SgBatchOpts), vp]
    lib.sg_batch_create.restype = st
    for name in ("sg_batch_solve", "sg_batch_solve_loop", "sg_batch_sync"):
        getattr(lib, name).argtypes = [vp, vp]
        getattr(lib, name).restype = st
    lib.sg_batch_release.argtypes = [vp]
    lib.sg_batch_release.restype = st
    lib.sg_batch_config.argtypes = [vp, ctypes.POINTER(SgBatchOpts), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                    ctypes.POINTER(ctypes.c_float)]
    lib.sg_batch_config.restype = st
    lib.sg_batch_tune_results.argtypes = [vp, i32, ctypes.POINTER(SgBatchOpts), ctypes.POINTER(ctypes.c_float)]
    lib.sg_batch_tune_results.restype = i32
    lib.sg_batch_destroy.argtypes = [vp]
    lib.sg_batch_destroy.restype = None
    lib.sg_batch_last_error.argtypes = [vp]
    lib.sg_batch_last_error.restype = ctypes.c_char_p
    lib.sg_set_column_engine.argtypes = [vp, i32]
    lib.sg_set_column_engine.restype = st
    lib.sg_tc_dft16.argtypes = [i32, ctypes.c_int64, vp, vp, i32, vp]
    lib.sg_tc_dft16.restype = st
    lib.sg_get_tiles.argtypes = [vp, ctypes.POINTER(SgTiles)]
    lib.sg_get_tiles.restype = st
    lib.sg_set_tiles.argtypes = [vp, ctypes.POINTER(SgTiles)]
    lib.sg_set_tiles.restype = st
    lib.sg_batch_tile_trials.argtypes = [vp, i32, ctypes.POINTER(SgTileTrial)]
    lib.sg_batch_tile_trials.restype = i32
    i64, f32 = ctypes.c_int64, ctypes.c_float
    nn = {
        "sg_nn_gemm": [i32, i32, i32, i32, f32, vp, i32, i64, i32, vp, i32, i64, f32, vp, i32, i64, vp, vp, vp],
        "sg_nn_spec_combine": [i32, i32, i32, i32, vp, vp, vp],
        "sg_nn_spec_combine_bwd": [i32, i32, i32, i32, vp, vp, vp],
        "sg_nn_modemix": [i32, i32, i32, i32, vp, vp, vp, vp],
        "sg_nn_modemix_bwd": [i32, i32, i32, i32, vp, vp, vp, vp, vp, vp],
        "sg_nn_act": [i64, vp, vp, i32, vp],
        "sg_nn_act_bwd": [i64, vp, vp, vp, vp, i32, vp],
        "sg_nn_colsum": [i64, i32, vp, vp, i32, vp],
        "sg_nn_rel_l2": [i32, i64, i32, vp, vp, vp, vp, vp],
        "sg_nn_adam": [i64, vp, vp, vp, vp, f32, f32, f32, f32, i32, vp, vp],
        "sg_nn_cast": [i64, vp, vp, vp],
        "sg_nn_transpose": [i32, i32, vp, vp, vp],
        "sg_nn_fields": [i32, i32, i32, vp, vp, vp, vp],
        "sg_nn_pack_inputs": [i32, i32, i32, vp, vp, vp, vp, vp],
        "sg_nn_pack_targets": [i32, i64, vp, vp, vp, vp, i32, vp],
    }
    lib.sg_nn_set_gemm_engine.argtypes = [i32]
    lib.sg_nn_set_gemm_engine.restype = st
    lib.sg_nn_check.argtypes = [vp]
    lib.sg_nn_check.restype = st
    for name, args in nn.items():
        getattr(lib, name).argtypes = args
        getattr(lib, name).restype = st
    lib.sg_launches_per_solve.argtypes = [vp, u32]
    lib.sg_launches_per_solve.restype = i32
    lib.sg_destroy.argtypes = [vp]
    lib.sg_destroy.restype = None
    lib.sg_status_string.argtypes = [st]
    lib.sg_status_string.restype = ctypes.c_char_p
    lib.sg_last_error.argtypes = [vp]
    lib.sg_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def check(status: int, plan_handle=None, what: str = "sg call", batch_handle=None) -> None:
    if status == SG_OK:
        return
    lib = load()
    msg = lib.sg_status_string(status).decode()
    if plan_handle or batch_handle:
        detail = (lib.sg_batch_last_error(batch_handle) if batch_handle else lib.sg_last_error(plan_handle)).decode()
        if detail:
            msg = f"{msg}: {detail}"
    raise SgError(status, f"{what}: {msg}")
