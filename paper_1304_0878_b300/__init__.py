"""b3t: a task-DAG executor for one B300 GPU.

The task-programming model of Courtes, "C Language Extensions for Hybrid
CPU/GPU Programming with StarPU" (Section 2): tasks declared with their
implementation and per-buffer access modes, registered buffers,
asynchronous submission, dependencies derived from the access modes in
submission order, and a wait.  The C-ABI library (include/b3t.h,
libb3t.so) does all of it; this package only marshals arguments.
"""
from ._lib import (Context, B3TError, Config, lib, strerror, q_bytes, header_symbols,  # noqa: F401
                   ir_work_elems, resid_part_elems, vec_args, TRSV_L, GEMV_L, TRSV_LT, GEMV_LT, AXPY, RESID, NRM,
                   VEC_F32, VEC_ASSIGN, VEC_LOWER_M, VEC_UPPER_M, TRTRI, TRMM_MX,
                   SLICE_A, SLICE_X, RESID_SL, SLICE_W, SLICE_U, TRMM_SL, ir_slice_bytes, slice_a_part_bytes,
                   slice_x_part_bytes, slice_w_bytes, slice_u_bytes, slice_args, TRTRI_COL,
                   pack_f32, pack_i32, R, W, RW, NOOP, SCAL_F32, POTRF, TRSM, SYRK, GEMM,
                   POTRF_MX, TRSM_MX, SYRK_MX, GEMM_MX, QUANT, FMT_BF16, FMT_E4M3,
                   PRIO_UPWARD, PRIO_DEPTH, PRIO_CRITICAL, POTRF_D, PANEL_TRSM, PANEL_UPD, CVT)
from . import tiles  # noqa: F401
