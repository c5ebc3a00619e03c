"""ctypes binding of libb3t.so: argument marshalling only.

Every function of include/b3t.h is reachable here under the same name
without the ``b3t_`` prefix, as a method of :class:`Context`.  Every step of
the task path (dependency derivation, task table build, scheduling, task
bodies) runs in the library; nothing here computes.  A negative return code
raises :class:`B3TError`.  The library must exist: there is no fallback.
"""
import ctypes
import errno
import os
import re
import struct

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libb3t.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "b3t.h")

R, W, RW = 1, 2, 3
NOOP, SCAL_F32, POTRF, TRSM, SYRK, GEMM = 0, 1, 2, 3, 4, 5
POTRF_MX, TRSM_MX, SYRK_MX, GEMM_MX, QUANT = 6, 7, 8, 9, 10
FMT_BF16, FMT_E4M3 = 0, 1
PRIO_CRITICAL, PRIO_DEPTH, PRIO_UPWARD = 0, 1, 2
TRSV_L, GEMV_L, TRSV_LT, GEMV_LT, AXPY, RESID, NRM = 11, 12, 13, 14, 15, 16, 17
VEC_F32, VEC_ASSIGN, VEC_LOWER_M, VEC_UPPER_M, VEC_KEEP_NORM = 1, 2, 4, 8, 16
POTRF_D, PANEL_TRSM, PANEL_UPD, CVT, TRTRI, TRMM_MX = 18, 19, 20, 21, 22, 23
SLICE_A, SLICE_X, RESID_SL, SLICE_W, SLICE_U, TRMM_SL = 24, 25, 26, 27, 28, 29
TRTRI_COL = 30


class B3TError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, strerror(code), code))


class Config(ctypes.Structure):
    _fields_ = [("timeout_ns", ctypes.c_int64), ("ctas_per_sm", ctypes.c_int32),
                ("prio_levels", ctypes.c_int32), ("debug_checks", ctypes.c_int32),
                ("host_only", ctypes.c_int32), ("prio_policy", ctypes.c_int32),
                ("stream_free_sms", ctypes.c_int32), ("stream_no_mx", ctypes.c_int32),
                ("item_chains", ctypes.c_int32)]


_lib = None
_i32, _i64, _vp, _sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t
_pi32, _pi64 = ctypes.POINTER(_i32), ctypes.POINTER(_i64)
_pu8 = ctypes.POINTER(ctypes.c_uint8)

_SIGS = {
    "b3t_q_bytes": (_sz, [ctypes.c_int, ctypes.c_int]),
    "b3t_init": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(Config), _vp]),
    "b3t_shutdown": (ctypes.c_int, [_vp]),
    "b3t_task_decl": (ctypes.c_int, [_vp, ctypes.c_char_p, ctypes.c_int, ctypes.c_int, _pu8, _sz, _pi32]),
    "b3t_data_register": (ctypes.c_int, [_vp, _vp, _sz, _sz, _i64, _pi32]),
    "b3t_data_lookup": (ctypes.c_int, [_vp, _vp, _pi32]),
    "b3t_data_partition": (ctypes.c_int, [_vp, _i32, _i32, _sz, _pi32]),
    "b3t_task_submit": (ctypes.c_int, [_vp, _i32, _pi32, _pu8, ctypes.c_int, _vp, _sz]),
    "b3t_task_submit_ptrs": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(_vp), ctypes.c_int, _vp, _sz]),
    "b3t_task_flush": (ctypes.c_int, [_vp]),
    "b3t_task_wait": (ctypes.c_int, [_vp, _i64]),
    "b3t_data_acquire": (ctypes.c_int, [_vp, _i32, ctypes.c_uint8]),
    "b3t_data_unregister": (ctypes.c_int, [_vp, _i32]),
    "b3t_last_error": (ctypes.c_int, [_vp, _pi32, _pi32]),
    "b3t_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "b3t_graph_capture_begin": (ctypes.c_int, [_vp]),
    "b3t_graph_capture_end": (ctypes.c_int, [_vp, _pi32]),
    "b3t_graph_replay": (ctypes.c_int, [_vp, _i32]),
    "b3t_graph_destroy": (ctypes.c_int, [_vp, _i32]),
    "b3t_dag_stats": (ctypes.c_int, [_vp, _pi64, _pi64]),
    "b3t_dag_edges": (ctypes.c_int, [_vp, _pi32, _pi32, _i64, _pi64]),
    "b3t_dag_levels": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_float), _pi32, _i64, _pi64]),
    "b3t_dag_item_chains": (ctypes.c_int, [_vp, _pi32, _i64, _pi64]),
    "b3t_last_launch": (ctypes.c_int, [_vp, _pi64, _pi64, _pi32, _pi64]),
    "b3t_debug_block_task": (ctypes.c_int, [_vp, _i64]),
    "b3t_cholesky_submit": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), _i32, _i32, _i32]),
    "b3t_cholesky_mx_submit": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                              ctypes.POINTER(_vp), _i32, _i32, _i32, _i32]),
    "b3t_cholesky_mx_inv_submit": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                                  ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i32, _i32, _i32,
                                                  _i32]),
    "b3t_tiles_unregister": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), _i32]),
    "b3t_scal_chains_noalloc": (ctypes.c_int, [_vp, _i64, _i32, _i32, _vp, _i64, _vp]),
    "b3t_stream_open": (ctypes.c_int, [_vp, _i64, _i64, _i32, _i64]),
    "b3t_stream_submit": (ctypes.c_int, [_vp, _pi32]),
    "b3t_stream_query": (ctypes.c_int, [_vp, _i32, _pi32]),
    "b3t_stream_close": (ctypes.c_int, [_vp]),
    "b3t_chol_solve_submit": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), _vp, _i32, _i32, _i32, _i64, _i32]),
    "b3t_ir_work_elems": (_sz, [_i32, _i32, _i32]),
    "b3t_resid_part_elems": (_sz, [_i32, _i32]),
    "b3t_chol_inv_submit": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i32, _i32]),
    "b3t_chol_solve_inv_submit": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp, _vp, _i32,
                                                 _i32, _i32, _i64, _i32]),
    "b3t_ir_release": (ctypes.c_int, [_vp, _vp, _i32, _i32, _i32]),
    "b3t_trace_start": (ctypes.c_int, [_vp, _i64]),
    "b3t_trace_read": (ctypes.c_int, [_vp, _vp, _i64, ctypes.POINTER(_i64)]),
    "b3t_trace_stop": (ctypes.c_int, [_vp]),
    "b3t_ir_step_submit": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(_vp), _vp, _vp, _vp, _vp, _i32, _i32,
                                          _i32, _i32, _i32]),
    "b3t_ir_solve": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(_vp), _vp, _vp, _vp, _vp, _i32, _i32, _i32,
                                    _i32, ctypes.c_double, _i32, _pi32, ctypes.POINTER(ctypes.c_double)]),
    "b3t_ir_slice_bytes": (_sz, [_i32, _i32]),
    "b3t_slice_a_part_bytes": (_sz, [_i32]),
    "b3t_slice_x_part_bytes": (_sz, [_i32]),
    "b3t_slice_w_bytes": (_sz, [_i32]),
    "b3t_slice_u_bytes": (_sz, [_i32]),
    "b3t_cholesky_mx_sliced_submit": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                                     ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                                     ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i32, _i32, _i32,
                                                     _i32]),
    "b3t_ir_solve_sliced": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(_vp), _vp, _vp, _vp, _vp, _vp, _i32, _i32,
                                           _i32, _i32, ctypes.c_double, _i32, _pi32,
                                           ctypes.POINTER(ctypes.c_double)]),
}


def header_symbols():
    """Names of every function include/b3t.h declares."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"B3T_API\s+[\w\s\*]*?\b(b3t_\w+)\s*\(", txt)))


def lib():
    """Load libb3t.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libb3t.so not built: run python -m paper_1304_0878_b300.build "
                              "(there is no fallback path)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(code):
    return lib().b3t_strerror(code).decode()


def _check(rc, where):
    if rc < 0:
        raise B3TError(rc, where)
    return rc


def _ptrs(seq):
    arr = (_vp * len(seq))()
    for i, p in enumerate(seq):
        arr[i] = int(p)
    return arr


def q_bytes(b, fmt):
    return int(lib().b3t_q_bytes(b, fmt))


def ir_work_elems(T, b, nrhs):
    return int(lib().b3t_ir_work_elems(T, b, nrhs))


def resid_part_elems(b, nrhs):
    return int(lib().b3t_resid_part_elems(b, nrhs))


def vec_args(nrhs, flags=0, i=0, T=1, b=64):
    return struct.pack("<5i", nrhs, flags, i, T, b)


def ir_slice_bytes(T, b):
    return int(lib().b3t_ir_slice_bytes(T, b))


def slice_a_part_bytes(b):
    return int(lib().b3t_slice_a_part_bytes(b))


def slice_x_part_bytes(b):
    return int(lib().b3t_slice_x_part_bytes(b))


def slice_w_bytes(b):
    return int(lib().b3t_slice_w_bytes(b))


def slice_u_bytes(b):
    return int(lib().b3t_slice_u_bytes(b))


def slice_args(i, j, T, b, nrhs):
    return struct.pack("<5i", i, j, T, b, nrhs)


class Context:
    """One b3t context bound to a CUDA stream (a raw cudaStream_t value such
    as ``torch.cuda.current_stream().cuda_stream``)."""

    def __init__(self, stream=0, timeout_ns=0, ctas_per_sm=0, prio_levels=0, debug=False,
                 host_only=False, prio_policy=0, stream_free_sms=0, stream_no_mx=False, item_chains=False):
        cfg = Config(timeout_ns, ctas_per_sm, prio_levels, 1 if debug else 0, 1 if host_only else 0,
                     prio_policy, stream_free_sms, 1 if stream_no_mx else 0, 1 if item_chains else 0)
        h = _vp()
        _check(lib().b3t_init(ctypes.byref(h), ctypes.byref(cfg), _vp(stream or 0)), "b3t_init")
        self._h = h

    def close(self):
        if self._h:
            h, self._h = self._h, None
            _check(lib().b3t_shutdown(h), "b3t_shutdown")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                lib().b3t_shutdown(self._h)
        except Exception:
            pass

    # -- task model (Section 2 of the paper) ----------------------------------
    def task_decl(self, name, kind, modes, scalar_bytes=0):
        out = _i32()
        m = (ctypes.c_uint8 * max(1, len(modes)))(*modes)
        _check(lib().b3t_task_decl(self._h, name.encode(), kind, len(modes), m, scalar_bytes,
                                   ctypes.byref(out)), "b3t_task_decl")
        return out.value

    def data_register(self, ptr, nelems, elemsize, ld=0):
        out = _i32()
        _check(lib().b3t_data_register(self._h, _vp(int(ptr)), nelems, elemsize, ld, ctypes.byref(out)),
               "b3t_data_register")
        return out.value

    def data_lookup(self, ptr):
        out = _i32()
        _check(lib().b3t_data_lookup(self._h, _vp(int(ptr)), ctypes.byref(out)), "b3t_data_lookup")
        return out.value

    def data_partition(self, h, nparts, part_nelems):
        out = (_i32 * nparts)()
        _check(lib().b3t_data_partition(self._h, h, nparts, part_nelems, out), "b3t_data_partition")
        return list(out)

    def task_submit(self, cl, handles, scalars=b"", modes=None):
        hs = (_i32 * max(1, len(handles)))(*handles)
        ms = (ctypes.c_uint8 * len(modes))(*modes) if modes is not None else None
        buf = ctypes.create_string_buffer(scalars, len(scalars)) if scalars else None
        _check(lib().b3t_task_submit(self._h, cl, hs, ms, len(handles), buf, len(scalars)),
               "b3t_task_submit")

    def task_submit_ptrs(self, cl, ptrs, scalars=b""):
        buf = ctypes.create_string_buffer(scalars, len(scalars)) if scalars else None
        _check(lib().b3t_task_submit_ptrs(self._h, cl, _ptrs(ptrs), len(ptrs), buf, len(scalars)),
               "b3t_task_submit_ptrs")

    def task_flush(self):
        _check(lib().b3t_task_flush(self._h), "b3t_task_flush")

    def task_wait(self, timeout_ns=0):
        _check(lib().b3t_task_wait(self._h, timeout_ns), "b3t_task_wait")

    def data_acquire(self, h, mode=R):
        _check(lib().b3t_data_acquire(self._h, h, mode), "b3t_data_acquire")

    def data_unregister(self, h):
        _check(lib().b3t_data_unregister(self._h, h), "b3t_data_unregister")

    def last_error(self):
        t, i = _i32(), _i32()
        lib().b3t_last_error(self._h, ctypes.byref(t), ctypes.byref(i))
        return t.value, i.value

    # -- repeated DAGs ----------------------------------------------------------
    def graph_capture_begin(self):
        _check(lib().b3t_graph_capture_begin(self._h), "b3t_graph_capture_begin")

    def graph_capture_end(self):
        out = _i32()
        _check(lib().b3t_graph_capture_end(self._h, ctypes.byref(out)), "b3t_graph_capture_end")
        return out.value

    def graph_replay(self, g):
        _check(lib().b3t_graph_replay(self._h, g), "b3t_graph_replay")

    def graph_destroy(self, g):
        _check(lib().b3t_graph_destroy(self._h, g), "b3t_graph_destroy")

    # -- introspection ----------------------------------------------------------
    def dag_stats(self):
        n, e = _i64(), _i64()
        _check(lib().b3t_dag_stats(self._h, ctypes.byref(n), ctypes.byref(e)), "b3t_dag_stats")
        return n.value, e.value

    def dag_edges(self):
        _, ne = self.dag_stats()
        p, s, cnt = (_i32 * max(ne, 1))(), (_i32 * max(ne, 1))(), _i64()
        _check(lib().b3t_dag_edges(self._h, p, s, ne, ctypes.byref(cnt)), "b3t_dag_edges")
        return [(p[i], s[i]) for i in range(cnt.value)]

    def dag_levels(self):
        """(rank, level) per pending task, as the next flush will use them."""
        nt, _ = self.dag_stats()
        rk, lv, cnt = (ctypes.c_float * max(nt, 1))(), (_i32 * max(nt, 1))(), _i64()
        _check(lib().b3t_dag_levels(self._h, rk, lv, nt, ctypes.byref(cnt)), "b3t_dag_levels")
        return [rk[i] for i in range(cnt.value)], [lv[i] for i in range(cnt.value)]

    def dag_item_chains(self):
        """Per pending task: k > 0 heads an item chain of k absorbed SCAL
        tasks, -1 absorbed, 0 neither (as the next flush will form them)."""
        nt, _ = self.dag_stats()
        aux, cnt = (_i32 * max(nt, 1))(), _i64()
        _check(lib().b3t_dag_item_chains(self._h, aux, nt, ctypes.byref(cnt)), "b3t_dag_item_chains")
        return [aux[i] for i in range(cnt.value)]

    def last_launch(self):
        nt, ni, nc, ns = _i64(), _i64(), _i32(), _i64()
        _check(lib().b3t_last_launch(self._h, ctypes.byref(nt), ctypes.byref(ni), ctypes.byref(nc),
                                     ctypes.byref(ns)), "b3t_last_launch")
        return {"ntasks": nt.value, "nitems": ni.value, "nctas": nc.value, "kernel_ns": ns.value}

    def debug_block_task(self, i):
        _check(lib().b3t_debug_block_task(self._h, i), "b3t_debug_block_task")

    # -- tiled Cholesky helpers -------------------------------------------------
    def cholesky_submit(self, tile_ptrs, T, b, col0=0):
        _check(lib().b3t_cholesky_submit(self._h, _ptrs(tile_ptrs), T, b, col0), "b3t_cholesky_submit")

    def cholesky_mx_submit(self, W_ptrs, L_ptrs, Q_ptrs, T, b, fmt, col0=0):
        _check(lib().b3t_cholesky_mx_submit(self._h, _ptrs(W_ptrs), _ptrs(L_ptrs), _ptrs(Q_ptrs),
                                            T, b, fmt, col0), "b3t_cholesky_mx_submit")

    # -- stream mode (continuous submission) --------------------------------------
    def cholesky_mx_inv_submit(self, W_ptrs, L_ptrs, Q_ptrs, U_ptrs, T, b, fmt, col0=0):
        _check(lib().b3t_cholesky_mx_inv_submit(self._h, _ptrs(W_ptrs), _ptrs(L_ptrs), _ptrs(Q_ptrs),
                                                _ptrs(U_ptrs), T, b, fmt, col0), "b3t_cholesky_mx_inv_submit")

    def cholesky_mx_sliced_submit(self, W_ptrs, L_ptrs, Q_ptrs, U_ptrs, WS_ptrs, US_ptrs, T, b, fmt, col0=0):
        _check(lib().b3t_cholesky_mx_sliced_submit(self._h, _ptrs(W_ptrs), _ptrs(L_ptrs), _ptrs(Q_ptrs),
                                                   _ptrs(U_ptrs), _ptrs(WS_ptrs), _ptrs(US_ptrs), T, b, fmt,
                                                   col0), "b3t_cholesky_mx_sliced_submit")

    def stream_open(self, max_tasks, max_edges, max_batches, deadline_ns):
        _check(lib().b3t_stream_open(self._h, max_tasks, max_edges, max_batches, deadline_ns),
               "b3t_stream_open")

    def stream_submit(self):
        out = _i32()
        _check(lib().b3t_stream_submit(self._h, ctypes.byref(out)), "b3t_stream_submit")
        return out.value

    def stream_query(self, batch):
        """(done, info): done is True when the batch has finished."""
        info = _i32(0)
        rc = _check(lib().b3t_stream_query(self._h, batch, ctypes.byref(info)), "b3t_stream_query")
        return rc == 1, info.value

    def stream_close(self):
        _check(lib().b3t_stream_close(self._h), "b3t_stream_close")

    def chol_solve_submit(self, L_ptrs, Y_ptr, T, b, nrhs, part_stride, flags=0):
        _check(lib().b3t_chol_solve_submit(self._h, _ptrs(L_ptrs), _vp(int(Y_ptr)), T, b, nrhs,
                                           part_stride, flags), "b3t_chol_solve_submit")

    def chol_inv_submit(self, L_ptrs, U_ptrs, T, b):
        _check(lib().b3t_chol_inv_submit(self._h, _ptrs(L_ptrs), _ptrs(U_ptrs), T, b), "b3t_chol_inv_submit")

    def chol_solve_inv_submit(self, L_ptrs, U_ptrs, Y_ptr, Z_ptr, T, b, nrhs, part_stride, flags=0):
        _check(lib().b3t_chol_solve_inv_submit(self._h, _ptrs(L_ptrs), _ptrs(U_ptrs), _vp(int(Y_ptr)),
                                               _vp(int(Z_ptr)), T, b, nrhs, part_stride, flags),
               "b3t_chol_solve_inv_submit")

    def trace_start(self, capacity=1 << 20):
        _check(lib().b3t_trace_start(self._h, int(capacity)), "b3t_trace_start")
        self._trace_cap = int(capacity)

    def trace_read(self):
        """The traced work items as a numpy structured array (task, item, sm,
        kind, t_start_ns, t_end_ns)."""
        import numpy as np
        dt = np.dtype([("task", np.int32), ("item", np.int32), ("sm", np.int32), ("kind", np.int32),
                       ("t_start_ns", np.uint64), ("t_end_ns", np.uint64)])
        cap = getattr(self, "_trace_cap", 0)
        buf = np.zeros(cap, dtype=dt)
        n = _i64(0)
        _check(lib().b3t_trace_read(self._h, _vp(buf.ctypes.data), cap, ctypes.byref(n)), "b3t_trace_read")
        return buf[:min(n.value, cap)]

    def trace_stop(self):
        _check(lib().b3t_trace_stop(self._h), "b3t_trace_stop")

    def ir_release(self, R_ptr, T, b, nrhs):
        _check(lib().b3t_ir_release(self._h, _vp(int(R_ptr)), T, b, nrhs), "b3t_ir_release")

    def ir_solve(self, A_ptr, L_ptrs, B_ptr, X_ptr, R_ptr, eta_ptr, T, b, nrhs, flags=0, tol=1e-12,
                 max_iter=30):
        """Returns (return code, iterations, eta list); -ERANGE is returned,
        not raised, so that a non-converged refinement can be reported."""
        it = _i32(0)
        eta = (ctypes.c_double * (nrhs + 1))()
        rc = lib().b3t_ir_solve(self._h, _vp(int(A_ptr)), _ptrs(L_ptrs), _vp(int(B_ptr)), _vp(int(X_ptr)),
                                _vp(int(R_ptr)), _vp(int(eta_ptr)), T, b, nrhs, flags, tol, max_iter,
                                ctypes.byref(it), eta)
        if rc < 0 and rc != ERANGE:
            raise B3TError(rc, "b3t_ir_solve")
        return rc, it.value, list(eta)

    def ir_solve_sliced(self, A_ptr, L_ptrs, B_ptr, X_ptr, R_ptr, S_ptr, eta_ptr, T, b, nrhs, flags=0,
                        tol=1e-12, max_iter=30):
        """ir_solve with the sliced FP64 residual; S_ptr: ir_slice_bytes(T, b)
        bytes of device memory.  Returns (return code, iterations, eta list)."""
        it = _i32(0)
        eta = (ctypes.c_double * (nrhs + 1))()
        rc = lib().b3t_ir_solve_sliced(self._h, _vp(int(A_ptr)), _ptrs(L_ptrs), _vp(int(B_ptr)),
                                       _vp(int(X_ptr)), _vp(int(R_ptr)), _vp(int(S_ptr)), _vp(int(eta_ptr)),
                                       T, b, nrhs, flags, tol, max_iter, ctypes.byref(it), eta)
        if rc < 0 and rc != ERANGE:
            raise B3TError(rc, "b3t_ir_solve_sliced")
        return rc, it.value, list(eta)

    def ir_step_submit(self, A_ptr, L_ptrs, B_ptr, X_ptr, R_ptr, eta_ptr, T, b, nrhs, flags=0, first=True):
        _check(lib().b3t_ir_step_submit(self._h, _vp(int(A_ptr)), _ptrs(L_ptrs), _vp(int(B_ptr)),
                                        _vp(int(X_ptr)), _vp(int(R_ptr)), _vp(int(eta_ptr)), T, b, nrhs,
                                        flags, 1 if first else 0), "b3t_ir_step_submit")

    def tiles_unregister(self, tile_ptrs, T):
        _check(lib().b3t_tiles_unregister(self._h, _ptrs(tile_ptrs), T), "b3t_tiles_unregister")


def pack_f32(x):
    return struct.pack("<f", x)


def pack_i32(x):
    return struct.pack("<i", x)


ENOENT, EINVAL, EEXIST, EBUSY = -errno.ENOENT, -errno.EINVAL, -errno.EEXIST, -errno.EBUSY
ENODEV, ETIMEDOUT, EDOM, EIO = -errno.ENODEV, -errno.ETIMEDOUT, -errno.EDOM, -errno.EIO
E2BIG, ERANGE = -errno.E2BIG, -errno.ERANGE
